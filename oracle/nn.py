"""FP64 reference for the network constraint and its derivatives.

TEST INFRASTRUCTURE ONLY (see the package docstring): never called by the CUDA library.

Notation follows Eq. 3: layer l = 1..L computes z_l = W_l a_{l-1} + b_l and a_l = sigma_l(z_l),
with a_0 = x and NN(x) = a_L.  The reduced-space constraint is g(x, y) = y - NN(x) (Section
3.2), so the solver needs NN(x), its Jacobian dNN/dx and, by Eq. 6, the n x n matrix
sum_i lambda_i d2 NN_i / dx2, which the paper obtains by differentiating the scalar
lambda^T NN(x) twice.
"""
import numpy as np

# ---------------------------------------------------------------- activations
# sigma, sigma' and sigma'' written out from their definitions.


def act_value(name, z):
    if name == "identity":
        return z.copy()
    if name == "softmax":
        e = np.exp(z - np.max(z))
        return e / np.sum(e)
    if name == "tanh":
        return np.tanh(z)
    if name == "sigmoid":
        return 1.0 / (1.0 + np.exp(-z))
    if name == "softplus":
        return np.logaddexp(0.0, z)
    if name == "gelu":
        from scipy.special import erf
        return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))
    raise ValueError(name)


def act_d1(name, z):
    if name == "identity":
        return np.ones_like(z)
    if name == "tanh":
        t = np.tanh(z)
        return 1.0 - t * t
    if name == "sigmoid":
        s = 1.0 / (1.0 + np.exp(-z))
        return s * (1.0 - s)
    if name == "softplus":
        return 1.0 / (1.0 + np.exp(-z))
    if name == "gelu":
        from scipy.special import erf
        phi = np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)
        return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * phi
    raise ValueError(name)


def act_d2(name, z):
    if name == "identity":
        return np.zeros_like(z)
    if name == "tanh":
        t = np.tanh(z)
        return -2.0 * t * (1.0 - t * t)
    if name == "sigmoid":
        s = 1.0 / (1.0 + np.exp(-z))
        return s * (1.0 - s) * (1.0 - 2.0 * s)
    if name == "softplus":
        s = 1.0 / (1.0 + np.exp(-z))
        return s * (1.0 - s)
    if name == "gelu":
        phi = np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)
        return phi * (2.0 - z * z)
    raise ValueError(name)


# Layer maps as operators.  An elementwise activation has the Jacobian diag(sigma'(z)) and, for
# an adjoint abar, the curvature matrix grad_z^2 (abar^T sigma(z)) = diag(sigma''(z) * abar).  The
# softmax output layer (Section 4.1's classifiers), p_i = exp(z_i) / sum_j exp(z_j), couples its
# outputs: dp_i/dz_j = p_i (delta_ij - p_j), and
#   d2 p_i / dz_j dz_k = p_i [(delta_ij - p_j)(delta_ik - p_k) - p_j (delta_jk - p_k)],
# so both are full matrices, written out below from these definitions.


def softmax_second(p):
    """The tensor D[i, j, k] = d2 p_i / dz_j dz_k of the softmax at probabilities p."""
    n = p.size
    I = np.eye(n)
    A = I - p[None, :]                                   # A[i, j] = delta_ij - p_j
    return p[:, None, None] * (A[:, :, None] * A[:, None, :] -
                               p[None, :, None] * (I - p[None, None, :]))


def jac_apply(name, z, M):
    """D sigma(z) @ M for a matrix (or vector) M."""
    if name == "softmax":
        p = act_value(name, z)
        return p[:, None] * M - np.outer(p, p @ M) if M.ndim == 2 else p * M - p * (p @ M)
    d1 = act_d1(name, z)
    return d1[:, None] * M if M.ndim == 2 else d1 * M


def jacT_apply(name, z, M):
    """D sigma(z)^T @ M (the softmax Jacobian is symmetric; elementwise ones are diagonal)."""
    return jac_apply(name, z, M)


def curvature(name, z, abar):
    """The matrix grad_z^2 (abar^T sigma(z)), or for an elementwise activation its diagonal."""
    if name == "softmax":
        return np.einsum("i,ijk->jk", abar, softmax_second(act_value(name, z)))
    return act_d2(name, z) * abar


def curv_apply(name, z, abar, Zdot):
    """grad_z^2 (abar^T sigma(z)) @ Zdot."""
    c = curvature(name, z, abar)
    return c @ Zdot if c.ndim == 2 else c[:, None] * Zdot


# ---------------------------------------------------------------- Eq. 3


def forward(net, x):
    """Eq. 3.  Returns (zs, as_) with zs[l-1] = z_l and as_[l] = a_l (as_[0] = x)."""
    a = np.asarray(x, dtype=np.float64)
    zs, as_ = [], [a]
    for W, b, act in zip(net.W, net.b, net.spec.acts):
        z = W @ a + b
        a = act_value(act, z)
        zs.append(z)
        as_.append(a)
    return zs, as_


def value(net, x):
    """NN(x) = a_L."""
    return forward(net, x)[1][-1]


# ---------------------------------------------------------------- Jacobian (reverse mode)


def jacobian(net, x):
    """dNN/dx, shape (n_out, n_in), by reverse mode with one seed per output.

    Seeds abar_L = e_i for every output i at once (columns of the identity); then
    zbar_l = D sigma_l(z_l)^T abar_l (sigma_l'(z_l) * abar_l for an elementwise activation) and
    abar_{l-1} = W_l^T zbar_l.  Row i of J is abar_0 of seed i.
    """
    zs, _ = forward(net, x)
    L = len(net.W)
    Abar = np.eye(net.spec.n_out)                       # columns are seeds
    for l in range(L, 0, -1):
        Zbar = jacT_apply(net.spec.acts[l - 1], zs[l - 1], Abar)
        Abar = net.W[l - 1].T @ Zbar
    return Abar.T.copy()


def vjp(net, x, lam):
    """lambda^T dNN/dx (the gradient of lambda^T NN), by one reverse sweep with seed lambda."""
    zs, _ = forward(net, x)
    abar = np.asarray(lam, dtype=np.float64)
    for l in range(len(net.W), 0, -1):
        abar = net.W[l - 1].T @ jacT_apply(net.spec.acts[l - 1], zs[l - 1], abar)
    return abar


def adjoints(net, zs, lam):
    """abar_l for l = 0..L of the reverse sweep with seed abar_L = lambda."""
    L = len(net.W)
    abars = [None] * (L + 1)
    abars[L] = np.asarray(lam, dtype=np.float64)
    for l in range(L, 0, -1):
        abars[l - 1] = net.W[l - 1].T @ jacT_apply(net.spec.acts[l - 1], zs[l - 1], abars[l])
    return abars


# ---------------------------------------------------------------- Eq. 6: Hessian of lambda^T NN


def hessian_lag_for(net, x, lam):
    """sum_i lambda_i d2 NN_i/dx2 by forward-over-reverse, the literal sweep.

    The reverse sweep of `adjoints` computes grad(lambda^T NN)(x) = abar_0.  Differentiating
    every step of it in the n_in directions e_1..e_n at once (forward mode, tangents carried
    as matrix columns) gives the Hessian:
      forward tangents:  Adot_0 = I,  Zdot_l = W_l Adot_{l-1},  Adot_l = D sigma_l(z_l) Zdot_l
      reverse tangents:  dabar_L = 0 (lambda is constant),
                         dzbar_l = D sigma_l(z_l)^T dabar_l + M_l(abar_l) Zdot_l,
                         dabar_{l-1} = W_l^T dzbar_l
    with M_l(abar) = grad_z^2 (abar^T sigma_l(z_l)) (diag(sigma_l'' * abar) when elementwise), and
    H = dabar_0.  The result is returned as computed (no symmetrisation).
    """
    zs, _ = forward(net, x)
    abars = adjoints(net, zs, lam)
    L = len(net.W)
    n = net.spec.n_in
    Adot = np.eye(n)
    Zdots = []
    for l in range(1, L + 1):
        Zdot = net.W[l - 1] @ Adot
        Adot = jac_apply(net.spec.acts[l - 1], zs[l - 1], Zdot)
        Zdots.append(Zdot)
    dabar = np.zeros((net.spec.n_out, n))
    for l in range(L, 0, -1):
        act = net.spec.acts[l - 1]
        dzbar = jacT_apply(act, zs[l - 1], dabar) + curv_apply(act, zs[l - 1], abars[l], Zdots[l - 1])
        dabar = net.W[l - 1].T @ dzbar
    return dabar


def hessian_lag_layers(net, x, lam):
    """The same Hessian as a sum over layers: H = sum_l Zdot_l^T M_l(abar_l) Zdot_l, where
    M_l(abar_l) = diag(sigma_l''(z_l) * abar_l) for an elementwise activation.

    Unrolling the reverse-tangent recursion of `hessian_lag_for` (the affine maps add no
    curvature) leaves one term per layer, where Zdot_l = dz_l/dx and abar_l is the adjoint of
    a_l.  This is the form the GPU path evaluates; the oracle keeps both so that a test can
    hold them equal.
    """
    zs, _ = forward(net, x)
    abars = adjoints(net, zs, lam)
    L = len(net.W)
    n = net.spec.n_in
    Adot = np.eye(n)
    H = np.zeros((n, n))
    for l in range(1, L + 1):
        act = net.spec.acts[l - 1]
        Zdot = net.W[l - 1] @ Adot
        H += Zdot.T @ curv_apply(act, zs[l - 1], abars[l], Zdot)
        Adot = jac_apply(act, zs[l - 1], Zdot)
    return H


def hessian_lag(net, x, lam):
    """The oracle's answer for nnc_hessian_lag: the forward-over-reverse Hessian, symmetrised."""
    H = hessian_lag_for(net, x, lam)
    return 0.5 * (H + H.T)


def all_outputs(net, x, lam):
    """(y, J, H, grad) at one point: value, Jacobian, Hessian of lambda^T NN and its gradient."""
    return value(net, x), jacobian(net, x), hessian_lag(net, x, lam), vjp(net, x, lam)


def hessian_lag_columns(net, x, lam, cols):
    """Columns `cols` of the forward-over-reverse Hessian: the same sweeps as `hessian_lag_for`
    with only the tangents e_j, j in cols (Adot_0 = I[:, cols]).  Used to sample large Hessians."""
    zs, _ = forward(net, x)
    abars = adjoints(net, zs, lam)
    L = len(net.W)
    n = net.spec.n_in
    cols = np.asarray(cols, dtype=np.int64)
    Adot = np.eye(n)[:, cols]
    Zdots = []
    for l in range(1, L + 1):
        Zdot = net.W[l - 1] @ Adot
        Adot = jac_apply(net.spec.acts[l - 1], zs[l - 1], Zdot)
        Zdots.append(Zdot)
    dabar = np.zeros((net.spec.n_out, cols.size))
    for l in range(L, 0, -1):
        act = net.spec.acts[l - 1]
        dzbar = jacT_apply(act, zs[l - 1], dabar) + curv_apply(act, zs[l - 1], abars[l], Zdots[l - 1])
        dabar = net.W[l - 1].T @ dzbar
    return dabar
