"""The test problems of Section 4 in the form of Eq. 1, built on the oracle network.

TEST INFRASTRUCTURE ONLY.

Adversarial problems.  `adversarial_l1` is Eq. 7 itself (L1 objective through split variables,
softmax confidence threshold) with the network in the reduced space (Eq. 5);
`adversarial_l1_fullspace` the same problem with the network in the full space (Eq. 4);
`adversarial` is a smooth variant (L2 objective, logit margins):
    variables v = (x in [0,1]^n_in, y in R^n_out, s in R^(n_out-1), s >= 0)
    min ||x - x0||^2
    s.t. y - NN(x) = 0                                   (the reduced-space constraint, Eq. 5)
         y_t - y_j - margin - s_j = 0   for j != t       (target class wins by `margin`)
Start: x = x0, y = NN(x0), s_j = max(y_t - y_j - margin, 1e-2).
"""
import numpy as np

from . import nn as onn
from .ipm import Problem
from synth.problems import scopf_first_bias, scopf_demand  # noqa: F401  (problem data)


def adversarial(mlp, x0, target=3, margin=0.1):
    n_in, n_out = mlp.spec.n_in, mlp.spec.n_out
    others = [j for j in range(n_out) if j != target]
    ns = len(others)
    nv = n_in + n_out + ns
    m = n_out + ns
    ix, iy, is_ = slice(0, n_in), slice(n_in, n_in + n_out), slice(n_in + n_out, nv)
    lb = np.concatenate([np.zeros(n_in), np.full(n_out, -np.inf), np.zeros(ns)])
    ub = np.concatenate([np.ones(n_in), np.full(n_out, np.inf), np.full(ns, np.inf)])
    y0 = onn.value(mlp, x0)
    s0 = np.maximum(np.array([y0[target] - y0[j] - margin for j in others]), 1e-2)
    v0 = np.concatenate([x0, y0, s0])
    E = np.zeros((ns, n_out))
    for r, j in enumerate(others):
        E[r, target] = 1.0
        E[r, j] = -1.0

    def f(v):
        d = v[ix] - x0
        return float(d @ d)

    def grad_f(v):
        g = np.zeros(nv)
        g[ix] = 2.0 * (v[ix] - x0)
        return g

    def hess_f(v):
        Hh = np.zeros((nv, nv))
        Hh[ix, ix] = 2.0 * np.eye(n_in)
        return Hh

    def c(v):
        return np.concatenate([v[iy] - onn.value(mlp, v[ix]), E @ v[iy] - margin - v[is_]])

    def jac_c(v):
        A = np.zeros((m, nv))
        A[:n_out, ix] = -onn.jacobian(mlp, v[ix])
        A[:n_out, iy] = np.eye(n_out)
        A[n_out:, iy] = E
        A[n_out:, is_] = -np.eye(ns)
        return A

    def hess_c(v, lam):
        Hh = np.zeros((nv, nv))
        Hh[ix, ix] = -onn.hessian_lag(mlp, v[ix], lam[:n_out])
        return Hh

    p = Problem(nv, m, lb, ub, v0, f, grad_f, hess_f, c, jac_c, hess_c)
    p.blocks = dict(n_in=n_in, n_out=n_out, ns=ns, target=target, margin=margin)
    return p


def adversarial_l1(mlp, x_ref, target, conf=0.6):
    """Eq. 7: the smallest L1 change to a reference image that makes a softmax classifier give the
    target class probability `conf` or more.  The L1 norm is written with split variables
    x - x_ref = p - q, p, q >= 0, so the objective is linear and smooth:
        variables v = (x in [0,1]^n, p >= 0, q >= 0, y with y_t >= conf)
        min sum(p) + sum(q)
        s.t. x - p + q - x_ref = 0,   y - NN(x) = 0.
    Start: x = x_ref, p = q = 0, y = NN(x_ref) (the solver pushes them into their bounds)."""
    n, n_out = mlp.spec.n_in, mlp.spec.n_out
    nv = 3 * n + n_out
    m = n + n_out
    ix, ip, iq, iy = (slice(0, n), slice(n, 2 * n), slice(2 * n, 3 * n), slice(3 * n, nv))
    lb = np.concatenate([np.zeros(3 * n), np.full(n_out, -np.inf)])
    ub = np.concatenate([np.ones(n), np.full(2 * n + n_out, np.inf)])
    lb[3 * n + target] = conf
    x_ref = np.asarray(x_ref, dtype=np.float64)
    v0 = np.concatenate([x_ref, np.zeros(2 * n), onn.value(mlp, x_ref)])

    def f(v):
        return float(np.sum(v[ip]) + np.sum(v[iq]))

    def grad_f(v):
        g = np.zeros(nv)
        g[ip] = 1.0
        g[iq] = 1.0
        return g

    def hess_f(v):
        return np.zeros((nv, nv))

    def c(v):
        return np.concatenate([v[ix] - v[ip] + v[iq] - x_ref, v[iy] - onn.value(mlp, v[ix])])

    def jac_c(v):
        A = np.zeros((m, nv))
        A[:n, ix] = np.eye(n)
        A[:n, ip] = -np.eye(n)
        A[:n, iq] = np.eye(n)
        A[n:, ix] = -onn.jacobian(mlp, v[ix])
        A[n:, iy] = np.eye(n_out)
        return A

    def hess_c(v, lam):
        Hh = np.zeros((nv, nv))
        Hh[ix, ix] = -onn.hessian_lag(mlp, v[ix], lam[n:])
        return Hh

    pr = Problem(nv, m, lb, ub, v0, f, grad_f, hess_f, c, jac_c, hess_c)
    pr.blocks = dict(n_in=n, n_out=n_out, target=target, conf=conf)
    return pr


def adversarial_l1_fullspace(mlp, x_ref, target, conf=0.6):
    """Eq. 7 with the network in the full-space form of Eq. 4: every layer's affine output z_l and
    activation output y_l are variables, tied by z_l - W_l y_{l-1} - b_l = 0 and
    y_l - sigma_l(z_l) = 0 (y_0 = x, y_L = y).  Same objective, bounds and split variables as
    `adversarial_l1`, so both forms have the same optima:
        v = (x, p, q, z_1, y_1, ..., z_L, y_L),  min sum(p) + sum(q)
        s.t. x - p + q - x_ref = 0,  z_l - W_l y_{l-1} - b_l = 0,  y_l - sigma_l(z_l) = 0.
    Start: x = x_ref, p = q = 0, (z_l, y_l) from the forward pass at x_ref."""
    n, L = mlp.spec.n_in, mlp.spec.n_layers
    widths, acts = mlp.spec.widths, mlp.spec.acts
    # variable offsets
    off_z, off_y = [], []
    k = 3 * n
    for l in range(L):
        off_z.append(k)
        k += widths[l + 1]
        off_y.append(k)
        k += widths[l + 1]
    nv = k
    m = n + 2 * sum(widths[1:])
    lb = np.full(nv, -np.inf)
    ub = np.full(nv, np.inf)
    lb[:3 * n] = 0.0
    ub[:n] = 1.0
    lb[off_y[-1] + target] = conf
    x_ref = np.asarray(x_ref, dtype=np.float64)
    zs, as_ = onn.forward(mlp, x_ref)
    v0 = np.zeros(nv)
    v0[:n] = x_ref
    for l in range(L):
        v0[off_z[l]:off_z[l] + widths[l + 1]] = zs[l]
        v0[off_y[l]:off_y[l] + widths[l + 1]] = as_[l + 1]

    def seg(v, off, l):
        return v[off[l]:off[l] + widths[l + 1]]

    def prev(v, l):
        return v[:n] if l == 0 else seg(v, off_y, l - 1)

    def f(v):
        return float(np.sum(v[n:3 * n]))

    def grad_f(v):
        g = np.zeros(nv)
        g[n:3 * n] = 1.0
        return g

    def hess_f(v):
        return np.zeros((nv, nv))

    def c(v):
        out = [v[:n] - v[n:2 * n] + v[2 * n:3 * n] - x_ref]
        for l in range(L):
            z = seg(v, off_z, l)
            out.append(z - mlp.W[l] @ prev(v, l) - mlp.b[l])
            out.append(seg(v, off_y, l) - onn.act_value(acts[l], z))
        return np.concatenate(out)

    def jac_c(v):
        A = np.zeros((m, nv))
        A[:n, :n] = np.eye(n)
        A[:n, n:2 * n] = -np.eye(n)
        A[:n, 2 * n:3 * n] = np.eye(n)
        r = n
        for l in range(L):
            w = widths[l + 1]
            z = seg(v, off_z, l)
            A[r:r + w, off_z[l]:off_z[l] + w] = np.eye(w)
            cols = slice(0, n) if l == 0 else slice(off_y[l - 1], off_y[l - 1] + widths[l])
            A[r:r + w, cols] = -mlp.W[l]
            r += w
            A[r:r + w, off_y[l]:off_y[l] + w] = np.eye(w)
            A[r:r + w, off_z[l]:off_z[l] + w] = -onn.jac_apply(acts[l], z, np.eye(w))
            r += w
        return A

    def hess_c(v, lam):
        # only y_l - sigma_l(z_l) is nonlinear: its multipliers mu_l give -grad^2 (mu_l^T sigma_l)
        Hh = np.zeros((nv, nv))
        r = n
        for l in range(L):
            w = widths[l + 1]
            r += w
            mu = lam[r:r + w]
            z = seg(v, off_z, l)
            C = onn.curvature(acts[l], z, mu)
            zz = slice(off_z[l], off_z[l] + w)
            Hh[zz, zz] = -(C if C.ndim == 2 else np.diag(C))
            r += w
        return Hh

    pr = Problem(nv, m, lb, ub, v0, f, grad_f, hess_f, c, jac_c, hess_c)
    pr.blocks = dict(n_in=n, n_out=widths[-1], target=target, conf=conf, off_z=off_z, off_y=off_y)
    return pr


def box_projection(x0):
    """min ||x - x0||^2 over [0,1]^n with no constraint: the solution is clip(x0, 0, 1)."""
    n = x0.size
    return Problem(n, 0, np.zeros(n), np.ones(n), np.full(n, 0.5),
                   lambda v: float((v - x0) @ (v - x0)), lambda v: 2.0 * (v - x0),
                   lambda v: 2.0 * np.eye(n), lambda v: np.zeros(0), lambda v: np.zeros((0, n)),
                   lambda v, lam: np.zeros((n, n)))


# ---------------------------------------------------------------- SCOPF-shaped batch (Eq. 8 variant)


def scopf_surrogate(data, k, d, calibrate=True):
    """The MLP of contingency k at load d, with its output bias calibrated so that the margin at
    the flat dispatch xbar = (D(d)/G) 1 equals delta_k (strictly feasible start)."""
    from copy import deepcopy
    net = deepcopy(data.nets[k])
    net.b[0] = scopf_first_bias(data, k, d)
    if calibrate:
        D = scopf_demand(data, d)
        xbar = np.full(len(data.subsets[k]), D / data.G)
        net.b[-1] = net.b[-1] - onn.value(net, xbar) + data.delta[k]
    return net


def scopf(data, d=None, nets=None):
    """min sum_i c_i x_i^2  s.t.  y_k - NN_k(x[S_k]) = 0 (k < K),  sum_i x_i - D(d) = 0,
    x in [0,1]^G, y_k >= 0 (every contingency keeps a non-negative stability margin).
    Variables v = (x in R^G, y in R^K).  Start: x = xbar, y_k = NN_k(xbar) = delta_k."""
    G, K = data.G, len(data.nets)
    d = np.ones(data.n_bus) if d is None else np.asarray(d, dtype=np.float64)
    nets = nets if nets is not None else [scopf_surrogate(data, k, d) for k in range(K)]
    D = scopf_demand(data, d)
    nv, m = G + K, K + 1
    lb = np.concatenate([np.zeros(G), np.zeros(K)])
    ub = np.concatenate([np.ones(G), np.full(K, np.inf)])
    xbar = np.full(G, D / G)
    v0 = np.concatenate([xbar, [onn.value(nets[k], xbar[data.subsets[k]])[0] for k in range(K)]])
    cost = data.cost

    def f(v):
        return float(cost @ (v[:G] ** 2))

    def grad_f(v):
        g = np.zeros(nv)
        g[:G] = 2.0 * cost * v[:G]
        return g

    def hess_f(v):
        Hh = np.zeros((nv, nv))
        Hh[:G, :G] = np.diag(2.0 * cost)
        return Hh

    def c(v):
        x = v[:G]
        out = np.empty(m)
        for k in range(K):
            out[k] = v[G + k] - onn.value(nets[k], x[data.subsets[k]])[0]
        out[K] = x.sum() - D
        return out

    def jac_c(v):
        x = v[:G]
        A = np.zeros((m, nv))
        for k in range(K):
            A[k, data.subsets[k]] = -onn.jacobian(nets[k], x[data.subsets[k]])[0]
            A[k, G + k] = 1.0
        A[K, :G] = 1.0
        return A

    def hess_c(v, lam):
        x = v[:G]
        Hh = np.zeros((nv, nv))
        for k in range(K):
            S = data.subsets[k]
            Hh[np.ix_(S, S)] -= onn.hessian_lag(nets[k], x[S], lam[k:k + 1])
        return Hh

    p = Problem(nv, m, lb, ub, v0, f, grad_f, hess_f, c, jac_c, hess_c)
    p.nets = nets
    p.demand = D
    return p


def scopf_raw_nets(data, d):
    """The surrogates with the load shift in the first-layer bias and no output calibration."""
    return [scopf_surrogate(data, k, d, calibrate=False) for k in range(len(data.nets))]
