"""Independent routes to the network's derivatives, used only to pin `oracle.nn`.

TEST INFRASTRUCTURE ONLY.  None of these routes uses the activation-derivative table of
`oracle.nn`: the activations are rebuilt from exp and log, so a wrong sigma' or sigma'' in
the table shows up as a mismatch.

* complex step (Squire & Trapp 1998): J[:, j] = Im NN(x + i h e_j) / h, exact to round-off;
* hyper-dual numbers (Fike & Alonso 2011): a + b e1 + c e2 + d e1 e2 with e1^2 = e2^2 = 0;
  evaluating lambda^T NN at x + e1 e_i + e2 e_j gives H_ij as the e1 e2 part, exactly;
* central finite differences of the value (for J) and of the gradient lambda^T J (for H);
* closed forms for one hidden layer.
"""
import numpy as np


def _act_complex(name, z):
    if name == "identity":
        return z
    if name == "softmax":
        e = np.exp(z)
        return e / np.sum(e)
    if name == "tanh":
        e = np.exp(2.0 * z)
        return (e - 1.0) / (e + 1.0)
    if name == "sigmoid":
        return 1.0 / (1.0 + np.exp(-z))
    if name == "softplus":
        return np.log(1.0 + np.exp(z))
    raise ValueError(name)


def value_complex(net, x):
    a = np.asarray(x, dtype=np.complex128)
    for W, b, act in zip(net.W, net.b, net.spec.acts):
        a = _act_complex(act, W @ a + b)
    return a


def jacobian_complex_step(net, x, h=1e-30):
    n = net.spec.n_in
    J = np.zeros((net.spec.n_out, n))
    for j in range(n):
        xc = np.asarray(x, dtype=np.complex128).copy()
        xc[j] += 1j * h
        J[:, j] = value_complex(net, xc).imag / h
    return J


class HyperDual:
    """Arrays of hyper-dual numbers a + b e1 + c e2 + d e1e2 (e1^2 = e2^2 = 0, e1e2 != 0)."""

    def __init__(self, a, b, c, d):
        self.a, self.b, self.c, self.d = a, b, c, d

    def __add__(self, o):
        if isinstance(o, HyperDual):
            return HyperDual(self.a + o.a, self.b + o.b, self.c + o.c, self.d + o.d)
        return HyperDual(self.a + o, self.b, self.c, self.d)

    __radd__ = __add__

    def __neg__(self):
        return HyperDual(-self.a, -self.b, -self.c, -self.d)

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if isinstance(o, HyperDual):
            return HyperDual(self.a * o.a, self.a * o.b + self.b * o.a, self.a * o.c + self.c * o.a,
                             self.a * o.d + self.b * o.c + self.c * o.b + self.d * o.a)
        return HyperDual(self.a * o, self.b * o, self.c * o, self.d * o)

    __rmul__ = __mul__

    def recip(self):
        # 1/u: value 1/a, first parts -b/a^2, -c/a^2, cross part -d/a^2 + 2bc/a^3
        ia = 1.0 / self.a
        return HyperDual(ia, -self.b * ia * ia, -self.c * ia * ia,
                         -self.d * ia * ia + 2.0 * self.b * self.c * ia * ia * ia)

    def __truediv__(self, o):
        if isinstance(o, HyperDual):
            return self * o.recip()
        return self * (1.0 / o)

    def __rtruediv__(self, o):
        return self.recip() * o

    def exp(self):
        e = np.exp(self.a)
        return HyperDual(e, e * self.b, e * self.c, e * (self.d + self.b * self.c))

    def log(self):
        return HyperDual(np.log(self.a), self.b / self.a, self.c / self.a,
                         self.d / self.a - self.b * self.c / (self.a * self.a))

    def matvec_left(self, W):
        """W @ self for a constant matrix W."""
        return HyperDual(W @ self.a, W @ self.b, W @ self.c, W @ self.d)

    def dot(self, v):
        return HyperDual(v @ self.a, v @ self.b, v @ self.c, v @ self.d)


def _act_hd(name, u):
    if name == "identity":
        return u
    if name == "softmax":
        e = u.exp()
        total = HyperDual(np.sum(e.a), np.sum(e.b), np.sum(e.c), np.sum(e.d))
        return e * total.recip()
    if name == "tanh":
        e = (u * 2.0).exp()
        return (e - 1.0) / (e + 1.0)
    if name == "sigmoid":
        return ((-u).exp() + 1.0).recip()
    if name == "softplus":
        return (u.exp() + 1.0).log()
    raise ValueError(name)


def lagrangian_hyperdual(net, x, lam, i, j):
    """lambda^T NN(x + e1 e_i + e2 e_j); its e1e2 part is H_ij exactly."""
    n = net.spec.n_in
    z = np.zeros(n)
    b = z.copy(); b[i] = 1.0
    c = z.copy(); c[j] = 1.0
    u = HyperDual(np.asarray(x, dtype=np.float64), b, c, z.copy())
    for W, bias, act in zip(net.W, net.b, net.spec.acts):
        u = _act_hd(act, u.matvec_left(W) + bias)
    return u.dot(np.asarray(lam, dtype=np.float64))


def hessian_hyperdual(net, x, lam):
    n = net.spec.n_in
    H = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            H[i, j] = H[j, i] = lagrangian_hyperdual(net, x, lam, i, j).d
    return H


def jacobian_fd(value_fn, x, h=None):
    x = np.asarray(x, dtype=np.float64)
    y0 = value_fn(x)
    J = np.zeros((y0.size, x.size))
    for j in range(x.size):
        hj = h if h is not None else 6e-6 * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += hj
        xm[j] -= hj
        J[:, j] = (value_fn(xp) - value_fn(xm)) / (2.0 * hj)
    return J


def hessian_fd_of_gradient(grad_fn, x, h=None):
    """Central differences of the gradient lambda^T J, column by column."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    H = np.zeros((n, n))
    for j in range(n):
        hj = h if h is not None else 6e-6 * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += hj
        xm[j] -= hj
        H[:, j] = (grad_fn(xp) - grad_fn(xm)) / (2.0 * hj)
    return H


def one_hidden_tanh_closed_form(W, b, V, c, x, lam):
    """NN(x) = V tanh(W x + b) + c.  Returns (y, J, H) from the textbook closed forms:
    J = V diag(1 - t^2) W and H = W^T diag((V^T lam) * (-2 t (1 - t^2))) W."""
    t = np.tanh(W @ x + b)
    y = V @ t + c
    J = V @ ((1.0 - t * t)[:, None] * W)
    w = (V.T @ lam) * (-2.0 * t * (1.0 - t * t))
    H = W.T @ (w[:, None] * W)
    return y, J, H
