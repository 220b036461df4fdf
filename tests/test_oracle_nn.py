"""Pins for the FP64 oracle of the network constraint (Eq. 3 and Eq. 6).

Each check reaches the same quantity by a route that does not share the oracle's
activation-derivative table or its sweep order, so a dropped term, a wrong sign, a
transposed operand or a wrong sigma'' in the oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import synth
from synth.nets import MLPSpec, make_mlp
from oracle import nn, checks

HERE = os.path.dirname(os.path.abspath(__file__))


def _net(widths, acts, seed=0, bias_std=0.3):
    return make_mlp(MLPSpec(widths, acts), seed=seed, tag="pin", bias_std=bias_std)


def _x(n, seed=1):
    return synth.uniform01(synth.derive_key(seed, "pin-x"), n) * 2.0 - 1.0


def _lam(m, seed=2):
    return synth.normal(synth.derive_key(seed, "pin-lam"), m)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("act", ["tanh"])
def test_one_hidden_layer_closed_form(act):
    net = _net([7, 9, 4], [act, "identity"])
    x, lam = _x(7), _lam(4)
    y, J, H = checks.one_hidden_tanh_closed_form(net.W[0], net.b[0], net.W[1], net.b[1], x, lam)
    assert _rel(nn.value(net, x), y) < 1e-15
    assert _rel(nn.jacobian(net, x), J) < 1e-14
    assert _rel(nn.hessian_lag(net, x, lam), H) < 1e-13
    assert _rel(nn.hessian_lag_layers(net, x, lam), H) < 1e-13


@pytest.mark.parametrize("acts", [
    ["tanh", "tanh", "identity"],
    ["sigmoid", "sigmoid", "sigmoid"],
    ["softplus", "tanh", "softplus"],
    ["tanh", "sigmoid", "tanh"],
])
def test_jacobian_complex_step(acts):
    net = _net([6, 8, 5, 3], acts)
    x = _x(6)
    J = nn.jacobian(net, x)
    Jc = checks.jacobian_complex_step(net, x)
    assert _rel(J, Jc) < 1e-13


@pytest.mark.parametrize("acts", [
    ["tanh", "tanh", "identity"],
    ["sigmoid", "sigmoid", "sigmoid"],
    ["softplus", "tanh", "softplus"],
    ["tanh", "sigmoid", "tanh"],
])
def test_hessian_hyperdual(acts):
    net = _net([5, 7, 6, 3], acts)
    x, lam = _x(5), _lam(3)
    Hh = checks.hessian_hyperdual(net, x, lam)
    assert _rel(nn.hessian_lag(net, x, lam), Hh) < 1e-12
    assert _rel(nn.hessian_lag_layers(net, x, lam), Hh) < 1e-12


def test_hessian_finite_differences_of_gradient():
    net = _net([9, 12, 12, 4], ["tanh", "tanh", "identity"])
    x, lam = _x(9), _lam(4)
    Hfd = checks.hessian_fd_of_gradient(lambda v: nn.vjp(net, v, lam), x)
    assert _rel(nn.hessian_lag(net, x, lam), Hfd) < 1e-7


def test_jacobian_finite_differences_and_vjp():
    net = _net([9, 12, 12, 4], ["tanh", "sigmoid", "identity"])
    x, lam = _x(9), _lam(4)
    Jfd = checks.jacobian_fd(lambda v: nn.value(net, v), x)
    J = nn.jacobian(net, x)
    assert _rel(J, Jfd) < 1e-8
    assert _rel(nn.vjp(net, x, lam), lam @ J) < 1e-14


def test_forward_over_reverse_is_symmetric_and_matches_layer_sum():
    net = make_mlp(synth.TINY, seed=0)
    d = synth.adversarial_data(seed=0)
    H_for = nn.hessian_lag_for(net, d.x0, d.lam)
    H_sum = nn.hessian_lag_layers(net, d.x0, d.lam)
    nrm = np.linalg.norm(H_for)
    assert np.linalg.norm(H_for - H_for.T) <= 1e-14 * nrm * 10  # round-off of two sweep orders
    assert _rel(H_sum, H_for) < 1e-12


def test_identity_activations_reduce_to_matrix_product():
    net = _net([6, 5, 4, 3], ["identity"] * 3)
    x, lam = _x(6), _lam(3)
    P = net.W[2] @ net.W[1] @ net.W[0]
    c = net.W[2] @ (net.W[1] @ net.b[0] + net.b[1]) + net.b[2]
    assert _rel(nn.value(net, x), P @ x + c) < 1e-14
    assert _rel(nn.jacobian(net, x), P) < 1e-14
    assert np.abs(nn.hessian_lag(net, x, lam)).max() == 0.0


def test_brute_force_symbolic_2_3_2():
    """A 2 -> 3 -> 2 net differentiated symbolically (sympy), evaluated exactly."""
    sp = pytest.importorskip("sympy")
    rng = np.random.default_rng(5)
    W1 = rng.integers(-3, 4, size=(3, 2)) / 4
    b1 = rng.integers(-3, 4, size=3) / 4
    W2 = rng.integers(-3, 4, size=(2, 3)) / 4
    b2 = rng.integers(-3, 4, size=2) / 4
    xv = np.array([0.25, -0.5])
    lv = np.array([1.5, -0.75])
    x1, x2 = sp.symbols("x1 x2")
    X = sp.Matrix([x1, x2])
    h = (sp.Matrix(W1.tolist()).applyfunc(sp.nsimplify) * X + sp.Matrix(b1.tolist()).applyfunc(sp.nsimplify))
    a1 = h.applyfunc(lambda u: 1 / (1 + sp.exp(-u)))     # sigmoid hidden layer
    out = sp.Matrix(W2.tolist()).applyfunc(sp.nsimplify) * a1 + sp.Matrix(b2.tolist()).applyfunc(sp.nsimplify)
    out = out.applyfunc(sp.tanh)                           # tanh output layer
    lagr = sum(sp.nsimplify(lv[i]) * out[i] for i in range(2))
    subs = {x1: sp.nsimplify(xv[0]), x2: sp.nsimplify(xv[1])}
    Jsym = np.array([[float(sp.diff(out[i], v).subs(subs).evalf(30)) for v in (x1, x2)] for i in range(2)])
    Hsym = np.array([[float(sp.diff(lagr, u, v).subs(subs).evalf(30)) for v in (x1, x2)] for u in (x1, x2)])
    ysym = np.array([float(out[i].subs(subs).evalf(30)) for i in range(2)])
    net = _net([2, 3, 2], ["sigmoid", "tanh"])
    net.W[0][:], net.b[0][:], net.W[1][:], net.b[1][:] = W1, b1, W2, b2
    assert _rel(nn.value(net, xv), ysym) < 1e-15
    assert _rel(nn.jacobian(net, xv), Jsym) < 1e-14
    assert _rel(nn.hessian_lag(net, xv, lv), Hsym) < 1e-13


def test_activation_derivative_table_against_complex_step():
    z = np.linspace(-4, 4, 41)
    for act in ["tanh", "sigmoid", "softplus"]:
        h = 1e-30
        d1 = checks._act_complex(act, z + 1j * h).imag / h
        assert np.allclose(nn.act_d1(act, z), d1, rtol=1e-13, atol=1e-15)
        d1fn = lambda u: nn.act_d1(act, u)  # noqa: E731
        d2 = (d1fn(z + 1e-6) - d1fn(z - 1e-6)) / 2e-6
        assert np.allclose(nn.act_d2(act, z), d2, rtol=1e-7, atol=1e-9)


def test_gelu_against_quadrature_definition():
    """GELU(z) = z * Phi(z); its derivatives against central differences."""
    z = np.linspace(-4, 4, 33)
    from scipy.stats import norm
    assert np.allclose(nn.act_value("gelu", z), z * norm.cdf(z), rtol=1e-14, atol=1e-15)
    f = lambda u: nn.act_value("gelu", u)  # noqa: E731
    g = lambda u: nn.act_d1("gelu", u)  # noqa: E731
    assert np.allclose(nn.act_d1("gelu", z), (f(z + 1e-6) - f(z - 1e-6)) / 2e-6, rtol=1e-7, atol=1e-9)
    assert np.allclose(nn.act_d2("gelu", z), (g(z + 1e-6) - g(z - 1e-6)) / 2e-6, rtol=1e-7, atol=1e-9)


def test_reduced_space_structure_matches_table2():
    """Table 2: the reduced-space MNIST Hessian has ~307k nonzeros whatever the network; the
    dense symmetric n_in x n_in Hessian of Eq. 6 stores n(n+1)/2 of them."""
    with open(os.path.join(HERE, "golden", "table2_reduced_structure.json")) as f:
        g = json.load(f)
    n = g["mnist"]["n_in"]
    assert (n * (n + 1) // 2) // 1000 == g["mnist"]["hess_nnz_thousands"]  # the table truncates
    net = make_mlp(synth.TINY, seed=0)
    d = synth.adversarial_data(seed=0)
    H = nn.hessian_lag(net, d.x0, d.lam)
    assert np.count_nonzero(np.tril(H)) == n * (n + 1) // 2


def test_hessian_columns_match_full_sweep():
    net = _net([11, 9, 8, 3], ["tanh", "softplus", "sigmoid"])
    x, lam = _x(11), _lam(3)
    cols = [0, 4, 10]
    assert _rel(nn.hessian_lag_columns(net, x, lam, cols), nn.hessian_lag_for(net, x, lam)[:, cols]) < 1e-15


# ---------------------------------------------------------------- softmax output layer
SOFTMAX_NETS = [([4, 5, 3], ["tanh", "softmax"]),
                ([3, 6, 4, 5], ["sigmoid", "softplus", "softmax"]),
                ([5, 4], ["softmax"])]


@pytest.mark.parametrize("case", range(len(SOFTMAX_NETS)))
def test_softmax_output_against_complex_step_and_hyperdual(case):
    """Softmax output layer (Section 4.1's classifiers): J by complex step, H by hyper-dual
    numbers (both from exp only), the literal sweep equal to the per-layer sum."""
    widths, acts = SOFTMAX_NETS[case]
    net = _net(widths, acts, seed=case)
    x, lam = _x(widths[0], seed=case + 3), _lam(widths[-1], seed=case + 4)
    p = nn.value(net, x)
    assert abs(p.sum() - 1.0) < 1e-14 and np.all(p > 0)
    J = nn.jacobian(net, x)
    assert np.max(np.abs(J - checks.jacobian_complex_step(net, x))) < 1e-13 * max(1.0, np.abs(J).max())
    assert np.allclose(nn.vjp(net, x, lam), lam @ J, rtol=0, atol=1e-14)
    H = nn.hessian_lag_for(net, x, lam)
    Hh = checks.hessian_hyperdual(net, x, lam)
    assert np.max(np.abs(H - Hh)) < 1e-12 * max(1.0, np.abs(Hh).max())
    assert np.max(np.abs(nn.hessian_lag_layers(net, x, lam) - Hh)) < 1e-12 * max(1.0, np.abs(Hh).max())


def test_softmax_invariants():
    """Probabilities sum to one, so the Jacobian's columns sum to zero and a multiplier vector
    proportional to (1, ..., 1) sees no curvature."""
    net = _net([6, 8, 5], ["tanh", "softmax"], seed=9)
    x = _x(6, seed=10)
    J = nn.jacobian(net, x)
    assert np.max(np.abs(J.sum(axis=0))) < 1e-15
    H = nn.hessian_lag(net, x, 2.5 * np.ones(5))
    assert np.max(np.abs(H)) < 1e-14
    # the softmax second-derivative tensor against central differences of its Jacobian
    z = synth.normal(synth.derive_key(11, "sm-z"), 5)
    D = nn.softmax_second(nn.act_value("softmax", z))
    h = 1e-5
    for k in range(5):
        e = np.zeros(5); e[k] = h
        pp, pm = nn.act_value("softmax", z + e), nn.act_value("softmax", z - e)
        Jp = np.diag(pp) - np.outer(pp, pp)
        Jm = np.diag(pm) - np.outer(pm, pm)
        assert np.max(np.abs((Jp - Jm) / (2 * h) - D[:, :, k])) < 1e-9
