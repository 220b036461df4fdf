"""Pins for the oracle interior-point method (Eq. 1 / Eq. 2 with IPOPT's barrier terms).

Pinned against closed forms (box projection), a one-dimensional reduction solved by scipy,
a QP special case (identity activations) solved by scipy's SLSQP, and the KKT conditions of
the adversarial problem recomputed from their definitions.
"""
import numpy as np
import pytest

import synth
from synth.nets import MLPSpec, make_mlp
from oracle import ipm, problems, nn as onn


def test_box_projection_closed_form():
    x0 = np.array([-0.7, 0.2, 1.3, 0.5, 2.0, -0.01])
    r = ipm.solve(problems.box_projection(x0), ipm.Options(tol=1e-10))
    assert r.status == ipm.OPTIMAL
    # an active bound is met to within mu / z with z = 2 |x0 - bound| (0.02 for x0 = -0.01)
    assert np.max(np.abs(r.v - np.clip(x0, 0.0, 1.0))) < 1e-7


def _one_dim_problem(a, b, w, b1, v, c):
    nn = lambda x: v * np.tanh(w * x + b1) + c  # noqa: E731
    dnn = lambda x: v * w * (1 - np.tanh(w * x + b1) ** 2)  # noqa: E731
    d2nn = lambda x: v * w * w * (-2 * np.tanh(w * x + b1) * (1 - np.tanh(w * x + b1) ** 2))  # noqa: E731
    p = ipm.Problem(
        2, 1, np.array([-2.0, -np.inf]), np.array([2.0, np.inf]), np.array([0.0, nn(0.0)]),
        lambda z: (z[0] - a) ** 2 + (z[1] - b) ** 2,
        lambda z: np.array([2 * (z[0] - a), 2 * (z[1] - b)]),
        lambda z: 2 * np.eye(2),
        lambda z: np.array([z[1] - nn(z[0])]),
        lambda z: np.array([[-dnn(z[0]), 1.0]]),
        lambda z, lam: np.array([[-lam[0] * d2nn(z[0]), 0.0], [0.0, 0.0]]))
    return p, nn


def test_one_dimensional_reduction_against_scipy():
    from scipy.optimize import minimize_scalar
    a, b, w, b1, v, c = 0.8, 1.5, 2.0, -0.3, 1.2, 0.1
    p, nn = _one_dim_problem(a, b, w, b1, v, c)
    r = ipm.solve(p)
    assert r.status == ipm.OPTIMAL
    h = lambda x: (x - a) ** 2 + (nn(x) - b) ** 2  # noqa: E731
    grid = np.linspace(-2, 2, 4001)
    x_best = grid[np.argmin(h(grid))]
    s = minimize_scalar(h, bounds=(max(-2, x_best - 0.01), min(2, x_best + 0.01)), method="bounded",
                        options={"xatol": 1e-12})
    assert abs(r.v[0] - s.x) < 1e-5
    assert abs(r.obj - s.fun) < 1e-8
    assert abs(r.v[1] - nn(r.v[0])) < 1e-7


def test_linear_network_qp_against_slsqp():
    from scipy.optimize import minimize
    spec = MLPSpec([30, 16, 4], ["identity", "identity"])
    mlp = make_mlp(spec, seed=4, tag="qp", bias_std=0.3)
    x0 = synth.uniform01(synth.derive_key(4, "qp-x0"), 30)
    t, margin = 1, 0.1      # class 1 loses at x0 and can win by 1.1 inside the box (LP check)
    r = ipm.solve(problems.adversarial(mlp, x0, target=t, margin=margin))
    assert r.status == ipm.OPTIMAL
    P = mlp.W[1] @ mlp.W[0]
    q = mlp.W[1] @ mlp.b[0] + mlp.b[1]
    cons = [{"type": "ineq", "fun": (lambda x, j=j: (P[t] - P[j]) @ x + q[t] - q[j] - margin),
             "jac": (lambda x, j=j: P[t] - P[j])} for j in range(4) if j != t]
    s = minimize(lambda x: (x - x0) @ (x - x0), x0, jac=lambda x: 2 * (x - x0), bounds=[(0, 1)] * 30,
                 constraints=cons, method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
    assert s.success
    assert abs(r.obj - s.fun) <= 1e-6 * max(1.0, abs(s.fun))
    assert np.max(np.abs(r.v[:30] - s.x)) < 1e-4


def test_adversarial_tiny_kkt_certificate():
    """784 -> 128 -> 128 -> 10 tanh: the solution satisfies the KKT conditions of Eq. 1 to 1e-6."""
    mlp = make_mlp(synth.TINY, seed=0)
    d = synth.adversarial_data(seed=0)
    p = problems.adversarial(mlp, d.x0, d.target, d.margin)
    r = ipm.solve(p)
    assert r.status == ipm.OPTIMAL, ipm.STATUS_NAMES[r.status]
    n_in, n_out = 784, 10
    x, y, s = r.v[:n_in], r.v[n_in:n_in + n_out], r.v[n_in + n_out:]
    # feasibility, from the definitions
    assert np.max(np.abs(y - onn.value(mlp, x))) < 1e-6
    others = [j for j in range(n_out) if j != d.target]
    assert np.all(y[d.target] - y[others] - d.margin - s > -1e-6)
    assert np.all(y[d.target] - y[others] - d.margin - s < 1e-6)
    assert np.all((x >= 0) & (x <= 1)) and np.all(s >= 0)
    # stationarity: 2(x - x0) - J^T lam_nn - zL + zU = 0, lam_nn + E^T lam_m = 0, -lam_m - zs = 0
    lam_nn, lam_m = r.lam[:n_out], r.lam[n_out:]
    J = onn.jacobian(mlp, x)
    rx = 2 * (x - d.x0) - J.T @ lam_nn - r.zL[:n_in] + r.zU[:n_in]
    E = np.zeros((len(others), n_out))
    for i, j in enumerate(others):
        E[i, d.target], E[i, j] = 1.0, -1.0
    ry = lam_nn + E.T @ lam_m
    rs = -lam_m - r.zL[n_in + n_out:]
    scale = max(100.0, (np.abs(r.lam).sum() + np.abs(r.zL).sum() + np.abs(r.zU).sum()) / (19 + 784 * 2 + 9)) / 100.0
    assert max(np.abs(rx).max(), np.abs(ry).max(), np.abs(rs).max()) / scale < 1e-6
    # complementarity
    assert np.max(np.abs(x * r.zL[:n_in])) < 1e-6 and np.max(np.abs((1 - x) * r.zU[:n_in])) < 1e-6
    assert r.iters < 100
    assert 0.0 < r.obj < 50.0


def test_status_codes():
    x0 = np.array([0.3, 1.4])
    r = ipm.solve(problems.box_projection(x0), ipm.Options(max_iter=2))
    assert r.status == ipm.MAX_ITER
    p = problems.box_projection(x0)
    p.f = lambda v: float("nan")
    assert ipm.solve(p).status == ipm.NONFINITE


def _l1_instance(seed, n=20, scale=4.0):
    """A small softmax classifier whose output layer is scaled so that its probabilities are as
    peaked as a trained classifier's (the 0.6 threshold of Eq. 7 is then reachable)."""
    mlp = make_mlp(MLPSpec([n, 16, 16, 5], ["tanh", "tanh", "softmax"]), seed=seed, tag="l1",
                   bias_std=0.3)
    mlp.W[-1] = mlp.W[-1] * scale
    x = synth.uniform01(synth.derive_key(seed, "l1-x"), n)
    p0 = onn.value(mlp, x)
    return mlp, x, int(np.argsort(p0)[-2])


@pytest.mark.parametrize("seed", [0, 1])
def test_l1_adversarial_against_slsqp(seed):
    """Eq. 7 with split variables: the IPM's optimum has p q = 0 componentwise, its objective is
    ||x - x_ref||_1, the confidence constraint is active, and scipy's SLSQP on the same smooth
    program from the same start reaches the same objective."""
    from scipy.optimize import minimize
    mlp, x_ref, t = _l1_instance(seed)
    n = x_ref.size
    pr = problems.adversarial_l1(mlp, x_ref, t, 0.6)
    r = ipm.solve(pr)
    assert r.status == ipm.OPTIMAL, r.status
    x, p, q = r.v[:n], r.v[n:2 * n], r.v[2 * n:3 * n]
    assert np.max(np.minimum(p, q)) < 1e-6
    # at the barrier optimum both split variables of an unchanged pixel sit at ~1e-7 (complementarity
    # mu <= tol / 10 with multipliers of order one), so sum(p + q) exceeds ||x - x_ref||_1 by
    # 2 sum(min(p, q)) <= 2 n 1e-7
    assert abs(r.obj - np.abs(x - x_ref).sum()) < 2e-7 * n + 1e-9
    assert abs(onn.value(mlp, x)[t] - 0.6) < 1e-6
    cons = [{"type": "eq", "fun": pr.c, "jac": pr.jac_c}]
    bounds = list(zip(np.where(np.isfinite(pr.lb), pr.lb, None), np.where(np.isfinite(pr.ub), pr.ub, None)))
    s = minimize(pr.f, pr.v0, jac=pr.grad_f, bounds=bounds, constraints=cons, method="SLSQP",
                 options={"ftol": 1e-12, "maxiter": 500})
    assert s.success, s.message
    assert abs(s.fun - r.obj) < 1e-5 * max(1.0, r.obj), (s.fun, r.obj)


def test_l1_adversarial_already_confident():
    """If the reference image already has target probability >= 0.6 the answer is x = x_ref with
    objective 0 (p = q = 0)."""
    mlp, x_ref, _ = _l1_instance(3)
    t = int(np.argmax(onn.value(mlp, x_ref)))
    conf = 0.5 * onn.value(mlp, x_ref)[t]
    r = ipm.solve(problems.adversarial_l1(mlp, x_ref, t, conf))
    assert r.status == ipm.OPTIMAL
    assert r.obj < 2e-7 * x_ref.size + 1e-9   # barrier floor of the split variables (see above)
    assert np.max(np.abs(r.v[:x_ref.size] - x_ref)) < 1e-5


@pytest.mark.parametrize("seed", [0, 1])
def test_l1_fullspace_matches_reduced(seed):
    """Eq. 7 with the network in the full space (Eq. 4: z_l and y_l as variables) is the same
    program as the reduced-space form (Eq. 5): the same optimum, reached from the same start."""
    mlp, x_ref, t = _l1_instance(seed)
    n = x_ref.size
    r = ipm.solve(problems.adversarial_l1(mlp, x_ref, t, 0.6))
    rf = ipm.solve(problems.adversarial_l1_fullspace(mlp, x_ref, t, 0.6))
    assert r.status == ipm.OPTIMAL and rf.status == ipm.OPTIMAL
    print(f"[l1 {seed}] reduced {r.iters} iterations, full space {rf.iters}")
    assert abs(rf.obj - r.obj) <= 1e-6 * max(1.0, abs(r.obj))
    assert np.max(np.abs(rf.v[:n] - r.v[:n])) < 1e-5
    pf = problems.adversarial_l1_fullspace(mlp, x_ref, t, 0.6)
    off_y = pf.blocks["off_y"]
    assert np.max(np.abs(rf.v[off_y[-1]:off_y[-1] + mlp.spec.n_out] - onn.value(mlp, rf.v[:n]))) < 1e-8


def test_l1_fullspace_derivatives():
    """The full-space constraint Jacobian against central differences of c, and the Hessian of
    the Lagrangian against central differences of lambda^T J (tanh, sigmoid and softmax layers);
    at the start point every layer constraint holds."""
    mlp = make_mlp(MLPSpec([3, 4, 5, 3], ["tanh", "sigmoid", "softmax"]), seed=4, tag="fs-d",
                   bias_std=0.3)
    x = synth.uniform01(synth.derive_key(4, "fs-x"), 3)
    pr = problems.adversarial_l1_fullspace(mlp, x, 1, 0.6)
    assert np.max(np.abs(pr.c(pr.v0))) < 1e-15
    v = pr.v0 + 0.05 * synth.normal(synth.derive_key(4, "fs-v"), pr.n)
    lam = synth.normal(synth.derive_key(4, "fs-lam"), pr.m)
    h = 1e-6
    A = pr.jac_c(v)
    Hl = pr.hess_c(v, lam)
    for k in range(pr.n):
        e = np.zeros(pr.n)
        e[k] = h
        fd = (pr.c(v + e) - pr.c(v - e)) / (2 * h)
        assert np.max(np.abs(fd - A[:, k])) < 1e-8, k
        fd2 = (pr.jac_c(v + e).T @ lam - pr.jac_c(v - e).T @ lam) / (2 * h)
        assert np.max(np.abs(fd2 - Hl[:, k])) < 1e-7, k


def test_structure_of_both_forms_matches_table2():
    """Table 2's structural counts for the 167k-parameter MNIST classifier ([784, 128 x 5, 10],
    tanh + softmax): variables, constraints and Jacobian nonzeros of the full-space form (Eq. 4)
    and the reduced-space form (Eq. 5) of Eq. 7, counted from the problems' own Jacobians and
    Hessians at the start point (the table truncates to thousands)."""
    import json
    import os
    from synth.nets import make_classifier
    with open(os.path.join(os.path.dirname(__file__), "golden", "table2_structure_167k.json")) as f:
        g = json.load(f)
    w = g["widths"]
    mlp = make_classifier(MLPSpec(w, ["tanh"] * (len(w) - 2) + ["softmax"]), seed=0)
    assert 166_000 < mlp.spec.n_params < 168_000
    x_ref = synth.uniform01(synth.derive_key(0, "t2-x"), w[0])
    for form, build in (("full_space", problems.adversarial_l1_fullspace),
                        ("reduced_space", problems.adversarial_l1)):
        pr = build(mlp, x_ref, 3, 0.6)
        A = pr.jac_c(pr.v0)
        H = pr.hess_c(pr.v0, np.ones(pr.m)) + pr.hess_f(pr.v0)
        counts = dict(n_var=pr.n, n_con=pr.m, jac_nnz=int(np.count_nonzero(A)),
                      hess_nnz=int(np.count_nonzero(np.tril(H))))
        print(form, counts)
        for key, val in g[form].items():
            assert counts[key.replace("_thousands", "")] // 1000 == val, (form, key, counts)
