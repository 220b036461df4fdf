"""Pins for two oracle parts that the interior-point pins reach only indirectly.

* `problems.scopf` (the SCOPF-shaped program, a variant of Eq. 8): its start is strictly feasible
  with the calibrated margins, each network row depends on exactly the setpoints its surrogate
  sees, the Jacobian and the Hessian of the Lagrangian match central differences of c and of
  lambda^T J, and the oracle's optimum of a small instance satisfies the KKT conditions of Eq. 1
  recomputed from their definitions and agrees with scipy's SLSQP on the program written without
  the margin variables.
* `ipm._inertia` (the inertia test of step 3 of the method): matrices of known inertia, namely
  random congruences Q diag(s) Q^T with chosen signs, KKT matrices of Eq. 2 whose barrier terms
  are 1e10 next to unit constraint rows (inertia (n, m, 0) by the Schur complement), and exactly
  singular KKT matrices (one zero eigenvalue).
"""
import numpy as np
import pytest

import synth
from oracle import ipm, problems, nn as onn


def _small_scopf(seed=3, K=4, G=12):
    data = synth.scopf_data(K=K, G=G, n_bus=20, seed=seed, n_min=3, n_max=9, hidden=16, depth=2,
                            n_load_buses=4)
    return data, problems.scopf(data)


def test_scopf_start_is_calibrated_and_feasible():
    data, pr = _small_scopf()
    G, K = data.G, len(data.nets)
    d = np.ones(data.n_bus)
    assert pr.n == G + K and pr.m == K + 1
    x0 = pr.v0[:G]
    # flat dispatch at half capacity on average: sum x = 0.5 G mean(d)
    assert np.allclose(x0, 0.5 * np.mean(d)) and abs(x0.sum() - pr.demand) < 1e-12
    # each margin starts at its calibration offset delta_k, and every constraint holds there
    assert np.max(np.abs(pr.v0[G:] - data.delta)) < 1e-12
    assert np.max(np.abs(pr.c(pr.v0))) < 1e-12
    assert np.all(pr.v0[G:] > 0) and np.all((x0 > 0) & (x0 < 1))


def test_scopf_rows_depend_on_their_subsets_only():
    """c_k = y_k - NN_k(x[S_k]): moving a setpoint outside S_k leaves row k unchanged, moving one
    inside S_k changes it, y_k enters row k alone with coefficient one, and the balance row is
    sum(x) - D."""
    data, pr = _small_scopf()
    G, K = data.G, len(data.nets)
    v = pr.v0 + 0.05 * synth.normal(synth.derive_key(3, "scopf-v"), pr.n)
    base = pr.c(v)
    for j in range(G):
        e = np.zeros(pr.n)
        e[j] = 0.3
        diff = pr.c(v + e) - base
        for k in range(K):
            inside = j in set(data.subsets[k].tolist())
            assert (abs(diff[k]) > 1e-12) == inside, (j, k, diff[k])
        assert abs(diff[K] - 0.3) < 1e-12
    for k in range(K):
        e = np.zeros(pr.n)
        e[G + k] = 0.7
        diff = pr.c(v + e) - base
        expect = np.zeros(K + 1)
        expect[k] = 0.7
        assert np.max(np.abs(diff - expect)) < 1e-12


def test_scopf_loads_enter_only_through_their_buses():
    """A load change at buses that surrogate k does not see leaves its first-layer bias alone."""
    data, _ = _small_scopf()
    d = np.ones(data.n_bus)
    for k in range(len(data.nets)):
        d2 = d.copy()
        outside = np.setdiff1d(np.arange(data.n_bus), data.load_buses[k])
        d2[outside] += 0.5
        b1 = problems.scopf_raw_nets(data, d)[k].b[0]
        b2 = problems.scopf_raw_nets(data, d2)[k].b[0]
        assert np.array_equal(b1, b2)
        d3 = d.copy()
        d3[data.load_buses[k][0]] += 0.5
        assert not np.array_equal(problems.scopf_raw_nets(data, d3)[k].b[0], b1)


def test_scopf_derivatives_central_differences():
    data, pr = _small_scopf()
    v = pr.v0 + 0.05 * synth.normal(synth.derive_key(3, "scopf-fd-v"), pr.n)
    lam = synth.normal(synth.derive_key(3, "scopf-fd-lam"), pr.m)
    A = pr.jac_c(v)
    Hl = pr.hess_c(v, lam)
    assert np.array_equal(Hl, Hl.T)
    h = 1e-6
    for j in range(pr.n):
        e = np.zeros(pr.n)
        e[j] = h
        fd = (pr.c(v + e) - pr.c(v - e)) / (2 * h)
        assert np.max(np.abs(fd - A[:, j])) < 1e-8, j
        fd2 = (pr.jac_c(v + e).T @ lam - pr.jac_c(v - e).T @ lam) / (2 * h)
        assert np.max(np.abs(fd2 - Hl[:, j])) < 1e-7, j
    # the objective's derivatives too
    for j in range(pr.n):
        e = np.zeros(pr.n)
        e[j] = h
        assert abs((pr.f(v + e) - pr.f(v - e)) / (2 * h) - pr.grad_f(v)[j]) < 1e-7
        fd3 = (pr.grad_f(v + e) - pr.grad_f(v - e)) / (2 * h)
        assert np.max(np.abs(fd3 - pr.hess_f(v)[:, j])) < 1e-7


def test_scopf_kkt_certificate_and_slsqp():
    """The oracle's optimum of a small instance: feasibility, stationarity and complementarity of
    Eq. 1 recomputed from their definitions (network values and Jacobians from oracle.nn, whose
    own pins are elsewhere), and the same objective as scipy's SLSQP on the program written
    without margin variables (min sum c_i x_i^2 s.t. NN_k(x[S_k]) >= 0, sum x = D, 0 <= x <= 1)."""
    from scipy.optimize import minimize
    data, pr = _small_scopf()
    G, K = data.G, len(data.nets)
    r = ipm.solve(pr)
    assert r.status == ipm.OPTIMAL, ipm.STATUS_NAMES[r.status]
    x, y = r.v[:G], r.v[G:]
    nets = pr.nets
    # feasibility
    for k in range(K):
        assert abs(y[k] - onn.value(nets[k], x[data.subsets[k]])[0]) < 1e-6
    assert abs(x.sum() - pr.demand) < 1e-6
    assert np.all(y >= 0) and np.all((x >= 0) & (x <= 1))
    # stationarity: grad f + A^T lam - zL + zU = 0 with A from the definitions
    lam_k, lam_d = r.lam[:K], r.lam[K]
    gx = 2.0 * data.cost * x + lam_d * np.ones(G) - r.zL[:G] + r.zU[:G]
    for k in range(K):
        S = data.subsets[k]
        gx[S] -= lam_k[k] * onn.jacobian(nets[k], x[S])[0]
    gy = lam_k - r.zL[G:]
    scale = max(100.0, (np.abs(r.lam).sum() + np.abs(r.zL).sum() + np.abs(r.zU[:G]).sum())
                / (K + 1 + 2 * G + K)) / 100.0
    assert max(np.abs(gx).max(), np.abs(gy).max()) / scale < 1e-6
    # complementarity
    assert np.max(np.abs(x * r.zL[:G])) < 1e-6 and np.max(np.abs((1 - x) * r.zU[:G])) < 1e-6
    assert np.max(np.abs(y * r.zL[G:])) < 1e-6
    # an independent solver on the program without margin variables
    cons = [{"type": "eq", "fun": lambda z: np.array([z.sum() - pr.demand]),
             "jac": lambda z: np.ones((1, G))}]
    for k in range(K):
        S = data.subsets[k]

        def fk(z, S=S, k=k):
            return onn.value(nets[k], z[S])

        def jk(z, S=S, k=k):
            row = np.zeros((1, G))
            row[0, S] = onn.jacobian(nets[k], z[S])[0]
            return row
        cons.append({"type": "ineq", "fun": fk, "jac": jk})
    s = minimize(lambda z: float(data.cost @ (z * z)), pr.v0[:G], jac=lambda z: 2 * data.cost * z,
                 bounds=[(0.0, 1.0)] * G, constraints=cons, method="SLSQP",
                 options={"ftol": 1e-14, "maxiter": 500})
    assert s.success, s.message
    assert abs(s.fun - r.obj) <= 1e-6 * max(1.0, abs(r.obj)), (s.fun, r.obj)
    assert np.max(np.abs(s.x - x)) < 1e-4


# ---------------------------------------------------------------- inertia


def _random_orthogonal(key, n):
    q, rr = np.linalg.qr(synth.normal(key, n * n).reshape(n, n))
    return q * np.sign(np.diag(rr))


@pytest.mark.parametrize("counts", [(5, 3, 0), (8, 0, 0), (0, 6, 0), (4, 4, 2), (3, 2, 3)])
def test_inertia_of_random_congruences(counts):
    """K = Q diag(s) Q^T with |s| spread over eight decades and the chosen sign counts; exact
    zeros in s give zero eigenvalues (Q orthogonal, so K's eigenvalues are s)."""
    npos, nneg, nzero = counts
    n = npos + nneg + nzero
    key = synth.derive_key(sum(counts) * 7 + npos, "inertia")
    mags = 10.0 ** (8.0 * synth.uniform01(key, n) - 4.0)
    s = np.concatenate([mags[:npos], -mags[npos:npos + nneg], np.zeros(nzero)])
    Q = _random_orthogonal(synth.derive_key(n, "inertia-q", npos), n)
    K = (Q * s) @ Q.T
    K = 0.5 * (K + K.T)
    assert ipm._inertia(K) == counts


def test_inertia_of_nonorthogonal_congruence():
    """Sylvester's law: any nonsingular congruence keeps the counts."""
    n = 9
    s = np.array([3.0, -1.0, 2e-3, -5e4, 7.0, -0.2, 1e-2, 4.0, -9.0])
    B = np.eye(n) + 0.3 * synth.normal(synth.derive_key(1, "inertia-b"), n * n).reshape(n, n)
    assert abs(np.linalg.det(B)) > 1e-3
    K = (B * s) @ B.T
    assert ipm._inertia(0.5 * (K + K.T)) == (5, 4, 0)


def _kkt(n, m, sigma, A, H=None):
    H = np.zeros((n, n)) if H is None else H
    K = np.zeros((n + m, n + m))
    K[:n, :n] = H + np.diag(sigma)
    K[n:, :n] = A
    K[:n, n:] = A.T
    return K


def test_inertia_of_badly_scaled_kkt():
    """[[H + Sigma, A^T], [A, 0]] with H + Sigma positive definite and A of full row rank has
    inertia (n, m, 0) (the Schur complement -A (H + Sigma)^-1 A^T is negative definite), even when
    Sigma holds barrier terms of 1e10 and the constraint rows touch only those variables: then the
    negative eigenvalues are about -1e-10 next to a largest one of 1e10."""
    n, m = 6, 2
    sigma = np.array([1e10, 1e10, 1.0, 2.0, 1.0, 3.0])
    A = np.zeros((m, n))
    A[0, 0] = 1.0
    A[1, 1] = 1.0
    K = _kkt(n, m, sigma, A)
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev < 0) == m and np.min(np.abs(ev)) < 1e-9   # tiny but negative
    assert ipm._inertia(K) == (n, m, 0)
    # a dense Hessian block and dense constraint rows with mixed 1e10 / unit barrier terms
    n, m = 12, 4
    Hh = synth.normal(synth.derive_key(2, "inertia-h"), n * n).reshape(n, n)
    Hh = Hh @ Hh.T / n
    sigma = np.where(np.arange(n) % 3 == 0, 1e10, 1.0)
    A = synth.normal(synth.derive_key(2, "inertia-a"), m * n).reshape(m, n)
    assert ipm._inertia(_kkt(n, m, sigma, A, Hh)) == (n, m, 0)


def test_inertia_of_indefinite_hessian_block():
    """An indefinite H + Sigma gives more than m negative eigenvalues: the inertia test must
    reject it (one negative direction of H inside the null space of A adds one)."""
    n, m = 5, 1
    H = np.diag([1.0, 1.0, -3.0, 1.0, 1.0])
    A = np.array([[1.0, 0.0, 0.0, 0.0, 0.0]])
    assert ipm._inertia(_kkt(n, m, np.zeros(n), A, H)) == (n - 1, m + 1, 0)


def test_inertia_of_singular_kkt():
    """Two equal constraint rows make the KKT matrix exactly singular: one zero eigenvalue, also
    next to barrier terms of 1e10."""
    n, m = 6, 3
    A = np.zeros((m, n))
    A[0, 2] = A[1, 2] = 1.0
    A[2, 4] = 1.0
    assert ipm._inertia(_kkt(n, m, np.ones(n), A)) == (n, m - 1, 1)
    A2 = np.zeros((m, n))
    A2[0, 0] = A2[1, 0] = 1.0
    A2[2, 1] = 1.0
    sigma = np.array([1e10, 1e10, 1.0, 1.0, 1.0, 1.0])
    assert ipm._inertia(_kkt(n, m, sigma, A2)) == (n, m - 1, 1)
