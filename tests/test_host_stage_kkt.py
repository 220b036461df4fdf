"""Block-tridiagonal sparse KKT factorization of the full-space problems (nnc_stage_kkt_solve,
FP64 on the host) against the plain definitions: inertia = signs of the eigenvalues of the
assembled matrix (numpy eigvalsh), solution = numpy solve.  The matrices have the full-space
structure of Eq. 4 (link rows, per layer affine and activation rows; free variables without
curvature, so zero diagonals that need 2 x 2 pivots) or are random block-tridiagonal."""
import numpy as np
import pytest

from paper_2509_22462_gb300 import build


@pytest.fixture(scope="module")
def nnc():
    build.build()
    from paper_2509_22462_gb300 import nnc as m
    return m


def _fullspace(widths, seed, softmax=False, dw=0.0, dc=0.0):
    """KKT pieces of the full-space L1 problem at a random point: returns n, m, stages, triplets
    and sigma.  Variables (x, p, q, z_1, y_1, ...), constraints (link, affine, activation)."""
    rng = np.random.default_rng(seed)
    n0, L = widths[0], len(widths) - 1
    vs, cs = [2] * n0 + [0] * (2 * n0), [1] * n0
    oz, oy, oa, oc = [], [], [], []
    nv, m = 3 * n0, n0
    for l in range(L):
        k = widths[l + 1]
        oz.append(nv); vs += [3 + 2 * l] * k; nv += k
        oy.append(nv); vs += [3 + 2 * l + 1] * k; nv += k
        oa.append(m); cs += [3 + 2 * l] * k; m += k
        oc.append(m); cs += [3 + 2 * l + 1] * k; m += k
    jr, jc, jv = [], [], []
    for i in range(n0):
        jr += [i, i, i]; jc += [i, n0 + i, 2 * n0 + i]; jv += [1.0, -1.0, 1.0]
    wr, wc, wv = [], [], []
    for l in range(L):
        k, kin = widths[l + 1], widths[l]
        prev = 0 if l == 0 else oy[l - 1]
        W = rng.standard_normal((k, kin)) / np.sqrt(kin)
        for j in range(k):
            jr.append(oa[l] + j); jc.append(oz[l] + j); jv.append(1.0)
            for c in range(kin):
                jr.append(oa[l] + j); jc.append(prev + c); jv.append(-W[j, c])
            jr.append(oc[l] + j); jc.append(oy[l] + j); jv.append(1.0)
        last_soft = softmax and l == L - 1
        if last_soft:
            P = rng.standard_normal((k, k)) * 0.3
            H = rng.standard_normal((k, k)) * 0.2
            H = H + H.T
            for j in range(k):
                for c in range(k):
                    jr.append(oc[l] + j); jc.append(oz[l] + c); jv.append(P[j, c])
                for c in range(j + 1):
                    wr.append(oz[l] + j); wc.append(oz[l] + c); wv.append(H[j, c])
        else:
            d1 = rng.uniform(0.1, 1.0, k)
            h = rng.standard_normal(k) * 0.5 * (rng.uniform(size=k) > 0.3)   # some exact zeros
            for j in range(k):
                jr.append(oc[l] + j); jc.append(oz[l] + j); jv.append(-d1[j])
                wr.append(oz[l] + j); wc.append(oz[l] + j); wv.append(h[j])
    sigma = np.zeros(nv)
    sigma[:3 * n0] = rng.uniform(0.05, 5.0, 3 * n0)          # bounded x, p, q
    sigma[oy[-1] + rng.integers(widths[-1])] = 0.7           # the bounded output
    return nv, m, np.array(vs), np.array(cs), (wr, wc, wv), (jr, jc, jv), sigma


def _assemble(n, m, W, A, sigma, dw, dc):
    K = np.zeros((n + m, n + m))
    for r, c, v in zip(*W):
        K[r, c] += v
        if r != c:
            K[c, r] += v
    K[np.arange(n), np.arange(n)] += sigma + dw
    for r, c, v in zip(*A):
        K[n + r, c] += v
        K[c, n + r] += v
    K[np.arange(n, n + m), np.arange(n, n + m)] -= dc
    return K


def _inertia(K, tol=1e-9):
    ev = np.linalg.eigvalsh(K)
    t = tol * max(1.0, np.abs(ev).max())
    return int((ev > t).sum()), int((ev < -t).sum()), int((np.abs(ev) <= t).sum())


@pytest.mark.parametrize("widths,softmax,dw,dc", [
    ([6, 5, 4, 3], False, 0.0, 0.0),
    ([10, 8, 8, 5], True, 0.0, 0.0),
    ([7, 12, 9, 9, 4], False, 1e-3, 1e-6),
    ([12, 20, 16, 10], True, 0.5, 0.0),
    ([30, 40, 40, 10], False, 0.0, 0.0),
    ([60, 100, 120, 20], True, 0.0, 0.0),     # multi-threaded solves and Schur updates
])
def test_fullspace_inertia_and_solution(nnc, widths, softmax, dw, dc):
    n, m, vs, cs, W, A, sigma = _fullspace(widths, seed=sum(widths), softmax=softmax)
    K = _assemble(n, m, W, A, sigma, dw, dc)
    rhs = np.random.default_rng(5).standard_normal(n + m)
    x, inert = nnc.stage_kkt_solve(n, m, vs, cs, W, A, sigma, rhs, delta_w=dw, delta_c=dc)
    assert inert == _inertia(K), (inert, _inertia(K))
    assert inert[2] == 0
    np.testing.assert_allclose(x, np.linalg.solve(K, rhs), rtol=1e-8, atol=1e-8 * np.abs(x).max())


def test_random_block_tridiagonal(nnc):
    """Dense random blocks of random sizes (indefinite), couplings between neighbours only."""
    rng = np.random.default_rng(11)
    sizes = [3, 7, 1, 5, 9, 2, 6]
    n = sum(sizes)                      # all unknowns as variables, no constraints
    st = np.repeat(np.arange(len(sizes)), sizes)
    off = np.concatenate([[0], np.cumsum(sizes)])
    wr, wc, wv = [], [], []
    for s, k in enumerate(sizes):
        B = rng.standard_normal((k, k))
        B = B + B.T
        for i in range(k):
            for j in range(i + 1):
                wr.append(off[s] + i); wc.append(off[s] + j); wv.append(B[i, j])
        if s > 0:
            C = rng.standard_normal((k, sizes[s - 1]))
            for i in range(k):
                for j in range(sizes[s - 1]):
                    wr.append(off[s] + i); wc.append(off[s - 1] + j); wv.append(C[i, j])
    sigma = np.zeros(n)
    K = _assemble(n, 0, (wr, wc, wv), ([], [], []), sigma, 0.0, 0.0)
    rhs = rng.standard_normal(n)
    x, inert = nnc.stage_kkt_solve(n, 0, st, [], (wr, wc, wv), ([], [], []), sigma, rhs)
    assert inert == _inertia(K)
    np.testing.assert_allclose(x, np.linalg.solve(K, rhs), rtol=1e-7, atol=1e-9 * np.abs(x).max())


def test_singular_and_bad_staging(nnc):
    n, m, vs, cs, W, A, sigma = _fullspace([5, 4, 3], seed=3)
    # a repeated link row (duplicate constraint): K singular, one zero eigenvalue
    jr, jc, jv = (list(a) for a in A)
    rows = [(r, c, v) for r, c, v in zip(jr, jc, jv) if r == 0]
    for r, c, v in rows:
        jr.append(m); jc.append(c); jv.append(v)
    cs2 = np.concatenate([cs, [cs[0]]])
    x, inert = nnc.stage_kkt_solve(n, m + 1, vs, cs2, W, (jr, jc, jv), sigma, np.ones(n + m + 1))
    K = _assemble(n, m + 1, W, (jr, jc, jv), sigma, 0.0, 0.0)
    assert _inertia(K)[2] == 1
    assert inert[2] >= 1 and x is None
    # a coupling between stages two apart is refused
    vs_bad = vs.copy()
    vs_bad[0] = vs[0] + 3          # x_0 away from its link row's neighbours
    with pytest.raises(nnc.NNCError):
        nnc.stage_kkt_solve(n, m, vs_bad, cs, W, A, sigma, np.ones(n + m))


def test_strongly_active_bounds(nnc):
    """Barrier terms from 1e-8 to 1e10 (bounds far away and strongly active side by side): the link
    multipliers' Schur complements are as small as 1e-10 and still regular.  Inertia against
    LAPACK's symmetric indefinite factorization (scipy.linalg.ldl) of the equilibrated matrix."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    n, m, vs, cs, W, A, sigma = _fullspace([40, 30, 30, 8], seed=21, softmax=True)
    rng = np.random.default_rng(2)
    sigma[:120] = 10.0 ** rng.uniform(-8, 10, 120)
    K = _assemble(n, m, W, A, sigma, 0.0, 0.0)
    d = 1.0 / np.sqrt(np.abs(K).max(axis=1))
    _, D, _ = scipy_linalg.ldl(d[:, None] * K * d[None, :])
    ev = np.linalg.eigvalsh(D)
    ref = (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    rhs = rng.standard_normal(n + m)
    x, inert = nnc.stage_kkt_solve(n, m, vs, cs, W, A, sigma, rhs)
    assert inert == ref
    res = K @ x - rhs
    assert np.abs(res).max() <= 1e-8 * (np.abs(K) @ np.abs(x) + np.abs(rhs)).max()
