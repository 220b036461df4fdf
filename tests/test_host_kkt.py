"""Host KKT solver of the interior-point driver (nnc_kkt_solve, FP64 on the CPU) against the plain
definitions: inertia = signs of the eigenvalues (numpy eigvalsh), solution = numpy solve."""
import numpy as np
import pytest

from paper_2509_22462_gb300 import build


@pytest.fixture(scope="module")
def nnc():
    build.build()
    from paper_2509_22462_gb300 import nnc as m
    return m


def _kkt(nd, ns, m, seed, indefinite=False, dw=0.0, dc=0.0):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((nd, nd))
    W = B @ B.T / nd + (0.5 if not indefinite else -0.8) * np.eye(nd)
    WSS = rng.uniform(0.0, 1.0, ns) * (rng.uniform(size=ns) > 0.5)
    sig = rng.uniform(0.01, 3.0, nd + ns)
    AD = rng.standard_normal((m, nd))
    AS = rng.standard_normal((m, ns))
    n = nd + ns
    K = np.zeros((n + m, n + m))
    K[:nd, :nd] = W
    K[:n, :n] += np.diag(sig + dw)
    K[nd:n, nd:n] += np.diag(WSS)
    K[n:, :nd] = AD
    K[n:, nd:n] = AS
    K[:n, n:] = K[n:, :n].T
    K[n:, n:] = -dc * np.eye(m)
    return W, WSS, sig, AD, AS, K


@pytest.mark.parametrize("nd,ns,m,indef", [(40, 7, 9, False), (130, 19, 19, False), (65, 3, 5, True),
                                           (12, 0, 4, False), (30, 10, 0, False), (200, 50, 51, True)])
def test_inertia_and_solution(nnc, nd, ns, m, indef):
    W, WSS, sig, AD, AS, K = _kkt(nd, ns, m, seed=nd + ns + m, indefinite=indef, dw=0.1, dc=1e-3)
    rhs = np.random.default_rng(1).standard_normal(K.shape[0])
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs, delta_w=0.1, delta_c=1e-3)
    ev = np.linalg.eigvalsh(K)
    assert (npos, nneg, nzero) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    assert full == 0           # small-block diagonals are >= 0: never the whole matrix
    ref = np.linalg.solve(K, rhs)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_singular_is_reported(nnc):
    W, WSS, sig, AD, AS, K = _kkt(20, 4, 3, seed=3)
    AD[2] = AD[1]
    AS[2] = AS[1]              # two equal constraint rows: K is singular without delta_c
    rhs = np.ones(20 + 4 + 3)
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs)
    assert nzero >= 1
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs, delta_c=1e-6)
    assert (npos, nneg, nzero) == (24, 3, 0)


@pytest.mark.parametrize("nd,ns,m,nz,indef", [(40, 30, 20, 3, False), (60, 125, 70, 9, False),
                                              (25, 12, 8, 1, False), (40, 30, 20, 3, True),
                                              (60, 125, 70, 9, True)])
def test_zero_diagonal_small_block(nnc, nd, ns, m, nz, indef):
    """Free variables without curvature (zero diagonal) in the small block, the shape of the L1
    problem's y (Eq. 7): they stay beside the multipliers in the reduced system (with the dense
    block too when that is indefinite); inertia and solution against the plain definitions."""
    W, WSS, sig, AD, AS, K = _kkt(nd, ns, m, seed=7 * nd + nz, indefinite=indef)
    n = nd + ns
    free = np.arange(nz) * (ns // nz)
    WSS[free] = 0.0
    sig[nd + free] = 0.0
    for j, a in enumerate(free):          # each free variable sits in one constraint row
        AS[:, a] = 0.0
        AS[j, a] = 1.0
    K = np.zeros((n + m, n + m))
    K[:nd, :nd] = W
    K[:n, :n] += np.diag(sig)
    K[nd:n, nd:n] += np.diag(WSS)
    K[n:, :nd] = AD
    K[n:, nd:n] = AS
    K[:n, n:] = K[n:, :n].T
    K[n:, n:] = -1e-8 * np.eye(m)
    rhs = np.random.default_rng(2).standard_normal(n + m)
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs, delta_c=1e-8)
    ev = np.linalg.eigvalsh(K)
    assert (npos, nneg, nzero) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    ref = np.linalg.solve(K, rhs)
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)


def _l1_kkt(n, n_out, seed, indefinite=False, dc=0.0):
    """The KKT matrix of the L1 problem (Eq. 7 with split variables): x (n, dense block), then
    p, q (n each) and y (n_out) in the small block; rows x - p + q (n) and y - NN(x) (n_out).
    p and q have bound terms; y is free except y_t."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    W = B @ B.T / n + (0.3 if not indefinite else -0.6) * np.eye(n)
    ns, m = 2 * n + n_out, n + n_out
    WSS = np.zeros(ns)
    sig = np.concatenate([rng.uniform(0.01, 2.0, n), 10.0 ** rng.uniform(-3, 6, 2 * n), np.zeros(n_out)])
    sig[3 * n + 1] = 5.0                          # y_t has a bound
    AD = np.zeros((m, n))
    AD[:n] = np.eye(n)
    AD[n:] = rng.standard_normal((n_out, n))
    AS = np.zeros((m, ns))
    AS[:n, :n] = -np.eye(n)
    AS[:n, n:2 * n] = np.eye(n)
    AS[n:, 2 * n:] = np.eye(n_out)
    N = n + ns
    K = np.zeros((N + m, N + m))
    K[:n, :n] = W
    K[:N, :N] += np.diag(sig)
    K[N:, :n] = AD
    K[N:, n:N] = AS
    K[:N, N:] = K[N:, :N].T
    K[N:, N:] = -dc * np.eye(m)
    return W, WSS, sig, AD, AS, K


@pytest.mark.parametrize("n,n_out,indef", [(30, 5, False), (64, 10, False), (40, 4, True)])
def test_pinning_rows_l1_structure(nnc, n, n_out, indef):
    """Rows that pin one dense variable through their own bounded slacks (x_i - p_i + q_i of the
    L1 problem) are eliminated first and leave a diagonal term on the dense block; inertia and
    solution against the plain definitions, also where the dense block alone is indefinite."""
    W, WSS, sig, AD, AS, K = _l1_kkt(n, n_out, seed=n + n_out, indefinite=indef, dc=1e-8)
    rhs = np.random.default_rng(5).standard_normal(K.shape[0])
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs, delta_c=1e-8)
    ev = np.linalg.eigvalsh(K)
    assert (npos, nneg, nzero) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    ref = np.linalg.solve(K, rhs)
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)


def test_pinning_row_without_dense_entry(nnc):
    """A row with slacks only (its A_D row is zero) is a pinning row too; mixed with ordinary
    rows that share no slack with it."""
    W, WSS, sig, AD, AS, K = _kkt(20, 8, 6, seed=11, dw=0.0, dc=0.0)
    AD[0] = 0.0
    AS[:, :2] = 0.0
    AS[0] = 0.0
    AS[0, :2] = [1.5, -0.5]                   # row 0 owns slack columns 0 and 1
    sig[20:22] = [0.7, 2.0]
    n = 28
    K = np.zeros((n + 6, n + 6))
    K[:20, :20] = W
    K[:n, :n] += np.diag(sig)
    K[20:n, 20:n] += np.diag(WSS)
    K[n:, :20] = AD
    K[n:, 20:n] = AS
    K[:n, n:] = K[n:, :n].T
    rhs = np.random.default_rng(9).standard_normal(n + 6)
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs)
    ev = np.linalg.eigvalsh(K)
    assert (npos, nneg, nzero) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    ref = np.linalg.solve(K, rhs)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_negative_small_block_diagonal_whole_matrix(nnc):
    """A negative small-block diagonal entry with an indefinite dense block: the whole matrix is
    factorized (the fourth inertia entry says so)."""
    W, WSS, sig, AD, AS, K = _kkt(30, 6, 5, seed=21, indefinite=True)
    WSS[2] = -5.0
    n = 36
    K[30 + 2, 30 + 2] = WSS[2] + sig[30 + 2]
    rhs = np.random.default_rng(4).standard_normal(n + 5)
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs)
    assert full == 1
    ev = np.linalg.eigvalsh(K)
    assert (npos, nneg, nzero) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    ref = np.linalg.solve(K, rhs)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_negative_small_block_diagonal_schur(nnc):
    """A negative small-block diagonal entry with a definite dense block: Cholesky of the dense
    block and Bunch-Kaufman of the whole reduced system of the small block and the multipliers."""
    W, WSS, sig, AD, AS, K = _kkt(40, 9, 7, seed=23, indefinite=False)
    WSS[[1, 4]] = [-6.0, -2.5]
    n = 49
    K[40 + 1, 40 + 1] = WSS[1] + sig[40 + 1]
    K[40 + 4, 40 + 4] = WSS[4] + sig[40 + 4]
    rhs = np.random.default_rng(8).standard_normal(n + 7)
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs)
    assert full == 0
    ev = np.linalg.eigvalsh(K)
    assert (npos, nneg, nzero) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    ref = np.linalg.solve(K, rhs)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,seed", [(5, 1), (37, 2), (300, 3)])
def test_bunch_kaufman_through_whole_matrix(nnc, n, seed):
    """Indefinite matrices of every size class through the whole-matrix factorization (negative
    small-block diagonal, indefinite dense block): inertia and solution."""
    W, WSS, sig, AD, AS, K = _kkt(n, 6, 4, seed=seed, indefinite=True)
    WSS[0] = -9.0
    K[n, n] = WSS[0] + sig[n]
    rhs = np.random.default_rng(seed).standard_normal(n + 10)
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs)
    assert full == 1
    ev = np.linalg.eigvalsh(K)
    assert (npos, nneg, nzero) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    ref = np.linalg.solve(K, rhs)
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)


def _check(nnc, W, WSS, sig, AD, AS, K, rhs, dw=0.0, dc=0.0, tol=1e-8):
    x, (npos, nneg, nzero, full) = nnc.kkt_solve(W, WSS, sig, AD, AS, rhs, delta_w=dw, delta_c=dc)
    ev = np.linalg.eigvalsh(K)
    assert (npos, nneg, nzero) == (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    ref = np.linalg.solve(K, rhs)
    assert np.linalg.norm(x - ref) <= tol * np.linalg.norm(ref)
    return full


@pytest.mark.parametrize("nd,ns,m", [(97, 11, 7), (600, 19, 19), (785, 9, 30)])
def test_bordered_cholesky_many_blocks(nnc, nd, ns, m):
    """Definite dense blocks spanning many column blocks with a ragged last block (the
    constraint rows below the block are carried through the same factorization): inertia
    (n, m, 0) and the solution against the plain definitions."""
    W, WSS, sig, AD, AS, K = _kkt(nd, ns, m, seed=nd + 3, indefinite=False, dw=0.05, dc=1e-6)
    rhs = np.random.default_rng(nd).standard_normal(nd + ns + m)
    assert _check(nnc, W, WSS, sig, AD, AS, K, rhs, dw=0.05, dc=1e-6) == 0


@pytest.mark.parametrize("nd,ns,m", [(400, 20, 15), (700, 12, 40)])
def test_indefinite_dense_block_parallel_path(nnc, nd, ns, m):
    """Indefinite dense blocks large enough for the multithreaded symmetric indefinite
    factorization (more than 256 rows with the multipliers): inertia and solution."""
    W, WSS, sig, AD, AS, K = _kkt(nd, ns, m, seed=nd + 5, indefinite=True, dw=0.0, dc=1e-6)
    WSS[:] = np.abs(WSS)
    K[nd:nd + ns, nd:nd + ns] = np.diag(WSS + sig[nd:])
    rhs = np.random.default_rng(nd + 1).standard_normal(nd + ns + m)
    assert _check(nnc, W, WSS, sig, AD, AS, K, rhs, dc=1e-6) == 0


@pytest.mark.parametrize("indef", [False, True])
def test_pinning_rows_l1_structure_large(nnc, indef):
    """The L1 structure (Eq. 7 with split variables) at 300 pixels: pinning-row elimination, then
    the bordered Cholesky or, with an indefinite dense block, the multithreaded indefinite
    factorization."""
    W, WSS, sig, AD, AS, K = _l1_kkt(300, 10, seed=301, indefinite=indef, dc=1e-8)
    rhs = np.random.default_rng(6).standard_normal(K.shape[0])
    assert _check(nnc, W, WSS, sig, AD, AS, K, rhs, dc=1e-8) == 0


def test_no_dense_block_and_no_constraints(nnc):
    """Degenerate shapes: no dense-block variables (nd = 0), and no constraints (m = 0, the KKT
    matrix is the positive definite Hessian block alone)."""
    W = np.zeros((0, 0))
    rng = np.random.default_rng(13)
    ns, m = 10, 5
    WSS = rng.uniform(0.1, 1.0, ns)
    sig = rng.uniform(0.1, 1.0, ns)
    AS = rng.standard_normal((m, ns))
    AD = np.zeros((m, 0))
    K = np.zeros((ns + m, ns + m))
    K[:ns, :ns] = np.diag(WSS + sig)
    K[ns:, :ns] = AS
    K[:ns, ns:] = AS.T
    K[ns:, ns:] = -1e-6 * np.eye(m)
    rhs = rng.standard_normal(ns + m)
    _check(nnc, W, WSS, sig, AD, AS, K, rhs, dc=1e-6)
    W, WSS, sig, AD, AS, K = _kkt(330, 4, 0, seed=17, indefinite=False)
    rhs = np.random.default_rng(17).standard_normal(334)
    _check(nnc, W, WSS, sig, AD, AS, K, rhs)
