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
    assert full == (1 if np.linalg.eigvalsh(W + np.diag(sig[:nd] + 0.1)).min() <= 0 else 0)
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
