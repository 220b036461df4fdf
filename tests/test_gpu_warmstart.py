"""The warm-start network's kernels against the FP64 oracle (gradients, Adam), and what the
trained network gains over the cold-started interior-point method on held-out loads.

Tolerances: FP32 operands 1e-5 relative (gradients) and 1e-6 (one Adam step); BF16 operands
3e-2 relative on the gradients (8-bit mantissas, FP32 accumulation)."""
import numpy as np
import pytest

import synth
from oracle import warmstart as ows, problems, ipm as oipm

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def nnc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22462_gb300 import build, nnc as m
    build.build()
    return m


def _data(seed=0, B=48, n_in=40, n_out=23):
    p = synth.warmstart_params(n_in, 64, 48, n_out, seed=seed)
    rng = np.random.default_rng(seed)
    for i in (1, 3, 5):
        p[i] = 0.1 * rng.standard_normal(p[i].shape)
    p = [np.float32(x).astype(np.float64) for x in p]      # exactly representable in FP32
    U = np.float32(rng.standard_normal((B, n_in))).astype(np.float64)
    T = np.float32(rng.standard_normal((B, n_out))).astype(np.float64)
    return p, U, T


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 3e-2)])
def test_gradients_match_oracle(nnc, prec, tol):
    p, U, T = _data()
    ws = nnc.WarmStart(p, precision=prec)
    loss, g = ws.loss_grad(U, T)
    lo = ows.loss(p, U, T)
    go = ows.grad(p, U, T)
    errs = [rel(a, b) for a, b in zip(g, go)]
    print(f"[warmstart {prec}] loss rel err {abs(loss - lo) / lo:.2e}, gradient rel errs "
          + " ".join(f"{e:.1e}" for e in errs))
    assert abs(loss - lo) <= tol * lo
    assert max(errs) < tol
    ws.free()


@pytest.mark.parametrize("shape", [(128, 128, 64, 23, 64),     # every product on the tensor cores
                                   (512, 256, 256, 713, 128),  # the warm-start network of the bench
                                   (128, 64, 64, 10, 48)])     # batch not a multiple of 64:
                                                               # tensor-core forward, CUDA-core backward
def test_tensor_core_gradients_match_oracle(nnc, shape):
    """The BF16 form on the tcgen05 path (widths multiples of 64): loss and every gradient against
    the FP64 oracle, and the prediction of the forward pass."""
    n_in, h1, h2, n_out, B = shape
    p = synth.warmstart_params(n_in, h1, h2, n_out, seed=5)
    rng = np.random.default_rng(5)
    for i in (1, 3, 5):
        p[i] = 0.1 * rng.standard_normal(p[i].shape)
    p = [np.float32(x).astype(np.float64) for x in p]
    U = np.float32(rng.standard_normal((B, n_in))).astype(np.float64)
    T = np.float32(rng.standard_normal((B, n_out))).astype(np.float64)
    ws = nnc.WarmStart(p, precision="bf16")
    loss, g = ws.loss_grad(U, T)
    lo = ows.loss(p, U, T)
    go = ows.grad(p, U, T)
    errs = [rel(a, b) for a, b in zip(g, go)]
    print(f"[warmstart tc {shape}] loss rel err {abs(loss - lo) / lo:.2e}, gradient rel errs "
          + " ".join(f"{e:.1e}" for e in errs))
    assert abs(loss - lo) <= 3e-2 * lo
    assert max(errs) < 3e-2
    P = ws.predict(U)
    assert rel(P, ows.forward(p, U)[0]) < 3e-2
    ws.free()


def test_adam_step_matches_oracle(nnc):
    p, U, T = _data(seed=1)
    ws = nnc.WarmStart(p, precision="fp32")
    _, g = ws.loss_grad(U, T)
    ws.adam_step(lr=1e-2)
    got = ws.params()
    ref = [x.copy() for x in p]
    ows.adam_step(ref, g, ows.init_state(ref), 1, lr=1e-2)
    for a, b in zip(got, ref):
        assert rel(a, b) < 1e-6
    ws.free()


def test_training_reduces_the_loss(nnc):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((7, 12)) * 0.4
    U = rng.standard_normal((512, 12))
    T = np.tanh(U @ A.T)
    ws = nnc.WarmStart(synth.warmstart_params(12, 64, 64, 7, seed=3), precision="bf16")
    l0 = ws.train(U, T, epochs=1, batch=64, lr=1e-3)
    l1 = ws.train(U, T, epochs=200, batch=64, lr=1e-3)
    assert l1 < 0.05 * l0
    P = ws.predict(U[:32])
    assert rel(P, T[:32]) < 0.15
    ws.free()


def test_warm_start_gain_on_held_out_loads(nnc):
    """Small SCOPF-shaped problem: the trained network must save iterations on held-out loads
    and reach the cold solve's objective."""
    from paper_2509_22462_gb300 import warmstart_experiment as wx
    rep, rows = wx.run(K=16, G=40, n_bus=64, hidden=128, depth=3, n_train=160, n_test=16, epochs=400,
                       batch_rows=32, lr=2e-3, seed=0, h1=128, h2=128, log=print)
    print("[warmstart gain]", rep)
    assert rep["warm_iters_mean"] < rep["cold_iters_mean"]
    assert rep["same_objective_frac"] >= 0.9


def test_warm_started_ipm_matches_oracle(nnc):
    """From the same predicted start, the library's warm-started solve and the oracle's reach the
    same objective."""
    data = synth.scopf_data(K=8, G=30, n_bus=64, n_min=5, n_max=20, hidden=64, depth=3, seed=1)
    d = synth.load_vectors(1, 64, seed=9)[0]
    po = problems.scopf(data, d)
    cold = oipm.solve(po)
    assert cold.status == oipm.OPTIMAL
    rng = np.random.default_rng(4)
    v0 = cold.v + 0.02 * rng.standard_normal(cold.v.size)
    l0 = cold.lam * (1 + 0.05 * rng.standard_normal(cold.lam.size))
    ro = oipm.solve(po, warm=(v0, l0))
    assert ro.status == oipm.OPTIMAL
    nets = [nnc.Net.from_mlp(m, precision="bf16x3") for m in problems.scopf_raw_nets(data, d)]
    b = nnc.Batch(nets)
    res, v, lam = nnc.ipm_scopf(b, data.G, data.subsets, data.cost, synth.scopf_demand(data, d), data.delta,
                                v_start=v0, lam_start=l0)
    print(f"[ipm warm] iters {res['iters']} (oracle {ro.iters}, cold {cold.iters}) obj {res['obj']:.12g} "
          f"(oracle {ro.obj:.12g})")
    assert res["status"] == 0 and res["kkt_error"] <= 1e-6
    assert abs(res["obj"] - ro.obj) <= 1e-6 * abs(ro.obj)
    b.free()
    for n in nets:
        n.free()
