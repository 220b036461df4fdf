"""Grouped batch of uneven surrogates (the SCOPF-shaped workload) against the FP64 oracle, and
the SCOPF-shaped interior-point solve against the oracle interior-point method.

Tolerances: value 1e-6 (relative over the batch), Jacobian 1e-3 and Hessian 1e-2 relative
Frobenius per network, FP64 residual 1e-10; IPM objective 1e-6 relative with KKT <= 1e-6."""
import numpy as np
import pytest

import synth
from synth.problems import scopf_data
from oracle import nn as onn, problems, ipm as oipm

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def nnc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22462_gb300 import build, nnc as m
    build.build()
    return m


def _raw_nets(data, d):
    """Surrogates with the load shift in the first-layer bias and no output calibration."""
    return [problems.scopf_surrogate(data, k, d, calibrate=False) for k in range(len(data.nets))]


@pytest.fixture(scope="module")
def small_batch(nnc):
    data = scopf_data(K=12, G=60, n_bus=64, n_min=5, n_max=60, hidden=256, depth=3, seed=3)
    d = np.ones(64)
    raw = _raw_nets(data, d)
    nets = [nnc.Net.from_mlp(m, precision="bf16x3") for m in raw]
    return data, raw, nets


def test_batch_matches_oracle(nnc, small_batch):
    data, raw, nets = small_batch
    b = nnc.Batch(nets)
    x = synth.uniform01(synth.derive_key(1, "bx"), data.G)
    xs = [x[S] for S in data.subsets]
    lams = [synth.normal(synth.derive_key(k, "blam"), 1) for k in range(len(raw))]
    ys, Js, Hs, gs = b.eval(xs, lams)
    yo = np.concatenate([onn.value(raw[k], xs[k]) for k in range(len(raw))])
    assert rel(np.concatenate(ys), yo) < 1e-6
    worst = dict(J=0.0, H=0.0, g=0.0)
    for k in range(len(raw)):
        Jo = onn.jacobian(raw[k], xs[k])
        Ho = onn.hessian_lag(raw[k], xs[k], lams[k])
        go = onn.vjp(raw[k], xs[k], lams[k])
        worst["J"] = max(worst["J"], rel(Js[k], Jo))
        worst["H"] = max(worst["H"], rel(Hs[k], Ho))
        worst["g"] = max(worst["g"], rel(gs[k], go))
        assert np.array_equal(Hs[k], Hs[k].T)
    print(f"[batch bf16x3] worst rel err J={worst['J']:.2e} H={worst['H']:.2e} g={worst['g']:.2e}")
    assert worst["J"] < 1e-3 and worst["H"] < 1e-2 and worst["g"] < 1e-3
    rs = b.residual(xs, [yo[k:k + 1] for k in range(len(raw))])
    assert np.max(np.abs(np.concatenate(rs))) < 1e-10 * max(1.0, np.max(np.abs(yo)))
    b.free()


def test_graph_replay_and_eval_batched_agree(nnc, small_batch):
    import torch
    data, raw, nets = small_batch
    b = nnc.Batch(nets)
    dev = torch.device("cuda:0")
    x = synth.uniform01(synth.derive_key(2, "bx"), data.G)
    xs = [x[S] for S in data.subsets]
    lams = [np.array([0.7 - 0.1 * k]) for k in range(len(raw))]
    xc = torch.tensor(b.concat(xs), device=dev)
    lc = torch.tensor(b.concat(lams), device=dev)
    outs = []
    for graph in (False, True, True):
        b.use_graph(graph)
        y = torch.empty(b.K, dtype=torch.float64, device=dev)
        J = torch.empty(b.n_sum, dtype=torch.float64, device=dev)
        H = torch.empty(b.h_sum, dtype=torch.float64, device=dev)
        g = torch.empty(b.n_sum, dtype=torch.float64, device=dev)
        b.eval_dev(xc, lc, y, J, H, g)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in (y, J, H, g)])
    for o in outs[1:]:
        for a, c in zip(o, outs[0]):
            assert np.array_equal(a, c)
    ys, Js, Hs = nnc.eval_batched(nets, xs, lams)
    yb, Jb, Hb, _ = b.split_outputs(*outs[0])
    for k in range(len(raw)):
        assert np.array_equal(ys[k], yb[k]) and np.array_equal(Js[k], Jb[k]) and np.array_equal(Hs[k], Hb[k])
    b.free()


def test_set_bias_changes_the_load(nnc, small_batch):
    data, raw, nets = small_batch
    b = nnc.Batch(nets)
    d2 = synth.load_vectors(1, 64, seed=5)[0]
    raw2 = _raw_nets(data, d2)
    b.set_bias(0, np.stack([m.b[0] for m in raw2]))
    x = synth.uniform01(synth.derive_key(3, "bx"), data.G)
    xs = [x[S] for S in data.subsets]
    ys, _, _, _ = b.eval(xs, None, want=("y",))
    yo = np.concatenate([onn.value(raw2[k], xs[k]) for k in range(len(raw2))])
    assert rel(np.concatenate(ys), yo) < 1e-6
    b.free()


def test_scopf_ipm_matches_oracle(nnc):
    data = scopf_data(K=16, G=40, n_bus=64, n_min=5, n_max=30, hidden=128, depth=3, seed=0)
    d = np.ones(64)
    po = problems.scopf(data, d)
    ro = oipm.solve(po)
    assert ro.status == oipm.OPTIMAL
    raw = _raw_nets(data, d)
    nets = [nnc.Net.from_mlp(m, precision="bf16x3") for m in raw]
    b = nnc.Batch(nets)
    res, v, lam = nnc.ipm_scopf(b, data.G, data.subsets, data.cost, problems.scopf_demand(data, d),
                                data.delta)
    print(f"[ipm scopf bf16x3] status={res['status_name']} iters={res['iters']} (oracle {ro.iters}) "
          f"obj={res['obj']:.12g} (oracle {ro.obj:.12g}) kkt={res['kkt_error']:.2e} t={res['solve_seconds']:.3f}s")
    assert res["status"] == 0 and res["kkt_error"] <= 1e-6
    assert abs(res["obj"] - ro.obj) <= 1e-6 * abs(ro.obj)
    b.free()
    for n in nets:
        n.free()


def test_fused_residual_matches_separate_calls(nnc, small_batch):
    """nnc_batch_eval_kkt_dev: the FP64-accurate residual, J, H and gradient of every net from one
    value pass, equal to the separate calls, with and without the CUDA graph."""
    import torch
    data, raw, nets = small_batch
    b = nnc.Batch(nets)
    dev = torch.device("cuda:0")
    x = synth.uniform01(synth.derive_key(4, "bx"), data.G)
    xs = [x[S] for S in data.subsets]
    lams = [np.array([0.3 + 0.05 * k]) for k in range(len(raw))]
    yv = np.array([0.1 * k - 0.4 for k in range(len(raw))])
    xc = torch.tensor(b.concat(xs), device=dev)
    lc = torch.tensor(b.concat(lams), device=dev)
    yc = torch.tensor(yv, device=dev)

    def bufs():
        return (torch.empty(b.K, dtype=torch.float64, device=dev),
                torch.empty(b.n_sum, dtype=torch.float64, device=dev),
                torch.empty(b.h_sum, dtype=torch.float64, device=dev),
                torch.empty(b.n_sum, dtype=torch.float64, device=dev))
    y, J, H, g = bufs()
    r_sep = torch.empty(b.K, dtype=torch.float64, device=dev)
    b.use_graph(False)
    b.eval_dev(xc, lc, y, J, H, g)
    b.residual_dev(xc, yc, r_sep)
    torch.cuda.synchronize()
    ref = [t.cpu().numpy() for t in (r_sep, J, H, g)]
    yo = np.concatenate([onn.value(raw[k], xs[k]) for k in range(len(raw))])
    assert np.max(np.abs(ref[0] - (yv - yo))) <= 1e-10 * max(1.0, np.max(np.abs(yo)))
    for graph in (False, True, True):
        b.use_graph(graph)
        r, J2, H2, g2 = bufs()
        b.eval_kkt_dev(xc, yc, lc, r, J2, H2, g2)
        torch.cuda.synchronize()
        for a, c in zip([t.cpu().numpy() for t in (r, J2, H2, g2)], ref):
            assert np.array_equal(a, c)
    b.free()


def test_syrk_splits_keep_results(nnc, small_batch):
    """nnc_batch_tune_set: split-K of the symmetric product changes only the FP32 summation order
    of H (relative change at FP32 rounding level); J and the gradient are untouched.  A graph
    replay counts its kernel nodes as launches."""
    import torch
    data, raw, nets = small_batch
    b = nnc.Batch(nets)
    dev = torch.device("cuda:0")
    x = synth.uniform01(synth.derive_key(5, "bx"), data.G)
    xc = torch.tensor(b.concat([x[S] for S in data.subsets]), device=dev)
    lc = torch.tensor(b.concat([np.array([0.5 + 0.1 * k]) for k in range(len(raw))]), device=dev)
    assert b.tuning() == 1
    outs = []
    for splits in (1, 3):
        b.tune_set(splits)
        assert b.tuning() == splits
        b.use_graph(True)
        y = torch.empty(b.K, dtype=torch.float64, device=dev)
        J = torch.empty(b.n_sum, dtype=torch.float64, device=dev)
        H = torch.empty(b.h_sum, dtype=torch.float64, device=dev)
        g = torch.empty(b.n_sum, dtype=torch.float64, device=dev)
        b.eval_dev(xc, lc, y, J, H, g)
        c0 = nnc.launch_count()
        b.eval_dev(xc, lc, y, J, H, g)
        torch.cuda.synchronize()
        assert nnc.launch_count() - c0 > 5
        outs.append([t.cpu().numpy() for t in (y, J, H, g)])
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert rel(outs[1][2], outs[0][2]) <= 1e-5
    with pytest.raises(nnc.NNCError):
        b.tune_set(0)
    assert b.tuning() == 3
    b.free()


def test_host_eval_kkt_matches_separate_calls(nnc, small_batch):
    """nnc_batch_eval_kkt (host arrays): the residual, J, H and gradient from one value pass equal
    nnc_batch_residual and nnc_batch_eval bit for bit, and the residual matches the oracle."""
    data, raw, nets = small_batch
    b = nnc.Batch(nets)
    x = synth.uniform01(synth.derive_key(6, "bx"), data.G)
    xs = [x[S] for S in data.subsets]
    lams = [np.array([0.2 + 0.03 * k]) for k in range(len(raw))]
    ys = [np.array([0.05 * k - 0.3]) for k in range(len(raw))]
    r, J, H, g = b.eval_kkt(xs, ys, lams)
    _, Js, Hs, gs = b.eval(xs, lams)        # per-net views of the concatenated outputs
    r_ref = np.concatenate(b.residual(xs, ys))
    _, J2, H2, g2 = b.split_outputs(None, J, H, g)
    assert np.array_equal(r, r_ref)
    for k in range(len(raw)):
        assert np.array_equal(J2[k], Js[k]) and np.array_equal(H2[k], Hs[k]) and np.array_equal(g2[k], gs[k])
    yo = np.concatenate([onn.value(raw[k], xs[k]) for k in range(len(raw))])
    assert np.max(np.abs(r - (np.concatenate(ys) - yo))) <= 1e-10 * max(1.0, np.max(np.abs(yo)))
    b.free()


def test_host_eval_kkt_pinned_outputs(nnc, small_batch):
    """nnc_batch_eval_kkt with outputs in page-locked memory (written in place by the kernels that
    form them) equals the call with pageable outputs bit for bit, with and without the CUDA graph,
    on repeated calls."""
    import torch
    data, raw, nets = small_batch
    b = nnc.Batch(nets)
    x = synth.uniform01(synth.derive_key(6, "bx"), data.G)
    xs = [x[S] for S in data.subsets]
    lams = [np.array([0.2 + 0.03 * k]) for k in range(len(raw))]
    ys = [np.array([0.05 * k - 0.3]) for k in range(len(raw))]
    ref = b.eval_kkt(xs, ys, lams)

    def pin(k):
        a = torch.empty(k, dtype=torch.float64, pin_memory=True).numpy()
        a[...] = np.nan
        return a

    outs = tuple(pin(a.size) for a in ref)
    for graph in (False, True, True):
        b.use_graph(graph)
        got = b.eval_kkt(xs, ys, lams, out=outs)
        for a, c in zip(got, ref):
            assert np.array_equal(a, c)
        for a in outs:
            a[...] = np.nan
    b.free()


def test_batch_bench_size_matches_oracle(nnc):
    """The batch the bench times: 256 surrogates n_k -> 1024 x 5 sigmoid -> 1 with n_k ~ U{20..200}
    (seed 0, loads d = 1), autotuned tiles, one fused evaluation per iterate replayed from the CUDA
    graph.  Nets
    with 128 < n_k <= 200 take three lower-triangle tiles of the grouped symmetric product and the
    persistent grouped tangent GEMM runs more than 13 tiles per CTA.  Every net's FP64 residual and
    the value are checked; J, gradient and the full H of 45 nets (the 16 with n_k > 190 and every
    eighth one) against the oracle, at the stated tolerances."""
    import torch
    data = scopf_data(K=256, G=200, n_bus=512, seed=0)
    d = np.ones(512)
    raw = _raw_nets(data, d)
    nets = [nnc.Net.from_mlp(m, precision="bf16x3") for m in raw]
    b = nnc.Batch(nets)
    for n in nets:
        n.free()
    bn, sp = b.autotune()                     # the tiling the bench runs with
    print(f"[batch bench size] autotuned tangent N tile {bn}, symmetric-product splits {sp}")
    assert bn >= 208 and 1 <= sp <= 3
    b.use_graph(True)
    dev = torch.device("cuda:0")
    x = synth.uniform01(synth.derive_key(9, "bench-bx"), data.G)
    xs = [x[S] for S in data.subsets]
    lams = [synth.normal(synth.derive_key(k, "bench-blam"), 1) for k in range(len(raw))]
    yo = np.concatenate([onn.value(raw[k], xs[k]) for k in range(len(raw))])
    xc = torch.tensor(b.concat(xs), device=dev)
    lc = torch.tensor(b.concat(lams), device=dev)
    yi = torch.tensor(yo, device=dev)
    outs = []
    for _ in range(2):          # capture, then replay
        r = torch.empty(b.K, dtype=torch.float64, device=dev)
        J = torch.empty(b.n_sum, dtype=torch.float64, device=dev)
        H = torch.empty(b.h_sum, dtype=torch.float64, device=dev)
        g = torch.empty(b.n_sum, dtype=torch.float64, device=dev)
        b.eval_kkt_dev(xc, yi, lc, r, J, H, g)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in (r, J, H, g)])
    for a, c in zip(outs[0], outs[1]):
        assert np.array_equal(a, c)
    r, J, H, g = outs[1]
    assert np.max(np.abs(r)) <= 1e-10 * max(1.0, np.max(np.abs(yo))), np.max(np.abs(r))
    ys, _, _, _ = b.eval(xs, None, want=("y",))
    assert rel(np.concatenate(ys), yo) < 1e-6
    _, Js, Hs, gs = b.split_outputs(None, J, H, g)
    n_in = np.array([len(S) for S in data.subsets])
    assert n_in.max() > 190 and (n_in > 128).sum() > 32
    sample = sorted(set(np.flatnonzero(n_in > 190).tolist()) | set(range(0, 256, 8)))
    worst = dict(J=0.0, H=0.0, g=0.0)
    for k in sample:
        Jo = onn.jacobian(raw[k], xs[k])
        Ho = onn.hessian_lag(raw[k], xs[k], lams[k])
        go = onn.vjp(raw[k], xs[k], lams[k])
        worst["J"] = max(worst["J"], rel(Js[k], Jo))
        worst["H"] = max(worst["H"], rel(Hs[k], Ho))
        worst["g"] = max(worst["g"], rel(gs[k], go))
        assert np.array_equal(Hs[k], Hs[k].T)
    print(f"[batch bench size, {len(sample)} nets] worst rel err J={worst['J']:.2e} "
          f"H={worst['H']:.2e} g={worst['g']:.2e}")
    assert worst["J"] < 1e-3 and worst["H"] < 1e-2 and worst["g"] < 1e-3
    b.free()
