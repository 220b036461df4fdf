#!/usr/bin/env python
"""Throughput of the reduced-space network-constraint oracles on one GB300 (or N replicas).

One step = everything one interior-point iteration asks of the network at one point x (with
multipliers lambda): the value NN(x), the Jacobian (n_out reverse seeds), the gradient
lambda^T J, the Hessian of lambda^T NN (n_in forward-over-reverse tangents, Eq. 6) and the FP64
residual y - NN(x).  The metric is Hessian-of-Lagrangian evaluations per second, i.e. steps/s,
with inputs resident in HBM; `e2e` is the same through the host-pointer C ABI (copies inside).

Workload: the ~104M-parameter MNIST-shaped net 784 -> 4096 x 7 -> 10 (tanh, N(0, 1/fan_in)
weights, seed 0), x0 ~ U[0,1]^784, lambda ~ N(0,1).  The packed weights (about 2 GB: double-float
pairs for the residual, FP32 for the reverse sweep, BF16 for the tangents) exceed the 129 MB L2,
so no flush is needed between steps.

The headline form is BF16 (one BF16 product per tensor-core tile, FP32 accumulation, the
double-float FP64-accurate residual and the FP32 reverse sweep); `forms` and `ipm_solve` report
the split-BF16x3 and FP8 forms and the FP64 GPU form beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--prec bf16|bf16x3|fp8|fp32|fp64]
Under torchrun each rank runs an independent replica (the path does not shard); rank 0 prints
one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hessian_lag_evals_per_s"

# DRAM bytes (read + write) of one tangent-GEMM launch per (M, N, K) shape, form and N tile, from
# the ncu capture summarised in profiles/k_tc_gemm_tangent_bf16_784x4096x4096.md (M = 4096,
# N = 784, K = 4096, the kernel with the shared-memory staged epilogue); an entry is valid only for
# the shape and kernel version it was taken on, other shapes and forms report null.
TANGENT_TRAFFIC = {((4096, 784, 4096), "bf16", 208): 40.16e6}
UNIT = "evals/s"
FP64_NOMINAL_TFLOPS = 1.25   # GB300's nominal dense FP64 rate


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="bf16", choices=["bf16", "bf16x3", "fp8", "fp32", "fp64"])
    p.add_argument("--workload", default="104m", choices=["104m", "87m", "tiny", "scopf68m", "scopf", "70m",
                                                              "274m", "warmstart", "fullspace"])
    p.add_argument("--scopf-k", type=int, default=256)
    p.add_argument("--ws-train", type=int, default=10000, help="warmstart: training loads (cold solves)")
    p.add_argument("--ws-test", type=int, default=1000, help="warmstart: held-out loads")
    p.add_argument("--ws-epochs", type=int, default=100)
    p.add_argument("--fs-widths", default="128,512,1024",
                   help="fullspace: hidden widths of the 784 -> w x 5 -> 10 classifiers")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-form", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-ipm", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the other tensor-core forms")
    p.add_argument("--oracle-step-probe", action="store_true", help=argparse.SUPPRESS)
    return p.parse_args()


def _workload(name):
    import synth
    spec = synth.spec_by_name(name)
    # the softmax classifiers (Eq. 7) use the trained-classifier stand-in; the rest plain N(0, 1/fan_in)
    mlp = synth.make_classifier(spec, seed=0) if spec.acts[-1] == "softmax" else synth.make_mlp(spec, seed=0)
    d = synth.adversarial_data(n_in=spec.n_in, n_out=spec.n_out, seed=0)
    return spec, mlp, d


def _workload_config(spec, name, prec):
    kind = "scopf_single" if name.startswith("scopf") else "mnist"
    acts = spec.acts[0] + ("+softmax" if spec.acts[-1] == "softmax" else "")
    weights = ("N(0,16/fan_in) sigmoid / N(0,1/fan_in) tanh hidden, logits x3 (classifier stand-in)"
               if spec.acts[-1] == "softmax" else "N(0,1/fan_in)")
    return {"workload": f"{kind}_{name}_{'x'.join(map(str, spec.widths))}_{acts}",
            "n_params": spec.n_params, "n_in": spec.n_in, "n_out": spec.n_out,
            "precision_form": prec,
            "inputs": f"x0~U[0,1]^{spec.n_in}, lambda~N(0,1), weights {weights} seed 0",
            "l2": "weights exceed L2 (no flush needed)"}


# ------------------------------------------------------------------ algorithmic work
def tangent_shape(spec):
    """(M, N, K) of the tangent GEMMs Zdot_l = W_l Adot_{l-1} (hidden layers 2 .. L-1, N = n_in),
    or None when the layers differ in shape."""
    w = spec.widths
    shapes = {(w[l], w[0], w[l - 1]) for l in range(2, len(w) - 1)}
    return shapes.pop() if len(shapes) == 1 else None


def hessian_flops(spec):
    """Algorithmic FLOPs of one Hessian by the per-layer sum form that the GPU runs, counted once
    (no padding, no x3): forward tangents 2 n m_l k_l for l >= 2, plus the lower triangle of each
    Zdot_l^T diag(c_l) Zdot_l, n (n+1) m_l, for layers with curvature."""
    n = spec.n_in
    f = 0
    L = spec.n_layers
    for l in range(L):
        m, k = spec.widths[l + 1], spec.widths[l]
        has_curv = spec.acts[l] != "identity"
        last = l == L - 1
        if l >= 1 and not (last and not has_curv):
            f += 2 * n * m * k
        if has_curv:
            f += n * (n + 1) * m
    return f


def tangent_gemm_flops(spec):
    """(flops per launch, launches) of the tangent GEMM Zdot_l = W_l Adot_{l-1}."""
    n = spec.n_in
    per = []
    L = spec.n_layers
    for l in range(1, L):
        last = l == L - 1
        if last and spec.acts[l] == "identity":
            continue
        per.append(2 * n * spec.widths[l + 1] * spec.widths[l])
    return per


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        with open(self.f.name) as fh:
            out = parse_clock_samples(fh)
        os.unlink(self.f.name)
        return out


def parse_clock_samples(lines):
    """nvidia-smi samples (csv, noheader, nounits, the Clocks.FIELDS order) -> the median SM clock
    under load, the maximum SM clock and the throttle reasons active in any sample; None without
    samples.  Malformed lines are skipped."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
        except ValueError:
            continue
    if not rows:
        return None
    sm = sorted(r[0] for r in rows)
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[2][i].lower().startswith("active")})
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
            "samples": len(rows)}


def _gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",")]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ multi-rank aggregation
def aggregate(el_ms, steps, world, device=None):
    """Whole-job throughput of `world` independent replicas: the timed region is the slowest
    rank's (max over ranks), every rank did `steps` units.  Returns (value, max_ms)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(el_ms)], device=device) if device is not None else torch.tensor([float(el_ms)])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el_ms = float(t.item())
    return world * steps / (el_ms / 1e3), el_ms


# ------------------------------------------------------------------ oracle timing
def oracle_step(mlp, x, lam, cols=None):
    from oracle import nn as onn
    y = onn.value(mlp, x)
    onn.jacobian(mlp, x)
    onn.vjp(mlp, x, lam)
    if cols is None:
        onn.hessian_lag(mlp, x, lam)
    else:
        onn.hessian_lag_columns(mlp, x, lam, cols)
    _ = y - onn.value(mlp, x)  # the residual y - NN(x) in FP64


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def time_oracle_single_thread(workload):
    """One full oracle step with every BLAS / OpenMP pool limited to one thread, in a child
    process (the thread limits must be set before numpy loads).  Returns seconds or None."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-step-probe",
                            "--workload", workload], capture_output=True, text=True, env=env,
                           timeout=600)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except Exception:
        return None


def _oracle_step_probe(args):
    spec, mlp, d = _workload(args.workload)
    t0 = time.perf_counter()
    oracle_step(mlp, d.x0, d.lam)
    print(time.perf_counter() - t0, flush=True)
    return 0


def time_oracle(mlp, d, budget_s=12.0, max_steps=20):
    """Bounded sample: full oracle steps until `budget_s` seconds (at least one)."""
    n_done, t0 = 0, time.perf_counter()
    while True:
        oracle_step(mlp, d.x0, d.lam)
        n_done += 1
        el = time.perf_counter() - t0
        if el > budget_s or n_done >= max_steps:
            break
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": n_done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_done} full oracle step(s) (value, Jacobian, gradient, forward-over-reverse "
                      f"Hessian, FP64 residual) in {el:.1f} s, numpy FP64 with multithreaded BLAS",
            "cpu_model": cpu_model()}


def time_oracle_ipm(mlp, d):
    """The oracle interior-point method (numpy FP64, eigenvalue inertia) on the adversarial
    problem, solved to KKT 1e-6 on the host cores: the CPU column of the IPM comparison."""
    from oracle import ipm as oipm, problems as oproblems
    t0 = time.perf_counter()
    r = oipm.solve(oproblems.adversarial(mlp, d.x0, d.target, d.margin))
    el = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"status": int(r.status), "iters": int(r.iters), "obj": float(r.obj),
            "kkt_error": float(r.kkt_error), "solve_seconds": el, "cores": cores,
            "kind": "oracle (numpy FP64 on the host cores: forward-over-reverse Hessian, "
                    "eigenvalue inertia)"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    spec, mlp, d = _workload(args.workload)
    cfg = _workload_config(spec, args.workload, "oracle-fp64")
    # Each reference step is one full oracle step when that is cheap enough; otherwise a sample
    # of 1/8 of the Hessian's tangent columns, whose time is scaled to a full evaluation.
    t0 = time.perf_counter()
    oracle_step(mlp, d.x0, d.lam)
    t_full = time.perf_counter() - t0
    budget = 150.0
    steps_total = args.steps + args.warmup
    sample_cols = None
    scale = 1.0
    if t_full * steps_total > budget:
        nc = max(1, spec.n_in // 8)
        sample_cols = np.arange(nc)
        t0 = time.perf_counter()
        oracle_step(mlp, d.x0, d.lam, cols=np.arange(1))
        t_fixed = time.perf_counter() - t0
        scale = None
    for _ in range(max(0, args.warmup - 1)):
        oracle_step(mlp, d.x0, d.lam, cols=sample_cols)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(mlp, d.x0, d.lam, cols=sample_cols)
    el = time.perf_counter() - t0
    per = el / args.steps
    if sample_cols is not None:
        # full eval ~ fixed part + 8 x (sampled-columns part)
        per = t_fixed + (spec.n_in / len(sample_cols)) * max(per - t_fixed, 0.0)
        sample = (f"{args.steps} oracle steps with {len(sample_cols)} of {spec.n_in} Hessian tangent "
                  f"columns, scaled to a full evaluation (fixed part {t_fixed:.2f} s)")
    else:
        sample = f"{args.steps} full oracle steps"
    value = 1.0 / per
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def _scopf_workload(K):
    """256 stability-margin surrogates n_k -> 1024 x 5 sigmoid -> 1, n_k ~ U{20..200}, G = 200,
    loads d = 1 entering each first-layer bias (the synthetic SCOPF-shaped batch)."""
    import copy
    import synth
    data = synth.scopf_data(K=K, G=200, n_bus=512, seed=0)
    d = np.ones(data.n_bus)
    raw = []
    for k in range(K):
        m = copy.copy(data.nets[k])
        m.b = list(m.b)
        m.b[0] = synth.scopf_first_bias(data, k, d)
        raw.append(m)
    return data, d, raw


def scopf_flops(n_in, hidden=1024, depth=5):
    """Algorithmic FLOPs of one batched Hessian (sum form): per net 2 n m k for the depth-1
    hidden-to-hidden tangent GEMMs plus n (n+1) m per sigmoid layer (lower triangles)."""
    f = 0
    for n in n_in:
        f += (depth - 1) * 2 * n * hidden * hidden + depth * n * (n + 1) * hidden
    return f


def scopf_weight_bytes(raw, prec):
    """Algorithmic DRAM bytes of one batched step: every weight is read by the double-float value
    pass (8 B: hi, lo FP32 pair), the FP32 reverse sweep (4 B) and the tangent sweep (the FP32
    first layer, 4 B; the hidden layers' tangent operand: BF16 hi + lo in the split form, 4 B,
    BF16 hi in the BF16 form, 2 B, e4m3 in the FP8 form, 1 B; a linear output layer takes no
    tangent)."""
    tb = {"bf16x3": 4, "bf16": 2, "fp8": 1}.get(prec, 4)
    b = 0
    for m in raw:
        P = sum(w.size for w in m.W)
        P1 = m.W[0].size
        b += 8 * P + 4 * P + 4 * P1 + tb * (P - P1 - m.W[-1].size)
    return b


def run_ours_scopf(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import synth

    data, d, raw = _scopf_workload(args.scopf_k)
    K = len(raw)
    n_in = [len(s) for s in data.subsets]
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import problems as oproblems, nn as onn
        sample = 8
        x = np.full(data.G, synth.scopf_demand(data, d) / data.G)
        t0 = time.perf_counter()
        for k in range(sample):
            xs = x[data.subsets[k]]
            onn.value(raw[k], xs)
            onn.jacobian(raw[k], xs)
            onn.vjp(raw[k], xs, np.ones(1))
            onn.hessian_lag(raw[k], xs, np.ones(1))
        el = time.perf_counter() - t0
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        cpu_baseline = {"value": 1.0 / (el * K / sample), "unit": UNIT, "cores": cores, "kind": "oracle",
                        "sample": f"value, Jacobian, gradient and Hessian of {sample} of the {K} surrogates "
                                  f"in {el:.1f} s, scaled by {K}/{sample} to one batched evaluation"}
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    from paper_2509_22462_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2509_22462_gb300 import nnc
    nets = [nnc.Net.from_mlp(m, precision=args.prec) for m in raw]
    batch = nnc.Batch(nets)
    for n in nets:
        n.free()      # the batch keeps its own stacked copy
    batch_tiling = batch.autotune(os.environ.get("NNC_BATCH_TUNE_CACHE"))
    batch.use_graph(True)
    x = np.full(data.G, synth.scopf_demand(data, d) / data.G)
    xc = torch.tensor(batch.concat([x[s] for s in data.subsets]), device=dev)
    lc = torch.ones(K, dtype=torch.float64, device=dev)
    y = torch.empty(K, dtype=torch.float64, device=dev)
    J = torch.empty(batch.n_sum, dtype=torch.float64, device=dev)
    H = torch.empty(batch.h_sum, dtype=torch.float64, device=dev)
    g = torch.empty(batch.n_sum, dtype=torch.float64, device=dev)
    r = torch.empty(K, dtype=torch.float64, device=dev)
    y_it = torch.zeros(K, dtype=torch.float64, device=dev)   # the iterate's margins y_k

    def step():
        # one interior-point iterate of every surrogate: FP64-accurate residual, J, H and
        # gradient from one value pass
        batch.eval_kkt_dev(xc, y_it, lc, r, J, H, g)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(_gpu_index(local_rank)) if rank == 0 else None
    launches0 = nnc.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = nnc.launch_count() - launches0
    clk = clocks.stop() if clocks else None
    value, el_ms = aggregate(e0.elapsed_time(e1), args.steps, world, dev)
    # end to end through the host-pointer batch call (the fused iterate call of the device step),
    # inputs and outputs in pinned host memory
    pin = lambda k: torch.empty(k, dtype=torch.float64, pin_memory=True).numpy()  # noqa: E731
    xh, yh, lh = pin(batch.n_sum), pin(K), pin(K)
    xh[:], yh[:], lh[:] = batch.concat([x[s] for s in data.subsets]), 0.0, 1.0
    outs = (pin(K), pin(batch.n_sum), pin(batch.h_sum), pin(batch.n_sum))
    batch.eval_kkt(xh, yh, lh, out=outs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        batch.eval_kkt(xh, yh, lh, out=outs)
    el = time.perf_counter() - t0
    e2e = {"value": world * args.steps / el, "unit": UNIT,
           "h2d_bytes_per_step": 8 * (batch.n_sum + K + K),
           "d2h_bytes_per_step": 8 * (K + batch.n_sum + batch.h_sum + batch.n_sum)}
    ipm = {}
    if rank == 0 and not args.no_ipm:
        res, v, lam = nnc.ipm_scopf(batch, data.G, data.subsets, data.cost, synth.scopf_demand(data, d),
                                    data.delta)
        ipm[args.prec] = res
    fl = scopf_flops(n_in)
    wb = scopf_weight_bytes(raw, args.prec)
    if rank == 0:
        out = {"metric": "batched_hessian_lag_evals_per_s", "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": el_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
               "data": "synthetic",
               "config": {"workload": f"scopf_{K}x(n_k->1024x5->1)_sigmoid", "n_params": int(sum(
                   sum(w.size + b.size for w, b in zip(m.W, m.b)) for m in raw)), "G": data.G,
                   "n_in_range": [min(n_in), max(n_in)], "precision_form": args.prec,
                   "l2": "weights exceed L2 (no flush needed)", "cuda_graph": True,
                   "autotuned": {"tangent_bn": batch_tiling[0], "syrk_splits": batch_tiling[1]}},
               "roofline": {"kernel": "whole step (grouped value pass, reverse sweep, persistent "
                                      "grouped tangent GEMM, symmetric product)",
                            "bound": "hbm", "achieved": wb / (el_ms / args.steps / 1e3) / 1e9,
                            "peak": _peaks()[0].get("hbm_gbs"), "unit": "GB/s",
                            "frac": wb / (el_ms / args.steps / 1e3) / 1e9 / _peaks()[0].get("hbm_gbs"),
                            "traffic": None, "algorithmic_bytes_per_step": wb,
                            "tensor_tflops_algorithmic": fl / (el_ms / args.steps / 1e3) / 1e12},
               "cpu_baseline": cpu_baseline, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
               "ipm_solve": ipm, "hessian_algorithmic_gflop": fl / 1e9}
        print(json.dumps(out), flush=True)
    batch.free()
    return 0


def timed_kernel_pass(net, step, steps, torch, kind="tangent_chain"):
    """K steps with one pair of events per step around the chain of tangent GEMMs (the library's
    "tangent_chain" span, counted as its launches, so that no event sits between launches that
    overlap through programmatic dependent launch; or another span kind); returns {kind: (ms,
    count)} and the pass's time per step in ms under "_ms_per_step"."""
    net.profile(True, kinds=[kind])
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record()
    for _ in range(steps):
        step()
    a1.record()
    torch.cuda.synchronize()
    out = net.profile_read()
    net.profile(False)
    out["_ms_per_step"] = (a0.elapsed_time(a1) / steps, steps)
    return out


def tangent_roofline(net, spec, prec, roof_pass, prof, peaks, peak_src):
    """Roofline of the dominant kernel, the tangent GEMM (the largest single kernel of a step):
    algorithmic FLOPs per launch over the average launch time of the timed kernel pass."""
    has_tan = prof.get("tangent_gemm", (0, 0))[1] > 0 or roof_pass.get("tangent_chain", (0, 0))[1] > 0
    dom_name = "tangent_gemm" if has_tan else max(prof.items(), key=lambda kv: kv[1][0])[0]
    if dom_name == "tangent_gemm" and roof_pass.get("tangent_chain", (0, 0))[1]:
        dom_ms, dom_cnt = roof_pass["tangent_chain"]
    else:
        dom_ms, dom_cnt = prof[dom_name]
    if dom_name == "tangent_gemm" and dom_cnt > 0:
        tangent_bn = net.tuning(1)[0] if len(spec.widths) > 3 else 0
        per = tangent_gemm_flops(spec)
        fl_per_launch = sum(per) / len(per)
        avg_s = dom_ms / dom_cnt / 1e3
        ach = fl_per_launch / avg_s / 1e12
        # the kernel is timed inside a step of well under a second: the burst peak applies
        # (for FP8 operands the measured BF16 peak times the nominal 2x of e4m3)
        pk = peaks.get("bf16_tflops") * (2.0 if prec == "fp8" else 1.0)
        kname = ("k_tc_chain (every tangent GEMM Zdot_l = W_l Adot_{l-1} of the step in one persistent "
                 "tcgen05 launch, fused sigma' / sigma'' epilogue; per-layer average)" if tangent_bn == 1 else
                 "k_tc_pair (tangent on SM pairs, tcgen05 cta_group::2: Zdot_l = W_l Adot_{l-1}, "
                 "fused sigma' / sigma'' epilogue)" if tangent_bn < 0 else
                 "k_tc_gemm (tangent: Zdot_l = W_l Adot_{l-1}, fused sigma' / sigma'' epilogue)")
        mult = {"bf16x3": 3, "bf16": 1, "fp8": 1}.get(prec, 1)
        return {"kernel": kname if prec in ("bf16", "bf16x3", "fp8") else "k_simt_gemm (tangent)",
                "timing": "average launch time over the chain of tangent GEMMs of each step "
                          "(one event pair per step, on the launch stream)",
                "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "traffic": TANGENT_TRAFFIC.get((tangent_shape(spec), prec, tangent_bn)),
                "tangent_bn": tangent_bn,
                "peak_source": f"{peak_src} bf16 burst" + (" x 2 (e4m3 nominal ratio)" if prec == "fp8" else ""),
                "executed_frac": ach * mult / pk, "products_per_tile": mult,
                "avg_launch_us": avg_s * 1e6, "launches": dom_cnt,
                "algorithmic_flops_per_launch": fl_per_launch,
                "timed_pass_ms_per_step": roof_pass.get("_ms_per_step", (None,))[0]}
    if dom_cnt > 0:
        avg_s = dom_ms / dom_cnt / 1e3
        return {"kernel": dom_name, "bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"),
                "unit": "GB/s", "frac": None, "traffic": None, "avg_launch_us": avg_s * 1e6}
    return None


def run_ours_warmstart(args, rank, world, local_rank):
    """The learned warm start on the SCOPF-shaped batch (256 surrogates): cold interior-point solves
    of --ws-train loads d ~ N(1, 0.1^2) per bus give the training data, the warm-start MLP
    (512 -> 256 -> 256 -> 713, GELU, BF16 on the tensor cores) is trained on the GPU, and
    --ws-test held-out loads are solved warm-started and cold to KKT 1e-6.  The metric is the mean
    warm-started solve time (fallbacks to a cold solve included); the cold mean sits beside it."""
    import torch
    if rank != 0:
        return 0
    torch.cuda.set_device(local_rank)
    from paper_2509_22462_gb300 import build as B
    B.build()
    from paper_2509_22462_gb300 import warmstart_experiment as wse
    t0 = time.perf_counter()
    rep, _ = wse.run(K=args.scopf_k, n_train=args.ws_train, n_test=args.ws_test, epochs=args.ws_epochs,
                     prec=args.prec if args.prec in ("bf16", "bf16x3") else "bf16x3", log=lambda *a: None)
    wall = time.perf_counter() - t0
    out = {"metric": "warm_started_ipm_solve_s", "value": rep["warm_seconds_mean"], "unit": "s",
           "n_gpus": 1, "steps": args.ws_test, "warmup": 0, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": f"scopf_{args.scopf_k}x(n_k->1024x5->1)_warmstart_512x256x256x713_gelu",
                      "train_loads": args.ws_train, "test_loads": args.ws_test, "epochs": args.ws_epochs,
                      "loads": "d ~ N(1, 0.1^2) per bus, 512 buses"},
           "cold_seconds_mean": rep["cold_seconds_mean"], "warm_start": rep, "wall_seconds": wall}
    print(json.dumps(out), flush=True)
    return 0


def run_ours_fullspace(args, rank, world, local_rank):
    """Tables 2-3's contrast on the MNIST-shaped classifiers 784 -> w x 5 -> 10 (tanh, softmax
    output; w = 128, 512, 1024 give the 167k, 1.46M and 5.0M parameter rows): Eq. 7 (L1 change
    of an image, target class at probability >= 0.6) solved to KKT 1e-6 in the reduced space (the
    network on the GPU, BF16 and FP64 forms) and in the full space of Eq. 4 (host functions, the
    sparse stage-by-stage KKT factorization), from the same start.  Weights N(0, 1/fan_in) with
    the output layer scaled by 4 (so that 0.6 is reachable, as for a trained classifier), x ~
    U[0,1]^784, target = the second most likely class.  The metric is the full-space solve time of
    the widest net; iterations, times and objectives of every form are beside it."""
    import torch
    if rank != 0:
        return 0
    torch.cuda.set_device(local_rank)
    from paper_2509_22462_gb300 import build as B, nnc
    B.build()
    import synth
    from synth.nets import MLPSpec
    rows = []
    for w in [int(v) for v in args.fs_widths.split(",") if v]:
        widths = [784] + [w] * 5 + [10]
        mlp = synth.make_mlp(MLPSpec(widths, ["tanh"] * 5 + ["softmax"]), seed=1, tag="table3",
                             bias_std=0.3)
        mlp.W[-1] = mlp.W[-1] * 4
        x = synth.uniform01(synth.derive_key(1, "table3-x"), 784)
        net = nnc.Net.from_mlp(mlp, precision="fp64")
        p0 = net.eval(x)
        t = int(np.argsort(p0)[-2])
        row = {"widths": widths, "n_params": int(sum(a.size for a in mlp.W) + sum(b.size for b in mlp.b)),
               "full_space_variables": 3 * 784 + 2 * (5 * w + 10),
               "full_space_constraints": 784 + 2 * (5 * w + 10)}
        keys = ("status_name", "iters", "obj", "kkt_error", "solve_seconds", "t_solver", "t_hessian")
        for prec in ("bf16", "fp64"):
            nr = net if prec == "fp64" else nnc.Net.from_mlp(mlp, precision=prec)
            r, _, _ = nnc.ipm_adversarial_l1(nr, x, t, 0.6)
            row["reduced_" + prec] = {k: r[k] for k in keys}
            if nr is not net:
                nr.free()
        r, _, _ = nnc.ipm_adversarial_l1_fullspace(net, x, t, 0.6, max_iter=3000)
        row["full_space"] = {k: r[k] for k in keys}
        net.free()
        rows.append(row)
    last = rows[-1]
    out = {"metric": "full_space_ipm_solve_s", "value": last["full_space"]["solve_seconds"], "unit": "s",
           "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "mnist_784_wx5_10_tanh_softmax_eq7_full_vs_reduced",
                      "widths": args.fs_widths, "target": "second most likely class, p >= 0.6"},
           "rows": rows}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    if args.workload == "scopf":
        return run_ours_scopf(args, rank, world, local_rank)
    if args.workload == "warmstart":
        return run_ours_warmstart(args, rank, world, local_rank)
    if args.workload == "fullspace":
        return run_ours_fullspace(args, rank, world, local_rank)

    spec, mlp, d = _workload(args.workload)
    cpu_baseline = None
    oracle_ipm = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_baseline = time_oracle(mlp, d)  # before the first GPU call
        t1 = time_oracle_single_thread(args.workload)
        cpu_baseline["single_thread"] = ({"value": 1.0 / t1, "unit": UNIT, "cores": 1,
                                          "sample": "1 full oracle step, BLAS and OpenMP limited to "
                                                    "one thread"} if t1 else None)
        if not args.no_ipm and spec.acts[-1] != "softmax":
            oracle_ipm = time_oracle_ipm(mlp, d)

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)   # every launch and both timing events go on this stream
    torch.cuda.set_stream(stream)
    from paper_2509_22462_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2509_22462_gb300 import nnc

    net = nnc.Net.from_mlp(mlp, precision=args.prec)
    net.autotune(os.environ.get("NNC_TUNE_CACHE"))
    n, m = spec.n_in, spec.n_out
    x = torch.tensor(d.x0, device=dev)
    lam = torch.tensor(d.lam, device=dev)
    y = torch.empty(m, dtype=torch.float64, device=dev)
    J = torch.empty(m, n, dtype=torch.float64, device=dev)
    H = torch.empty(n, n, dtype=torch.float64, device=dev)
    g = torch.empty(n, dtype=torch.float64, device=dev)
    r = torch.empty(m, dtype=torch.float64, device=dev)
    y_it = torch.zeros(m, dtype=torch.float64, device=dev)   # the iterate's y of g(x, y) = y - NN(x)

    def step():
        # one interior-point iterate: FP64-accurate residual, J, H and gradient from one value pass
        net.eval_kkt_dev(x, y_it, lam, r, J, H, g)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(_gpu_index(local_rank)) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    # the headline: K steps with no event inside the timed region
    launches0 = nnc.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = nnc.launch_count() - launches0
    value, el_ms = aggregate(e0.elapsed_time(e1), args.steps, world, dev)
    # the roofline kernel's launch time: a second timed pass of K steps with the library's events
    # around each tangent-GEMM launch only, on the stream the kernel runs on
    roof_pass = timed_kernel_pass(net, step, args.steps, torch)
    # the double-float value pass (the step's HBM-bound part on its critical path), the same way
    value_pass = timed_kernel_pass(net, step, args.steps, torch, kind="value_pass") \
        if args.prec != "fp64" else None
    clk = clocks.stop() if clocks else None
    # per-kind breakdown (events around every launch, outside the timed region)
    net.profile(True)
    for _ in range(min(args.steps, 10)):
        step()
    torch.cuda.synchronize()
    prof = net.profile_read()
    net.profile(False)
    n_prof = min(args.steps, 10)

    peaks, peak_src = _peaks()
    roof = tangent_roofline(net, spec, args.prec, roof_pass, prof, peaks, peak_src)
    kernel_ms = {k: {"ms_per_step": v[0] / n_prof, "launches_per_step": v[1] / n_prof}
                 for k, v in prof.items() if v[1] > 0}

    # end to end through the host-pointer C ABI (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        # inputs and outputs in pinned host memory
        pin = lambda *shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        xh, lh, yh = pin(n), pin(m), pin(m)
        xh[:], lh[:], yh[:] = d.x0, d.lam, 0.0
        outs = (pin(m), pin(m, n), pin(n, n), pin(n))
        for _ in range(2):
            net.eval_kkt(xh, yh, lh, out=outs)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            net.eval_kkt(xh, yh, lh, out=outs)
        el = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        h2d = 8 * (n + m + m)                    # x, lambda, y
        d2h = 8 * (m + m * n + n * n + n)        # r, J, H, grad
        e2e = {"value": world * args.steps / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # IPM solve of the adversarial problem to KKT tolerance 1e-6 with this form
    # (Eq. 7 with its L1 objective and 0.6 confidence for a softmax classifier, else the
    # margin form of the adversarial problem)
    def solve(nt):
        if spec.acts[-1] == "softmax":
            return nnc.ipm_adversarial_l1(nt, d.x0, d.target, 0.6)[0]
        return nnc.ipm_adversarial(nt, d.x0, d.target, d.margin)[0]

    ipm = {}
    if rank == 0 and not args.no_ipm:
        ipm[args.prec] = solve(net)
    if oracle_ipm is not None:
        ipm["oracle"] = oracle_ipm

    # the other tensor-core forms, each timed like the headline (K steps, no events) plus its
    # own tangent-kernel pass, and solved with the same interior-point driver
    hf = hessian_flops(spec)
    forms = {args.prec: {"evals_per_s": value / world, "ms_per_eval": el_ms / args.steps,
                         "tangent_roofline_frac": roof.get("frac") if roof else None}}
    others = [] if (args.no_forms or rank != 0) else \
        [f for f in ("bf16x3", "bf16", "fp8") if f != args.prec and args.prec in ("bf16x3", "bf16", "fp8")]
    net.free()
    for f in others:
        nf = nnc.Net.from_mlp(mlp, precision=f)
        nf.autotune(os.environ.get("NNC_TUNE_CACHE"))

        def stepf(nf=nf):
            nf.eval_kkt_dev(x, y_it, lam, r, J, H, g)

        for _ in range(args.warmup):
            stepf()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(args.steps):
            stepf()
        a1.record()
        torch.cuda.synchronize()
        msf = a0.elapsed_time(a1) / args.steps
        rp = timed_kernel_pass(nf, stepf, args.steps, torch)
        rf = tangent_roofline(nf, spec, f, rp, rp, peaks, peak_src)
        forms[f] = {"evals_per_s": 1e3 / msf, "ms_per_eval": msf,
                    "tangent_roofline_frac": rf.get("frac") if rf else None,
                    "tangent_avg_launch_us": rf.get("avg_launch_us") if rf else None,
                    "tangent_bn": rf.get("tangent_bn") if rf else None}
        if not args.no_ipm:
            ipm[f] = solve(nf)
        nf.free()

    # the FP64 form on the same GPU, for the TC-vs-FP64 comparison of the metric; its Hessian runs
    # on FP64 CUDA cores, reported against the nominal FP64 rate (no measured FP64 peak exists)
    if rank == 0 and not args.no_fp64_form and args.prec != "fp64":
        n64 = nnc.Net.from_mlp(mlp, precision="fp64")
        if not args.no_ipm:
            ipm["fp64"] = solve(n64)

        def step64():
            n64.eval_kkt_dev(x, y_it, lam, r, J, H, g)

        step64()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k64 = 3
        a0.record()
        for _ in range(k64):
            step64()
        a1.record()
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1) / k64
        fp64_tflops = hf / (ms64 / 1e3) / 1e12
        forms["fp64"] = {"evals_per_s": 1e3 / ms64, "ms_per_eval": ms64, "steps": k64,
                         "hessian_tflops_algorithmic": fp64_tflops,
                         "fp64_peak_frac": fp64_tflops / FP64_NOMINAL_TFLOPS,
                         "fp64_peak": FP64_NOMINAL_TFLOPS,
                         "fp64_peak_source": "nominal GB300 FP64 rate (not measured)"}
        n64.free()

    if rank == 0:
        roof_value = None
        if value_pass and value_pass.get("value_pass", (0, 0))[1] > 0:
            vms, vcnt = value_pass["value_pass"]
            vbytes = 8 * sum(a * b for a, b in zip(spec.widths[1:], spec.widths[:-1]))
            vgbs = vbytes / (vms / 1e3 / (vcnt / (len(spec.widths) - 1))) / 1e9
            roof_value = {"kernel": "k_gemv_stream (double-float value pass, every layer)", "bound": "hbm",
                          "achieved": vgbs, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                          "frac": vgbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                          "traffic": None, "algorithmic_bytes_per_pass": vbytes,
                          "ms_per_pass": vms / (vcnt / (len(spec.widths) - 1)),
                          "timing": "one event pair per step around the pass's layers, on the launch stream"}
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.prec.startswith("bf16") else
               {"fp32": "f32", "fp8": "e4m3"}.get(args.prec, "f64"),
               "data": "synthetic", "config": _workload_config(spec, args.workload, args.prec),
               "roofline": roof, "roofline_value_pass": roof_value, "cpu_baseline": cpu_baseline,
               "e2e": e2e, "gpu_launches": launches,
               "clocks": clk, "kernels": kernel_ms, "forms": forms, "ipm_solve": ipm,
               "hessian_algorithmic_gflop": hessian_flops(spec) / 1e9}
        print(json.dumps(out), flush=True)
    return 0


def main():
    args = _args()
    if args.oracle_step_probe:
        return _oracle_step_probe(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
