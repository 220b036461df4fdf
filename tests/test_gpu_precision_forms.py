"""The precision forms on the ~104M-parameter net over 32 reference images.

For x0 ~ U[0,1]^784 with seeds 0..31 (lambda ~ N(0,1) of the same seed), the BF16, split-BF16x3
and FP8-e4m3 forms are compared with the FP64 oracle on the value, the Jacobian and the full
784 x 784 Hessian of lambda^T NN, and each form's interior-point solve of the adversarial problem
(min ||x - x0||^2 s.t. y = NN(x), y_3 >= y_j + 0.1, 0 <= x <= 1) to KKT 1e-6 is compared with the
FP64 GPU form's solve from the same start (whose iterates follow the oracle interior-point
method, tests/test_gpu_ipm.py).  Tolerances: BF16 and BF16x3 value 1e-6, Jacobian 1e-3, Hessian
1e-2 (relative Frobenius), converged objective 1e-6 relative with both KKT certificates <= 1e-6;
FP8 is reported (its Hessian bound 0.3 only catches a broken kernel), its solves must certify
KKT <= 1e-6 when they converge.
"""
import numpy as np
import pytest

import synth
from synth.nets import make_mlp
from oracle import nn as onn

pytestmark = pytest.mark.gpu

SEEDS = range(32)
FORMS = ("bf16", "bf16x3", "fp8")
TOL = {"bf16": dict(y=1e-6, J=1e-3, H=1e-2), "bf16x3": dict(y=1e-6, J=1e-3, H=1e-2),
       "fp8": dict(y=1e-6, J=1e-3, H=0.3)}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_precision_forms_over_32_seeds():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_22462_gb300 import build, nnc
    build.build()
    mlp = make_mlp(synth.PAPER_104M, seed=0)
    data = [synth.adversarial_data(seed=s) for s in SEEDS]
    errs = {f: {"y": [], "J": [], "H": []} for f in FORMS}
    outs = {}
    for f in FORMS:
        net = nnc.Net.from_mlp(mlp, precision=f)
        net.autotune()
        outs[f] = []
        for d in data:
            y = net.eval(d.x0)
            J = net.jacobian(d.x0)
            H = net.hessian_lag(d.x0, d.lam)
            outs[f].append((y, J, H))
        net.free()
    for i, d in enumerate(data):
        yo, Jo, Ho, _ = onn.all_outputs(mlp, d.x0, d.lam)
        for f in FORMS:
            y, J, H = outs[f][i]
            errs[f]["y"].append(rel(y, yo))
            errs[f]["J"].append(rel(J, Jo))
            errs[f]["H"].append(rel(H, Ho))
    del outs
    print("\nform    quantity  median      max        (relative Frobenius vs the FP64 oracle, 32 seeds)")
    for f in FORMS:
        for q in ("y", "J", "H"):
            v = np.array(errs[f][q])
            print(f"{f:7s} {q:8s}  {np.median(v):.3e}  {v.max():.3e}")
            assert v.max() < TOL[f][q], (f, q, v.max())

    # converged objectives: each form against the FP64 GPU form from the same start
    results = {}
    for f in ("fp64",) + FORMS:
        net = nnc.Net.from_mlp(mlp, precision=f)
        net.autotune()
        results[f] = [nnc.ipm_adversarial(net, d.x0, d.target, d.margin)[0] for d in data]
        net.free()
    print("form    solved  iters(mean)  seconds(mean)  max |obj - obj_fp64| / |obj_fp64|")
    for f in ("fp64",) + FORMS:
        rs = results[f]
        ok = [r["status"] == 0 and r["kkt_error"] <= 1e-6 for r in rs]
        dobj = [abs(r["obj"] - r64["obj"]) / abs(r64["obj"]) for r, r64 in zip(rs, results["fp64"])
                if r["status"] == 0]
        print(f"{f:7s} {sum(ok):3d}/32  {np.mean([r['iters'] for r in rs]):8.2f}  "
              f"{np.mean([r['solve_seconds'] for r in rs]):12.4f}  {max(dobj) if dobj else float('nan'):.3e}")
    for i in range(len(data)):
        r64 = results["fp64"][i]
        assert r64["status"] == 0 and r64["kkt_error"] <= 1e-6, (i, r64)
        for f in FORMS:
            r = results[f][i]
            if f == "fp8" and r["status"] != 0:
                continue          # reported above
            assert r["status"] == 0 and r["kkt_error"] <= 1e-6, (f, i, r)
            if f != "fp8":
                assert abs(r["obj"] - r64["obj"]) <= 1e-6 * abs(r64["obj"]), (f, i, r["obj"], r64["obj"])
