"""A small, self-contained workload for kernel profiling (ncu) and quick timing.

  python -m paper_2509_22462_gb300.profile_case --widths 784,4096,4096,4096,10 --prec bf16x3 --reps 2
  python -m paper_2509_22462_gb300.profile_case --widths 784,128,128,10 --prec bf16 --ipm --kkt-device 1

Builds a tanh MLP with N(0, 1/fan_in) weights (seed 0) and runs `reps` full oracle calls
(value, Jacobian, gradient and Hessian of lambda^T NN, then the FP64 residual) on device-resident
inputs, then prints
the per-kernel-kind times of the last call.  With the default widths every tangent GEMM has the
shape of the 104M network's (M = 4096, N = 784, K = 4096).  --bn pins the tangent tiling (1: the
persistent chain).  --ipm instead solves the adversarial problem (x0 ~ U[0,1]^n_in, target 3,
margin 0.1) with the host interior-point driver, the KKT dense block on the device with
--kkt-device 1, and prints the per-iteration timing.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--widths", default="784,4096,4096,4096,10")
    ap.add_argument("--act", default="tanh")
    ap.add_argument("--prec", default="bf16x3")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--bn", type=int, default=0, help="pin the tangent N tile (0: the load-time plan)")
    ap.add_argument("--ipm", action="store_true", help="solve the adversarial problem instead")
    ap.add_argument("--kkt-device", type=int, default=0)
    a = ap.parse_args()
    import torch
    import synth
    from synth.nets import MLPSpec
    from paper_2509_22462_gb300 import build, nnc

    build.build()
    widths = [int(w) for w in a.widths.split(",")]
    spec = MLPSpec(widths, [a.act] * (len(widths) - 2) + ["identity"])
    mlp = synth.make_mlp(spec, seed=0)
    d = synth.adversarial_data(n_in=widths[0], n_out=widths[-1], seed=0)
    dev = torch.device("cuda:0")
    st = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(st)
    net = nnc.Net.from_mlp(mlp, precision=a.prec)
    if a.bn:
        net.tune_set(tangent_bn=a.bn)
    if a.ipm:
        res, _, _ = nnc.ipm_adversarial(net, d.x0, 3, 0.1, kkt_on_device=a.kkt_device, verbose=1)
        print({k: res[k] for k in ("status_name", "iters", "obj", "solve_seconds", "t_solver", "t_hessian")})
        net.free()
        return
    n, m = widths[0], widths[-1]
    x = torch.tensor(d.x0, device=dev)
    lam = torch.tensor(d.lam, device=dev)
    y = torch.empty(m, dtype=torch.float64, device=dev)
    J = torch.empty(m, n, dtype=torch.float64, device=dev)
    H = torch.empty(n, n, dtype=torch.float64, device=dev)
    g = torch.empty(n, dtype=torch.float64, device=dev)
    r = torch.empty(m, dtype=torch.float64, device=dev)
    for i in range(a.reps):
        if i == a.reps - 1:
            net.profile(True)
        net.eval_all_dev(x, lam, y, J, H, g)
        net.residual_dev(x, y, r)
    torch.cuda.synchronize()
    prof = net.profile_read()
    for k, (ms, cnt) in prof.items():
        if cnt:
            print(f"{k:14s} {cnt:3d} launches  {ms * 1e3 / cnt:9.1f} us/launch  {ms:8.3f} ms")
    assert bool(torch.isfinite(H).all())
    net.free()


if __name__ == "__main__":
    main()
