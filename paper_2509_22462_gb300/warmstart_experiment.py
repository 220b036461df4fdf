"""Learned warm start for the SCOPF-shaped problem (the synthetic Eq. 8 variant).

1. Data: for load vectors d ~ N(1, 0.1^2) per bus, solve the problem cold with the interior-point
   driver (nnc_ipm_scopf); record d -> (x*, y*, lambda*).
2. Train the warm-start MLP (512 -> 256 -> 256 -> G + K + K + 1, GELU) on the GPU with the
   library's forward / backward / Adam kernels (nnc_ws_*).
3. On held-out loads, predict (x, y, lambda), solve warm-started (nnc_ipm_scopf_warm); if the
   warm solve fails or needs more iterations than the cold cap, fall back to a cold solve and
   count both.  The cold solve of the same instance is the reference it is measured against.

  python -m paper_2509_22462_gb300.warmstart_experiment --K 256 --train 512 --test 64
"""
import argparse
import copy
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def build_problem(K, G, n_bus, hidden, depth, seed, prec, n_min=20, n_max=200):
    import synth
    from paper_2509_22462_gb300 import nnc
    data = synth.scopf_data(K=K, G=G, n_bus=n_bus, seed=seed, n_min=n_min, n_max=n_max, hidden=hidden,
                            depth=depth)
    d1 = np.ones(n_bus)
    nets = []
    for k in range(K):
        m = copy.copy(data.nets[k])
        m.b = list(m.b)
        m.b[0] = synth.scopf_first_bias(data, k, d1)
        nets.append(nnc.Net.from_mlp(m, precision=prec))
    batch = nnc.Batch(nets)
    for n in nets:
        n.free()
    return data, batch


def set_loads(data, batch, d):
    import synth
    batch.set_bias(0, np.stack([synth.scopf_first_bias(data, k, d) for k in range(len(data.nets))]))
    return synth.scopf_demand(data, d)


def run(K=256, G=200, n_bus=512, hidden=1024, depth=5, n_train=512, n_test=64, epochs=300, batch_rows=64,
        lr=1e-3, seed=0, prec="bf16x3", ws_prec="bf16", h1=256, h2=256, log=print):
    import synth
    from paper_2509_22462_gb300 import nnc
    data, batch = build_problem(K, G, n_bus, hidden, depth, seed, prec,
                                n_min=min(20, G), n_max=min(200, G))
    loads = synth.load_vectors(n_train + n_test, n_bus, seed=seed, tag="warmstart-loads")
    # 1. data by cold solves
    U, T, cold = [], [], []
    t0 = time.perf_counter()
    for i in range(n_train + n_test):
        D = set_loads(data, batch, loads[i])
        res, v, lam = nnc.ipm_scopf(batch, data.G, data.subsets, data.cost, D, data.delta)
        cold.append(res)
        U.append(loads[i])
        T.append(np.concatenate([v, lam]))
    t_data = time.perf_counter() - t0
    U, T = np.array(U), np.array(T)
    ok = np.array([c["status"] == 0 for c in cold])
    tr = np.arange(n_train)[ok[:n_train]]
    te = np.arange(n_train, n_train + n_test)
    log(f"data: {len(tr)}/{n_train} training solves optimal, {t_data:.1f} s")
    # 2. training on the GPU
    params = synth.warmstart_params(n_bus, h1, h2, T.shape[1], seed=seed)
    ws = nnc.WarmStart(params, precision=ws_prec)
    t0 = time.perf_counter()
    final = ws.train(U[tr], T[tr], epochs=epochs, batch=batch_rows, lr=lr, seed=seed)
    t_train = time.perf_counter() - t0
    log(f"training: final loss {final:.3e} (standardized MSE), {t_train:.1f} s")
    # 3. held-out comparison
    P = ws.predict(U[te])
    cap = max(c["iters"] for c in cold)
    rows = []
    for j, i in enumerate(te):
        D = set_loads(data, batch, loads[i])
        v0, l0 = P[j, :G + K], P[j, G + K:]
        rw, vw, lw = nnc.ipm_scopf(batch, data.G, data.subsets, data.cost, D, data.delta, v_start=v0, lam_start=l0)
        fallback = rw["status"] != 0 or rw["iters"] > cap
        iters, secs = rw["iters"], rw["solve_seconds"]
        if fallback:
            rc, _, _ = nnc.ipm_scopf(batch, data.G, data.subsets, data.cost, D, data.delta)
            iters += rc["iters"]
            secs += rc["solve_seconds"]
        c = cold[i]
        rows.append(dict(cold_iters=c["iters"], cold_s=c["solve_seconds"], warm_iters=iters, warm_s=secs,
                         fallback=bool(fallback), obj_cold=c["obj"], obj_warm=rw["obj"],
                         same_obj=bool(abs(rw["obj"] - c["obj"]) <= 1e-6 * abs(c["obj"]))))
    ws.free()
    batch.free()
    ci = np.array([r["cold_iters"] for r in rows], float)
    wi = np.array([r["warm_iters"] for r in rows], float)
    cs = np.array([r["cold_s"] for r in rows])
    wsec = np.array([r["warm_s"] for r in rows])
    rep = {"K": K, "G": G, "hidden": hidden, "depth": depth, "n_train": int(len(tr)), "n_test": n_test,
           "epochs": epochs, "final_train_loss": final, "data_seconds": t_data, "train_seconds": t_train,
           "cold_iters_mean": float(ci.mean()), "warm_iters_mean": float(wi.mean()),
           "cold_seconds_mean": float(cs.mean()), "warm_seconds_mean": float(wsec.mean()),
           "iters_saved_frac": float(1 - wi.sum() / ci.sum()), "fallbacks": int(sum(r["fallback"] for r in rows)),
           "wins": int((wi < ci).sum()), "losses": int((wi > ci).sum()),
           "same_objective_frac": float(np.mean([r["same_obj"] for r in rows]))}
    return rep, rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--K", type=int, default=256)
    ap.add_argument("--G", type=int, default=200)
    ap.add_argument("--hidden", type=int, default=1024)
    ap.add_argument("--depth", type=int, default=5)
    ap.add_argument("--train", type=int, default=512)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    from paper_2509_22462_gb300 import build
    build.build()
    rep, rows = run(K=a.K, G=a.G, hidden=a.hidden, depth=a.depth, n_train=a.train, n_test=a.test, epochs=a.epochs)
    print(json.dumps(rep))
    if a.out:
        with open(a.out, "w") as f:
            json.dump({"report": rep, "rows": rows}, f, indent=1)


if __name__ == "__main__":
    main()
