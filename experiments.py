"""Measurement runs of the configurations other than the default bench workload.

    python experiments.py c3            # FP64 vs mixed FP32 / BF16 solves
    python experiments.py c5 [ntrain] [ntest] [steps] [mg]   # learned warm start
    python experiments.py c4 [nsys] [batch] [solo]   # uneven systems (64, in batches of 16)

Each prints one JSON line.  Times are wall-clock around the C-ABI solve calls (the calls
synchronise), with setup excluded and reported separately.
"""

from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _solve_one(sg, torch, d):
    t0 = time.time()
    h = sg.sg_setup(sg.sg_default_params(**d))
    torch.cuda.synchronize()
    setup = time.time() - t0
    N, P, _ = sg.sg_dims(h)
    F = torch.empty(N, P, dtype=torch.float64, device="cuda")
    sg.sg_rhs(h, 0, F)
    X = torch.zeros_like(F)
    torch.cuda.synchronize()
    t0 = time.time()
    rc, info = sg.sg_gmres_solve(h, [F], [X], raise_on_error=False)
    secs = time.time() - t0
    return h, F, X, rc, info[0], secs, setup


def run_c3():
    import torch
    from paper_1910_11505_gb300 import sg, workloads as W
    out = {"config": "c3: 256x256 Q1, M=6, p=3 (P=84, L=924), sigma=1, ell=0.5, mean-based ILU(0), "
                     "GMRES(100), relative residual 1e-8"}
    ref = None
    for prec in ("fp64", "fp32", "bf16"):
        d = W.c3_params(prec)
        if prec == "bf16":
            d["max_iters"] = 600
        h, F, X, rc, info, secs, setup = _solve_one(sg, torch, d)
        rec = {"rc": rc, "iters": info["iters"], "refinements": info["restarts"],
               "rel_resid": info["rel_resid"], "solve_s": secs, "setup_s": setup,
               "solves_per_s": (1.0 / secs) if rc == 0 else 0.0}
        if prec == "fp64":
            ref = X.clone()
        elif rc == 0:
            rec["rel_err_vs_fp64"] = float((X - ref).norm() / ref.norm())
        out[prec] = rec
        h.close()
        del F, X
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def run_c5(ntrain=4096, ntest=256, steps=3000, mg=1):
    """Learned warm start at c5; ``mg`` = 1 solves with the paper's multigrid preconditioner
    (G-M-Fg-I), 0 with the mean-based ILU(0)."""
    import numpy as np
    import torch
    from paper_1910_11505_gb300 import learned, sg, workloads as W
    draws = W.c5_draws(ntrain + ntest)
    base = dict(n=64, M=4, p=3, precond="mean")
    if mg:
        base.update(precond="mg", mg_smoother="fg", fg_rule="paper", ilu_order="color4")
    tr = [dict(base, sigma=s, ell=l) for s, l in draws[:ntrain]]
    te = [dict(base, sigma=s, ell=l) for s, l in draws[ntrain:]]
    Z, T, gen = learned.generate(tr, chunk=64, precision="fp32", rtol=1e-6)
    net = sg.SGNet(Z.shape[1], 64, 64, T.shape[1], max_batch=256, bf16=True, seed=1910)
    net.set_stats(Z, T)
    net.set_basis(T)
    torch.cuda.synchronize()
    t0 = time.time()
    losses = learned.train(net, Z, T, steps=steps, batch=256, lr=1e-3, log_every=max(1, steps // 10))
    torch.cuda.synchronize()
    train_s = time.time() - t0
    res = {}
    for prec in ("fp64", "fp32"):
        zi, wi, zs, ws, zr, wr = [], [], 0.0, 0.0, [], []
        for c0 in range(0, len(te), 64):
            ev = learned.warm_start_eval(net, te[c0:c0 + 64], precision=prec, rtol=1e-8)
            zi += ev["zero_iters"]
            wi += ev["warm_iters"]
            zr += ev["zero_resid"]
            wr += ev["warm_resid"]
            zs += ev["zero_seconds"]
            ws += ev["warm_seconds"]
        res[prec] = {"zero_mean_iters": float(np.mean(zi)), "warm_mean_iters": float(np.mean(wi)),
                     "zero_solves_per_s": len(te) / zs, "warm_solves_per_s": len(te) / ws,
                     "max_zero_resid": max(zr), "max_warm_resid": max(wr)}
    print(json.dumps({"config": "c5: 64x64 Q1, M=4, p=3 (D=4225x35), sigma~U[0.1,1.5], "
                                "ell~U[0.25,2]; MLP 6-64-64-D (tanh), BF16 output layer, Adam; "
                                + ("G-M-Fg-I" if mg else "mean-based ILU(0)"),
                      "ntrain": ntrain, "ntest": ntest, "steps": steps,
                      "generation": gen, "train_seconds": train_s, "losses": losses,
                      "eval": res}), flush=True)
    net.close()


def _c4_case(sg, d):
    fits = max(f1 - f0 for f0, f1 in sg.sg_fg_splits(d["M"], d["p"], "paper")) <= 96
    d.update(precond="mg", mg_smoother="fg" if fits else "fs_gs", ilu_order="color4",
             restart=30, graphs=1, max_iters=3000)
    return d


def _c4_solve(sg, torch, ps):
    """Set up the systems ps in one handle and solve them together; returns (setup s, solve s,
    per-system info)."""
    t0 = time.time()
    h = sg.sg_setup([sg.sg_default_params(**d) for d in ps])
    torch.cuda.synchronize()
    setup = time.time() - t0
    Fs, Xs = [], []
    for i in range(h.nsys):
        N, P, _ = sg.sg_dims(h, i)
        F = torch.empty(N, P, dtype=torch.float64, device="cuda")
        sg.sg_rhs(h, i, F)
        Fs.append(F)
        Xs.append(torch.zeros_like(F))
    torch.cuda.synchronize()
    t0 = time.time()
    rc, info = sg.sg_gmres_solve(h, Fs, Xs, raise_on_error=False)
    torch.cuda.synchronize()
    secs = time.time() - t0
    h.close()
    del Fs, Xs
    torch.cuda.empty_cache()
    return setup, secs, info


def run_c4(nsys=64, batch=16, solo=1):
    """The first ``nsys`` seeded c4 systems, each with the paper's multigrid preconditioner:
    G-M-Fg-I where every split of the paper's rule has at most 96 fields, else G-M-F-I (FP32
    inner solves, the four-colour ILU(0) ordering).  They are solved ``batch`` at a time in one
    handle (one stream per system, GMRES cycles replayed from captured graphs; the batch size
    bounds device memory), and with ``solo`` each system also alone, for the batch's gain."""
    import torch
    from paper_1910_11505_gb300 import sg, workloads as W
    ps = [_c4_case(sg, d) for d in W.c4_params(nsys)]
    setup = secs = 0.0
    info = []
    for b0 in range(0, nsys, batch):
        su, se, inf = _c4_solve(sg, torch, ps[b0:b0 + batch])
        setup += su
        secs += se
        info += inf
    ok = sum(1 for i in info if i["status"] == 0)
    out = {"config": f"c4: {nsys} seeded systems in batches of {batch}, mixed FP32, G-M-Fg-I "
                     "(G-M-F-I where a split exceeds 96 fields), GMRES(30), 1e-8, each cycle a "
                     "captured CUDA graph",
           "smoothers": [d["mg_smoother"] for d in ps],
           "sizes": [[d["n"], d["M"], d["p"]] for d in ps],
           "setup_s": setup, "solve_s": secs, "converged": ok, "solves_per_s": ok / secs,
           "iters": [i["iters"] for i in info],
           "max_rel_resid": max(i["rel_resid"] for i in info)}
    if solo:
        alone = [_c4_solve(sg, torch, [d])[1] for d in ps]
        out["solo_solve_s"] = sum(alone)
        out["solo_solves_per_s"] = nsys / sum(alone)
        out["batch_over_solo"] = sum(alone) / secs
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    from paper_1910_11505_gb300 import build as B
    B.build()
    what = sys.argv[1] if len(sys.argv) > 1 else "c3"
    args = [int(a) for a in sys.argv[2:]]
    {"c3": run_c3, "c5": run_c5, "c4": run_c4}[what](*args)
