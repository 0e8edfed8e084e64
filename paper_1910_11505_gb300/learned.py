"""Learned warm start: data generation with the SG solver, training and evaluation loops.

The network and its training run in ``libsg_gb300.so`` (include/sgnet.h); this module only sets
up systems, moves device pointers and loops.  Features of a system: (sigma, ell,
sqrt(lambda_1..M)) with lambda the KL eigenvalues the library computed for it.
"""

from __future__ import annotations

import math
import time

import numpy as np

from . import sg


def features(h: sg.SGHandle, sys: int):
    prm = h.params[sys]
    lam = sg.sg_export(h, sys, 3)
    return [prm.sigma, prm.ell] + [math.sqrt(max(l, 0.0)) for l in lam]


def generate(param_dicts, chunk: int = 32, precision: str = "fp32", rtol: float = 1e-6,
             restart: int = 100, max_iters: int = 4000, graphs: int = 1):
    """Solve every system (x0 = 0) and return (Z, T, stats): Z n x in float32 features, T n x D
    float32 solutions (device tensors), stats of the solves."""
    import torch
    Zs, Ts, iters = [], [], []
    t0 = time.time()
    for c0 in range(0, len(param_dicts), chunk):
        part = [dict(d, precision=precision, rtol=rtol, restart=restart, max_iters=max_iters,
                     graphs=graphs) for d in param_dicts[c0:c0 + chunk]]
        h = sg.sg_setup([sg.sg_default_params(**d) for d in part])
        Fs, Xs = [], []
        for i in range(h.nsys):
            N, P, _ = sg.sg_dims(h, i)
            F = torch.empty(N, P, dtype=torch.float64, device="cuda")
            sg.sg_rhs(h, i, F)
            Fs.append(F)
            Xs.append(torch.zeros_like(F))
        rc, info = sg.sg_gmres_solve(h, Fs, Xs)
        for i in range(h.nsys):
            Zs.append(features(h, i))
            Ts.append(Xs[i].reshape(-1).float())
            iters.append(info[i]["iters"])
        h.close()
    Z = torch.tensor(np.array(Zs, dtype=np.float32), device="cuda")
    T = torch.stack(Ts).contiguous()
    return Z, T, {"seconds": time.time() - t0, "mean_iters": float(np.mean(iters))}


def train(net: sg.SGNet, Z, T, steps: int, batch: int, lr: float, seed: int = 7,
          log_every: int = 0):
    """Adam on contiguous mini-batches visited in a seeded random order (the rows themselves are
    already in random draw order).  Returns the list of sampled losses."""
    n = Z.shape[0]
    nb = max(1, n // batch)
    rng = np.random.default_rng(seed)
    order = []
    losses = []
    for s in range(steps):
        if not order:
            order = list(rng.permutation(nb))
        k = order.pop()
        z = Z[k * batch:(k + 1) * batch]
        t = T[k * batch:(k + 1) * batch]
        want = log_every and (s % log_every == 0 or s == steps - 1)
        loss = net.train_step(z, t, lr, want_loss=bool(want))
        if want:
            losses.append((s, loss))
    return losses


def warm_start_eval(net: sg.SGNet, param_dicts, precision: str = "fp64", rtol: float = 1e-8,
                    restart: int = 100, max_iters: int = 4000, graphs: int = 1):
    """Solve each system from x0 = 0 and from the network's prediction; returns per-system
    iterations, residuals and the two wall times.  Both timed solves use the same F and X
    buffers after one untimed solve, so captured cycle graphs serve both alike."""
    import torch
    part = [dict(d, precision=precision, rtol=rtol, restart=restart, max_iters=max_iters,
                 graphs=graphs) for d in param_dicts]
    h = sg.sg_setup([sg.sg_default_params(**d) for d in part])
    Fs, Xs, feats = [], [], []
    for i in range(h.nsys):
        N, P, _ = sg.sg_dims(h, i)
        F = torch.empty(N, P, dtype=torch.float64, device="cuda")
        sg.sg_rhs(h, i, F)
        Fs.append(F)
        Xs.append(torch.zeros_like(F))
        feats.append(features(h, i))
    Z = torch.tensor(np.array(feats, dtype=np.float32), device="cuda")
    sg.sg_gmres_solve(h, Fs, Xs)  # untimed: captures the cycle graphs
    for x in Xs:
        x.zero_()
    torch.cuda.synchronize()
    t0 = time.time()
    rc0, info0 = sg.sg_gmres_solve(h, Fs, Xs)
    t_zero = time.time() - t0
    torch.cuda.synchronize()
    t0 = time.time()
    for i in range(h.nsys):
        net.predict(Z[i:i + 1], Xs[i].view(1, -1))
    rcw, infow = sg.sg_gmres_solve(h, Fs, Xs)
    t_warm = time.time() - t0
    h.close()
    return {"zero_iters": [d["iters"] for d in info0], "warm_iters": [d["iters"] for d in infow],
            "zero_resid": [d["rel_resid"] for d in info0],
            "warm_resid": [d["rel_resid"] for d in infow],
            "zero_seconds": t_zero, "warm_seconds": t_warm, "rc": (rc0, rcw)}
