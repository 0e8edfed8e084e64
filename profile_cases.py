"""Small, self-contained cases of single kernels for profiling (e.g. under ``ncu``).

    python profile_cases.py precond [fs_gs|fs_jacobi|mean] [n]
    python profile_cases.py sweep [n] [M] [p] [fp32|fp64]   # four-colour FS-GS sweep as in c3
    python profile_cases.py vcycle [reps] [fg|fs_gs]   # the c3 mixed solve's V-cycle preconditioner
    python profile_cases.py smoother [fg|fs_gs] [n]     # the c3 smoother alone on an n x n mesh
    python profile_cases.py matvec [fp64|fp32|bf16] [n] [M] [p] [pairs|tile [kappa] [ctas]]
    python profile_cases.py gmres [n] [iters]      # Arnoldi kernels
    python profile_cases.py net [batch] [basis]    # network training step (basis 1: fixed output layer)
    python profile_cases.py stamp CLASS RATIO SUMMARY SRC...   # record a capture's DRAM ratio

``stamp`` writes profiles/traffic.json's entry for a kernel class: the measured DRAM bytes per
algorithmic byte of a captured launch, the summary that documents the capture and the SHA-256
of the kernel's source files (bench.py reports the traffic only while they are unchanged).

Each case builds one SG system, runs three applications of the chosen operation on seeded
inputs and exits 0.  Sizes stay at a few GB of device memory.
"""

from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def stamp(argv):
    import hashlib
    import json
    cls, ratio, summary, srcs = argv[2], float(argv[3]), argv[4], argv[5:]
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        rec = {}
    h = hashlib.sha256()
    for src in srcs:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    rec[cls] = {"dram_per_algorithmic_byte": ratio, "capture": summary, "sources": srcs,
                "sha256": h.hexdigest()}
    with open(path, "w") as f:
        json.dump(rec, f, indent=1, sort_keys=True)
        f.write("\n")


def main(argv):
    if len(argv) > 1 and argv[1] == "stamp":
        return stamp(argv)
    import torch

    from paper_1910_11505_gb300 import build as B
    B.build()
    from paper_1910_11505_gb300 import sg, workloads as W

    what = argv[1] if len(argv) > 1 else "precond"
    if what == "precond":
        pc = argv[2] if len(argv) > 2 else "fs_gs"
        n = int(argv[3]) if len(argv) > 3 else 128
        h = sg.sg_setup(sg.sg_default_params(n=n, M=4, p=3, sigma=0.5, ell=0.5, precond=pc))
        N, P, _ = sg.sg_dims(h)
        R = torch.from_numpy(W.random_field(N, P, seed=1)).cuda()
        Z = torch.empty_like(R)
        for _ in range(3):
            sg.sg_precond_apply(h, 0, R, Z)
    elif what == "sweep":
        # the field-split Gauss-Seidel sweep of the c3 smoother (four-colour ILU(0); the FP32
        # form couples from the BF16 stiffness copy)
        n = int(argv[2]) if len(argv) > 2 else 128
        M = int(argv[3]) if len(argv) > 3 else 6
        p = int(argv[4]) if len(argv) > 4 else 3
        prec = argv[5] if len(argv) > 5 else "fp32"
        h = sg.sg_setup(sg.sg_default_params(n=n, M=M, p=p, sigma=1.0, ell=0.5, precond="fs_gs",
                                             precision=prec, ilu_order="color4",
                                             coupling_bf16=1 if prec == "fp32" else 0))
        N, P, _ = sg.sg_dims(h)
        R = torch.from_numpy(W.random_field(N, P, seed=1)).cuda()
        if prec == "fp32":
            R = R.float()
        Z = torch.empty_like(R)
        apply = sg.sg_precond_apply_lowp if prec == "fp32" else sg.sg_precond_apply
        for _ in range(3):
            apply(h, 0, R, Z)
    elif what == "vcycle":
        # applications of the c3 multigrid preconditioner as the mixed solver's inner FGMRES
        # runs it (FP32, G-M-F-I with four-colour ILU(0) and BF16 coupling); prints the library's
        # launch count after setup and after each application (for a profiler's -s / -c)
        reps = int(argv[2]) if len(argv) > 2 else 2
        smoother = argv[3] if len(argv) > 3 else "fg"
        h = sg.sg_setup(sg.sg_default_params(**W.c3_mg_params("fp32", smoother)))
        N, P, _ = sg.sg_dims(h)
        R = torch.from_numpy(W.random_field(N, P, seed=1)).float().cuda()
        Z = torch.empty_like(R)
        torch.cuda.synchronize()
        print("launches after setup", sg.sg_launch_count(), flush=True)
        for _ in range(reps):
            sg.sg_precond_apply_lowp(h, 0, R, Z)
            torch.cuda.synchronize()
            print("launches", sg.sg_launch_count(), flush=True)
    elif what == "smoother":
        # three applications of the c3 smoother (FP32) alone on an n x n mesh
        smoother = argv[2] if len(argv) > 2 else "fg"
        n = int(argv[3]) if len(argv) > 3 else 128
        h = sg.sg_setup(sg.sg_default_params(**dict(W.c3_smoother_params(smoother), n=n)))
        N, P, _ = sg.sg_dims(h)
        R = torch.from_numpy(W.random_field(N, P, seed=1)).float().cuda()
        Z = torch.empty_like(R)
        for _ in range(3):
            sg.sg_precond_apply_lowp(h, 0, R, Z)
    elif what == "matvec":
        prec = argv[2] if len(argv) > 2 else "fp64"
        n = int(argv[3]) if len(argv) > 3 else 128
        M = int(argv[4]) if len(argv) > 4 else 6
        p = int(argv[5]) if len(argv) > 5 else 3
        op = {}
        if len(argv) > 6:  # operator kernel: pairs | tile [kappa] [ctas]
            op["op_kernel"] = argv[6]
            if len(argv) > 7:
                op["op_kappa"] = int(argv[7])
            if len(argv) > 8:
                op["op_ctas"] = int(argv[8])
        h = sg.sg_setup(sg.sg_default_params(n=n, M=M, p=p, sigma=1.0, ell=0.5, precond="none",
                                             precision=prec, **op))
        N, P, _ = sg.sg_dims(h)
        X = torch.from_numpy(W.random_field(N, P, seed=2)).cuda()
        if prec == "fp64":
            Y = torch.empty_like(X)
            for _ in range(3):
                sg.sg_matvec(h, 0, X, Y)
        else:
            X32 = X.float()
            Y32 = torch.empty_like(X32)
            for _ in range(3):
                sg.sg_matvec_lowp(h, 0, X32, Y32)
    elif what == "gmres":
        n = int(argv[2]) if len(argv) > 2 else 128
        iters = int(argv[3]) if len(argv) > 3 else 40
        h = sg.sg_setup(sg.sg_default_params(n=n, M=4, p=3, sigma=0.5, ell=0.5, precond="mean",
                                             restart=64, max_iters=iters))
        N, P, _ = sg.sg_dims(h)
        F = torch.empty(N, P, dtype=torch.float64, device="cuda")
        sg.sg_rhs(h, 0, F)
        X = torch.zeros_like(F)
        sg.sg_gmres_solve(h, [F], [X], raise_on_error=False)
    elif what == "net":
        B = int(argv[2]) if len(argv) > 2 else 256
        basis = int(argv[3]) if len(argv) > 3 else 1
        D = 4225 * 35
        net = sg.SGNet(6, 64, 64, D, max_batch=B, bf16=True, seed=1)
        Z = torch.from_numpy(W.random_field(B, 6, seed=3)).float().cuda()
        T = 0.01 * torch.from_numpy(W.random_field(B, D, seed=4)).float().cuda()
        net.set_stats(Z, T)
        if basis:  # the c5 network: fixed output layer (the tensor-core residual epilogue)
            net.set_basis(T)
        for _ in range(3):
            net.train_step(Z, T, 1e-3)
        torch.cuda.synchronize()
        net.close()
        print("ok", what)
        return 0
    else:
        raise SystemExit(f"unknown case {what}")
    torch.cuda.synchronize()
    h.close()
    print("ok", what)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
