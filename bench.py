"""Benchmark of the SG-GMRES hot path on GB300.

Workload (one step): solve the four field-split Gauss-Seidel SG systems of the 128 x 128 Q1 mesh,
M = 4 KL terms, p = 3 (P = 35, L = 210), ell = 0.5, sigma in {0.25, 0.5, 1.0, 1.5}, FP64,
relative residual 1e-10, from a zero initial guess.  value = solved systems per second over all
ranks (each rank solves its own copy of the four systems: weak scaling, no collective on the
data path).

Also reported: the roofline of the dominant kernel (live CUDA-event timing inside the library on
the stream each kernel is launched on), the SG operator's own throughput, the end-to-end rate
through the C ABI with host buffers, SM clocks sampled during the timed region, and the FP64
CPU oracle timed on the host cores on a bounded sample (``cpu_baseline``).

``--impl reference`` times the oracle alone (the CPU reference of this project) on a bounded
sample of the same workload and prints the same JSON line with "impl": "reference".
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SG solves/sec & matvec HBM GB/s, mixed/learned vs FP64 GMRES at 1e-8 residual"
WORKLOAD = ("c2: 128x128 Q1 mesh, M=4, p=3 (P=35, L=210), ell=0.5, sigma in {0.25,0.5,1.0,1.5}, "
            "FP64 GMRES(300) with field-split Gauss-Seidel + ILU(0), rel. residual 1e-10, x0 = 0")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
DFMA_PEAK_GFLOPS = 1192.0   # measured FP64 FMA loop on GB300 (2 DFMA per clock per SM, 2 flops each)
ITERS_FILE = os.path.join(ROOT, "oracle", "c2_iterations.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SOURCES = {"ilu_solve": "paper_1910_11505_gb300/csrc/k_precond.cu",
                  "apply_f64": "paper_1910_11505_gb300/csrc/k_matvec.cu"}


def measured_traffic(kernel):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, or None when the
    kernel's source has changed since the counters were taken."""
    import hashlib
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        return rec["bytes_per_launch"] if sha == rec["sha256"] else None
    except Exception:
        return None


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle (CPU) timing

def cpu_oracle_sample(iters_cap: int, sigma: float):
    """Time the FP64 oracle's GMRES on one c2 system for ``iters_cap`` iterations (setup excluded);
    runs in a fresh single-threaded process.  Returns seconds per GMRES iteration."""
    code = (
        "import os,sys,time,json\n"
        f"sys.path.insert(0,{ROOT!r})\n"
        "import numpy as np\n"
        "import oracle as O\n"
        f"prob=O.build_problem(128,4,3,sigma={sigma},ell=0.5)\n"
        "blocks=O.fs_blocks(prob)\n"
        "N,P=prob.N,prob.P\n"
        "K=lambda v:O.sg_matvec(prob,v.reshape(N,P)).ravel()\n"
        "M=lambda v:O.fs_precond(prob,v.reshape(N,P),blocks=blocks).ravel()\n"
        "t=time.perf_counter()\n"
        f"x,info=O.gmres(K,M,prob.F.ravel(),rtol=1e-10,restart=300,max_iters={iters_cap})\n"
        "dt=time.perf_counter()-t\n"
        "print(json.dumps({'seconds':dt,'iters':info['iters']}))\n")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["seconds"] / max(1, d["iters"]), d


C2_RESTART = 300


def oracle_iterations():
    """GMRES iteration counts of the oracle on the four c2 systems (written by
    oracle/c2_iterations.py) for the restart length the bench uses, or None."""
    try:
        with open(ITERS_FILE) as f:
            d = json.load(f)
        return d if d.get("restart") == C2_RESTART else None
    except Exception:
        return None


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1910_11505_gb300 import workloads as W
    its = oracle_iterations()
    cap = 2
    per_solve = []
    for k in range(args.warmup + args.steps):
        sig = W.C2_SIGMAS[k % 4]
        t_it, d = cpu_oracle_sample(cap, sig)
        if k >= args.warmup:
            n_it = its["iters"][str(sig)] if its else None
            per_solve.append(t_it * (n_it if n_it else 1))
    total = sum(per_solve)
    value = len(per_solve) / total
    unit = "solves/s" if its else "GMRES iterations/s"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / len(per_solve), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                             "sample": f"{cap} GMRES iterations of one c2 system per step (setup "
                                       "excluded), scaled by the oracle's own iteration count to "
                                       "a full solve"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- multi-rank aggregation

def aggregate_ranks(ms_local: float, systems_local: int, device="cpu"):
    """Whole-job figures over the ranks of the default process group (if any): the slowest
    rank's time and the systems solved by all ranks.  Only these two numbers cross ranks; the
    data path has no collective (every rank solves its own systems)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local, systems_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    n = torch.tensor([systems_local], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


# ---------------------------------------------------------------- GPU arm

def algorithmic_bytes_apply(nnzA, N, P, L, s):
    return nnzA * L * s + 4 * nnzA + 4 * (N + 1) + 2 * N * P * s


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--timing-stride", type=int, default=4)
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    # the CPU oracle sample runs in a child process started before any GPU work
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu_t_iter, cpu_info = cpu_oracle_sample(3, 0.5)
        cpu = (cpu_t_iter, cpu_info)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_11505_gb300 import sg, workloads as W

    stream = torch.cuda.current_stream()
    params = [sg.sg_default_params(**d) for d in W.c2_params()]
    h = sg.sg_setup(params, stream)
    ns = h.nsys
    Fs, Xs = [], []
    for i in range(ns):
        N, P, L = sg.sg_dims(h, i)
        F = torch.empty(N, P, dtype=torch.float64, device="cuda")
        sg.sg_rhs(h, i, F, stream)
        Fs.append(F)
        Xs.append(torch.zeros_like(F))
    nnzA, nnzG = sg.sg_nnz(h, 0)

    def step():
        for X in Xs:
            X.zero_()
        return sg.sg_gmres_solve(h, Fs, Xs, stream)

    for _ in range(args.warmup):
        rc, info = step()
        assert rc == sg.SG_OK, info

    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    sg.sg_timing_start(h, args.timing_stride)
    l0 = sg.sg_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        rc, info = step()
        assert rc == sg.SG_OK, info
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = sg.sg_launch_count() - l0
    ktimes = sg.sg_timing_stop(h)
    clk = clocks.stop()
    ms, systems = aggregate_ranks(ms, ns * args.steps, device="cuda")
    if world > 1:
        dist.barrier()
    value = systems / (ms / 1000.0)

    # dominant kernel class by estimated total time
    est = {c: (v[0] / v[1] * v[2] if v[1] else 0.0) for c, v in ktimes.items()}
    dom = max(est, key=est.get)
    d_ms, d_timed, d_launch = ktimes[dom]
    d_avg_s = d_ms / max(1, d_timed) / 1000.0
    hbm, peak_kind = _peaks()
    N, P, L = sg.sg_dims(h, 0)
    if dom == "ilu_solve":
        # one block solve: 9 factor values per row (lower 4, upper 4, 1/u_ii), the right-hand
        # side column and z, and the level table
        m = int(round(N ** 0.5))
        alg_bytes = 9 * N * 8 + 2 * N * 8 + 4 * (3 * m - 1)
    elif dom == "apply_f64":
        alg_bytes = algorithmic_bytes_apply(nnzA, N, P, L, 8)
    else:
        alg_bytes = None
    roof = {"kernel": dom, "bound": "hbm",
            "achieved": (alg_bytes / d_avg_s / 1e9) if alg_bytes else None,
            "peak": hbm, "unit": "GB/s", "peak_kind": peak_kind,
            "frac": (alg_bytes / d_avg_s / 1e9 / hbm) if alg_bytes else None,
            "traffic": measured_traffic(dom), "avg_launch_us": d_avg_s * 1e6,
            "launches_timed": d_timed, "share_of_timed_gpu_time": est[dom] / max(1e-30, sum(est.values()))}
    if dom == "ilu_solve":
        # the block solve is bound by its dependency chain: two sweeps of 3m - 8 interior
        # wavefront levels, one barrier step each plus two, and per step two dependent FP64 FMAs
        # (64 cycles each on this GPU), a shared-memory load and store (~50 cycles) and the
        # barrier (~50 cycles): an estimated floor of ~230 cycles per step at 2.07 GHz
        m = int(round(N ** 0.5))
        steps = 2 * (3 * m - 8) + 4
        roof["critical_path_steps"] = steps
        roof["ns_per_step"] = d_avg_s * 1e9 / steps
        roof["ns_per_step_floor_est"] = (2 * 64 + 50 + 50) / 2.07

    # the SG operator alone (K1): FP64 DFMA-bound, reported against the DFMA peak as well
    X = torch.from_numpy(W.random_field(N, P, seed=7)).cuda()
    Y = torch.empty_like(X)
    for _ in range(3):
        sg.sg_matvec(h, 1, X, Y, stream)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    ea.record(stream)
    for _ in range(reps):
        sg.sg_matvec(h, 1, X, Y, stream)
    eb.record(stream)
    torch.cuda.synchronize()
    mv_s = ea.elapsed_time(eb) / 1000.0 / reps
    ops = sg.sg_launch_count()  # noqa: F841
    # flops: 9 U + nnz_G FMAs per interior row (U = (k, b) pairs), 2 flops each
    trip = sg.sg_export(h, 1, 5).reshape(-1, 4)
    U = len({(int(k), int(b)) for k, _, b in trip[:, :3]})
    flops = 2.0 * N * (9 * U + nnzG)
    matvec = {"ms": mv_s * 1e3,
              "gbs": algorithmic_bytes_apply(nnzA, N, P, L, 8) / mv_s / 1e9,
              "hbm_frac": algorithmic_bytes_apply(nnzA, N, P, L, 8) / mv_s / 1e9 / hbm,
              "gflops": flops / mv_s / 1e9, "bound": "alu",
              "dfma_peak_gflops": DFMA_PEAK_GFLOPS, "alu_frac": flops / mv_s / 1e9 / DFMA_PEAK_GFLOPS}

    # end to end through the C ABI with pinned host buffers
    Fh = [F.cpu().pin_memory() for F in Fs]
    Xh = [torch.empty_like(F).pin_memory() for F in Fh]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    ea.record(stream)
    for _ in range(e2e_steps):
        for i in range(ns):
            Fs[i].copy_(Fh[i], non_blocking=True)
            Xs[i].zero_()
        rc, _ = sg.sg_gmres_solve(h, Fs, Xs, stream)
        for i in range(ns):
            Xh[i].copy_(Xs[i], non_blocking=True)
    eb.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ea.elapsed_time(eb) / e2e_steps
    bytes_np = sum(F.numel() * 8 for F in Fh)
    e2e = {"value": ns * world / (e2e_ms / 1000.0), "unit": "solves/s",
           "h2d_bytes_per_step": bytes_np, "d2h_bytes_per_step": bytes_np}

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "systems_per_step_per_gpu": ns,
                       "l2": "inputs larger than L2 (four 249 MB FP64 stiffness stacks)",
                       "iters": [i["iters"] for i in infos[-1]],
                       "rel_resid": [i["rel_resid"] for i in infos[-1]]},
            "roofline": roof, "matvec": matvec, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk,
            "kernel_ms": {c: {"timed_ms": v[0], "timed": v[1], "launches": v[2]}
                          for c, v in ktimes.items()}}
    if cpu is not None:
        t_it, info = cpu
        its = oracle_iterations()
        n_it = its["iters"]["0.5"] if its else infos[-1][1]["iters"]
        src = "the oracle's own count" if its else "the GPU path's count (same algorithm)"
        line["cpu_baseline"] = {
            "value": 1.0 / (t_it * n_it), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{info['iters']} FP64 GMRES iterations of the sigma=0.5 c2 system in "
                      f"{info['seconds']:.1f} s (setup excluded), scaled to {n_it} iterations "
                      f"per solve ({src})"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
