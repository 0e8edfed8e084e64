"""Seeded synthetic workloads (parameters and random inputs) shared by tests and the bench.

This module holds no arithmetic of the method: only parameter sets of the configurations and
seeded random numbers.  The problem itself is synthetic (f = 1 on the unit square), so nothing
stands in for a dataset.

Configurations (sizes N nodes, P and L chaos terms):
  c1  n=16,  M=2, p=2 (P=6,  L=15),  sigma=0.5, ell=1,   mean-based preconditioner, rtol 1e-10
  c2  n=128, M=4, p=3 (P=35, L=210), sigma in {0.25, 0.5, 1, 1.5}, ell=0.5, field-split
      Gauss-Seidel, rtol 1e-10 (four independent systems, one per sigma); GMRES restart 300
      (sigma = 1.5 needs 979 iterations; restart 30 stagnates above 2000, 64 needs 1609; 1024
      needs 805 but its longer Arnoldi steps make the solve no faster)
  c3  n=256, M=6, p=3 (P=84, L=924), sigma=1, ell=0.5, mixed precision vs FP64, rtol 1e-8
  c4  64 systems, n in {32, 64, 128, 256}, M in {2..6}, p in {2, 3, 4}, sigma ~ U[0.1, 1.5],
      ell ~ U[0.25, 2], drawn with splitmix64 from the seed in the order (n, M, p, sigma, ell)
  c5  n=64, M=4, p=3, sigma ~ U[0.1, 1.5], ell ~ U[0.25, 2] (learned warm start)
"""

from __future__ import annotations

import numpy as np

DEFAULT_SEED = 1910115050
MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """One step of the splitmix64 generator (Steele, Lea, Flood 2014): returns (value, state)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31), state


class SplitMix:
    def __init__(self, seed: int = DEFAULT_SEED):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        v, self.state = splitmix64(self.state)
        return v

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def choice(self, seq):
        return seq[self.next_u64() % len(seq)]


def c1_params():
    return dict(n=16, M=2, p=2, sigma=0.5, ell=1.0, precond="mean", rtol=1e-10)


C2_SIGMAS = (0.25, 0.5, 1.0, 1.5)


def c2_params(sigma=None):
    sig = C2_SIGMAS if sigma is None else (sigma,)
    return [dict(n=128, M=4, p=3, sigma=s, ell=0.5, precond="fs_gs", rtol=1e-10, restart=300,
                 max_iters=4000) for s in sig]


def c3_mg_params(precision="fp64", smoother="fg"):
    """c3 with the paper's multigrid preconditioners (one pre- and one post-smoothing step, 2 x 2
    coarsest mesh, ILU(0) in the four-colour node order): by default G-M-Fg-I — the grouped
    field split with the paper's split rule, which at M = 6, p = 3 forms one split of all 84
    fields, so the smoother is the ILU(0) of each level's whole K (in the mixed form its factors
    are stored in BF16); smoother="fs_gs" gives G-M-F-I (one split per field), whose mixed form
    couples from a BF16 stiffness copy."""
    d = dict(n=256, M=6, p=3, sigma=1.0, ell=0.5, precond="mg", mg_smoother=smoother,
             rtol=1e-8, restart=50, max_iters=400, precision=precision, graphs=1,
             ilu_order="color4")
    if smoother == "fg":
        d["fg_rule"] = "paper"
        if precision == "fp32":
            d["fg_bf16"] = 1  # the block ILU(0) factors stored in BF16, applied in FP32
    if smoother == "fs_gs" and precision == "fp32":
        d["coupling_bf16"] = 1  # the smoother's Gauss-Seidel coupling from a BF16 copy
    return d


def c3_smoother_params(smoother="fg"):
    """The finest level's smoother of c3_mg_params("fp32", smoother) on its own: one application
    of the grouped field split (or of the field-split Gauss-Seidel sweep)."""
    d = dict(n=256, M=6, p=3, sigma=1.0, ell=0.5, precond=smoother, precision="fp32",
             ilu_order="color4")
    if smoother == "fg":
        d["fg_rule"] = "paper"
        d["fg_bf16"] = 1
    else:
        d["coupling_bf16"] = 1
    return d


def c3_params(precision="fp64"):
    return dict(n=256, M=6, p=3, sigma=1.0, ell=0.5, precond="mean", rtol=1e-8, restart=100,
                max_iters=6000, precision=precision)


def c4_params(nsys: int = 64, seed: int = DEFAULT_SEED, precision="fp32"):
    rng = SplitMix(seed)
    out = []
    for _ in range(nsys):
        n = rng.choice((32, 64, 128, 256))
        M = rng.choice((2, 3, 4, 5, 6))
        p = rng.choice((2, 3, 4))
        sigma = rng.uniform(0.1, 1.5)
        ell = rng.uniform(0.25, 2.0)
        out.append(dict(n=n, M=M, p=p, sigma=sigma, ell=ell, precond="mean", rtol=1e-8,
                        precision=precision))
    return out


def c5_draws(count: int, seed: int = DEFAULT_SEED + 5):
    rng = SplitMix(seed)
    return [(rng.uniform(0.1, 1.5), rng.uniform(0.25, 2.0)) for _ in range(count)]


def c5_params(sigma, ell):
    return dict(n=64, M=4, p=3, sigma=sigma, ell=ell, precond="mean", rtol=1e-8)


def random_field(N: int, P: int, seed: int = DEFAULT_SEED, scale: float = 1.0) -> np.ndarray:
    """Seeded N x P float64 test vector with independent N(0, scale^2) entries."""
    return scale * np.random.default_rng(seed).standard_normal((N, P))
