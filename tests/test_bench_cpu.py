"""The byte and cost models behind bench.py's roofline and CPU-baseline estimate, on the CPU:
the c3 operator bytes (the table of algorithmic work per application), the smoother's bytes per
colour-phase launch, the multigrid level list and the oracle solve estimate's level sum."""

import math

import bench


def test_operator_bytes_match_the_c3_table():
    # c3: n = 256 (N = 66 049), nnz_A = (3m - 2)^2 = 591 361, P = 84, L = 924
    N, nnzA, P, L = 257 * 257, (3 * 257 - 2) ** 2, 84, 924
    assert nnzA == 591361
    b64 = bench.algorithmic_bytes_apply(nnzA, N, P, L, 8)
    b32 = bench.algorithmic_bytes_apply(nnzA, N, P, L, 4)
    assert b32 == 2232684828          # the figure the bench's roofline divides by
    assert round(b64 / 1e6) == 4463   # ~4 462 MB: the stack twice as wide
    # the stack dominates: X and Y together are 2 N P s
    assert b32 - nnzA * L * 4 == 4 * nnzA + 4 * (N + 1) + 2 * N * P * 4


def test_smoothing_levels_are_the_hierarchy_above_the_coarsest_mesh():
    lv = bench.smoothing_levels(256, 2)
    assert [N for N, _ in lv] == [(n + 1) ** 2 for n in (256, 128, 64, 32, 16, 8, 4)]
    assert all(nnz == (3 * math.isqrt(N) - 2) ** 2 for N, nnz in lv)


def test_grouped_split_bytes_per_phase_launch():
    # one split of all P fields: every node's 9 blocks of P x P factor values (sf bytes) once per
    # application of 8 colour phases, plus the right-hand side read and the result written
    N, P = 257 * 257, 84
    per_launch = bench.fg_solve_bytes([(N, 0)], P, 4, 2)
    assert per_launch == N * (9 * P * P * 2 + 2 * P * 4) / 8
    two = bench.fg_solve_bytes([(N, 0), (129 * 129, 0)], P, 4, 2)
    assert two == (N + 129 * 129) * (9 * P * P * 2 + 2 * P * 4) / 16


def test_oracle_solve_estimate_sums_the_levels():
    # unit costs: per level two smoother applications (per node) and two residual operators
    # (three on the finest level, which adds the outer operator), times the iterations
    sample = {"bilu_solve_s_per_node": 1.0, "row_s_single": 10.0, "row_s_allcores": 1.0}
    one, allc = bench.oracle_solve_estimate(sample, 1, n=8, coarse=2)
    Ns = [(8 + 1) ** 2, (4 + 1) ** 2]
    assert one == 2 * sum(Ns) + 10.0 * (3 * Ns[0] + 2 * Ns[1])
    assert allc == 2 * sum(Ns) + 1.0 * (3 * Ns[0] + 2 * Ns[1])
    seven, _ = bench.oracle_solve_estimate(sample, 7, n=8, coarse=2)
    assert seven == 7 * one
