"""Pins of the oracle's grouped field split and multi-field ILU(0) (readings R20, R21): the
paper's worked grouping example, the defining property of ILU(0) (L U equals the matrix on its
pattern), and reductions to the already pinned single-field ILU(0) and field-split routines."""

import os

import numpy as np
import pytest

from oracle import sg_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_splits():
    rows = []
    with open(os.path.join(GOLDEN, "fg_splits_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                _, groups, count = line.split()
                rows.append(([int(g) for g in groups.split(",")], int(count)))
    return rows


def test_fg_splits_paper_example():
    Jp = O.multi_indices(2, 4)
    splits = O.fg_splits(Jp, "paper")
    gold = _golden_splits()
    assert [f1 - f0 for f0, f1 in splits] == [c for _, c in gold]
    for (f0, f1), (groups, _) in zip(splits, gold):
        assert sorted(set(Jp[f0:f1, 0].tolist())) == groups


def test_fg_splits_rules():
    Jp = O.multi_indices(6, 3)                      # c3: only Group0 holds an all-equal index
    assert O.fg_splits(Jp, "paper") == [(0, 84)]
    assert O.fg_splits(Jp, "groups") == [(0, 56), (56, 77), (77, 83), (83, 84)]
    assert O.fg_splits(Jp, "whole") == [(0, 84)]
    assert O.fg_splits(Jp, "fields")[:2] == [(0, 1), (1, 2)]
    Jp = O.multi_indices(2, 2)                      # (0,0), (1,1) open splits; Group2 joins
    assert O.fg_splits(Jp, "paper") == [(0, 3), (3, 6)]


def _lu_dense(LU):
    Lo, Up, order = LU
    return (Lo @ Up).toarray(), order


@pytest.mark.parametrize("ordering", ["color4", "natural"])
def test_bilu0_matches_the_block_on_its_pattern(ordering):
    prob = O.build_problem(4, 2, 1, sigma=0.8, ell=0.6)
    for f0, f1 in [(0, 3), (1, 3)]:
        A = O.block_pattern_matrix(prob, f0, f1)
        LU = O.bilu0(prob, f0, f1, ordering)
        prod, order = _lu_dense(LU)
        Ap = A[order][:, order].toarray()
        stored = A[order][:, order].tocoo()       # every position of the pattern, zeros kept
        err = abs(prod[stored.row, stored.col] - stored.data).max()
        assert err <= 1e-12 * abs(Ap).max()
        # and the factorisation is not the exact LU (fill outside the pattern was dropped)
        assert abs(prod - Ap).max() > 1e-8 * abs(Ap).max()


def test_block_pattern_matrix_is_K_in_node_major_order():
    prob = O.build_problem(4, 2, 2, sigma=0.7, ell=0.5)
    A = O.block_pattern_matrix(prob, 0, prob.P).toarray()
    K = sum(np.kron(prob.G[k], prob.A[k].toarray()) for k in range(prob.L))  # field-major
    N, P = prob.N, prob.P
    perm = (np.arange(N)[:, None] + N * np.arange(P)[None, :]).ravel()   # node-major -> field-major
    assert np.allclose(A, K[np.ix_(perm, perm)], rtol=0, atol=1e-14 * abs(K).max())


def test_single_field_splits_equal_the_field_split():
    prob = O.build_problem(6, 2, 2, sigma=0.6, ell=0.7)
    R = np.random.default_rng(3).standard_normal((prob.N, prob.P))
    splits = O.fg_splits(prob.Jp, "fields")
    Z = O.fg_precond(prob, R, splits, O.fg_blocks(prob, splits, "color4"))
    ref = O.fs_precond(prob, R, mode="gs", blocks=O.fs_blocks(prob, ordering="color4"))
    assert np.abs(Z - ref).max() <= 1e-12 * np.abs(ref).max()


def test_whole_split_solves_exactly_without_dropped_fill():
    # a 2 x 2-cell mesh: one interior node; every other row is a Dirichlet identity row, so no
    # fill is dropped and ILU(0) of K is its exact LU
    prob = O.build_problem(2, 2, 1, sigma=0.9, ell=0.5)
    R = np.random.default_rng(4).standard_normal((prob.N, prob.P))
    Z = O.fg_precond(prob, R, [(0, prob.P)])
    K = sum(np.kron(prob.G[k], prob.A[k].toarray()) for k in range(prob.L))
    ref = np.linalg.solve(K, R.T.ravel()).reshape(prob.P, prob.N).T
    assert np.abs(Z - ref).max() <= 1e-12 * np.abs(ref).max()


def test_gmres_with_whole_K_ilu_converges_faster_than_field_split():
    prob = O.build_problem(8, 2, 2, sigma=1.0, ell=0.5)
    F = prob.F
    K = lambda x: O.sg_matvec(prob, x.reshape(prob.N, prob.P)).ravel()
    whole = O.fg_blocks(prob, [(0, prob.P)])
    fsb = O.fs_blocks(prob, ordering="color4")
    _, i1 = O.gmres(K, lambda v: O.fg_precond(prob, v.reshape(prob.N, prob.P), [(0, prob.P)],
                                              whole).ravel(), F.ravel(), restart=50, rtol=1e-10)
    _, i2 = O.gmres(K, lambda v: O.fs_precond(prob, v.reshape(prob.N, prob.P),
                                              blocks=fsb).ravel(), F.ravel(), restart=50, rtol=1e-10)
    assert i1["converged"] and i2["converged"]
    assert i1["iters"] < i2["iters"]
