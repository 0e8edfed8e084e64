"""The grouped field split (Sec. 3, Eq. P_group) and the ILU(0) of multi-field blocks of K
(readings R20, R21) through the C ABI against the oracle: G-I (one split of all fields), the
paper's split rule and one split per group, alone and as the multigrid smoother (G-M-I,
G-M-Fg-I), and GMRES with them against the direct solution.

Tolerances: 1e-12 relative per FP64 application (the block factorisation takes the diagonal
blocks' exact inverses with partial pivoting where the oracle eliminates without pivoting: the
same factors up to rounding, amplified by at most the blocks' condition numbers, ~1e2 here);
FP32 applications against the FP64 oracle at 1e-5, scaled by Q / 8 for splits of Q > 8 fields.
Outputs start as NaN, so an entry read before the sweep writes it shows.
"""

import numpy as np
import pytest

import oracle as O
from paper_1910_11505_gb300 import sg, workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11505_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()


def _relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _kw(case):
    return {k: case[k] for k in ("sigma", "ell", "a_min") if k in case}


FG_CASES = [
    (dict(n=6, M=2, p=2, sigma=0.7, ell=0.6), "whole"),     # G-I, Q = 6
    (dict(n=6, M=2, p=2, sigma=0.7, ell=0.6), "paper"),     # splits (0, 3), (3, 6)
    (dict(n=7, M=2, p=2, sigma=0.7, ell=0.6), "groups"),    # (0, 3), (3, 5), (5, 6); odd mesh
    (dict(n=9, M=3, p=2, sigma=0.9, ell=0.5, a_min=0.01), "whole"),   # Q = 10
    (dict(n=5, M=4, p=2, sigma=0.5, ell=0.8), "groups"),    # Q = 10 + 4 + 1
    (dict(n=4, M=2, p=6, sigma=0.6, ell=0.6), "whole"),     # Q = 28: three lanes' groups
    (dict(n=3, M=3, p=4, sigma=0.6, ell=0.6), "whole"),     # Q = 35: two warps per node
    (dict(n=3, M=4, p=4, sigma=0.6, ell=0.6), "whole"),     # Q = 70: three warps per node
    (dict(n=3, M=4, p=5, sigma=0.5, ell=0.8), "paper"),     # splits of 56 and 70 fields
    (dict(n=4, M=6, p=3, sigma=1.0, ell=0.5), "paper"),     # the c3 chaos basis: one split of 84
]


@pytest.mark.parametrize("case,rule", FG_CASES)
def test_fg_matches_oracle(case, rule):
    h = sg.sg_setup(sg.sg_default_params(**case, precond="fg", fg_rule=rule, ilu_order="color4"))
    N, P, _ = sg.sg_dims(h)
    prob = O.build_problem(case["n"], case["M"], case["p"], **_kw(case))
    splits = O.fg_splits(prob.Jp, rule)
    facs = O.fg_blocks(prob, splits, "color4")
    R = W.random_field(N, P, seed=61)
    # the output starts as NaN: no entry may be read before the sweep writes it
    Z = torch.full((N, P), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        sg.sg_precond_apply(h, 0, torch.from_numpy(R).cuda(), Z)
    ref = O.fg_precond(prob, R, splits, facs)
    assert _relerr(Z.cpu().numpy(), ref) <= 1e-12
    h.close()


@pytest.mark.parametrize("case,rule", [(dict(n=16, M=2, p=2, sigma=0.8, ell=0.5), "paper"),
                                       (dict(n=3, M=4, p=4, sigma=0.6, ell=0.6), "whole"),
                                       (dict(n=5, M=4, p=3, sigma=0.6, ell=0.6), "whole")])
def test_fg_fp32_against_fp64_oracle(case, rule):
    # FP32 factors and sweeps; n = 3 and 5 give meshes of 4 and 6 nodes per side, where the
    # edge nodes of odd colours have neighbour slots outside the mesh
    h = sg.sg_setup(sg.sg_default_params(**case, precond="fg", fg_rule=rule, ilu_order="color4",
                                         precision="fp32"))
    N, P, _ = sg.sg_dims(h)
    prob = O.build_problem(case["n"], case["M"], case["p"], **_kw(case))
    splits = O.fg_splits(prob.Jp, rule)
    R = W.random_field(N, P, seed=62).astype(np.float32).astype(np.float64)
    Z = torch.full((N, P), float("nan"), dtype=torch.float32, device="cuda")
    sg.sg_precond_apply_lowp(h, 0, torch.from_numpy(R).float().cuda(), Z)
    ref = O.fg_precond(prob, R, splits, O.fg_blocks(prob, splits, "color4"))
    # FP32 Gauss-Jordan inverses of the diagonal blocks: ~Q roundings per entry
    q = max(f1 - f0 for f0, f1 in splits)
    assert _relerr(Z.double().cpu().numpy(), ref) <= 1e-5 * max(1.0, q / 8.0)
    h.close()


@pytest.mark.parametrize("rule", ["whole", "paper"])
def test_fg_vcycle_matches_oracle(rule):
    case = dict(n=8, M=2, p=2, sigma=0.6, ell=0.8)
    h = sg.sg_setup(sg.sg_default_params(**case, precond="mg", mg_smoother="fg", fg_rule=rule,
                                         ilu_order="color4"))
    N, P, _ = sg.sg_dims(h)
    levels = O.mg_levels(8, 2, 2, coarse=2, **_kw(case))
    data = O.mg_setup(levels, "fg:" + rule, "color4")
    R = W.random_field(N, P, seed=63)
    R[levels[-1].boundary] = 0.0
    Z = torch.full((N, P), float("nan"), dtype=torch.float64, device="cuda")
    sg.sg_precond_apply(h, 0, torch.from_numpy(R).cuda(), Z)
    ref = O.mg_vcycle(levels, data, R, "fg:" + rule)
    assert _relerr(Z.cpu().numpy(), ref) <= 1e-12
    h.close()


@pytest.mark.parametrize("pc,extra", [("fg", dict(fg_rule="whole")),
                                      ("mg", dict(mg_smoother="fg", fg_rule="whole")),
                                      ("mg", dict(mg_smoother="fg", fg_rule="paper"))])
def test_gmres_with_grouped_split_solves(pc, extra):
    case = dict(n=8, M=2, p=2, sigma=0.9, ell=0.5)
    h = sg.sg_setup(sg.sg_default_params(**case, precond=pc, ilu_order="color4", rtol=1e-10,
                                         restart=40, max_iters=200, **extra))
    N, P, _ = sg.sg_dims(h)
    F = torch.empty(N, P, dtype=torch.float64, device="cuda")
    sg.sg_rhs(h, 0, F)
    X = torch.zeros_like(F)
    rc, info = sg.sg_gmres_solve(h, [F], [X])
    assert rc == sg.SG_OK, info
    prob = O.build_problem(8, 2, 2, **_kw(case))
    K = sum(np.kron(prob.G[k], prob.A[k].toarray()) for k in range(prob.L))
    ref = np.linalg.solve(K, prob.F.T.ravel()).reshape(prob.P, prob.N).T
    assert np.linalg.norm(X.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    h.close()


def test_grouped_split_refusals():
    with pytest.raises(RuntimeError):  # only the four-colour ordering is built
        sg.sg_setup(sg.sg_default_params(n=8, M=2, p=2, precond="fg", ilu_order="natural"))
    with pytest.raises(RuntimeError):  # a split of 210 fields
        sg.sg_setup(sg.sg_default_params(n=4, M=6, p=4, precond="fg", fg_rule="whole",
                                         ilu_order="color4"))


@pytest.mark.parametrize("case,rule", [(dict(n=5, M=4, p=4, sigma=0.6, ell=0.6), "whole"),
                                       (dict(n=4, M=7, p=3, sigma=0.5, ell=0.8), "groups"),
                                       (dict(n=9, M=3, p=2, sigma=0.7, ell=0.6), "groups")])
def test_bf16_factor_layout_wide_blocks(case, rule):
    # BF16 factors in columns of four: one split of Q = 70; splits of 84, 28, 7 and 1 fields
    # (zero-padded columns for 7 and 1); splits of 6, 3 and 1; against the same factors applied
    # in FP32 the difference is the BF16 rounding of the factors, amplified by the sweeps
    hs = [sg.sg_setup(sg.sg_default_params(**case, precond="fg", fg_rule=rule,
                                           ilu_order="color4", precision="fp32", fg_bf16=b))
          for b in (0, 1)]
    N, P, _ = sg.sg_dims(hs[0])
    R = torch.from_numpy(W.random_field(N, P, seed=65)).float().cuda()
    Z = [torch.full_like(R, float("nan")) for _ in hs]
    for h, z in zip(hs, Z):
        sg.sg_precond_apply_lowp(h, 0, R, z)
    d = float((Z[1] - Z[0]).abs().max() / Z[0].abs().max())
    assert 1e-6 < d < 5e-2, d
    for h in hs:
        h.close()


def test_bf16_factor_storage():
    # rounding the stored factors to BF16 changes the preconditioner by about the BF16 unit
    # round-off (2^-8) amplified by the sweeps; the solution of the mixed solve does not change
    case = dict(n=16, M=2, p=2, sigma=0.8, ell=0.5)
    hs = [sg.sg_setup(sg.sg_default_params(**case, precond="fg", fg_rule="paper",
                                           ilu_order="color4", precision="fp32", fg_bf16=b))
          for b in (0, 1)]
    N, P, _ = sg.sg_dims(hs[0])
    R = torch.from_numpy(W.random_field(N, P, seed=64)).float().cuda()
    Z = [torch.full_like(R, float("nan")) for _ in hs]
    for h, z in zip(hs, Z):
        sg.sg_precond_apply_lowp(h, 0, R, z)
    d = float((Z[1] - Z[0]).abs().max() / Z[0].abs().max())
    assert 1e-5 < d < 5e-2, d
    for h in hs:
        h.close()
    h = sg.sg_setup(sg.sg_default_params(**case, precond="mg", mg_smoother="fg", fg_rule="paper",
                                         ilu_order="color4", precision="fp32", fg_bf16=1,
                                         rtol=1e-10, restart=40, max_iters=200))
    F = torch.empty(N, P, dtype=torch.float64, device="cuda")
    sg.sg_rhs(h, 0, F)
    X = torch.zeros_like(F)
    rc, info = sg.sg_gmres_solve(h, [F], [X])
    assert rc == sg.SG_OK, info
    prob = O.build_problem(16, 2, 2, **_kw(case))
    K = sum(np.kron(prob.G[k], prob.A[k].toarray()) for k in range(prob.L))
    ref = np.linalg.solve(K, prob.F.T.ravel()).reshape(prob.P, prob.N).T
    assert np.linalg.norm(X.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    h.close()
    with pytest.raises(RuntimeError):  # BF16 factors only in the mixed form
        sg.sg_setup(sg.sg_default_params(**case, precond="fg", ilu_order="color4", fg_bf16=1))
