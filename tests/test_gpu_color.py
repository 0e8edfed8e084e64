"""The four-colour ILU(0) ordering (reading R18) through the C ABI against the oracle: the factors
themselves, every block preconditioner at small and large meshes, and the multigrid V-cycle with
these smoothers.  Block solves run on one CTA with the column in shared memory up to ~8 k nodes,
on a thread-block cluster of 2, 4 or 8 CTAs beyond.  Tolerances as in test_gpu_parity (1e-12
FP64)."""

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


def test_color4_factors_match_oracle():
    d = dict(n=9, M=2, p=1, sigma=0.7, ell=0.6, a_min=0.02)
    h = sg.sg_setup(sg.sg_default_params(**d, precond="mean", ilu_order="color4"))
    prob = O.build_problem(9, 2, 1, sigma=0.7, ell=0.6, a_min=0.02)
    Lo, Up, order = O.ilu0(prob.A[0], O.color4_order(9))
    LUp = Lo.toarray() - np.eye(prob.N) + Up.toarray()
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    LU = LUp[np.ix_(inv, inv)]               # back to natural node numbering
    rowptr, col = sg.sg_export(h, 0, 1), sg.sg_export(h, 0, 2)
    vals = sg.sg_export(h, 0, 4)
    for r in range(prob.N):
        for e in range(rowptr[r], rowptr[r + 1]):
            assert abs(vals[e] - LU[r, col[e]]) <= 1e-13 * np.abs(LU).max(), (r, col[e])
    h.close()


@pytest.mark.parametrize("d,pc", [
    (dict(n=6, M=3, p=2, sigma=0.5, ell=1.0, a_min=0.01), "mean"),
    (dict(n=6, M=3, p=2, sigma=0.5, ell=1.0, a_min=0.01), "fs_gs"),
    (dict(n=7, M=2, p=2, sigma=0.8, ell=0.6), "fs_jacobi"),
    (dict(n=256, M=2, p=2, sigma=0.8, ell=0.5), "fs_gs"),      # cluster of 16 (where offered)
    (dict(n=200, M=2, p=1, sigma=0.8, ell=0.5), "fs_gs"),      # cluster of 8 CTAs per column
    (dict(n=200, M=2, p=1, sigma=0.8, ell=0.5), "mean"),
    (dict(n=128, M=2, p=1, sigma=0.6, ell=0.5), "fs_gs"),      # cluster of 4
    (dict(n=100, M=2, p=1, sigma=0.6, ell=0.5), "fs_jacobi"),  # cluster of 2
])
def test_color4_preconditioners_match_oracle(d, pc):
    h = sg.sg_setup(sg.sg_default_params(**d, precond=pc, ilu_order="color4"))
    N, P, _ = sg.sg_dims(h)
    kw = {k: d[k] for k in ("sigma", "ell", "a_min") if k in d}
    prob = O.build_problem(d["n"], d["M"], d["p"], **kw)
    R = W.random_field(N, P, seed=51)
    Z = torch.full((N, P), float("nan"), dtype=torch.float64, device="cuda")
    sg.sg_precond_apply(h, 0, torch.from_numpy(R).cuda(), Z)
    if pc == "mean":
        ref = O.mean_precond(prob, R, ordering="color4")
    else:
        ref = O.fs_precond(prob, R, mode="gs" if pc == "fs_gs" else "jacobi",
                           blocks=O.fs_blocks(prob, ordering="color4"))
    assert _relerr(Z.cpu().numpy(), ref) <= 1e-12
    h.close()


def test_color4_fp32_large_mesh():
    d = dict(n=256, M=2, p=1, sigma=0.8, ell=0.5)              # cluster of 16 or 8, FP32
    h = sg.sg_setup(sg.sg_default_params(**d, precond="fs_gs", ilu_order="color4",
                                         precision="fp32"))
    N, P, _ = sg.sg_dims(h)
    prob = O.build_problem(256, 2, 1, sigma=0.8, ell=0.5)
    R = W.random_field(N, P, seed=52)
    Z = torch.full((N, P), float("nan"), dtype=torch.float32, device="cuda")
    sg.sg_precond_apply_lowp(h, 0, torch.from_numpy(R).float().cuda(), Z)
    ref = O.fs_precond(prob, R.astype(np.float32).astype(np.float64),
                       blocks=O.fs_blocks(prob, ordering="color4"))
    assert _relerr(Z.double().cpu().numpy(), ref) <= 1e-6
    h.close()


@pytest.mark.parametrize("smoother", ["fs_gs", "fs_jacobi"])
def test_color4_vcycle_matches_oracle(smoother):
    case = dict(n=16, M=3, p=2, sigma=0.7, ell=0.6)
    h = sg.sg_setup(sg.sg_default_params(**case, precond="mg", mg_smoother=smoother,
                                         ilu_order="color4"))
    N, P, _ = sg.sg_dims(h)
    levels = O.mg_levels(16, 3, 2, sigma=0.7, ell=0.6)
    data = O.mg_setup(levels, smoother, ordering="color4")
    R = W.random_field(N, P, seed=53)
    R[levels[-1].boundary] = 0.0
    Z = torch.full((N, P), float("nan"), dtype=torch.float64, device="cuda")
    sg.sg_precond_apply(h, 0, torch.from_numpy(R).cuda(), Z)
    ref = O.mg_vcycle(levels, data, R, smoother)
    assert _relerr(Z.cpu().numpy(), ref) <= 1e-12
    h.close()


def test_color4_refuses_inner_iterations():
    with pytest.raises(sg.SGError) as ei:
        sg.sg_setup(sg.sg_default_params(n=8, M=2, p=1, precond="mean", ilu_order="color4",
                                         inner_iters=2))
    assert ei.value.code == sg.SG_ERR_ARG


def _bf16_round(x):
    """Round-to-nearest-even of FP64 values to BF16 (8 significant bits), written out."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def test_bf16_coupling_sweep_matches_oracle_with_rounded_coupling():
    # the FP32 Gauss-Seidel sweep whose coupling reads BF16 stiffness values, against the oracle
    # sweep with the coupling matrices rounded the same way (FP32 arithmetic bound 1e-6 as for the
    # other FP32 sweeps, plus ties that FP32 rounding of the products may resolve differently)
    import scipy.sparse
    d = dict(n=40, M=3, p=2, sigma=0.9, ell=0.5)
    h = sg.sg_setup(sg.sg_default_params(**d, precond="fs_gs", precision="fp32", coupling_bf16=1))
    N, P, _ = sg.sg_dims(h)
    prob = O.build_problem(40, 3, 2, sigma=0.9, ell=0.5)
    coupling = []
    for A in prob.A:
        Ar = A.copy()
        Ar.data = _bf16_round(Ar.data)
        coupling.append(Ar)
    R = W.random_field(N, P, seed=54)
    Z = torch.full((N, P), float("nan"), dtype=torch.float32, device="cuda")
    sg.sg_precond_apply_lowp(h, 0, torch.from_numpy(R).float().cuda(), Z)
    Rr = R.astype(np.float32).astype(np.float64)
    ref = O.fs_precond(prob, Rr, coupling=coupling)
    ref_exact = O.fs_precond(prob, Rr)
    err = _relerr(Z.double().cpu().numpy(), ref)
    assert err <= 1e-5, err
    assert _relerr(ref, ref_exact) > 10 * err  # the rounding is visible: the test sees the copy
    h.close()
    with pytest.raises(sg.SGError):
        sg.sg_setup(sg.sg_default_params(**d, precond="fs_gs", precision="fp64", coupling_bf16=1))
