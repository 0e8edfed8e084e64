"""The multigrid V-cycle preconditioner (Sec. 3; V-cycle 1/1 on the hierarchy of Sec. 4) through the
C ABI against the oracle's V-cycle, and MG-preconditioned GMRES against the direct solution.

Tolerance: 1e-12 relative per V-cycle application in FP64 (each level adds a few operator and
block-solve applications, each already within 1e-14 relative of the oracle); FP32 V-cycles are
checked against the FP64 oracle at 1e-5 (the FP32 operator's 2e-5 bound per application, with the
coarse corrections damped by the smoothers).
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


MG_CASES = [
    (dict(n=8, M=2, p=2, sigma=0.6, ell=0.8), "fs_gs", 2),
    (dict(n=8, M=2, p=2, sigma=0.6, ell=0.8), "fs_jacobi", 2),
    (dict(n=8, M=2, p=2, sigma=0.6, ell=0.8), "mean", 2),
    (dict(n=16, M=3, p=2, sigma=0.9, ell=0.5, a_min=0.01), "fs_gs", 2),
    (dict(n=4, M=2, p=1, sigma=0.5, ell=1.0), "fs_gs", 2),     # one smoothing level
    (dict(n=12, M=2, p=2, sigma=0.5, ell=1.0), "fs_gs", 3),    # coarsest 3 x 3 cells
    (dict(n=16, M=1, p=3, sigma=0.7, ell=0.6), "fs_jacobi", 4),
]


@pytest.mark.parametrize("case,smoother,coarse", MG_CASES)
def test_vcycle_matches_oracle(case, smoother, coarse):
    h = sg.sg_setup(sg.sg_default_params(**case, precond="mg", mg_smoother=smoother,
                                         mg_coarse=coarse))
    N, P, _ = sg.sg_dims(h)
    kw = {k: case[k] for k in ("sigma", "ell", "a_min") if k in case}
    levels = O.mg_levels(case["n"], case["M"], case["p"], coarse=coarse, **kw)
    data = O.mg_setup(levels, smoother)
    R = W.random_field(N, P, seed=41)
    R[levels[-1].boundary] = 0.0
    Z = torch.full((N, P), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):  # a second application reuses every level's buffers
        sg.sg_precond_apply(h, 0, torch.from_numpy(R).cuda(), Z)
    ref = O.mg_vcycle(levels, data, R, smoother)
    assert _relerr(Z.cpu().numpy(), ref) <= 1e-12
    h.close()


def test_vcycle_fp32_matches_oracle():
    case = dict(n=16, M=3, p=2, sigma=0.9, ell=0.5)
    h = sg.sg_setup(sg.sg_default_params(**case, precond="mg", precision="fp32"))
    N, P, _ = sg.sg_dims(h)
    levels = O.mg_levels(16, 3, 2, sigma=0.9, ell=0.5)
    data = O.mg_setup(levels, "fs_gs")
    R = W.random_field(N, P, seed=42)
    R[levels[-1].boundary] = 0.0
    Z = torch.full((N, P), float("nan"), dtype=torch.float32, device="cuda")
    sg.sg_precond_apply_lowp(h, 0, torch.from_numpy(R).float().cuda(), Z)
    ref = O.mg_vcycle(levels, data, R.astype(np.float32).astype(np.float64), "fs_gs")
    assert _relerr(Z.double().cpu().numpy(), ref) <= 1e-5
    h.close()


# the block-Jacobi smoother ignores the coupling between chaos modes, so it serves smaller sigma
# (at sigma = 0.6 the oracle's GMRES with it stalls too)
@pytest.mark.parametrize("smoother,sigma", [("fs_gs", 0.6), ("fs_jacobi", 0.3), ("mean", 0.3)])
def test_mg_gmres_solution_and_mesh_independent_iterations(smoother, sigma):
    its = []
    for n in (8, 16, 32, 64):
        case = dict(n=n, M=2, p=2, sigma=sigma, ell=0.8)
        h = sg.sg_setup(sg.sg_default_params(**case, precond="mg", mg_smoother=smoother,
                                             rtol=1e-12, restart=30, max_iters=300))
        N, P, _ = sg.sg_dims(h)
        F = torch.full((N, P), float("nan"), dtype=torch.float64, device="cuda")
        sg.sg_rhs(h, 0, F)
        X = torch.zeros_like(F)
        rc, info = sg.sg_gmres_solve(h, [F], [X])
        assert rc == sg.SG_OK, info
        its.append(info[0]["iters"])
        if n == 8:
            prob = O.build_problem(8, 2, 2, sigma=sigma, ell=0.8)
            K = sum(np.kron(prob.G[k], prob.A[k].toarray()) for k in range(prob.L))
            ref = np.linalg.solve(K, prob.F.T.ravel()).reshape(prob.P, prob.N).T
            assert np.linalg.norm(X.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
        h.close()
    # Table 1's trend: with the field-split smoothers the MG-preconditioned iteration count does
    # not grow with the mesh; the mean-based smoother (not one of the paper's) ignores the coupling
    # between chaos modes and is only held to bounded growth over the 8x refinement
    if smoother == "mean":
        assert max(its) <= 1.5 * min(its), its
    else:
        assert max(its) - min(its) <= 3, its


def test_mg_refuses_what_it_cannot_build():
    for kw in (dict(n=12, mg_coarse=2), dict(n=10, mg_coarse=4), dict(n=2, mg_coarse=2),
               dict(n=8, mg_smoother="none")):
        with pytest.raises(sg.SGError) as ei:
            sg.sg_setup(sg.sg_default_params(M=2, p=1, precond="mg", **kw))
        assert ei.value.code == sg.SG_ERR_ARG
