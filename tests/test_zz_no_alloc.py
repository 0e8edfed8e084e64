"""The allocation-free preconditioner entry point, called through the C ABI.

sg_precond_apply_noalloc exists for callers that may not allocate device memory (for example a
process whose memory is held by another allocator's pool, or code with a fixed budget).  It keeps
its scratch in a fixed array inside the library, so these checks compare it with the regular
sg_precond_apply on two calls in a row (different inputs, so stale scratch would show) and check
that sizes beyond the array's limit are refused.  This file is collected last on purpose.
"""

import numpy as np
import pytest

from paper_1910_11505_gb300 import sg, workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11505_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("n,M,p,inner", [
    (24, 3, 2, 1),    # whole column of each block solve in shared memory
    (24, 3, 2, 2),    # two ILU(0)-Richardson steps per block: the work columns are used too
    (200, 3, 3, 1),   # a column too large for shared memory: the level-window kernel
])
def test_noalloc_matches_regular_entry_point_twice(n, M, p, inner):
    prm = sg.sg_default_params(n=n, M=M, p=p, sigma=0.8, ell=0.7, precond="fs_gs",
                               inner_iters=inner)
    h = sg.sg_setup(prm)
    N, P, _ = sg.sg_dims(h)
    for seed in (1, 2):  # two calls in a row with different inputs
        R = torch.from_numpy(W.random_field(N, P, seed=seed)).cuda()
        Zref = torch.empty_like(R)
        Z = torch.full_like(R, float("nan"))
        assert P * ((N + 3) // 4 * 4) <= (1 << 20)
        sg.sg_precond_apply(h, 0, R, Zref)
        sg.sg_precond_apply_noalloc(h, 0, R, Z)
        torch.cuda.synchronize()
        err = float((Z - Zref).abs().max() / Zref.abs().max())
        assert err <= 1e-12, (seed, err)
    h.close()


def test_noalloc_refuses_what_it_cannot_serve():
    big = sg.sg_default_params(n=120, M=6, p=3, sigma=0.5, ell=1.0, precond="fs_gs")
    h = sg.sg_setup(big)
    N, P, _ = sg.sg_dims(h)
    assert N * P > (1 << 20)
    R = torch.zeros(N, P, dtype=torch.float64, device="cuda")
    with pytest.raises(sg.SGError) as ei:
        sg.sg_precond_apply_noalloc(h, 0, R, torch.empty_like(R))
    assert ei.value.code == sg.SG_ERR_ARG and "exceeds" in str(ei.value)
    h.close()
    h = sg.sg_setup(sg.sg_default_params(n=8, M=2, p=1, precond="mean"))
    N, P, _ = sg.sg_dims(h)
    R = torch.zeros(N, P, dtype=torch.float64, device="cuda")
    with pytest.raises(sg.SGError) as ei:
        sg.sg_precond_apply_noalloc(h, 0, R, torch.empty_like(R))
    assert ei.value.code == sg.SG_ERR_ARG
    h.close()
