"""CPU checks of the row-tiled operator's planner (host code of the library, no device work).

The planner groups the coefficient chaos indices k, cuts the groups into chunks that fit the
shared-memory budget and places every (k, b) pair of a nonzero G_k[a, b] in exactly one T slot and
every nonzero G_k[a, b] in exactly one stage-2 entry.  The counts are checked against the oracle's
triple products, and the budget rule against the stated shared-memory limit.
"""

import math

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def sg():
    from paper_1910_11505_gb300 import build as B
    B.build()
    from paper_1910_11505_gb300 import sg as _sg
    return _sg


@pytest.mark.parametrize("M,p", [(2, 2), (4, 3), (3, 1), (1, 4), (2, 0)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plan_places_every_pair_and_entry_once(sg, M, p, precision):
    G = O.triple_products(O.multi_indices(M, 2 * p), O.multi_indices(M, p))
    pairs = int(np.count_nonzero(np.any(G != 0, axis=1)))   # (k, b) with some a
    entries = int(np.count_nonzero(G))
    ks = int(np.count_nonzero(np.any(G != 0, axis=(1, 2))))
    plan = sg.sg_tune_plan(64, M, p, 0, precision)
    elem = 8 if precision == "fp64" else 4
    P = G.shape[1]
    for pl in plan:
        if not pl["fits"]:
            continue
        assert pl["verified"], pl
        assert pl["pairs"] == pairs and pl["entries"] == entries and pl["k_kept"] == ks
        assert pl["groups"] >= math.ceil(ks / pl["kappa"])
        assert pl["smem"] <= pl["budget"]
        # the stated layout: barriers, two stack chunk slots and two side-table slots, T slots (or
        # the Y staging of P outputs), the three grid lines of X with an odd stride
        slab = 3 * 34 * (P | 1)
        assert pl["smem"] >= 128 + elem * (slab + 32 * max(pl["max_slots"], P))
    assert plan[0]["fits"]


def test_plan_respects_the_shared_memory_budget(sg):
    big = sg.sg_tune_plan(128, 4, 3, 0, "fp64")
    for pl in big:
        if pl["fits"]:
            small = sg.sg_tune_plan(128, 4, 3, 0, "fp64", smem_max=pl["smem"] - 1)
            assert all(q["smem"] <= q["budget"] for q in small if q["fits"])
    tiny = sg.sg_tune_plan(128, 4, 3, 0, "fp64", smem_max=16 * 1024)
    assert not any(q["fits"] for q in tiny)


@pytest.mark.parametrize("n,M,p,precision", [(128, 4, 3, "fp64"), (128, 4, 3, "fp32"),
                                             (256, 6, 3, "fp32"), (256, 6, 3, "fp64"),
                                             (16, 8, 2, "fp32")])
def test_plans_at_solver_sizes_decode_to_the_triple_products(sg, n, M, p, precision):
    plan = sg.sg_tune_plan(n, M, p, 0, precision)
    assert any(pl["fits"] for pl in plan)
    for pl in plan:
        if pl["fits"]:
            assert pl["verified"], pl


def test_plan_refuses_invalid_sizes(sg):
    with pytest.raises(sg.SGError):
        sg.sg_tune_plan(1, 2, 2)
    with pytest.raises(sg.SGError):
        sg.sg_tune_plan(16, 9, 2)
