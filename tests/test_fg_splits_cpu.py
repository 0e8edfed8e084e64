"""CPU check of the library's split rule of the grouped field split (host code, no device
work) against the oracle's (reading R21; the oracle's rule is pinned to the paper's worked
example in test_oracle_fg.py)."""

import pytest

import oracle as O


@pytest.fixture(scope="module")
def sg():
    from paper_1910_11505_gb300 import build as B
    B.build()
    from paper_1910_11505_gb300 import sg as _sg
    return _sg


@pytest.mark.parametrize("M,p", [(2, 4), (2, 2), (6, 3), (4, 3), (3, 3), (5, 4), (1, 3), (4, 0)])
@pytest.mark.parametrize("rule", ["paper", "groups", "whole"])
def test_library_splits_equal_the_oracle(sg, M, p, rule):
    assert sg.sg_fg_splits(M, p, rule) == O.fg_splits(O.multi_indices(M, p), rule)


def test_split_rule_refusals(sg):
    with pytest.raises(RuntimeError):
        sg.sg_fg_splits(9, 2, "paper")
    with pytest.raises(RuntimeError):
        sg.sg_fg_splits(2, 7, "paper")
