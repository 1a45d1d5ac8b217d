"""Host logic of the autotuner (no GPU): the choice among timed configurations under the error
tolerances, and the depth candidates."""
from paper_2410_01626_b300.autotune import depth_candidates, select_within_tolerance


def test_fastest_within_tolerance_wins():
    table = {(2, 0, 0): {"ms": 3.0, "err_F": 2e-5, "err_dVdl": 1e-5},
             (3, 0, 0): {"ms": 1.0, "err_F": 1.3e-4, "err_dVdl": 2e-5},   # fastest, force error too large
             (4, 0, 0): {"ms": 2.0, "err_F": 6e-5, "err_dVdl": 3e-5}}
    assert select_within_tolerance(table) == (4, 0, 0)
    # a dV/dlambda error beyond safety x tolerance also disqualifies
    table[(4, 0, 0)]["err_dVdl"] = 8e-5
    assert select_within_tolerance(table) == (2, 0, 0)


def test_most_accurate_when_none_meets_the_tolerance():
    table = {(2, 0, 0): {"ms": 3.0, "err_F": 3e-4, "err_dVdl": 1e-5},
             (3, 0, 0): {"ms": 1.0, "err_F": 2e-4, "err_dVdl": 5e-4}}
    assert select_within_tolerance(table) == (2, 0, 0)  # max(3, 0.1) < max(2, 5)


def test_depth_candidates():
    assert depth_candidates(500000, True) == [4, 5]          # clamped at the deepest supported tree
    assert depth_candidates(6000, True) == [2, 3, 4]
    assert depth_candidates(1000, False) == [2, 3]            # open boxes start at depth 2
