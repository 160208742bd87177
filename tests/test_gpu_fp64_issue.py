"""The FP64 pipe property the refinement's work distribution rests on: a dependent chain
of FP64 FMAs takes the same time whether 1, 8 or 32 lanes of the warp run it, so lanes
left idle by a pass of fewer propagations than lanes can take extra propagations for
free; warps on different sub-partitions of one SM run their chains side by side."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_chain_cost_does_not_depend_on_active_lanes():
    from paper_2207_13175_gb300 import api
    full = api.selftest_fp64_issue(1, 32)
    for lanes in (1, 8, 13):
        c = api.selftest_fp64_issue(1, lanes)
        assert abs(c - full) <= 0.05 * full, (lanes, c, full)


def test_two_warps_run_side_by_side():
    from paper_2207_13175_gb300 import api
    one = api.selftest_fp64_issue(1, 32)
    two = api.selftest_fp64_issue(2, 32)
    assert two <= 1.1 * one, (one, two)
