"""The measurement probes behind the rooflines: the INT32 rate of the fill's instruction mixes and the dependency
floor of one fill step. Checked for plausibility against the device's own limits (a rate cannot exceed what its SMs
issue; a step of B rows cannot take fewer cycles than its B dependent row updates)."""

import pytest

pytestmark = pytest.mark.gpu


def test_int_rate_plausible():
    from paper_1306_4627_gb300 import lcs
    for mix, ops in ((0, 5), (1, 6), (2, 1)):
        r = lcs.probe_int_rate(0, mix, 20000)
        assert r["ops_per_chain"] == ops
        assert r["sms"] > 0 and r["blocks_per_sm"] > 0
        # four schedulers per SM issue at most one warp instruction (32 lanes) per clock each: <= 128 lane-ops
        assert 8.0 < r["ops_per_clk_sm"] <= 128.0, r
        assert 300.0 < r["sm_clock_mhz"] < 3000.0, r
        assert r["ops_per_s"] > 1e12, r


def test_step_floor_plausible():
    from paper_1306_4627_gb300 import lcs
    for b in (8, 16):
        for tb in (False, True):
            c = lcs.probe_step_floor(0, b, tb, 2048)
            # each row is a dependent chain of at least three instructions (mask AND, add with carry, OR)
            assert 3 * b < c < 100 * b, (b, tb, c)
    with pytest.raises(lcs.LCSError):
        lcs.probe_step_floor(0, 12, False, 100)


def test_step_mask_sources_plausible():
    from paper_1306_4627_gb300 import lcs
    cyc = [lcs.probe_step_masks(0, k, 2048) for k in range(len(lcs.MASK_SOURCES))]
    for c in cyc:
        assert 3 * 8 < c < 100 * 8, cyc
    # source 0 is the traceback step floor itself, measured the same way
    floor = lcs.probe_step_floor(0, 8, True, 2048)
    assert abs(cyc[0] - floor) < 0.25 * floor, (cyc, floor)
    with pytest.raises(lcs.LCSError):
        lcs.probe_step_masks(0, 4, 100)
