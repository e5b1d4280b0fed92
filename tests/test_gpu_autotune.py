"""Fill configurations and the autotuner: every configuration gives the oracle's results; the autotuner keeps
one of them per mode."""

import pytest

from paper_1306_4627_gb300 import gen

pytestmark = pytest.mark.gpu

CONFIGS = [(8, 0), (8, 1), (16, 0), (16, 1)]


@pytest.fixture(scope="module")
def ctx():
    from paper_1306_4627_gb300 import lcs
    c = lcs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("rows,vg", CONFIGS)
def test_every_fill_config_is_exact(ctx, oracle, rows, vg):
    x, y = gen.pair_uniform(3001, 9000, 4, seed=61)
    want_len, want_s = oracle.lcs_length(x, y), oracle.lcs_traceback(x, y)
    for tb in (False, True):
        ctx.set_fill_config(rows, vg, traceback=tb)
        assert ctx.get_fill_config(traceback=tb) == {"rows_per_step": rows, "vg_select": vg}
    assert ctx.length(x, y) == want_len
    assert ctx.traceback(x, y) == want_s


def test_set_fill_config_rejects_bad_values(ctx):
    from paper_1306_4627_gb300 import lcs
    with pytest.raises(lcs.LCSError):
        ctx.set_fill_config(12, 0)
    with pytest.raises(lcs.LCSError):
        ctx.set_fill_config(8, 3)


def test_autotune_keeps_a_valid_config(ctx, oracle):
    import torch
    d = torch.device("cuda", 0)
    x, y = gen.pair_uniform(8192, 8192, 4, seed=62)
    dx, dy = torch.from_numpy(x.copy()).to(d), torch.from_numpy(y.copy()).to(d)
    for tb in (False, True):
        best = ctx.autotune_dev(dx, dy, traceback=tb)
        assert (best["rows_per_step"], best["vg_select"]) in CONFIGS and best["ms"] > 0
        assert ctx.get_fill_config(traceback=tb) == {"rows_per_step": best["rows_per_step"],
                                                     "vg_select": best["vg_select"]}
    assert ctx.length(x, y) == oracle.lcs_length(x, y)
    assert ctx.traceback(x, y) == oracle.lcs_traceback(x, y)
