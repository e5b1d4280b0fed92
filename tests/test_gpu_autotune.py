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


# ---- batch configurations -----------------------------------------------------------------------------------------
BATCH_CONFIGS = [(k, sp, bp) for k in (2, 4, 8) for sp in (50, 100, 0) for bp in (1, 2)]


@pytest.fixture(scope="module")
def mixed_batch(oracle):
    """Pairs whose rows span every words-per-lane class (row widths around 32, 64, 128, 256 and 4096 columns),
    short and tall pairs (split and not split), alphabets 4, 20 and 256 in one batch."""
    import numpy as np
    rng = np.random.default_rng(77)
    widths = [1, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 1024, 2047, 2048, 2049, 4095, 4096]
    heights = [1, 7, 255, 256, 257, 600, 3000]
    shapes = [(h, w) for w in widths for h in heights[:: 1 + (w % 3)]]
    shapes += [(int(rng.integers(1, 3000)), int(rng.integers(1, 4097))) for _ in range(60)]
    pairs = [gen.pair_uniform(m, n, [4, 20, 256][k % 3], seed=7000 + k) for k, (m, n) in enumerate(shapes)]
    return pairs, [oracle.lcs_length(x, y) for x, y in pairs]


@pytest.mark.parametrize("k,sp,bp", BATCH_CONFIGS)
def test_every_batch_config_is_exact(ctx, mixed_batch, k, sp, bp):
    pairs, want = mixed_batch
    ctx.set_batch_config(k, sp, bp)
    assert ctx.get_batch_config() == {"words_per_lane": k, "split_pct": sp, "blocks_per_sm": bp}
    assert [int(v) for v in ctx.batch(pairs)] == want  # planned and launched
    assert [int(v) for v in ctx.batch(pairs)] == want  # the same batch again: replayed as a CUDA graph


def test_set_batch_config_rejects_bad_values(ctx):
    from paper_1306_4627_gb300 import lcs
    for bad in [(3, 100, 1), (16, 100, 1), (4, 2000, 1), (4, 100, 0), (4, 100, 3)]:
        with pytest.raises(lcs.LCSError):
            ctx.set_batch_config(*bad)


def test_batch_autotune_keeps_a_valid_config(ctx, mixed_batch):
    import numpy as np
    import torch
    pairs, want = mixed_batch
    d = torch.device("cuda", 0)
    xs = np.concatenate([x for x, _ in pairs])
    ys = np.concatenate([y for _, y in pairs])
    xo = np.zeros(len(pairs) + 1, np.int64)
    yo = np.zeros(len(pairs) + 1, np.int64)
    xo[1:] = np.cumsum([len(x) for x, _ in pairs])
    yo[1:] = np.cumsum([len(y) for _, y in pairs])
    out = torch.zeros(len(pairs), dtype=torch.int64, device=d)
    best = ctx.autotune_batch_dev(torch.from_numpy(xs).to(d), torch.from_numpy(xo).to(d), torch.from_numpy(ys).to(d),
                                  torch.from_numpy(yo).to(d), len(pairs), out)
    assert (best["words_per_lane"], best["split_pct"], best["blocks_per_sm"]) in [(k, sp, bp) for k in (2, 4, 8)
                                                                               for sp in (50, 100, 200, 0)
                                                                               for bp in (1, 2)]
    assert best["ms"] > 0
    assert ctx.get_batch_config() == {k: best[k] for k in ("words_per_lane", "split_pct", "blocks_per_sm")}
    assert [int(v) for v in out.cpu().numpy()] == want
    assert [int(v) for v in ctx.batch(pairs)] == want
