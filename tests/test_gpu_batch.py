"""lcs_batch: many independent pairs in one persistent launch, every length exact vs the CPU oracle."""

import numpy as np
import pytest

from paper_1306_4627_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1306_4627_gb300 import lcs
    c = lcs.Context(0)
    yield c
    c.close()


def test_batch_edge_shapes(ctx, oracle):
    shapes = [(0, 5), (5, 0), (1, 1), (1, 31), (31, 32), (33, 33), (64, 127), (100, 128), (129, 129), (7, 512),
              (513, 1000), (2000, 4096), (300, 4097), (50, 5000), (4096, 64)]
    pairs = []
    for k, (m, n) in enumerate(shapes):
        pairs.append(gen.pair_uniform(m, n, 4, seed=900 + k))
    got = ctx.batch(pairs)
    for (x, y), g in zip(pairs, got):
        assert int(g) == oracle.lcs_length(x, y), (len(x), len(y))


# alphabets by the 32-value blocks of byte values they occupy (the prep's alphabet pass has a path for one block,
# one for two and one for more): "AB", DNA and protein letters one block each, mixed-case DNA two, digits with
# mixed-case letters three, all bytes eight
ALPHABETS = {2: b"AB", 4: gen.DNA, 20: gen.PROTEIN, 256: gen.BYTES, "2blk": b"ACGTacgt", "3blk": b"09AZaz"}


@pytest.mark.parametrize("sigma", [2, 4, 20, 256, "2blk", "3blk"])
def test_batch_random_mixed(ctx, oracle, sigma):
    rng = np.random.default_rng(len(ALPHABETS[sigma]))
    pairs = []
    for k in range(300):
        m = int(rng.integers(1, 700))
        n = int(rng.integers(1, 1500))
        alpha = ALPHABETS[sigma]
        pairs.append((gen.random_string(5000 + 2 * k, m, alpha), gen.random_string(5001 + 2 * k, n, alpha)))
    got = ctx.batch(pairs)
    want = [oracle.lcs_length(x, y) for x, y in pairs]
    assert [int(v) for v in got] == want


def test_batch_mixed_alphabets_in_one_launch(ctx, oracle):
    pairs = [gen.pair_uniform(200 + 13 * k, 3000 - 11 * k, [4, 20, 256][k % 3], seed=70 + k) for k in range(60)]
    got = ctx.batch(pairs)
    assert [int(v) for v in got] == [oracle.lcs_length(x, y) for x, y in pairs]


def test_batch_dev_and_host_offsets_vs_oracle(ctx, oracle):
    """lcs_batch_dev (offsets on the device) and lcs_batch_dev_hoff (offsets in host memory, starting past a few
    leading bytes of the buffers), each called twice (a planning call, then the cached plan replayed as a graph),
    every length against the oracle."""
    import torch
    pairs = gen.batch_pairs(count=500, seed=123)
    want = np.array([oracle.lcs_length(x, y) for x, y in pairs], np.int64)
    lead_x, lead_y = 7, 3  # bytes in front of the first pair
    xs = np.concatenate([np.full(lead_x, 65, np.uint8)] + [x for x, _ in pairs])
    ys = np.concatenate([np.full(lead_y, 67, np.uint8)] + [y for _, y in pairs])
    xo = np.zeros(len(pairs) + 1, np.int64)
    yo = np.zeros(len(pairs) + 1, np.int64)
    xo[1:] = np.cumsum([len(x) for x, _ in pairs])
    yo[1:] = np.cumsum([len(y) for _, y in pairs])
    xo += lead_x
    yo += lead_y
    d = torch.device("cuda", 0)
    dxs, dys = torch.from_numpy(xs).to(d), torch.from_numpy(ys).to(d)
    out = torch.zeros(len(pairs), dtype=torch.int64, device=d)
    for _ in range(2):
        out.zero_()
        ctx.batch_dev(dxs, torch.from_numpy(xo).to(d), dys, torch.from_numpy(yo).to(d), len(pairs), out)
        ctx.sync()
        assert np.array_equal(out.cpu().numpy(), want)
    for _ in range(2):
        out.zero_()
        ctx.batch_dev_hoff(dxs, xo.astype(np.uint64), dys, yo.astype(np.uint64), len(pairs), out)
        ctx.sync()
        assert np.array_equal(out.cpu().numpy(), want)


def test_batch_dev_hoff_rejects_bad_offsets(ctx):
    import torch
    from paper_1306_4627_gb300 import lcs
    d = torch.device("cuda", 0)
    buf = torch.zeros(16, dtype=torch.uint8, device=d)
    out = torch.zeros(2, dtype=torch.int64, device=d)
    with pytest.raises(lcs.LCSError):  # decreasing offsets
        ctx.batch_dev_hoff(buf, np.array([0, 8, 4], np.uint64), buf, np.array([0, 4, 8], np.uint64), 2, out)


def test_batch_matches_single_pair_path(ctx):
    pairs = gen.batch_pairs(count=200, seed=321)
    got = ctx.batch(pairs)
    for (x, y), g in zip(pairs[:60], got[:60]):
        assert int(g) == ctx.length(x, y)


@pytest.mark.slow
def test_batch_10000_pairs_vs_oracle(ctx, oracle):
    """The batched workload: 10000 pairs, m and n log-uniform in [64, 4096], alphabet 4 for half the pairs and
    20 for the other half; every length exact vs the oracle."""
    pairs = gen.batch_pairs()
    got = ctx.batch(pairs)
    want = np.array([oracle.lcs_length(x, y) for x, y in pairs])
    assert np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("sigma", [4, 20, 256])
def test_batch_split_pairs(ctx, oracle, sigma):
    """Pairs with many rows run as a forward top half and a reversed bottom half, joined at the middle row
    (c[mt, j] + LCS of the bottom rows with Y[j+1..n], maximised over j): odd and even m, ragged n, unrelated and
    closely related strings."""
    shapes = [(256, 300), (257, 257), (258, 31), (301, 4096), (511, 1000), (1024, 33), (2047, 2049), (4096, 4096),
              (3000, 129)]
    pairs = []
    for k, (m, n) in enumerate(shapes):
        pairs.append(gen.pair_uniform(m, n, sigma, seed=4400 + 10 * sigma + k))
        x, _ = gen.pair_uniform(m, 1, sigma, seed=4500 + 10 * sigma + k)
        pairs.append((x, gen.mutate(x, seed=4600 + 10 * sigma + k, alphabet=gen.ALPHABETS[sigma], out_len=min(m, 4096))))
    want = [oracle.lcs_length(x, y) for x, y in pairs]
    for _ in range(3):  # first call plans and launches; the repeats replay the recorded launches
        got = ctx.batch(pairs)
        assert [int(v) for v in got] == want


def test_batch_page_locked_buffers_read_in_place(ctx, oracle):
    """lcs_batch on page-locked host buffers, which the kernels read in place over the host link instead of a copy
    into device buffers: bytes in front of the first pair, empty pairs, a pair wider than 4096 columns (it takes the
    single-pair path, reading in place as well); the first call plans and the repeats replay the recorded launches.
    Every length equals the oracle's and the same batch's from pageable buffers."""
    import torch
    pairs = gen.batch_pairs(count=300, seed=77)
    pairs += [gen.pair_uniform(900, 5000, 4, seed=78), gen.pair_uniform(0, 40, 4, seed=79),
              gen.pair_uniform(35, 0, 20, seed=80)]
    want = np.array([oracle.lcs_length(x, y) for x, y in pairs], np.uint64)
    lead_x, lead_y = 5, 11
    xs = np.concatenate([np.full(lead_x, 71, np.uint8)] + [x for x, _ in pairs])
    ys = np.concatenate([np.full(lead_y, 84, np.uint8)] + [y for _, y in pairs])
    xo = np.zeros(len(pairs) + 1, np.uint64)
    yo = np.zeros(len(pairs) + 1, np.uint64)
    xo[1:] = np.cumsum([len(x) for x, _ in pairs])
    yo[1:] = np.cumsum([len(y) for _, y in pairs])
    xo += lead_x
    yo += lead_y
    xs_pinned = torch.from_numpy(xs).pin_memory()
    ys_pinned = torch.from_numpy(ys).pin_memory()
    for _ in range(3):
        assert np.array_equal(ctx.batch_concat(xs_pinned.numpy(), xo, ys_pinned.numpy(), yo), want)
    assert np.array_equal(ctx.batch_concat(xs, xo, ys, yo), want)
