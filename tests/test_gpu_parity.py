"""CUDA path vs the CPU oracle, element by element (length and LCS string must be identical)."""

import os
import random

import numpy as np
import pytest

from paper_1306_4627_gb300 import gen
from tests.conftest import read_golden_cases

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "clrs_tiebreak.txt")


@pytest.fixture(scope="module")
def ctx():
    from paper_1306_4627_gb300 import lcs
    c = lcs.Context(0)
    yield c
    c.close()


def check_pair(ctx, oracle, x, y, traceback=True):
    x = np.ascontiguousarray(x, dtype=np.uint8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    L = oracle.lcs_length(x, y)
    assert ctx.length(x, y) == L, (len(x), len(y))
    if traceback:
        s = ctx.traceback(x, y)
        assert s == oracle.lcs_traceback(x, y), (len(x), len(y))


def test_golden_cases(ctx, oracle):
    cases, _ = read_golden_cases(GOLDEN)
    for x, y, L, s in cases:
        assert ctx.length(x, y) == L
        assert ctx.traceback(x, y) == s


def test_empty(ctx):
    assert ctx.length(b"", b"ACGT") == 0
    assert ctx.length(b"ACGT", b"") == 0
    assert ctx.traceback(b"", b"") == b""
    assert ctx.traceback(b"AC", b"") == b""


@pytest.mark.parametrize("sigma", [2, 4, 20, 256])
def test_random_small(ctx, oracle, sigma):
    rng = random.Random(sigma)
    alpha = {2: b"AB", 4: gen.DNA, 20: gen.PROTEIN, 256: gen.BYTES}[sigma]
    for k in range(40):
        m, n = rng.randint(1, 300), rng.randint(1, 300)
        x = gen.random_string(1000 * sigma + 2 * k, m, alpha)
        y = gen.random_string(1000 * sigma + 2 * k + 1, n, alpha)
        check_pair(ctx, oracle, x, y)


@pytest.mark.parametrize("m", [1, 7, 8, 9, 31, 32, 33, 1023, 1024, 1025])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 63, 64, 4095, 4096, 4097])
def test_edge_shapes(ctx, oracle, m, n):
    x, y = gen.pair_uniform(m, n, 4, seed=m * 10007 + n)
    check_pair(ctx, oracle, x, y)


def test_multi_block_columns(ctx, oracle):
    # n spans several 4096-column blocks (global carry hand-off) and a ragged last word
    for m, n in [(700, 9000), (2050, 12289), (64, 20000)]:
        x, y = gen.pair_uniform(m, n, 4, seed=m + n)
        check_pair(ctx, oracle, x, y)


def test_identical_and_disjoint(ctx):
    x = gen.random_string(3, 5000, gen.DNA)
    assert ctx.length(x, x) == 5000
    assert ctx.traceback(x, x) == x.tobytes()
    a = gen.random_string(4, 3000, b"AC")
    b = gen.random_string(5, 3100, b"GT")
    assert ctx.length(a, b) == 0
    assert ctx.traceback(a, b) == b""


def test_single_pair_2048_dna(ctx, oracle):
    x, y = gen.pair_uniform(2048, 2048, 4, seed=gen.BASE_SEED + 0)
    check_pair(ctx, oracle, x, y)


@pytest.mark.parametrize("variant", ["uniform", "mutated"])
def test_pair_16384(ctx, oracle, variant):
    if variant == "uniform":
        x, y = gen.pair_uniform(16384, 16384, 4, seed=77)
    else:
        x, y = gen.pair_mutated(16384, 4, seed=78)
    check_pair(ctx, oracle, x, y)


@pytest.mark.parametrize("sigma", [20, 256])
def test_pair_large_alphabets(ctx, oracle, sigma):
    x, y = gen.pair_uniform(5000, 7000, sigma, seed=sigma)
    check_pair(ctx, oracle, x, y)


def test_capacity_error(ctx):
    from paper_1306_4627_gb300 import lcs
    with pytest.raises(lcs.LCSError) as e:
        ctx.traceback(b"ACGTACGT", b"ACGTTTTT", out_cap=2)
    assert e.value.code == lcs.ERR_CAPACITY


# ---- full-size workloads ---------------------------------------------------------------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("variant", ["uniform", "mutated"])
def test_full_pair_65536_traceback(ctx, oracle, variant):
    """m = n = 65536 DNA with traceback (1-bit bitmap of 537 MB), the single-pair benchmark size; exact vs oracle."""
    if variant == "uniform":
        x, y = gen.pair_uniform(65536, 65536, 4, seed=gen.BASE_SEED + 1)
    else:
        x, y = gen.pair_mutated(65536, 4, seed=gen.BASE_SEED + 1)
    s = ctx.traceback(x, y)
    assert s == oracle.lcs_traceback(x, y)
    assert ctx.length(x, y) == len(s)


@pytest.mark.slow
@pytest.mark.parametrize("sigma", [4, 20])
def test_full_length_262144_properties(ctx, oracle, sigma):
    """m = n = 262144, length only (multi-block wavefront, meet-in-the-middle). Properties that hold at any size:
    the split length equals the forward-only length of the traceback path, and is symmetric and reversal
    invariant; the traced string is a common subsequence of that length. Exact vs the oracle on a sub-problem
    that spans all column blocks (the first 4096 rows of X against all of Y)."""
    x, y = gen.pair_uniform(262144, 262144, sigma, seed=gen.BASE_SEED + 2)
    L = ctx.length(x, y)
    assert L == ctx.length(y, x)
    assert L == ctx.length(x[::-1].copy(), y[::-1].copy())
    s = ctx.traceback(x, y)
    assert len(s) == L
    assert oracle.is_subsequence(s, x.tobytes()) and oracle.is_subsequence(s, y.tobytes())
    xs = x[:4096].copy()
    assert ctx.length(xs, y) == oracle.lcs_length(xs, y)
    assert ctx.traceback(xs, y) == oracle.lcs_traceback(xs, y)


@pytest.mark.slow
@pytest.mark.parametrize("sigma", [4, 20])
def test_full_length_262144_oracle(ctx, oracle, sigma):
    """The full 262144^2 length against the oracle's recurrence, filled in column blocks on all host cores (the
    serial oracle takes minutes per pair; LCS_SERIAL_ORACLE=1 uses it)."""
    x, y = gen.pair_uniform(262144, 262144, sigma, seed=gen.BASE_SEED + 2)
    if os.environ.get("LCS_SERIAL_ORACLE") == "1":
        want = oracle.lcs_length(x, y)
    else:
        want = oracle.lcs_length_par(x, y, os.cpu_count() or 1)
    assert ctx.length(x, y) == want


@pytest.mark.parametrize("n", [(1 << 18), (1 << 18) + 1])
def test_alphabet_paths_around_one_block_limit(ctx, oracle, n):
    """Y up to 2^18 symbols: the alphabet in one block; longer: the multi-block presence. Both give the oracle's
    length and string; all 256 byte values present exercises the largest alphabet."""
    x, y = gen.pair_uniform(600, n, 256, seed=4100 + n % 7)
    assert ctx.length(x, y) == oracle.lcs_length(x, y)
    assert ctx.traceback(x, y) == oracle.lcs_traceback(x, y)


def test_reused_context_after_alphabet_change(ctx, oracle):
    """Consecutive calls on one context with different alphabets: no state of one call leaks into the next (the
    masks are rewritten in full, the scratch words cleared in the row-offset launch)."""
    for k, sigma in enumerate([256, 4, 20, 4, 256]):
        x, y = gen.pair_uniform(1500 + 17 * k, 3000 - 31 * k, sigma, seed=4200 + k)
        assert ctx.length(x, y) == oracle.lcs_length(x, y)
        assert ctx.traceback(x, y) == oracle.lcs_traceback(x, y)


# The shapes of the paper's Table 1 (parent length M rows, child length N columns). The tall ones make corridors of
# hundreds of columns (a thread per walker in the traceback); the square-ish ones make narrow corridors (a warp
# per walker).
TABLE1_SHAPES = [(10, 5), (100, 10), (200, 30), (500, 80), (800, 100), (1000, 150), (2000, 200), (5000, 200),
                 (5000, 400), (5000, 800), (5000, 1000), (10000, 1000), (10000, 1500)]


@pytest.mark.parametrize("k", range(len(TABLE1_SHAPES)))
def test_table1_shapes(ctx, oracle, k):
    m, n = TABLE1_SHAPES[k]
    x, y = gen.pair_uniform(m, n, 4, seed=gen.BASE_SEED + 100 + k)
    check_pair(ctx, oracle, x, y)


@pytest.mark.parametrize("m,n", [(20000, 3000), (3000, 20000), (12000, 12000)])
def test_wide_and_narrow_corridors(ctx, oracle, m, n):
    """Tall, wide and square pairs of related strings (Y a mutated piece of X, or the other way round)."""
    base = gen.random_string(77, max(m, n), gen.DNA)
    longer = base[: max(m, n)]
    shorter = gen.mutate(longer, seed=78, alphabet=gen.DNA, out_len=min(m, n))
    x, y = (longer, shorter) if m >= n else (shorter, longer)
    check_pair(ctx, oracle, x, y)


# ---- small pairs: the one-launch path and the general path --------------------------------------------------------
@pytest.fixture(scope="module")
def ctx_general():
    """A context whose small pairs take the general (multi-kernel) path as well (test hook LCS_NO_SMALL_PATH)."""
    from paper_1306_4627_gb300 import lcs
    os.environ["LCS_NO_SMALL_PATH"] = "1"
    try:
        c = lcs.Context(0)
    finally:
        del os.environ["LCS_NO_SMALL_PATH"]
    yield c
    c.close()


@pytest.mark.parametrize("m", [1, 9, 33, 1023, 1024, 1025])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 991, 992, 993])
def test_small_shapes_both_paths(ctx, ctx_general, oracle, m, n):
    """Around the limits of the one-launch path (m <= 1024, n <= 992; 992 = 31 words, so the carry for column n
    has its own word), on both paths."""
    x, y = gen.pair_uniform(m, n, 4, seed=5000 + 7 * m + n)
    check_pair(ctx, oracle, x, y)
    check_pair(ctx_general, oracle, x, y)


@pytest.mark.parametrize("sigma", [2, 20, 256])
def test_small_path_alphabets_and_related(ctx, ctx_general, oracle, sigma):
    alpha = {2: b"AB", 20: gen.PROTEIN, 256: gen.BYTES}[sigma]
    x = gen.random_string(6000 + sigma, 700, alpha)
    y = gen.mutate(x, seed=6001 + sigma, alphabet=alpha, out_len=640)
    for c in (ctx, ctx_general):
        check_pair(c, oracle, x, y)
        check_pair(c, oracle, y, x)


@pytest.mark.parametrize("m,n,sigma", [(2048, 2048, 4), (3001, 1500, 20), (1200, 5000, 256), (70000, 300, 4)])
def test_repeated_arguments_replay_a_graph(ctx, oracle, m, n, sigma):
    """Calls that repeat the previous call's arguments: the second one captures its launches as a CUDA graph and
    later ones replay it. New strings written into the same device buffers between calls, four traceback calls in a
    row, then four length calls in a row, then host-buffer calls of one shape; every result equals the oracle's."""
    import torch
    d = torch.device("cuda", 0)
    dx = torch.empty(m, dtype=torch.uint8, device=d)
    dy = torch.empty(n, dtype=torch.uint8, device=d)
    out = torch.zeros(min(m, n), dtype=torch.uint8, device=d)
    out_len = torch.zeros(1, dtype=torch.int64, device=d)
    pairs = [gen.pair_uniform(m, n, sigma, seed=7700 + 10 * k + sigma) for k in range(4)]
    for x, y in pairs:
        dx.copy_(torch.from_numpy(x))
        dy.copy_(torch.from_numpy(y))
        ctx.traceback_dev(dx, dy, out, out_len)
        ctx.sync()
        L = int(out_len.item())
        assert bytes(out[:L].cpu().numpy()) == oracle.lcs_traceback(x, y)
    for x, y in pairs:
        dx.copy_(torch.from_numpy(x))
        dy.copy_(torch.from_numpy(y))
        ctx.length_dev(dx, dy, out_len)
        ctx.sync()
        assert int(out_len.item()) == oracle.lcs_length(x, y)
    for x, y in pairs[:3]:
        assert ctx.traceback(x, y) == oracle.lcs_traceback(x, y)


def test_direct_launches_match_replayed_graph(oracle):
    """The same repeated calls on a context that never captures (LCS_NO_PAIR_GRAPH=1) give the same results."""
    from paper_1306_4627_gb300 import lcs
    os.environ["LCS_NO_PAIR_GRAPH"] = "1"
    try:
        direct = lcs.Context(0)
    finally:
        del os.environ["LCS_NO_PAIR_GRAPH"]
    pairs = [gen.pair_uniform(4000, 3000, 4, seed=7800 + k) for k in range(3)]
    with lcs.Context(0) as graphed:
        for x, y in pairs:
            want = oracle.lcs_traceback(x, y)
            assert direct.traceback(x, y) == want
            assert graphed.traceback(x, y) == want
        for x, y in pairs:
            assert direct.length(y, x) == graphed.length(y, x) == oracle.lcs_length(x, y)
    direct.close()


def test_segment_geometries_agree(oracle):
    """Small traceback pairs walk segments of 8 row-blocks and up (the fill snapshots every 8 row-blocks); a context
    with LCS_NO_DENSE_SNAP=1 keeps segments of 32 row-blocks and up. Both give the oracle's string."""
    from paper_1306_4627_gb300 import lcs
    os.environ["LCS_NO_DENSE_SNAP"] = "1"
    try:
        sparse = lcs.Context(0)
    finally:
        del os.environ["LCS_NO_DENSE_SNAP"]
    with lcs.Context(0) as dense:
        for k, (m, n, sigma) in enumerate([(2048, 2048, 4), (1000, 1500, 20), (5000, 400, 4), (8192, 2048, 4),
                                           (3001, 3001, 256), (700, 4000, 4)]):
            x, y = gen.pair_uniform(m, n, sigma, seed=7900 + k)
            want = oracle.lcs_traceback(x, y)
            assert dense.traceback(x, y) == want, (m, n)
            assert sparse.traceback(x, y) == want, (m, n)
    sparse.close()


def test_profiled_repeated_calls_replay_with_stage_times(oracle):
    """With stage timing on, repeated calls replay a graph that records the stage events: every call's result equals
    the oracle's, and every call's profile has its fill and traceback stages inside its total."""
    import torch
    from paper_1306_4627_gb300 import lcs
    d = torch.device("cuda", 0)
    m, n = 3000, 2500
    dx = torch.empty(m, dtype=torch.uint8, device=d)
    dy = torch.empty(n, dtype=torch.uint8, device=d)
    out = torch.zeros(min(m, n), dtype=torch.uint8, device=d)
    out_len = torch.zeros(1, dtype=torch.int64, device=d)
    with lcs.Context(0) as ctx:
        ctx.set_profiling(True)
        for k in range(4):
            x, y = gen.pair_uniform(m, n, 4, seed=8100 + k)
            dx.copy_(torch.from_numpy(x))
            dy.copy_(torch.from_numpy(y))
            ctx.traceback_dev(dx, dy, out, out_len)
            p = ctx.last_profile()
            ctx.sync()
            L = int(out_len.item())
            assert bytes(out[:L].cpu().numpy()) == oracle.lcs_traceback(x, y)
            assert p["fill_ms"] > 0 and p["trace_ms"] > 0 and p["prep_ms"] >= 0
            assert p["fill_ms"] + p["trace_ms"] <= p["total_ms"] * 1.001
            assert p["cells"] == m * n
        ctx.set_profiling(False)
