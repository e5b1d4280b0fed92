"""Serving (continuous batching): every result equals the same request run alone; back-pressure, HBM admission
and bounded device waits report errors instead of hanging."""

import os
import random

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


def make_requests(count, seed, lo=32, hi=65536, tb_max=16384):
    """Requests shaped like the serving workload: m and n log-uniform in [lo, hi], alphabet 4, 20 or 256 with equal
    probability, a quarter of them with traceback (tracebacks drawn with both sides <= tb_max so that the oracle's
    full b table stays small)."""
    rng = random.Random(seed)
    reqs = []
    for k in range(count):
        sigma = rng.choice([4, 20, 256])
        tb = rng.random() < 0.25
        top = min(hi, tb_max) if tb else hi
        m = int(np.exp(rng.uniform(np.log(lo), np.log(top))))
        n = int(np.exp(rng.uniform(np.log(lo), np.log(top))))
        x, y = gen.pair_uniform(m, n, sigma, seed=10_000 + 7 * k + seed)
        reqs.append((x, y, tb))
    return reqs


def oracle_answer(oracle, x, y, tb):
    threads = min(16, os.cpu_count() or 1)
    if tb:
        s = oracle.lcs_traceback_par(x, y, threads) if len(x) * len(y) > 1 << 22 else oracle.lcs_traceback(x, y)
        return len(s), s
    L = oracle.lcs_length_par(x, y, threads) if len(x) * len(y) > 1 << 22 else oracle.lcs_length(x, y)
    return L, None


def test_mix_equals_alone_and_oracle(ctx, oracle):
    """Every request of a mixed stream (short and long pairs, all three alphabets, tracebacks of every alphabet)
    gives the oracle's length, and its string when a traceback was asked for, both in the mix and run alone."""
    from paper_1306_4627_gb300 import lcs
    reqs = make_requests(240, seed=1)
    assert any(tb and len(set(x.tolist())) > 20 for x, _, tb in reqs)  # a traceback over the 256-symbol alphabet
    srv = lcs.Server(ctx, max_batch=64)
    tickets = [srv.submit(x, y, traceback=tb) for x, y, tb in reqs]
    results = [srv.wait(t, timeout_s=120.0) for t in tickets]
    srv.close()
    for (x, y, tb), r in zip(reqs, results):
        L, s = oracle_answer(oracle, x, y, tb)
        assert r is not None and r["status"] == 0
        assert r["length"] == L, (len(x), len(y))
        assert ctx.length(x, y) == L
        if tb:
            assert r["lcs"] == s, (len(x), len(y))
            assert ctx.traceback(x, y) == s
        assert r["latency_s"] > 0


def test_poll_and_release(ctx):
    from paper_1306_4627_gb300 import lcs
    srv = lcs.Server(ctx)
    t = srv.submit(b"ACGTACGT", b"TTACG", traceback=True)
    r = srv.wait(t, timeout_s=30.0)
    assert r["length"] == 4 and r["lcs"] == b"ACGT"[:0] + r["lcs"] and len(r["lcs"]) == 4
    with pytest.raises(lcs.LCSError):
        srv.poll(t)  # released by wait()
    with pytest.raises(lcs.LCSError):
        srv.poll(987654321)
    t2 = srv.submit(b"", b"ACGT")
    assert srv.wait(t2, timeout_s=30.0)["length"] == 0
    srv.close()


def test_backpressure(ctx):
    from paper_1306_4627_gb300 import lcs
    srv = lcs.Server(ctx, max_queue=4)
    x, y = gen.pair_uniform(60000, 60000, 4, seed=3)
    codes, tickets = [], []
    for _ in range(40):
        rc, t = srv.try_submit(x, y)
        codes.append(rc)
        if rc == lcs.OK:
            tickets.append(t)
    assert lcs.ERR_BUSY in codes and lcs.OK in codes
    for t in tickets:
        assert srv.wait(t, timeout_s=120.0)["status"] == 0
    rc, t = srv.try_submit(b"AC", b"CA")
    assert rc == lcs.OK
    srv.wait(t, timeout_s=30.0)
    srv.close()


def test_hbm_admission(ctx):
    from paper_1306_4627_gb300 import lcs
    srv = lcs.Server(ctx, hbm_budget_bytes=96 << 20)
    x, y = gen.pair_uniform(65536, 65536, 4, seed=4)
    rc, _ = srv.try_submit(x, y, traceback=True)   # needs ~540 MB of bitmap: can never fit
    assert rc == lcs.ERR_NOMEM
    rc, t = srv.try_submit(x, y, traceback=False)  # length only needs no bitmap
    assert rc == lcs.OK
    xs, ys = gen.pair_uniform(8000, 8000, 4, seed=5)
    ts = [srv.submit(xs, ys, traceback=True) for _ in range(6)]  # each fits alone; they queue for the budget
    assert srv.wait(t, timeout_s=120.0)["length"] == ctx.length(x, y)
    want = ctx.traceback(xs, ys)
    for tt in ts:
        assert srv.wait(tt, timeout_s=120.0)["lcs"] == want
    srv.close()


def test_bounded_wait_reports_timeout():
    """A carry hand-off that is never published: the waiting warps give up after a short limit, the call returns
    LCS_ERR_TIMEOUT, and a fresh context computes correctly afterwards (no hang, no fault)."""
    from paper_1306_4627_gb300 import lcs
    x, y = gen.pair_uniform(3000, 20000, 4, seed=6)
    os.environ["LCS_SPIN_LIMIT"] = "4096"
    os.environ["LCS_DEBUG_DROP_HANDOFF"] = "1"
    try:
        bad = lcs.Context(0)
    finally:
        del os.environ["LCS_SPIN_LIMIT"]
        del os.environ["LCS_DEBUG_DROP_HANDOFF"]
    with pytest.raises(lcs.LCSError) as e:
        bad.length(x, y)
    assert e.value.code == lcs.ERR_TIMEOUT
    with pytest.raises(lcs.LCSError) as e:
        bad.traceback(x, y)
    assert e.value.code in (lcs.ERR_TIMEOUT, lcs.ERR_INTERNAL)
    bad.close()
    with lcs.Context(0) as good:
        assert good.length(x, y) == good.length(y, x)
