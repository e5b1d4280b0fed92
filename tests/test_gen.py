"""The seeded input generators: determinism, published splitmix64 values, and the workload distributions."""

import numpy as np

from paper_1306_4627_gb300 import gen


def test_splitmix64_published_values():
    # splitmix64 with state 0: the first outputs of the reference sequence (Vigna's splitmix64.c, seed 0).
    v = gen.splitmix64(0, 3)
    assert [int(a) for a in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_deterministic_and_seed_sensitive():
    a = gen.pair_uniform(1000, 900, 4, seed=3)
    b = gen.pair_uniform(1000, 900, 4, seed=3)
    c = gen.pair_uniform(1000, 900, 4, seed=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    assert len(a[0]) == 1000 and len(a[1]) == 900


def test_uniform_symbol_frequencies():
    x = gen.random_string(17, 200000, gen.DNA)
    counts = np.array([(x == s).sum() for s in gen.DNA])
    assert set(np.unique(x).tolist()) == set(gen.DNA)
    assert np.all(np.abs(counts / 200000 - 0.25) < 0.005)
    z = gen.random_string(18, 256 * 400, gen.BYTES)
    assert len(np.unique(z)) == 256


def test_mutation_rates():
    x = gen.random_string(5, 200000, gen.DNA)
    y = gen.mutate(x, 6, gen.DNA)  # cut/extended to len(x)
    assert len(y) == len(x)
    # with no indels the substitution rate is visible position by position
    ys = gen.mutate(x, 7, gen.DNA, p_del=0.0, p_ins=0.0, p_sub=0.10)
    diff = (ys != x).mean()
    assert abs(diff - 0.10) < 0.005
    # substitutions always change the symbol
    yd = gen.mutate(x, 8, gen.DNA, p_del=0.0, p_ins=0.0, p_sub=1.0)
    assert np.all(yd != x)
    # deletion-only shortens by about p_del before the final extension
    yl = gen.mutate(x, 9, gen.DNA, p_del=0.02, p_ins=0.0, p_sub=0.0, out_len=10**7)
    assert len(yl) == 10**7


def test_loguniform_lengths_and_batch():
    v = gen.loguniform_lengths(1, 100000, 64, 4096)
    assert v.min() >= 64 and v.max() <= 4096
    med = np.median(v)
    assert abs(np.log(med) - 0.5 * (np.log(64) + np.log(4096))) < 0.05
    pairs = gen.batch_pairs(count=200)
    assert len(pairs) == 200
    sig4 = sum(1 for x, y in pairs if set(np.unique(np.concatenate([x, y])).tolist()) <= set(gen.DNA))
    assert 90 <= sig4 <= 110


def test_serve_stream():
    reqs = gen.serve_requests(rate=1000.0, count=2000)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 2000 - 1e-3) < 1e-4
    tb = np.mean([r["traceback"] for r in reqs])
    assert abs(tb - 0.2) < 0.03
    assert {r["sigma"] for r in reqs} == {4, 20, 256}
