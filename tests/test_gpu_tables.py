"""lcs_tables: the full c and b tables of LCS-length (§I.C) from the GPU, cell by cell equal to the oracle's."""

import os

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


def test_tables_golden_textbook(ctx):
    _, tables = read_golden_cases(GOLDEN)
    sym = {"D": 1, "U": 2, "L": 3}
    for (x, y), t in tables.items():
        c, b = ctx.tables(x, y)
        assert c.tolist() == t["c"]
        assert b.tolist() == [[sym[v] for v in row] for row in t["b"]]


@pytest.mark.parametrize("m,n,sigma", [(1, 1, 4), (1, 200, 4), (200, 1, 4), (31, 33, 4), (64, 64, 20),
                                       (65, 127, 20), (300, 4095, 4), (513, 4097, 20), (129, 9000, 256),
                                       (1000, 1000, 4), (2049, 700, 256)])
def test_tables_vs_oracle(ctx, oracle, m, n, sigma):
    """Several row chunks and fill blocks, ragged last words, every alphabet size."""
    x, y = gen.pair_uniform(m, n, sigma, seed=7000 + m + 3 * n + sigma)
    c, b = ctx.tables(x, y)
    co, bo = oracle.lcs_tables(x, y)
    assert np.array_equal(c, co)
    assert np.array_equal(b, bo)


def test_tables_related_strings(ctx, oracle):
    x = gen.random_string(4242, 1500, gen.DNA)
    y = gen.mutate(x, seed=4243, alphabet=gen.DNA)
    c, b = ctx.tables(x, y)
    co, bo = oracle.lcs_tables(x, y)
    assert np.array_equal(c, co)
    assert np.array_equal(b, bo)
    assert int(c[-1, -1]) == ctx.length(x, y)


def test_tables_empty(ctx):
    c, b = ctx.tables(b"", b"ACGT")
    assert c.shape == (1, 5) and not c.any() and b.shape == (0, 4)
    c, b = ctx.tables(b"ACG", b"")
    assert c.shape == (4, 1) and not c.any() and b.shape == (3, 0)


def test_tables_dev_matches_host(ctx):
    import torch
    x, y = gen.pair_uniform(700, 900, 4, seed=77)
    c, b = ctx.tables(x, y)
    d = torch.device("cuda", 0)
    dx, dy = torch.from_numpy(x.copy()).to(d), torch.from_numpy(y.copy()).to(d)
    dc = torch.zeros(701 * 901, dtype=torch.int32, device=d)
    db = torch.zeros(700 * 900, dtype=torch.uint8, device=d)
    ctx.tables_dev(dx, dy, dc, db)
    ctx.sync()
    assert np.array_equal(dc.cpu().numpy().view(np.uint32).reshape(701, 901), c)
    assert np.array_equal(db.cpu().numpy().reshape(700, 900), b)
