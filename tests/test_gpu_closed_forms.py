"""CUDA path against answers the mathematics fixes exactly (and against the oracle where it is fast enough).

* LCS(a^p, a^q) = min(p, q), the string a^min(p, q).
* LCS(a^p b^q, b^r a^s) = max(min(p, s), min(q, r)); the string is fixed by Print-LCS's tie-break (§I.D), see
  runs_lcs_string (pinned against the oracle on every small case in test_oracle_pins.py).
* X = a^m against Y = a b^(n-1): the first row's add carries from column 1 through every later column, so the
  carry crosses every warp and block boundary of the row in one row (and Y = b^(n-1) a does the same in the table
  of the reversed strings that length-only calls fill at the same time). LCS = 1, the string "a".
Widths 4095, 4097 and 70000 straddle the 4096-column block of the fill and span 18 blocks.
"""

import itertools

import pytest

from tests.test_oracle_pins import runs_lcs_string

pytestmark = pytest.mark.gpu

SIZES = [4095, 4097, 70000]


@pytest.fixture(scope="module")
def ctx():
    from paper_1306_4627_gb300 import lcs
    c = lcs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("p,q", list(itertools.product([1] + SIZES, SIZES)))
def test_one_symbol_runs(ctx, oracle, p, q):
    x, y = b"A" * p, b"A" * q
    assert ctx.length(x, y) == min(p, q)
    assert ctx.traceback(x, y) == b"A" * min(p, q)
    if p * q <= 1 << 25:
        assert oracle.lcs_traceback(x, y) == b"A" * min(p, q)


@pytest.mark.parametrize("p,q,r,s", list(itertools.product(SIZES, repeat=4)))
def test_two_runs_closed_form(ctx, oracle, p, q, r, s):
    x = b"A" * p + b"B" * q
    y = b"B" * r + b"A" * s
    want = runs_lcs_string(p, q, r, s)
    assert ctx.length(x, y) == len(want) == max(min(p, s), min(q, r))
    assert ctx.length(y, x) == len(want)
    assert ctx.traceback(x, y) == want
    if max(p, q, r, s) < 70000:  # at most 8194 x 8194 cells: the oracle as well
        assert oracle.lcs_length(x, y) == len(want)
        assert oracle.lcs_traceback(x, y) == want


@pytest.mark.parametrize("m", [1, 8, 1000, 70000])
@pytest.mark.parametrize("n", [12289, 20000, 70000])
def test_carry_ripples_through_every_block(ctx, oracle, m, n):
    x = b"A" * m
    for y in (b"A" + b"B" * (n - 1), b"B" * (n - 1) + b"A"):
        assert ctx.length(x, y) == 1
        assert ctx.length(y, x) == 1
        assert ctx.traceback(x, y) == b"A"
        if m * n <= 1 << 25:
            assert oracle.lcs_traceback(x, y) == b"A"
