"""Pins for the CPU oracle against facts fixed outside it (CPU only).

* Brute force (paper §I, §I.A): the exhaustive search over all 2^m subsequences of X gives the exact length and the
  set of all LCSs; the oracle's length must equal it and its string must be one of the set.
* Hand-derived worked examples of LCS-length / Print-LCS with the paper's tie-break (§I.C-D), including full c and
  b tables (tests/golden/clrs_tiebreak.txt).
* The c table, filled by the oracle, against brute-force lengths of every pair of prefixes: c[i,j] is by definition
  the LCS length of X_i and Y_j (§I.B).
* Closed forms and invariants that follow from the definition and the optimal-substructure theorem (§I.A).
"""

import os
import random

import numpy as np
import pytest

from tests.conftest import read_golden_cases
from paper_1306_4627_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "clrs_tiebreak.txt")


def rand_str(rng, length, alphabet):
    return bytes(rng.choice(alphabet) for _ in range(length))


# ----------------------------------------------------------------------------------------------------------------
# Brute force
# ----------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("alphabet", [b"AB", b"ABC", b"ACGT", gen.PROTEIN])
def test_length_and_string_vs_brute_force(oracle, alphabet):
    rng = random.Random(1306 + len(alphabet))
    for _ in range(60):
        x = rand_str(rng, rng.randint(0, 10), alphabet)
        y = rand_str(rng, rng.randint(0, 12), alphabet)
        L, lcs_set = oracle.brute_force(x, y)
        assert oracle.lcs_length(x, y) == L, (x, y)
        s = oracle.lcs_traceback(x, y)
        assert len(s) == L and s in lcs_set, (x, y, s, lcs_set)


def test_brute_force_m16(oracle):
    rng = random.Random(4627)
    for _ in range(3):
        x = rand_str(rng, 16, b"ACGT")
        y = rand_str(rng, 20, b"ACGT")
        L, lcs_set = oracle.brute_force(x, y)
        assert oracle.lcs_length(x, y) == L
        assert oracle.lcs_traceback(x, y) in lcs_set


def test_c_table_is_prefix_lcs(oracle):
    """c[i,j] = |LCS(X_i, Y_j)| for every prefix pair (definition of c in §I.B), checked by brute force."""
    rng = random.Random(7)
    for _ in range(6):
        x = rand_str(rng, rng.randint(1, 7), b"ACG")
        y = rand_str(rng, rng.randint(1, 8), b"ACG")
        c, b = oracle.lcs_tables(x, y)
        for i in range(len(x) + 1):
            for j in range(len(y) + 1):
                assert c[i, j] == oracle.brute_force(x[:i], y[:j])[0], (x, y, i, j)


def test_b_table_rule(oracle):
    """b is DIAG exactly on matches; on a mismatch UP exactly when c[i-1,j] >= c[i,j-1] (§I.C)."""
    rng = random.Random(11)
    for _ in range(20):
        x = rand_str(rng, rng.randint(1, 30), b"ACGT")
        y = rand_str(rng, rng.randint(1, 30), b"ACGT")
        c, b = oracle.lcs_tables(x, y)
        for i in range(1, len(x) + 1):
            for j in range(1, len(y) + 1):
                if x[i - 1] == y[j - 1]:
                    assert b[i - 1, j - 1] == oracle.DIAG
                elif c[i - 1, j] >= c[i, j - 1]:
                    assert b[i - 1, j - 1] == oracle.UP
                else:
                    assert b[i - 1, j - 1] == oracle.LEFT


# ----------------------------------------------------------------------------------------------------------------
# Hand-derived worked examples (tie-break direction)
# ----------------------------------------------------------------------------------------------------------------

def test_golden_tiebreak_cases(oracle):
    cases, _ = read_golden_cases(GOLDEN)
    assert len(cases) >= 5
    for x, y, L, s in cases:
        assert oracle.lcs_length(x, y) == L, (x, y)
        assert oracle.lcs_traceback(x, y) == s, (x, y)


def test_golden_tables(oracle):
    _, tables = read_golden_cases(GOLDEN)
    sym = {"D": oracle.DIAG, "U": oracle.UP, "L": oracle.LEFT}
    assert tables
    for (x, y), t in tables.items():
        c, b = oracle.lcs_tables(x, y)
        assert c.tolist() == t["c"]
        assert b.tolist() == [[sym[v] for v in row] for row in t["b"]]


# ----------------------------------------------------------------------------------------------------------------
# Closed forms and invariants
# ----------------------------------------------------------------------------------------------------------------

def test_empty(oracle):
    assert oracle.lcs_length(b"", b"ACGT") == 0
    assert oracle.lcs_length(b"ACGT", b"") == 0
    assert oracle.lcs_traceback(b"", b"") == b""
    assert oracle.lcs_traceback(b"A", b"") == b""


def test_identical(oracle):
    x, _ = gen.pair_uniform(700, 1, 4, seed=5)
    x = x.tobytes()
    assert oracle.lcs_length(x, x) == len(x)
    assert oracle.lcs_traceback(x, x) == x


def test_disjoint_alphabets(oracle):
    x = bytes(gen.random_string(1, 300, b"AC"))
    y = bytes(gen.random_string(2, 257, b"GT"))
    assert oracle.lcs_length(x, y) == 0
    assert oracle.lcs_traceback(x, y) == b""


def test_subsequence_gives_full_length(oracle):
    y = gen.random_string(3, 900, gen.DNA)
    keep = gen.uniform01(4, 900) < 0.6
    x = y[keep].tobytes()
    assert oracle.lcs_length(x, y.tobytes()) == len(x)
    assert oracle.lcs_traceback(x, y.tobytes()) == x


def test_runs_closed_form(oracle):
    """LCS(a^p, a^q) = min(p, q); LCS(a^p b^q, b^r a^s) = max(min(p, s), min(q, r))."""
    for p, q in [(0, 5), (3, 3), (7, 2), (40, 65)]:
        assert oracle.lcs_length(b"A" * p, b"A" * q) == min(p, q)
    for p, q, r, s in [(3, 4, 5, 2), (10, 1, 1, 10), (6, 6, 6, 6), (0, 3, 2, 9), (33, 31, 32, 34)]:
        x = b"A" * p + b"B" * q
        y = b"B" * r + b"A" * s
        assert oracle.lcs_length(x, y) == max(min(p, s), min(q, r))


def runs_lcs_string(p, q, r, s):
    """The string Print-LCS (§I.D) traces for X = a^p b^q, Y = b^r a^s. A common subsequence is a^k or b^k (X has
    its a's first, Y its b's), so with A = min(p, s) and B = min(q, r) the LCS is unique unless A = B. On a tie the
    walk starts at (m, n) on a mismatch (x_m = b, y_n = a) whose up and left neighbours both hold A, so it steps
    up; down column n every neighbour pair stays tied or favours up until row p, where x_p = y_n = a, and from there
    it matches a's on the diagonal: a^A."""
    A, B = min(p, s), min(q, r)
    return b"A" * A if A >= B else b"B" * B


def test_runs_closed_form_strings(oracle):
    """The traced string of the two-run closed form, every (p, q, r, s) in 0..5 (ties included), and the carry that
    ripples along the whole first row: X = a^m against Y = a b^(n-1) (and the mirror image)."""
    for p in range(6):
        for q in range(6):
            for r in range(6):
                for s in range(6):
                    x = b"A" * p + b"B" * q
                    y = b"B" * r + b"A" * s
                    assert oracle.lcs_traceback(x, y) == runs_lcs_string(p, q, r, s), (p, q, r, s)
    for m, n in [(1, 1), (1, 70), (9, 70), (70, 3)]:
        assert oracle.lcs_traceback(b"A" * m, b"A" + b"B" * (n - 1)) == b"A"
        assert oracle.lcs_traceback(b"A" * m, b"B" * (n - 1) + b"A") == b"A"


def test_theorem_case1_append(oracle):
    """Optimal substructure case 1 (§I.A): if x_m = y_n the LCS is an LCS of the prefixes plus that symbol."""
    for seed in range(5):
        x, y = gen.pair_uniform(150 + seed, 170, 4, seed=seed)
        x, y = x.tobytes(), y.tobytes()
        for ch in b"AT":
            assert oracle.lcs_length(x + bytes([ch]), y + bytes([ch])) == oracle.lcs_length(x, y) + 1
            assert oracle.lcs_traceback(x + bytes([ch]), y + bytes([ch]))[-1] == ch


@pytest.mark.parametrize("sigma", [4, 20, 256])
def test_invariants_random(oracle, sigma):
    for seed in range(4):
        x, y = gen.pair_uniform(300 + 37 * seed, 260 + 41 * seed, sigma, seed=100 + seed)
        xb, yb = x.tobytes(), y.tobytes()
        L = oracle.lcs_length(xb, yb)
        assert L == oracle.lcs_length(yb, xb)                      # symmetric
        assert L == oracle.lcs_length(xb[::-1], yb[::-1])          # reversal
        assert L <= min(len(xb), len(yb))
        s = oracle.lcs_traceback(xb, yb)
        assert len(s) == L
        assert oracle.is_subsequence(s, xb) and oracle.is_subsequence(s, yb)
        # a bijection of the alphabet maps the LCS string symbol by symbol (equality is all the method uses)
        perm = np.random.default_rng(seed).permutation(256).astype(np.uint8)
        assert oracle.lcs_traceback(perm[x].tobytes(), perm[y].tobytes()) == perm[np.frombuffer(s, np.uint8)].tobytes()


def test_chvatal_sankoff_plausibility(oracle):
    """Plausibility only: for uniform DNA the ratio L/n approaches the Chvatal-Sankoff constant (about 0.654)."""
    x, y = gen.pair_uniform(4000, 4000, 4, seed=9)
    r = oracle.lcs_length(x, y) / 4000
    assert 0.62 < r < 0.67


def test_traceback_capacity_error(oracle):
    import ctypes
    lib = oracle._load()
    x = np.frombuffer(b"ACGTACGT", np.uint8)
    y = np.frombuffer(b"ACGTTTTT", np.uint8)
    out = np.zeros(2, np.uint8)
    n_out = ctypes.c_uint64(0)
    u8 = ctypes.POINTER(ctypes.c_uint8)
    rc = lib.oracle_lcs_traceback(x.ctypes.data_as(u8), 8, y.ctypes.data_as(u8), 8, out.ctypes.data_as(u8), 2,
                                  ctypes.byref(n_out))
    assert rc == -2 and n_out.value == 5


# ----------------------------------------------------------------------------------------------------------------
# The multi-threaded oracle (column blocks over host threads, §II.A-B) gives the serial oracle's results
# ----------------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("threads", [1, 2, 3, 5, 16])
def test_parallel_oracle_equals_serial(oracle, threads):
    rng = np.random.default_rng(31 + threads)
    for k in range(25):
        m = int(rng.integers(1, 300))
        n = int(rng.integers(1, 200))
        alpha = [b"AB", b"ACGT", bytes(range(20))][k % 3]
        x = bytes(rng.choice(list(alpha), m).astype(np.uint8))
        y = bytes(rng.choice(list(alpha), n).astype(np.uint8))
        assert oracle.lcs_traceback_par(x, y, threads) == oracle.lcs_traceback(x, y), (m, n)


def test_parallel_oracle_edges(oracle):
    assert oracle.lcs_traceback_par(b"", b"ACGT", 4) == b""
    assert oracle.lcs_traceback_par(b"A", b"A", 8) == b"A"  # more threads than columns
    x = b"ACGTTGCA" * 40
    assert oracle.lcs_traceback_par(x, x, 4) == x
    for x, y, L, s in read_golden_cases(GOLDEN)[0]:
        assert oracle.lcs_traceback_par(x, y, 3) == s


@pytest.mark.parametrize("threads", [1, 2, 7])
def test_parallel_length_oracle_equals_serial(oracle, threads):
    rng = np.random.default_rng(90 + threads)
    for k in range(20):
        m = int(rng.integers(1, 700))
        n = int(rng.integers(1, 400))
        alpha = [b"AB", b"ACGT", bytes(range(20))][k % 3]
        x = bytes(rng.choice(list(alpha), m).astype(np.uint8))
        y = bytes(rng.choice(list(alpha), n).astype(np.uint8))
        assert oracle.lcs_length_par(x, y, threads) == oracle.lcs_length(x, y), (m, n)
    assert oracle.lcs_length_par(b"", b"ACGT", 3) == 0
    assert oracle.lcs_length_par(b"ACGT" * 100, b"ACGT" * 100, 64) == 400  # more threads than needed
