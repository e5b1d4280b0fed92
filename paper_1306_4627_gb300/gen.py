"""Seeded synthetic inputs for the LCS workloads (shared by the CUDA path's tests/bench and the oracle tests).

This module holds random-number generation and string assembly only: none of the LCS arithmetic lives here, so
that the CPU oracle and the CUDA path can both draw inputs from it without sharing any of the method's code.

Every stream is splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
state_k = seed + (k + 1) * 0x9E3779B97F4A7C15 (mod 2^64), followed by the published 64-bit finaliser. Streams are
separated by mixing a stream tag into the seed, so every draw is a pure function of (seed, tag, index) and the
same inputs come out on any machine and in any order of generation.

The paper (§I, §II) motivates LCS with DNA strands over {A, C, G, T} and describes its parent/child strings only by
their lengths (its Table 1 gives (M, N) shapes and no contents), so every input here is synthetic:
  * uniform i.i.d. symbols over a named alphabet (DNA, the 20 amino-acid letters, or all 256 byte values);
  * a mutated copy (substitutions, single-symbol insertions and deletions) for related-string workloads;
  * log-uniform lengths and Poisson arrival times for batched and served workloads.
"""

from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)

DNA = b"ACGT"
PROTEIN = b"ACDEFGHIKLMNPQRSTVWY"
BYTES = bytes(range(256))
ALPHABETS = {4: DNA, 20: PROTEIN, 256: BYTES}

# Base seed of every named workload; a workload adds its own small offset.
BASE_SEED = 0x13064627

# Stream tags (arbitrary distinct constants) so that different uses of one seed never share draws.
_TAG_X, _TAG_Y, _TAG_MUT_U, _TAG_MUT_SYM, _TAG_EXT = 0x11, 0x22, 0x33, 0x44, 0x55
_TAG_LEN_M, _TAG_LEN_N, _TAG_SHUF, _TAG_ARR, _TAG_SIG, _TAG_TB = 0x66, 0x77, 0x88, 0x99, 0xAA, 0xBB


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
        return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, tag: int) -> int:
    """Seed of an independent sub-stream: the splitmix64 finaliser applied to seed ^ (tag * golden)."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(tag) * GOLDEN)
    return int(_mix(np.array([s], dtype=np.uint64))[0])


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws start .. start+count-1 of the splitmix64 sequence for `seed` (uint64 array)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN
    return _mix(state)


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def below(seed: int, count: int, bound: int) -> np.ndarray:
    """Integers in [0, bound) by multiply-shift of the high 32 bits (bound <= 2^32)."""
    hi = splitmix64(seed, count) >> np.uint64(32)
    return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


def random_string(seed: int, length: int, alphabet: bytes) -> np.ndarray:
    """`length` symbols drawn i.i.d. uniform from `alphabet`, as a uint8 array."""
    table = np.frombuffer(alphabet, dtype=np.uint8)
    return table[below(seed, length, len(alphabet))]


def mutate(x: np.ndarray, seed: int, alphabet: bytes, p_del: float = 0.02, p_ins: float = 0.02,
           p_sub: float = 0.10, out_len: int | None = None) -> np.ndarray:
    """A related copy of `x`: walk x; per position draw u: u < p_del deletes x_i; u < p_del+p_ins inserts a uniform
    symbol before x_i and keeps x_i; u < p_del+p_ins+p_sub replaces x_i by a uniform *different* symbol; otherwise
    x_i is kept. The result is then cut, or extended with uniform symbols, to `out_len` (default len(x))."""
    m = len(x)
    sig = len(alphabet)
    table = np.frombuffer(alphabet, dtype=np.uint8)
    lut = np.full(256, 0, dtype=np.int64)
    lut[table] = np.arange(sig)
    u = uniform01(stream_seed(seed, _TAG_MUT_U), m)
    draw = below(stream_seed(seed, _TAG_MUT_SYM), m, sig)
    other = below(stream_seed(seed, _TAG_MUT_SYM + 1), m, max(sig - 1, 1))
    a_del, a_ins, a_sub = p_del, p_del + p_ins, p_del + p_ins + p_sub
    keep = u >= a_del
    ins = (u >= a_del) & (u < a_ins)
    sub = (u >= a_ins) & (u < a_sub)
    xi = lut[x]
    body = np.where(sub, table[(xi + 1 + other) % sig], x)
    # Assemble: for each kept position, an optional inserted symbol followed by the (possibly substituted) symbol.
    counts = keep.astype(np.int64) + ins.astype(np.int64)
    out = np.empty(int(counts.sum()), dtype=np.uint8)
    ends = np.cumsum(counts)
    pos_body = ends[keep] - 1
    out[pos_body] = body[keep]
    pos_ins = ends[ins] - 2
    out[pos_ins] = table[draw[ins]]
    target = m if out_len is None else out_len
    if len(out) >= target:
        return out[:target].copy()
    ext = random_string(stream_seed(seed, _TAG_EXT), target - len(out), alphabet)
    return np.concatenate([out, ext])


def loguniform_lengths(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """floor(exp(U(ln lo, ln hi))), clipped to [lo, hi]."""
    u = uniform01(seed, count)
    v = np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    return np.clip(v, lo, hi)


# ---------------------------------------------------------------------------------------------------------------
# Named workloads (sizes and distributions of the single-pair, long-pair, batched and served LCS workloads)
# ---------------------------------------------------------------------------------------------------------------

def pair_uniform(m: int, n: int, sigma: int = 4, seed: int = BASE_SEED) -> tuple[np.ndarray, np.ndarray]:
    """Independent uniform strings X (length m) and Y (length n) over the sigma-letter alphabet."""
    alpha = ALPHABETS[sigma]
    return (random_string(stream_seed(seed, _TAG_X), m, alpha), random_string(stream_seed(seed, _TAG_Y), n, alpha))


def pair_mutated(n: int, sigma: int = 4, seed: int = BASE_SEED) -> tuple[np.ndarray, np.ndarray]:
    """X uniform of length n; Y = X with 10% substitutions, 2% insertions and 2% deletions, cut/extended to n."""
    alpha = ALPHABETS[sigma]
    x = random_string(stream_seed(seed, _TAG_X), n, alpha)
    return x, mutate(x, stream_seed(seed, _TAG_Y), alpha, out_len=n)


def batch_pairs(count: int = 10000, lo: int = 64, hi: int = 4096, sigmas: tuple[int, ...] = (4, 20),
                seed: int = BASE_SEED + 3) -> list[tuple[np.ndarray, np.ndarray]]:
    """`count` independent pairs; m and n drawn independently log-uniform in [lo, hi]; the first half of the pairs
    use sigmas[0] and the second half sigmas[1]; the order is then shuffled by the seed."""
    ms = loguniform_lengths(stream_seed(seed, _TAG_LEN_M), count, lo, hi)
    ns = loguniform_lengths(stream_seed(seed, _TAG_LEN_N), count, lo, hi)
    order = np.argsort(splitmix64(stream_seed(seed, _TAG_SHUF), count), kind="stable")
    pairs = []
    for k in range(count):
        sig = sigmas[0] if k < count // 2 else sigmas[-1]
        pairs.append(pair_uniform(int(ms[k]), int(ns[k]), sig, seed=stream_seed(seed, 0x1000 + k)))
    return [pairs[int(i)] for i in order]


def serve_requests(rate: float, count: int, lo: int = 32, hi: int = 65536, p_traceback: float = 0.2,
                   seed: int = BASE_SEED + 4) -> list[dict]:
    """A Poisson request stream: arrival times (seconds, exponential gaps at `rate` per second), m and n
    log-uniform in [lo, hi], alphabet 4, 20 or 256 with equal probability, traceback with probability
    p_traceback (length only otherwise)."""
    gaps = -np.log1p(-uniform01(stream_seed(seed, _TAG_ARR), count)) / rate
    t = np.cumsum(gaps)
    ms = loguniform_lengths(stream_seed(seed, _TAG_LEN_M), count, lo, hi)
    ns = loguniform_lengths(stream_seed(seed, _TAG_LEN_N), count, lo, hi)
    sig = np.array([4, 20, 256])[below(stream_seed(seed, _TAG_SIG), count, 3)]
    tb = uniform01(stream_seed(seed, _TAG_TB), count) < p_traceback
    out = []
    for k in range(count):
        x, y = pair_uniform(int(ms[k]), int(ns[k]), int(sig[k]), seed=stream_seed(seed, 0x2000 + k))
        out.append({"t": float(t[k]), "x": x, "y": y, "sigma": int(sig[k]), "traceback": bool(tb[k])})
    return out
