"""Python face of the CPU oracle — TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may import this module. It shares
no code with the CUDA library and never calls it.

* `lcs_length`, `lcs_traceback`, `lcs_tables`: ctypes calls into `lcs_oracle.c`, the literal LCS-length (§I.C)
  and Print-LCS (§I.D) of Dash & Nayak with the paper's tie-break (UP when c[i-1,j] >= c[i,j-1]).
* `lcs_traceback_par`, `lcs_length_par`: `lcs_oracle_par.c`, the same fill split into column blocks over host
  threads (the paper's parallel algorithm, §II.A-B); a CPU baseline for the paper's own experiment (Table 1), and
  the length at sizes the serial loop takes minutes for.
* `brute_force`: the exhaustive method the paper contrasts with dynamic programming (§I and §I.A): enumerate all
  2^m subsequences of X, keep those that are also subsequences of Y, and return the largest length together with
  the set of all common subsequences of that length. Exponential; only for m <= 16.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcs_oracle.c")
_SRC_PAR = os.path.join(_HERE, "lcs_oracle_par.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblcs_oracle.so")
_lock = threading.Lock()
_lib = None

DIAG, UP, LEFT = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile lcs_oracle.c and lcs_oracle_par.c with gcc into oracle/_build/liblcs_oracle.so (plain -O2, no
    tuning)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_PAR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-pthread", "-shared", "-fPIC", "-o", tmp, _SRC,
                               _SRC_PAR])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p, u64 = ctypes.POINTER(ctypes.c_uint8), ctypes.c_uint64
            lib.oracle_lcs_length.argtypes = [u8p, u64, u8p, u64]
            lib.oracle_lcs_length.restype = u64
            lib.oracle_lcs_traceback.argtypes = [u8p, u64, u8p, u64, u8p, u64, ctypes.POINTER(u64)]
            lib.oracle_lcs_traceback.restype = ctypes.c_int
            lib.oracle_lcs_tables.argtypes = [u8p, u64, u8p, u64, ctypes.POINTER(ctypes.c_uint32), u8p]
            lib.oracle_lcs_tables.restype = ctypes.c_int
            lib.oracle_lcs_traceback_par.argtypes = [u8p, u64, u8p, u64, u8p, u64, ctypes.POINTER(u64), ctypes.c_int]
            lib.oracle_lcs_traceback_par.restype = ctypes.c_int
            lib.oracle_lcs_length_par.argtypes = [u8p, u64, u8p, u64, ctypes.c_int]
            lib.oracle_lcs_length_par.restype = u64
            _lib = lib
    return _lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    return np.ascontiguousarray(a, dtype=np.uint8)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def lcs_length(x, y) -> int:
    """c[m, n] of LCS-length (§I.C)."""
    x, y = _u8(x), _u8(y)
    v = _load().oracle_lcs_length(_ptr(x), len(x), _ptr(y), len(y))
    if v == 2**64 - 1:
        raise MemoryError("oracle: out of memory")
    return int(v)


def lcs_traceback(x, y) -> bytes:
    """The LCS that Print-LCS (§I.D) emits from the b table of LCS-length (§I.C)."""
    x, y = _u8(x), _u8(y)
    cap = max(1, min(len(x), len(y)))
    out = np.zeros(cap, dtype=np.uint8)
    n_out = ctypes.c_uint64(0)
    rc = _load().oracle_lcs_traceback(_ptr(x), len(x), _ptr(y), len(y), _ptr(out), cap, ctypes.byref(n_out))
    if rc == -1:
        raise MemoryError("oracle: out of memory")
    if rc != 0:
        raise RuntimeError(f"oracle_lcs_traceback failed: {rc}")
    return out[: n_out.value].tobytes()


def lcs_tables(x, y) -> tuple[np.ndarray, np.ndarray]:
    """(c, b): c of shape (m+1, n+1) and b of shape (m, n) with values DIAG=1, UP=2, LEFT=3 (§I.C)."""
    x, y = _u8(x), _u8(y)
    m, n = len(x), len(y)
    c = np.zeros((m + 1) * (n + 1), dtype=np.uint32)
    b = np.zeros(max(1, m * n), dtype=np.uint8)
    _load().oracle_lcs_tables(_ptr(x), m, _ptr(y), n, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _ptr(b))
    return c.reshape(m + 1, n + 1), b[: m * n].reshape(m, n)


def lcs_traceback_par(x, y, threads: int) -> bytes:
    """The same LCS as lcs_traceback, with the table filled by `threads` host threads in column blocks (the
    paper's parallel algorithm, §II.A-B). Returns the string; its length is c[m, n]."""
    x, y = _u8(x), _u8(y)
    cap = max(1, min(len(x), len(y)))
    out = np.zeros(cap, dtype=np.uint8)
    n_out = ctypes.c_uint64(0)
    rc = _load().oracle_lcs_traceback_par(_ptr(x), len(x), _ptr(y), len(y), _ptr(out), cap, ctypes.byref(n_out),
                                          int(threads))
    if rc == -1:
        raise MemoryError("oracle: out of memory")
    if rc != 0:
        raise RuntimeError(f"oracle_lcs_traceback_par failed: {rc}")
    return out[: n_out.value].tobytes()


def lcs_length_par(x, y, threads: int) -> int:
    """c[m, n] with the fill split into column blocks over `threads` host threads (§II.A-B), length only."""
    x, y = _u8(x), _u8(y)
    v = _load().oracle_lcs_length_par(_ptr(x), len(x), _ptr(y), len(y), int(threads))
    if v == 2**64 - 1:
        raise MemoryError("oracle: out of memory")
    return int(v)


def is_subsequence(z: bytes, s: bytes) -> bool:
    """True when z can be obtained from s by deleting symbols (greedy left-to-right scan)."""
    it = iter(s)
    return all(ch in it for ch in z)


def brute_force(x: bytes, y: bytes) -> tuple[int, set[bytes]]:
    """Exhaustive LCS (§I, §I.A): try every subset of X's positions, longest first; return (length, all LCSs)."""
    x, y = bytes(x), bytes(y)
    m = len(x)
    if m > 16:
        raise ValueError("brute force is limited to m <= 16")
    by_size: dict[int, list[int]] = {}
    for mask in range(1 << m):
        by_size.setdefault(bin(mask).count("1"), []).append(mask)
    for size in range(m, -1, -1):
        found = set()
        for mask in by_size.get(size, []):
            z = bytes(x[k] for k in range(m) if mask >> k & 1)
            if z not in found and is_subsequence(z, y):
                found.add(z)
        if found:
            return size, found
    return 0, {b""}
