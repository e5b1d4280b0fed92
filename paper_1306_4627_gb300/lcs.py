"""Thin Python binding of liblcs.so (include/lcs.h): argument marshalling only, every step runs in the library.

Functions keep the C names without the `lcs_` prefix. Host inputs are bytes, bytearray or uint8 numpy arrays;
"_dev" inputs are uint8 CUDA tensors (torch is used only for device memory and streams). When the library cannot
be loaded this module raises at import: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblcs.so")

OK, PENDING = 0, 1
ERR_INVALID, ERR_NOMEM, ERR_CAPACITY, ERR_BUSY, ERR_TIMEOUT, ERR_CUDA, ERR_INTERNAL = -1, -2, -3, -4, -5, -6, -7
TRACEBACK = 1

# Every function declared in include/lcs.h.
EXPORTS = (
    "lcs_strerror", "lcs_ctx_create", "lcs_ctx_destroy", "lcs_ctx_sync", "lcs_length", "lcs_length_dev",
    "lcs_traceback", "lcs_traceback_dev", "lcs_batch", "lcs_batch_dev", "lcs_batch_dev_hoff", "lcs_serve_create", "lcs_serve_submit",
    "lcs_serve_poll", "lcs_serve_wait", "lcs_result_release", "lcs_serve_destroy", "lcs_ctx_set_profiling",
    "lcs_ctx_last_profile", "lcs_tables", "lcs_tables_dev", "lcs_ctx_get_fill_config", "lcs_ctx_set_fill_config",
    "lcs_ctx_autotune_dev", "lcs_ctx_get_batch_config", "lcs_ctx_set_batch_config", "lcs_ctx_autotune_batch_dev",
    "lcs_probe_int_rate", "lcs_probe_step_floor", "lcs_probe_step_masks",
)


class LCSError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


class ServeCfg(ctypes.Structure):
    _fields_ = [("max_queue", ctypes.c_uint32), ("max_batch", ctypes.c_uint32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("long_pair_cells_log2", ctypes.c_uint32), ("pair_workers", ctypes.c_uint32)]


class Profile(ctypes.Structure):
    _fields_ = [("prep_ms", ctypes.c_double), ("fill_ms", ctypes.c_double), ("trace_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("fill_blocks", ctypes.c_uint64), ("cells", ctypes.c_uint64)]


class FillConfig(ctypes.Structure):
    _fields_ = [("rows_per_step", ctypes.c_uint32), ("vg_select", ctypes.c_uint32)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("words_per_lane", ctypes.c_uint32), ("split_pct", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class IntRate(ctypes.Structure):
    _fields_ = [("ops_per_s", ctypes.c_double), ("ops_per_clk_sm", ctypes.c_double), ("sm_clock_mhz", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("sms", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("ops_per_chain", ctypes.c_uint32), ("threads", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("flags", ctypes.c_uint32), ("length", ctypes.c_uint64),
                ("lcs", ctypes.POINTER(ctypes.c_uint8)), ("lcs_len", ctypes.c_uint64),
                ("submit_to_done_s", ctypes.c_double)]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"liblcs.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, u64, u32, u8p = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint8)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    sig = {
        "lcs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lcs_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp)]),
        "lcs_ctx_destroy": (None, [vp]),
        "lcs_ctx_sync": (ctypes.c_int, [vp]),
        "lcs_length": (ctypes.c_int, [vp, u8p, u64, u8p, u64, u64p]),
        "lcs_length_dev": (ctypes.c_int, [vp, vp, u64, vp, u64, vp, vp]),
        "lcs_traceback": (ctypes.c_int, [vp, u8p, u64, u8p, u64, u8p, u64, u64p]),
        "lcs_traceback_dev": (ctypes.c_int, [vp, vp, u64, vp, u64, vp, u64, vp, vp]),
        "lcs_batch": (ctypes.c_int, [vp, u8p, u64p, u8p, u64p, u64, u64p]),
        "lcs_batch_dev": (ctypes.c_int, [vp, vp, vp, vp, vp, u64, vp, vp]),
        "lcs_batch_dev_hoff": (ctypes.c_int, [vp, vp, vp, vp, vp, u64, vp, vp]),
        "lcs_serve_create": (ctypes.c_int, [vp, ctypes.POINTER(ServeCfg), ctypes.POINTER(vp)]),
        "lcs_serve_submit": (ctypes.c_int, [vp, u8p, u64, u8p, u64, u32, u64p]),
        "lcs_serve_poll": (ctypes.c_int, [vp, u64, ctypes.POINTER(Result)]),
        "lcs_serve_wait": (ctypes.c_int, [vp, u64, ctypes.c_double, ctypes.POINTER(Result)]),
        "lcs_result_release": (None, [vp, u64]),
        "lcs_serve_destroy": (None, [vp]),
        "lcs_ctx_set_profiling": (ctypes.c_int, [vp, ctypes.c_int]),
        "lcs_ctx_last_profile": (ctypes.c_int, [vp, ctypes.POINTER(Profile)]),
        "lcs_tables": (ctypes.c_int, [vp, u8p, u64, u8p, u64, ctypes.POINTER(ctypes.c_uint32), u8p]),
        "lcs_tables_dev": (ctypes.c_int, [vp, vp, u64, vp, u64, vp, vp, vp]),
        "lcs_ctx_get_fill_config": (ctypes.c_int, [vp, u32, ctypes.POINTER(FillConfig)]),
        "lcs_ctx_set_fill_config": (ctypes.c_int, [vp, u32, ctypes.POINTER(FillConfig)]),
        "lcs_ctx_autotune_dev": (ctypes.c_int, [vp, vp, u64, vp, u64, u32, vp, ctypes.POINTER(FillConfig),
                                                 ctypes.POINTER(ctypes.c_double)]),
        "lcs_ctx_get_batch_config": (ctypes.c_int, [vp, ctypes.POINTER(BatchConfig)]),
        "lcs_ctx_set_batch_config": (ctypes.c_int, [vp, ctypes.POINTER(BatchConfig)]),
        "lcs_ctx_autotune_batch_dev": (ctypes.c_int, [vp, vp, vp, vp, vp, u64, vp, vp, ctypes.POINTER(BatchConfig),
                                                       ctypes.POINTER(ctypes.c_double)]),
        "lcs_probe_int_rate": (ctypes.c_int, [ctypes.c_int, u32, u32, ctypes.POINTER(IntRate)]),
        "lcs_probe_step_floor": (ctypes.c_int, [ctypes.c_int, u32, ctypes.c_int, u32, ctypes.POINTER(ctypes.c_double)]),
        "lcs_probe_step_masks": (ctypes.c_int, [ctypes.c_int, u32, u32, ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load()


def strerror(code: int) -> str:
    return _lib.lcs_strerror(code).decode()


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise LCSError(rc, what)


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    return np.ascontiguousarray(a, dtype=np.uint8)


def probe_int_rate(device: int = 0, mix: int = 0, iters: int = 200000) -> dict:
    """INT32 throughput of the device for an instruction mix (0: the row update, 1: with the traceback word,
    2: three-input logic), see lcs_probe_int_rate."""
    r = IntRate()
    _check(_lib.lcs_probe_int_rate(device, mix, iters, ctypes.byref(r)), "lcs_probe_int_rate")
    return {k: getattr(r, k) for k, _ in IntRate._fields_}


def probe_step_floor(device: int = 0, rows_per_step: int = 8, traceback: bool = False, steps: int = 4096) -> float:
    """Clock cycles of one fill step's row arithmetic and carry shuffles alone (lcs_probe_step_floor)."""
    c = ctypes.c_double(0.0)
    _check(_lib.lcs_probe_step_floor(device, rows_per_step, 1 if traceback else 0, steps, ctypes.byref(c)),
           "lcs_probe_step_floor")
    return c.value


MASK_SOURCES = ("registers", "shared_table", "planes_prmt", "planes_expanded")


def probe_step_masks(device: int = 0, source: int = 0, steps: int = 4096) -> float:
    """Clock cycles of one 8-row traceback fill step with its match masks from `source` (0..3, MASK_SOURCES)
    (lcs_probe_step_masks)."""
    c = ctypes.c_double(0.0)
    _check(_lib.lcs_probe_step_masks(device, source, steps, ctypes.byref(c)), "lcs_probe_step_masks")
    return c.value


def _p8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(None)
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class Context:
    """An lcs_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check(_lib.lcs_ctx_create(device, ctypes.byref(h)), "lcs_ctx_create")
        self._h = h
        self.device = device

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def close(self) -> None:
        if self._h:
            _lib.lcs_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sync(self) -> None:
        _check(_lib.lcs_ctx_sync(self._h), "lcs_ctx_sync")

    def set_profiling(self, enable: bool = True) -> None:
        _check(_lib.lcs_ctx_set_profiling(self._h, 1 if enable else 0), "lcs_ctx_set_profiling")

    def last_profile(self) -> dict:
        p = Profile()
        _check(_lib.lcs_ctx_last_profile(self._h, ctypes.byref(p)), "lcs_ctx_last_profile")
        return {k: getattr(p, k) for k, _ in Profile._fields_}

    def get_fill_config(self, traceback: bool = False) -> dict:
        f = FillConfig()
        _check(_lib.lcs_ctx_get_fill_config(self._h, 1 if traceback else 0, ctypes.byref(f)), "lcs_ctx_get_fill_config")
        return {"rows_per_step": f.rows_per_step, "vg_select": f.vg_select}

    def set_fill_config(self, rows_per_step: int, vg_select: int = 0, traceback: bool = False) -> None:
        f = FillConfig(rows_per_step, vg_select)
        _check(_lib.lcs_ctx_set_fill_config(self._h, 1 if traceback else 0, ctypes.byref(f)), "lcs_ctx_set_fill_config")

    def autotune_dev(self, x, y, traceback: bool = False, stream=None) -> dict:
        """Times every fill configuration on the CUDA tensors x, y and keeps the fastest (lcs_ctx_autotune_dev)."""
        f = FillConfig()
        ms = ctypes.c_double(0.0)
        rc = _lib.lcs_ctx_autotune_dev(self._h, ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(y.data_ptr()),
                                       y.numel(), 1 if traceback else 0, _stream_ptr(stream), ctypes.byref(f),
                                       ctypes.byref(ms))
        _check(rc, "lcs_ctx_autotune_dev")
        return {"rows_per_step": f.rows_per_step, "vg_select": f.vg_select, "ms": ms.value}

    def get_batch_config(self) -> dict:
        b = BatchConfig()
        _check(_lib.lcs_ctx_get_batch_config(self._h, ctypes.byref(b)), "lcs_ctx_get_batch_config")
        return {"words_per_lane": b.words_per_lane, "split_pct": b.split_pct, "blocks_per_sm": b.blocks_per_sm}

    def set_batch_config(self, words_per_lane: int = 4, split_pct: int = 100, blocks_per_sm: int = 1) -> None:
        b = BatchConfig(words_per_lane, split_pct, blocks_per_sm, 0)
        _check(_lib.lcs_ctx_set_batch_config(self._h, ctypes.byref(b)), "lcs_ctx_set_batch_config")

    def autotune_batch_dev(self, xs, x_off, ys, y_off, count: int, out, stream=None) -> dict:
        """Times every batch configuration on the batch given as for batch_dev and keeps the fastest
        (lcs_ctx_autotune_batch_dev); out receives the lengths."""
        b = BatchConfig()
        ms = ctypes.c_double(0.0)
        rc = _lib.lcs_ctx_autotune_batch_dev(self._h, ctypes.c_void_p(xs.data_ptr()), ctypes.c_void_p(x_off.data_ptr()),
                                             ctypes.c_void_p(ys.data_ptr()), ctypes.c_void_p(y_off.data_ptr()), count,
                                             ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream), ctypes.byref(b),
                                             ctypes.byref(ms))
        _check(rc, "lcs_ctx_autotune_batch_dev")
        return {"words_per_lane": b.words_per_lane, "split_pct": b.split_pct, "blocks_per_sm": b.blocks_per_sm,
                "ms": ms.value}

    # -- host buffers -------------------------------------------------------------------------------------------
    def length(self, x, y) -> int:
        x, y = _u8(x), _u8(y)
        out = ctypes.c_uint64(0)
        _check(_lib.lcs_length(self._h, _p8(x), len(x), _p8(y), len(y), ctypes.byref(out)), "lcs_length")
        return int(out.value)

    def traceback(self, x, y, out_cap: int | None = None) -> bytes:
        x, y = _u8(x), _u8(y)
        cap = min(len(x), len(y)) if out_cap is None else out_cap
        out = np.empty(max(cap, 1), dtype=np.uint8)
        n_out = ctypes.c_uint64(0)
        rc = _lib.lcs_traceback(self._h, _p8(x), len(x), _p8(y), len(y), _p8(out), cap, ctypes.byref(n_out))
        _check(rc, "lcs_traceback")
        return out[: n_out.value].tobytes()

    def tables(self, x, y) -> tuple[np.ndarray, np.ndarray]:
        """(c, b) of LCS-length: c of shape (m+1, n+1) uint32, b of shape (m, n) uint8 (1 DIAG, 2 UP, 3 LEFT)."""
        x, y = _u8(x), _u8(y)
        m, n = len(x), len(y)
        c = np.zeros((m + 1) * (n + 1), dtype=np.uint32)
        b = np.zeros(max(m * n, 1), dtype=np.uint8)
        rc = _lib.lcs_tables(self._h, _p8(x) if m else None, m, _p8(y) if n else None, n,
                             c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _p8(b))
        _check(rc, "lcs_tables")
        return c.reshape(m + 1, n + 1), b[: m * n].reshape(m, n)

    def batch(self, pairs) -> np.ndarray:
        xs = [_u8(x) for x, _ in pairs]
        ys = [_u8(y) for _, y in pairs]
        x_off = np.zeros(len(pairs) + 1, dtype=np.uint64)
        y_off = np.zeros(len(pairs) + 1, dtype=np.uint64)
        x_off[1:] = np.cumsum([len(a) for a in xs])
        y_off[1:] = np.cumsum([len(a) for a in ys])
        xcat = np.concatenate(xs) if xs else np.zeros(0, np.uint8)
        ycat = np.concatenate(ys) if ys else np.zeros(0, np.uint8)
        xcat = xcat if len(xcat) else np.zeros(1, np.uint8)
        ycat = ycat if len(ycat) else np.zeros(1, np.uint8)
        out = np.zeros(max(len(pairs), 1), dtype=np.uint64)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        rc = _lib.lcs_batch(self._h, _p8(xcat), x_off.ctypes.data_as(u64p), _p8(ycat), y_off.ctypes.data_as(u64p),
                            len(pairs), out.ctypes.data_as(u64p))
        _check(rc, "lcs_batch")
        return out[: len(pairs)]

    def batch_concat(self, xs, x_off, ys, y_off) -> np.ndarray:
        """lcs_batch on already concatenated host buffers with count+1 offsets each."""
        xs, ys = _u8(xs), _u8(ys)
        x_off = np.ascontiguousarray(x_off, dtype=np.uint64)
        y_off = np.ascontiguousarray(y_off, dtype=np.uint64)
        count = len(x_off) - 1
        out = np.zeros(max(count, 1), dtype=np.uint64)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        xs1 = xs if len(xs) else np.zeros(1, np.uint8)
        ys1 = ys if len(ys) else np.zeros(1, np.uint8)
        rc = _lib.lcs_batch(self._h, _p8(xs1), x_off.ctypes.data_as(u64p), _p8(ys1), y_off.ctypes.data_as(u64p), count,
                            out.ctypes.data_as(u64p))
        _check(rc, "lcs_batch")
        return out[:count]

    # -- device buffers (torch uint8 CUDA tensors) ---------------------------------------------------------------
    def length_dev(self, x, y, out, stream=None) -> None:
        """x, y: uint8 CUDA tensors; out: a uint64/int64 CUDA tensor with at least one element."""
        rc = _lib.lcs_length_dev(self._h, ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(y.data_ptr()),
                                 y.numel(), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
        _check(rc, "lcs_length_dev")

    def traceback_dev(self, x, y, out, out_len, stream=None) -> None:
        rc = _lib.lcs_traceback_dev(self._h, ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(y.data_ptr()),
                                    y.numel(), ctypes.c_void_p(out.data_ptr()), out.numel(),
                                    ctypes.c_void_p(out_len.data_ptr()), _stream_ptr(stream))
        _check(rc, "lcs_traceback_dev")

    def tables_dev(self, x, y, c, b, stream=None) -> None:
        """c: int32/uint32 CUDA tensor of (m+1)*(n+1) elements; b: uint8 CUDA tensor of m*n elements."""
        rc = _lib.lcs_tables_dev(self._h, ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(y.data_ptr()),
                                 y.numel(), ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                 _stream_ptr(stream))
        _check(rc, "lcs_tables_dev")

    def batch_dev(self, xs, x_off, ys, y_off, count: int, out, stream=None) -> None:
        rc = _lib.lcs_batch_dev(self._h, ctypes.c_void_p(xs.data_ptr()), ctypes.c_void_p(x_off.data_ptr()),
                                ctypes.c_void_p(ys.data_ptr()), ctypes.c_void_p(y_off.data_ptr()), count,
                                ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
        _check(rc, "lcs_batch_dev")

    def batch_dev_hoff(self, xs, x_off, ys, y_off, count: int, out, stream=None) -> None:
        """xs, ys, out: CUDA tensors; x_off, y_off: host uint64 arrays of count + 1 offsets (lcs_batch_dev_hoff)."""
        xo = np.ascontiguousarray(x_off, dtype=np.uint64)
        yo = np.ascontiguousarray(y_off, dtype=np.uint64)
        rc = _lib.lcs_batch_dev_hoff(self._h, ctypes.c_void_p(xs.data_ptr()), xo.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.c_void_p(ys.data_ptr()), yo.ctypes.data_as(ctypes.c_void_p), count,
                                     ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
        _check(rc, "lcs_batch_dev_hoff")


class Server:
    """lcs_server: continuous batching of requests submitted over time."""

    def __init__(self, ctx: Context, max_queue: int = 0, max_batch: int = 0, hbm_budget_bytes: int = 0,
                 long_pair_cells_log2: int = 0, pair_workers: int = 0):
        cfg = ServeCfg(max_queue, max_batch, hbm_budget_bytes, long_pair_cells_log2, pair_workers)
        h = ctypes.c_void_p()
        _check(_lib.lcs_serve_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)), "lcs_serve_create")
        self._h = h
        self._ctx = ctx

    def close(self) -> None:
        if self._h:
            _lib.lcs_serve_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, x, y, traceback: bool = False) -> int:
        x, y = _u8(x), _u8(y)
        t = ctypes.c_uint64(0)
        rc = _lib.lcs_serve_submit(self._h, _p8(x), len(x), _p8(y), len(y), TRACEBACK if traceback else 0,
                                   ctypes.byref(t))
        _check(rc, "lcs_serve_submit")
        return int(t.value)

    def try_submit(self, x, y, traceback: bool = False) -> tuple[int, int]:
        x, y = _u8(x), _u8(y)
        t = ctypes.c_uint64(0)
        rc = _lib.lcs_serve_submit(self._h, _p8(x), len(x), _p8(y), len(y), TRACEBACK if traceback else 0,
                                   ctypes.byref(t))
        return rc, int(t.value)

    def _take(self, ticket: int, r: Result) -> dict:
        d = {"status": r.status, "length": int(r.length), "latency_s": float(r.submit_to_done_s),
             "lcs": ctypes.string_at(r.lcs, r.lcs_len) if r.lcs and r.lcs_len else (b"" if r.flags & 1 else None)}
        _lib.lcs_result_release(self._h, ticket)
        return d

    def poll(self, ticket: int):
        r = Result()
        rc = _lib.lcs_serve_poll(self._h, ticket, ctypes.byref(r))
        if rc == PENDING:
            return None
        _check(rc, "lcs_serve_poll")
        return self._take(ticket, r)

    def wait(self, ticket: int, timeout_s: float = -1.0):
        r = Result()
        rc = _lib.lcs_serve_wait(self._h, ticket, timeout_s, ctypes.byref(r))
        if rc == PENDING:
            return None
        _check(rc, "lcs_serve_wait")
        return self._take(ticket, r)
