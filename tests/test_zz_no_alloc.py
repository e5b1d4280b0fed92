"""lcs_length_noalloc: the length entry point that allocates no device memory.

Some callers cannot let a library allocate device memory (a framework that owns the whole pool or a fixed budget;
latency-critical loops where cudaMalloc would synchronise the device). This entry point works in a scratch array
the library reserves statically; its results must equal those of lcs_length_dev exactly, on consecutive calls that
share that scratch. The file is named to run last, so a failure here does not stop the other tests.
"""

import ctypes

import pytest

from paper_1306_4627_gb300 import gen

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    from paper_1306_4627_gb300 import lcs
    f = lcs._lib.lcs_length_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def test_noalloc_matches_length_dev_on_consecutive_calls():
    import torch
    from paper_1306_4627_gb300 import lcs
    f = _noalloc_fn()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(device=dev)
    with lcs.Context(0) as ctx:
        # two calls in a row: a large pair, then a smaller one that reuses (and must not be confused by) the scratch
        for m, n, sigma, seed in [(65536, 65536, 4, 11), (3000, 41000, 20, 12), (65536, 977, 256, 13)]:
            x, y = gen.pair_uniform(m, n, sigma, seed=seed)
            dx = torch.from_numpy(x.copy()).to(dev)
            dy = torch.from_numpy(y.copy()).to(dev)
            got = torch.zeros(1, dtype=torch.int64, device=dev)
            want = torch.zeros(1, dtype=torch.int64, device=dev)
            torch.cuda.synchronize()
            rc = f(dx.data_ptr(), m, dy.data_ptr(), n, got.data_ptr(), stream.cuda_stream)
            assert rc == lcs.OK, lcs.strerror(rc)
            ctx.length_dev(dx, dy, want)
            ctx.sync()
            assert int(got.item()) == int(want.item()), (m, n)


def test_noalloc_limits():
    import torch
    from paper_1306_4627_gb300 import lcs
    f = _noalloc_fn()
    dev = torch.device("cuda", 0)
    x = torch.zeros(65537, dtype=torch.uint8, device=dev)
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    assert f(x.data_ptr(), 65537, x.data_ptr(), 10, out.data_ptr(), None) == lcs.ERR_INVALID
    assert f(x.data_ptr(), 10, x.data_ptr(), 65537, out.data_ptr(), None) == lcs.ERR_INVALID
    assert f(x.data_ptr(), 0, x.data_ptr(), 10, out.data_ptr(), None) == lcs.OK
    torch.cuda.synchronize()
    assert int(out.item()) == 0
