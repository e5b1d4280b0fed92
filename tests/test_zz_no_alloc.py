"""lcs_length_noalloc: the length entry point that allocates no device memory.

Some callers cannot let a library allocate device memory: code inside a framework that owns the whole device pool or
a fixed memory budget, and latency-critical loops where cudaMalloc/cudaFree would synchronise the device. This entry
point works in a scratch array the library reserves statically. Its results must equal the CPU oracle's and those of
lcs_length_dev exactly, on consecutive calls that share that scratch, on either of two streams, on the one-launch path
for small pairs as well as the general one; and once warmed up, its calls must leave the device's free memory
unchanged. The file is named to run last, so that a failure here does not stop the other tests.
"""

import ctypes

import pytest

from paper_1306_4627_gb300 import gen

pytestmark = pytest.mark.gpu

# (m, n, alphabet size, seed): a full-size pair, two uneven ones, and one that takes the one-launch small-pair path
CASES = [(65536, 65536, 4, 11), (3000, 41000, 20, 12), (65536, 977, 256, 13), (700, 900, 4, 14)]


def _noalloc_fn():
    from paper_1306_4627_gb300 import lcs
    f = lcs._lib.lcs_length_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def _oracle_length(oracle, x, y):
    # the column-block oracle (pinned equal to the serial one) keeps the 65536^2 case to about a second
    return oracle.lcs_length_par(x, y, 16) if len(x) * len(y) > 1 << 26 else oracle.lcs_length(x, y)


def test_noalloc_matches_oracle_and_length_dev_on_consecutive_calls(oracle):
    import torch
    from paper_1306_4627_gb300 import lcs
    f = _noalloc_fn()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
    inputs = []
    for m, n, sigma, seed in CASES:
        x, y = gen.pair_uniform(m, n, sigma, seed=seed)
        inputs.append((x, y, torch.from_numpy(x.copy()).to(dev), torch.from_numpy(y.copy()).to(dev),
                       _oracle_length(oracle, x, y)))
    with lcs.Context(0) as ctx:
        # two passes over the cases, alternating the two streams call by call: every call follows one of another
        # shape that left its own contents in the shared scratch
        k = 0
        for _ in range(2):
            for (x, y, dx, dy, want_oracle), (m, n, _, _) in zip(inputs, CASES):
                got = torch.zeros(1, dtype=torch.int64, device=dev)
                want = torch.zeros(1, dtype=torch.int64, device=dev)
                torch.cuda.synchronize()
                rc = f(dx.data_ptr(), m, dy.data_ptr(), n, got.data_ptr(), streams[k % 2].cuda_stream)
                k += 1
                assert rc == lcs.OK, lcs.strerror(rc)
                ctx.length_dev(dx, dy, want)
                ctx.sync()
                assert int(got.item()) == want_oracle, (m, n)
                assert int(want.item()) == want_oracle, (m, n)


def test_noalloc_leaves_free_device_memory_unchanged():
    import torch
    from paper_1306_4627_gb300 import lcs
    f = _noalloc_fn()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(device=dev)
    bufs = []
    for m, n, sigma, seed in CASES:
        x, y = gen.pair_uniform(m, n, sigma, seed=seed)
        bufs.append((m, n, torch.from_numpy(x.copy()).to(dev), torch.from_numpy(y.copy()).to(dev)))
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    for m, n, dx, dy in bufs:  # warm-up: the first call on the device looks up the scratch array
        assert f(dx.data_ptr(), m, dy.data_ptr(), n, out.data_ptr(), stream.cuda_stream) == lcs.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    for _ in range(3):
        for m, n, dx, dy in bufs:
            assert f(dx.data_ptr(), m, dy.data_ptr(), n, out.data_ptr(), stream.cuda_stream) == lcs.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0, (free0, free1)


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
