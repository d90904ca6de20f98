"""fz_compress_noalloc: compression for callers that cannot allocate GPU
memory (a pool that already holds the free HBM, latency-critical loops that
cannot pay for cudaMalloc, fixed memory plans).

The entry point keeps its scratch in a static device array instead of a
context, so these tests check that its streams, sizes and statuses equal
the regular fz_compress entry point's, over consecutive calls that share the
array (each call must clear what the previous one left behind).  The file
sorts last so that a run stopping at its first failure has run every other
test before it.
"""
import ctypes

import numpy as np
import pytest

import paper_2304_12557_gb300 as fz
from paper_2304_12557_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12557_gb300 import build
    build.build()
    lib = fz.load_library()
    codec = fz.Codec(0)
    yield torch, lib, codec
    codec.close()


def _cap(dims, ndim, n):
    return fz.stream_min_bytes(dims, ndim) + 16 * 256 * (n // 2048 + 64)


def noalloc_call(torch, lib, x_t, ndim, mode, eb, cap=None):
    """(status, out_size, stream bytes) through the C ABI."""
    dims = list(x_t.shape[::-1])[:ndim]
    cap = cap if cap is not None else _cap(dims, ndim, x_t.numel())
    out = torch.empty(max(cap, 16), dtype=torch.uint8, device=x_t.device)
    size = ctypes.c_uint64(0)
    d = (ctypes.c_uint64 * 3)(*(list(dims) + [1] * (3 - ndim)))
    st = lib.fz_compress_noalloc(ctypes.c_void_p(x_t.data_ptr()), d, ndim, mode,
                                 float(eb), ctypes.c_void_p(out.data_ptr()), cap,
                                 ctypes.byref(size),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    data = out[: size.value].cpu().numpy().tobytes() if st == fz.OK else b""
    return st, int(size.value), data


def regular_call(torch, codec, x_t, ndim, mode, eb, cap=None):
    dims = list(x_t.shape[::-1])[:ndim]
    cap = cap if cap is not None else _cap(dims, ndim, x_t.numel())
    out = torch.empty(max(cap, 16), dtype=torch.uint8, device=x_t.device)
    st, size = codec.compress_into(x_t, out[:cap], mode, eb, ndim,
                                   raise_on_error=False)
    torch.cuda.synchronize()
    data = out[:size].cpu().numpy().tobytes() if st == fz.OK else b""
    return st, size, data


def test_noalloc_matches_fz_compress_over_consecutive_calls(env):
    torch, lib, codec = env
    rng = np.random.default_rng(12)
    a = fields.grf((24, 96, 64), -3.0, 21).astype(np.float32)
    a.reshape(-1)[rng.choice(a.size, 30, replace=False)] = 5e4   # outliers
    b = fields.climate2d(257, 300)
    c = np.cumsum(rng.normal(0, 1, 100_003)).astype(np.float32)  # 1-D, ragged tail
    cases = [(a, 3, fz.EB_ABS, 0.25), (b, 2, fz.EB_REL, 1e-3), (c, 1, fz.EB_REL, 1e-4),
             (a, 3, fz.EB_ABS, 0.25), (c, 1, fz.EB_ABS, 0.01)]
    for x, ndim, mode, eb in cases:
        xt = torch.from_numpy(x).cuda()
        got = noalloc_call(torch, lib, xt, ndim, mode, eb)
        want = regular_call(torch, codec, xt, ndim, mode, eb)
        assert got[0] == fz.OK
        assert got == want


def test_noalloc_capacity_errors_report_the_needed_size(env):
    torch, lib, codec = env
    x = fields.grf((20, 70, 90), -3.0, 5).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    dims = list(x.shape[::-1])
    full = regular_call(torch, codec, xt, 3, fz.EB_REL, 1e-3)
    assert full[0] == fz.OK
    min_bytes = fz.stream_min_bytes(dims, 3)
    # below the flags section: refused before any launch
    got = noalloc_call(torch, lib, xt, 3, fz.EB_REL, 1e-3, cap=min_bytes - 16)
    want = regular_call(torch, codec, xt, 3, fz.EB_REL, 1e-3, cap=min_bytes - 16)
    assert got[0] == fz.ERR_CAPACITY and got[:2] == want[:2] and got[1] == min_bytes
    # room for the flags but not the payload: found by the kernel
    cap = (min_bytes + full[1]) // 2 // 16 * 16
    got = noalloc_call(torch, lib, xt, 3, fz.EB_REL, 1e-3, cap=cap)
    want = regular_call(torch, codec, xt, 3, fz.EB_REL, 1e-3, cap=cap)
    assert got[0] == fz.ERR_CAPACITY and got[:2] == want[:2] and got[1] == full[1]
    # the next call with room is unaffected by the failed ones
    assert noalloc_call(torch, lib, xt, 3, fz.EB_REL, 1e-3) == full


def test_noalloc_nonfinite_after_a_relative_bound_call(env):
    """An absolute bound over an input with NaN/Inf runs a second range pass
    on the shared range block right after a relative-bound call used it."""
    torch, lib, codec = env
    x = fields.grf((16, 64, 64), -3.0, 9).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    ok = noalloc_call(torch, lib, xt, 3, fz.EB_REL, 1e-3)
    assert ok[0] == fz.OK
    for bad in (np.nan, np.inf):
        y = x.copy()
        y[3, 17, 40] = bad
        yt = torch.from_numpy(y).cuda()
        got = noalloc_call(torch, lib, yt, 3, fz.EB_ABS, 1e-3)
        want = regular_call(torch, codec, yt, 3, fz.EB_ABS, 1e-3)
        assert got[0] == fz.ERR_NONFINITE and got[:2] == want[:2]
        assert noalloc_call(torch, lib, xt, 3, fz.EB_REL, 1e-3) == ok
    # and an absolute bound too small for a finite field: EB_RANGE
    got = noalloc_call(torch, lib, xt, 3, fz.EB_ABS, 1e-9)
    assert got[0] == fz.ERR_EB_RANGE == regular_call(torch, codec, xt, 3, fz.EB_ABS, 1e-9)[0]
    assert noalloc_call(torch, lib, xt, 3, fz.EB_REL, 1e-3) == ok


def test_noalloc_rejects_fields_beyond_its_scratch(env):
    torch, lib, _ = env
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.empty(64, dtype=torch.uint8, device="cuda")
    size = ctypes.c_uint64(0)
    too_big = (ctypes.c_uint64 * 3)(1024, 1024, 129)      # > FZ_NOALLOC_MAX_CODES
    st = lib.fz_compress_noalloc(ctypes.c_void_p(x.data_ptr()), too_big, 3,
                                 fz.EB_REL, 1e-3, ctypes.c_void_p(out.data_ptr()),
                                 64, ctypes.byref(size), None)
    assert st == fz.ERR_ARG and size.value == 0
