"""fz_compress_noalloc: compression for callers that cannot allocate GPU
memory (a pool that already holds the free HBM, latency-critical loops that
cannot pay for cudaMalloc, fixed memory plans).

The entry point keeps its scratch in a static device array instead of a
context, so these tests check that its streams are byte-identical to the
regular fz_compress entry point's, over consecutive calls that share the
array (each call must clear what the previous one left behind).
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


def noalloc_compress(torch, lib, x_t, ndim, mode, eb):
    dims = list(x_t.shape[::-1])[:ndim]
    cap = fz.stream_min_bytes(dims, ndim) + 16 * 256 * (x_t.numel() // 2048 + 64)
    out = torch.empty(cap, dtype=torch.uint8, device=x_t.device)
    size = ctypes.c_uint64(0)
    d = (ctypes.c_uint64 * 3)(*(list(dims) + [1] * (3 - ndim)))
    st = lib.fz_compress_noalloc(ctypes.c_void_p(x_t.data_ptr()), d, ndim, mode,
                                 float(eb), ctypes.c_void_p(out.data_ptr()), cap,
                                 ctypes.byref(size),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, out[: size.value].cpu().numpy().tobytes()


def test_noalloc_matches_fz_compress_over_consecutive_calls(env):
    torch, lib, codec = env
    rng = np.random.default_rng(12)
    a = fields.grf((24, 96, 64), -3.0, 21).astype(np.float32)
    a.reshape(-1)[rng.choice(a.size, 30, replace=False)] = 5e4   # outliers
    b = fields.climate2d(257, 300)
    cases = [(a, 3, fz.EB_ABS, 0.25), (b, 2, fz.EB_REL, 1e-3),
             (a, 3, fz.EB_ABS, 0.25)]
    for x, ndim, mode, eb in cases:
        xt = torch.from_numpy(x).cuda()
        st, got = noalloc_compress(torch, lib, xt, ndim, mode, eb)
        assert st == fz.OK
        want = codec.compress(xt, mode=mode, eb=eb, ndim=ndim).cpu().numpy().tobytes()
        assert got == want


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
