"""GPU: a field split into slabs, compressed slab by slab on one GPU (as the
ranks of a sharded run would, one after another) with the range pass, the
supplied-range compression and the device concatenation; the result must be
the single-shot stream byte for byte (the GPU's and the oracle's)."""
import numpy as np
import pytest

import oracle
import paper_2304_12557_gb300 as fz
from paper_2304_12557_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    return t


@pytest.fixture(scope="module")
def codec(torch):
    from paper_2304_12557_gb300 import build
    build.build()
    c = fz.Codec(0)
    yield c
    c.close()


def _outliers(shape, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, shape).astype(np.float32)
    flat = x.reshape(-1)
    idx = rng.choice(flat.size, n, replace=False)
    flat[idx] = rng.choice([-1, 1], n) * rng.uniform(2e4, 9e4, n)
    return x


CASES = {
    "bumps3d_64_rel": (lambda: fields.bumps3d(64), 3, "rel", 1e-3),
    "grf3d_ragged_rel": (lambda: fields.grf((41, 70, 33), -3.0, 5).astype(np.float32),
                         3, "rel", 1e-4),
    "climate2d_rel": (lambda: fields.climate2d(1800, 3600), 2, "rel", 1e-3),
    "climate2d_abs": (lambda: fields.climate2d(300, 500), 2, "abs", 0.01),
    "grf1d_rel": (lambda: fields.grf((300001,), -2.0, 6).astype(np.float32), 1, "rel", 1e-3),
    "outliers3d_abs": (lambda: _outliers((40, 67, 96), 80, 8), 3, "abs", 0.5),
    "outliers2d_rel": (lambda: _outliers((520, 130), 80, 9), 2, "rel", 1e-6),
}


def _sharded(codec, torch, xt, ndim, mode, eb, world):
    dims = list(xt.shape[::-1])[:ndim]
    slabs = []
    for r in range(world):
        b, e = fz.shard_extent(dims, ndim, world, r)
        if b < e:
            slabs.append(xt[b:e])
    rng = None
    if mode == "rel":
        los, his = [], []
        for s in slabs:
            lo, hi, bad = codec.value_range(s)
            assert not bad
            los.append(lo)
            his.append(hi)
        rng = (min(los), max(his))                   # the all-reduce's result
    parts = []
    for s in slabs:
        sd = list(s.shape[::-1])[:ndim]
        out = torch.empty(fz.compress_bound(sd, ndim), dtype=torch.uint8, device="cuda")
        if rng is None:
            _, size = codec.compress_into(s, out, "abs", eb, ndim)
        else:
            _, size = codec.compress_ranged_into(s, out, eb, rng[0], rng[1], ndim)
        parts.append(out[:size])
    total = sum(p.numel() for p in parts)
    out = torch.empty(total + 64, dtype=torch.uint8, device="cuda")
    _, size = codec.concat_into(parts, out)
    torch.cuda.synchronize()
    return out[:size].cpu().numpy().tobytes()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("world", [2, 3, 8])
def test_sharded_equals_single_stream(codec, torch, name, world):
    make, ndim, mode, eb = CASES[name]
    x = np.ascontiguousarray(make(), dtype=np.float32)
    xt = torch.from_numpy(x).cuda()
    single = codec.compress(xt, mode=mode, eb=eb, ndim=ndim).cpu().numpy().tobytes()
    st, ostream = oracle.compress(x, ndim, fz.EB_REL if mode == "rel" else fz.EB_ABS, eb)
    assert st == 0 and single == ostream
    assert _sharded(codec, torch, xt, ndim, mode, eb, world) == single


def test_value_range(codec, torch):
    x = fields.grf((33, 70, 41), -3.0, 5).astype(np.float32)
    x[3, 4, 5] = -0.0
    xt = torch.from_numpy(x).cuda()
    lo, hi, bad = codec.value_range(xt)
    assert (lo, hi, bad) == (float(x.min()), float(x.max()), False)
    x[0, 0, 7] = np.nan
    assert codec.value_range(torch.from_numpy(x).cuda())[2]
    z = torch.zeros(1000, device="cuda") * -1.0               # -0.0 everywhere
    lo, hi, _ = codec.value_range(z)
    assert np.signbit(lo) == False and np.signbit(hi) == False  # noqa: E712


def test_ranged_errors(codec, torch):
    x = fields.bumps3d(64)
    xt = torch.from_numpy(x).cuda()
    out = torch.empty(fz.compress_bound((64, 64, 64), 3), dtype=torch.uint8, device="cuda")
    lo, hi = float(x.min()), float(x.max())
    st, _ = codec.compress_ranged_into(xt, out, 1e-3, hi, lo, 3, raise_on_error=False)
    assert st == fz.ERR_ARG                                     # inverted range
    st, _ = codec.compress_ranged_into(xt, out, 1e-3, lo, float("nan"), 3,
                                       raise_on_error=False)
    assert st == fz.ERR_ARG
    # a range far narrower than the data: some element quantises too large
    st, _ = codec.compress_ranged_into(xt, out, 1e-7, 0.0, 1e-3, 3, raise_on_error=False)
    assert st == fz.ERR_EB_RANGE
    y = x.copy()
    y[10, 11, 12] = np.inf
    st, _ = codec.compress_ranged_into(torch.from_numpy(y).cuda(), out, 1e-3, lo, hi, 3,
                                       raise_on_error=False)
    assert st == fz.ERR_NONFINITE
    # a wider range than the data's: the oracle's supplied-range stream
    st, size = codec.compress_ranged_into(xt, out, 1e-3, lo - 2.0, hi + 5.0, 3)
    _, o = oracle.compress_ranged(x, 3, 1e-3, lo - 2.0, hi + 5.0)
    assert out[:size].cpu().numpy().tobytes() == o


def test_concat_device_rejects_and_reports_capacity(codec, torch):
    x = fields.bumps3d(64)
    xt = torch.from_numpy(x).cuda()
    parts = []
    for b, e in [(0, 32), (32, 64)]:
        out = torch.empty(fz.compress_bound((64, 64, e - b), 3), dtype=torch.uint8,
                          device="cuda")
        _, size = codec.compress_into(xt[b:e], out, "abs", 1e-3, 3)
        parts.append(out[:size])
    total = sum(p.numel() for p in parts)
    small = torch.empty(total - 64 - 1, dtype=torch.uint8, device="cuda")
    st, need = codec.concat_into(parts, small, raise_on_error=False)
    assert st == fz.ERR_CAPACITY and need == total - 64
    st, _ = codec.concat_into([parts[0][:-8], parts[1]], small, raise_on_error=False)
    assert st == fz.ERR_CORRUPT
