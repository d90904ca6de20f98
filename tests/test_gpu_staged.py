"""GPU: the unfused kernel sequence (codes and shuffled words in HBM) gives
byte for byte the oracle's stream and the fused kernel's, with either
bitshuffle (the register transpose or Listing 1's warp ballots), including
escapes, unaligned inputs, ragged shapes and errors."""
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


def _outliers(shape, n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    x = (rng.normal(0, 1, shape) * scale).astype(np.float32)
    flat = x.reshape(-1)
    idx = rng.choice(flat.size, n, replace=False)
    flat[idx] = rng.choice([-1, 1], n) * rng.uniform(2e4, 9e4, n)
    return x


CASES = [
    (lambda: fields.bumps3d(64), "rel", 1e-3),
    (lambda: fields.grf((33, 70, 41), -3.0, 71).astype(np.float32), "rel", 1e-4),
    (lambda: fields.climate2d(300, 500), "rel", 1e-3),
    (lambda: fields.grf((257, 301), -2.5, 72).astype(np.float32), "abs", 0.01),
    (lambda: fields.grf((30001,), -2.0, 73).astype(np.float32), "rel", 1e-3),
    (lambda: _outliers((40, 64, 96), 60, 74), "abs", 0.5),
    (lambda: _outliers((16, 96, 64), 10, 75, 3e4), "abs", 0.5),      # > 10000 escapes
    (lambda: np.zeros((16, 32, 32), np.float32), "rel", 1e-3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("shuffle", ["register", "ballot"])
def test_staged_equals_oracle_and_fused(codec, torch, case, offset, shuffle):
    make, mode, eb = CASES[case]
    x = np.ascontiguousarray(make(), dtype=np.float32)
    xt = torch.from_numpy(x).cuda()
    if offset:                                  # an input off its 16-byte boundary
        buf = torch.empty(x.size + offset, dtype=torch.float32, device="cuda")
        buf[offset:] = xt.reshape(-1)
        xt = buf[offset:].view(x.shape)
    fused = codec.compress(xt, mode=mode, eb=eb, ndim=x.ndim).cpu().numpy().tobytes()
    out = torch.zeros(fz.compress_bound(list(x.shape[::-1]), x.ndim), dtype=torch.uint8,
                      device="cuda")
    codec.set_staged_shuffle(shuffle)
    try:
        st, size, ms = codec.compress_staged_into(xt, out, mode, eb, x.ndim)
    finally:
        codec.set_staged_shuffle("register")
    got = out[:size].cpu().numpy().tobytes()
    ost, want = oracle.compress(x, x.ndim, oracle.EB_ABS if mode == "abs" else oracle.EB_REL, eb)
    assert ost == oracle.OK
    assert st == fz.OK and got == want
    assert got == fused
    assert all(t >= 0 for t in ms) and ms[1] > 0


def test_staged_errors(codec, torch):
    x = fields.bumps3d(64)
    bad = x.copy()
    bad[3, 4, 5] = np.nan
    out = torch.zeros(fz.compress_bound((64, 64, 64), 3), dtype=torch.uint8, device="cuda")
    st, _, _ = codec.compress_staged_into(torch.from_numpy(bad).cuda(), out, "rel", 1e-3,
                                          raise_on_error=False)
    assert st == fz.ERR_NONFINITE
    st, _, _ = codec.compress_staged_into(torch.from_numpy(x).cuda(), out, "abs", 1e-9,
                                          raise_on_error=False)
    assert st == fz.ERR_EB_RANGE
    small = torch.zeros(fz.stream_min_bytes((64, 64, 64), 3) + 16, dtype=torch.uint8,
                        device="cuda")
    st, need, _ = codec.compress_staged_into(torch.from_numpy(x).cuda(), small, "rel", 1e-3,
                                             raise_on_error=False)
    fused = codec.compress(torch.from_numpy(x).cuda(), mode="rel", eb=1e-3)
    assert st == fz.ERR_CAPACITY and need == fused.numel()
    # the context still serves the fused path afterwards
    again = codec.compress(torch.from_numpy(x).cuda(), mode="rel", eb=1e-3)
    assert torch.equal(again, fused)
