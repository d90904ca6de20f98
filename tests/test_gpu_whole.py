"""GPU: whole-field Lorenzo (stream version 2) against the oracle.

fz_compress_whole must give the oracle's fzo_compress_whole stream byte for
byte, and fz_decompress must read it back bit-identical to the oracle's
reconstruction, which is also the version-1 reconstruction (both streams are
lossless on the quantised values q, Sec. 2.2).  The shapes put several
chunks, with ragged tails, along every axis, so that every cross-chunk scan
of the decompressor (and both of its block shapes) is exercised; fields with
escaped residuals cover the outlier path in both passes.  At full size the
oracle runs in one thread, so 512^3 is checked through that last property.
"""
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


def _escapes(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(0, 1, shape) * 3e4).astype(np.float32)


CASES = [
    ("3d_ragged", lambda: fields.grf((41, 97, 70), -3.0, 71).astype(np.float32), 3, "rel", 1e-3),
    ("3d_bumps", lambda: fields.bumps3d(64), 3, "rel", 1e-4),
    ("3d_one_chunk", lambda: fields.grf((5, 20, 17), -3.0, 72).astype(np.float32), 3, "abs", 1e-3),
    ("3d_escapes", lambda: _escapes((19, 70, 45), 73), 3, "abs", 0.5),
    ("3d_cosmo", lambda: fields.cosmo3d(128), 3, "rel", 1e-3),
    ("2d_climate", lambda: fields.climate2d(300, 500), 2, "rel", 1e-3),
    ("2d_ragged", lambda: fields.grf((517, 203), -2.5, 74).astype(np.float32), 2, "abs", 1e-2),
    ("2d_escapes", lambda: _escapes((260, 150), 75), 2, "abs", 0.5),
    ("1d_short", lambda: fields.grf((30001,), -2.0, 76).astype(np.float32), 1, "rel", 1e-3),
    # 513 chunks: the one-word scan takes three steps of 256 chunks
    ("1d_long", lambda: fields.grf((513 * 8192 - 7,), -2.0, 77).astype(np.float32), 1, "rel", 1e-4),
    ("1d_escapes", lambda: _escapes((20000,), 78), 1, "abs", 0.5),
]


def _mode(m):
    return oracle.EB_ABS if m == "abs" else oracle.EB_REL


@pytest.mark.parametrize("name,make,ndim,mode,eb", CASES, ids=[c[0] for c in CASES])
def test_whole_stream_and_reconstruction_match_the_oracle(codec, torch, name, make, ndim, mode, eb):
    x = make()
    ost, ostream = oracle.compress(x, ndim, _mode(mode), eb, whole=True)
    assert ost == oracle.OK
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    s = codec.compress(xt, mode=mode, eb=eb, ndim=ndim, whole=True)
    g = s.cpu().numpy().tobytes()
    assert fz.inspect(g[:64])["version"] == 2
    assert len(g) == len(ostream)
    if g != ostream:
        a, b = np.frombuffer(g, np.uint8), np.frombuffer(ostream, np.uint8)
        bad = np.flatnonzero(a != b)
        raise AssertionError(f"stream differs at {bad.size} bytes, first {bad[:8]}")
    if "escapes" in name:
        assert fz.inspect(g[:64])["n_outliers"] > 0
    y = codec.decompress(s).cpu().numpy().ravel()
    st, want = oracle.decompress(ostream)
    assert st == oracle.OK
    np.testing.assert_array_equal(y.view(np.uint32), want.view(np.uint32))
    # the same reconstruction as the chunk-local stream's
    y1 = codec.decompress(codec.compress(xt, mode=mode, eb=eb, ndim=ndim)).cpu().numpy().ravel()
    np.testing.assert_array_equal(y.view(np.uint32), y1.view(np.uint32))


def test_whole_full_size_512_cubed_reconstructs_like_version_1(codec, torch):
    """A smooth 512^3 field (running sums of Gaussian noise along the three
    axes) at rel 1e-3, the size of the 3-D workload: the version-2
    reconstruction equals the version-1 one bit for bit and stays within the
    bound; the oracle checks the stream of a 64^3 corner box separately (the
    whole-field residuals of a box at the origin read only inside it)."""
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn((512, 512, 512), generator=g, device="cuda")
    x = x.cumsum(2).cumsum(1).cumsum(0)
    x = (x / x.abs().max()).float().contiguous()
    s2 = codec.compress(x, mode="rel", eb=1e-3, whole=True)
    s1 = codec.compress(x, mode="rel", eb=1e-3)
    assert fz.inspect(s2[:64].cpu().numpy().tobytes())["version"] == 2
    y2 = codec.decompress(s2)
    y1 = codec.decompress(s1)
    assert torch.equal(y2.view(torch.int32), y1.view(torch.int32))
    info = fz.inspect(s1[:64].cpu().numpy().tobytes())
    # the bound up to the fp32 rounding of x (as the version-1 parity tests)
    slack = 2.0 ** -22 * torch.maximum(x.abs(), y2.abs()).double()
    assert bool(((y2.double() - x.double()).abs() <= info["eb"] + slack).all())
    del y1, y2
    # the stream of the field's first 64^3 corner (whole-field residuals of
    # a sub-box that starts at the origin only read inside it)
    corner = x[:64, :64, :64].contiguous()
    ost, ostream = oracle.compress(corner.cpu().numpy(), 3, oracle.EB_ABS, info["eb"], whole=True)
    assert ost == oracle.OK
    sc = codec.compress(corner, mode="abs", eb=info["eb"], whole=True)
    assert sc.cpu().numpy().tobytes() == ostream


def test_whole_errors_and_version_checks(codec, torch):
    x = fields.bumps3d(64)
    xt = torch.from_numpy(x).cuda()
    s = codec.compress(xt, mode="rel", eb=1e-3, whole=True)
    # a corrupt flag bit fails like version 1's
    bad = s.clone()
    bad[64] ^= 1
    out = torch.empty(x.size, dtype=torch.float32, device="cuda")
    assert codec.decompress_into(bad, out, raise_on_error=False) == fz.ERR_CORRUPT
    # too small an output
    small = torch.empty(x.size - 1, dtype=torch.float32, device="cuda")
    assert codec.decompress_into(s, small, raise_on_error=False) == fz.ERR_CAPACITY
    # the next call still works
    y = codec.decompress(s).cpu().numpy().ravel()
    st, want = oracle.decompress(oracle.compress(x, 3, oracle.EB_REL, 1e-3, whole=True)[1])
    np.testing.assert_array_equal(y.view(np.uint32), want.view(np.uint32))
    # NaN input: the same error as version 1
    xn = x.copy()
    xn[3, 4, 5] = np.nan
    st, _ = codec.compress_into(torch.from_numpy(xn).cuda(), torch.empty(1 << 22, dtype=torch.uint8,
                                device="cuda"), mode="rel", eb=1e-3, raise_on_error=False,
                                whole=True)
    assert st == fz.ERR_NONFINITE
    # the server reads version-1 streams only
    srv = fz.Server(0, pool_bytes=64 << 20)
    try:
        with pytest.raises(fz.FZError) as e:
            srv.submit_decompress(s.cpu().numpy())
        assert e.value.status == fz.ERR_VERSION
    finally:
        srv.close()
