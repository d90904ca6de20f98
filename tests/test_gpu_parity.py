"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Streams must be byte-identical to the oracle's and reconstructions
bit-identical (integer codes and compressed bytes are exact; the only
floating point is the fp32 quantiser multiply and the fp32 dequantiser
multiply, which both sides perform identically).  Inputs are the seeded
synthetic fields of paper_2304_12557_gb300.fields at the workloads' full
sizes, plus small ragged shapes, outliers, errors and corrupt streams.
"""
import struct

import numpy as np
import pytest

import oracle
import paper_2304_12557_gb300 as fz
from golden_io import expected_bytes, load
from paper_2304_12557_gb300 import fields

pytestmark = pytest.mark.gpu

GOLDEN = ["g1_1d_basic.txt", "g2_1d_escape.txt", "g3_2d_basic.txt",
          "g4_3d_rel.txt"]


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


def gpu_compress(codec, torch, x, ndim, mode, eb, offset=0):
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    if offset:
        # an input that starts off a 16-byte boundary (generic load path)
        buf = torch.empty(x.size + offset, dtype=torch.float32, device="cuda")
        buf[offset:] = xt.reshape(-1)
        xt = buf[offset:].view(x.shape)
    s = codec.compress(xt, mode=mode, eb=eb, ndim=ndim)
    torch.cuda.synchronize()
    return s.cpu().numpy().tobytes()


def gpu_decompress(codec, torch, s):
    st = torch.from_numpy(np.frombuffer(s, np.uint8).copy()).cuda()
    y = codec.decompress(st)
    torch.cuda.synchronize()
    return y.cpu().numpy().ravel()


def check_parity(codec, torch, x, ndim, mode, eb, offset=0, all_cores=False):
    """all_cores: the oracle's all-cores variant (bit-identical to the
    one-thread oracle, checked on the CPU) for the full-size fields"""
    ost, ostream = oracle.compress(x, ndim, mode, eb, all_cores=all_cores)
    assert ost == oracle.OK
    g = gpu_compress(codec, torch, x, ndim, mode, eb, offset)
    assert len(g) == len(ostream)
    if g != ostream:
        a = np.frombuffer(g, np.uint8)
        b = np.frombuffer(ostream, np.uint8)
        bad = np.flatnonzero(a != b)
        raise AssertionError(f"stream differs at {bad.size} bytes, first {bad[:8]}")
    xr_gpu = gpu_decompress(codec, torch, g)
    st, xr_or = oracle.decompress(ostream, all_cores=all_cores)
    assert st == oracle.OK
    np.testing.assert_array_equal(xr_gpu.view(np.uint32), xr_or.view(np.uint32))
    return g, xr_gpu


# ------------------------------------------------------------ hand-worked
@pytest.mark.parametrize("name", GOLDEN)
def test_golden_streams_on_gpu(codec, torch, name):
    rec = load(name)
    g = gpu_compress(codec, torch, rec["x"], rec["ndim"], rec["mode"], rec["eb"])
    assert g == expected_bytes(rec)
    np.testing.assert_array_equal(gpu_decompress(codec, torch, g), rec["x"].ravel())


# ------------------------------------------------------------ small ragged
@pytest.mark.parametrize("shape,ndim", fields.small_cases())
@pytest.mark.parametrize("mode,eb", [(fz.EB_REL, 1e-2), (fz.EB_REL, 1e-4),
                                     (fz.EB_ABS, 0.37)])
def test_small_shapes(codec, torch, shape, ndim, mode, eb):
    if min(shape) > 2:
        x = fields.grf(shape, -3.0, 17).astype(np.float32) * 10 + 3
    else:
        x = np.random.default_rng(4).standard_normal(shape).astype(np.float32)
    check_parity(codec, torch, x, ndim, mode, eb)


@pytest.mark.parametrize("shape,ndim", [((20, 64, 96), 3), ((257, 300), 2),
                                        ((30001,), 1)])
def test_unaligned_input_pointer(codec, torch, shape, ndim):
    x = fields.grf(shape, -3.0, 5).astype(np.float32)
    check_parity(codec, torch, x, ndim, fz.EB_REL, 1e-3, offset=1)


# ------------------------------------------------------------ full workloads
@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4])
def test_bumps3d_64(codec, torch, eb):
    check_parity(codec, torch, fields.bumps3d(), 3, fz.EB_REL, eb)


# the paper's five relative bounds (Sec. 4.1)
PAPER_EBS = [1e-2, 5e-3, 1e-3, 5e-4, 1e-4]


@pytest.mark.parametrize("eb", PAPER_EBS)
def test_climate2d_1800x3600(codec, torch, eb):
    check_parity(codec, torch, fields.climate2d(), 2, fz.EB_REL, eb, all_cores=True)


@pytest.fixture(scope="module")
def cosmo512():
    return fields.cosmo3d(512)


@pytest.mark.parametrize("eb", PAPER_EBS)
def test_cosmo3d_512(codec, torch, cosmo512, eb):
    g, xr = check_parity(codec, torch, cosmo512, 3, fz.EB_REL, eb, all_cores=True)
    info = fz.inspect(g[:64])
    x = cosmo512.ravel().astype(np.float64)
    err = np.abs(x - xr.astype(np.float64))
    slack = 2.0 ** -22 * np.maximum(np.abs(x), np.abs(xr.astype(np.float64)))
    assert np.all(err <= info["eb"] + slack)


@pytest.mark.parametrize("rel", [1e-3, 1e-5])
def test_cosmo3d_512_absolute_bound(codec, torch, cosmo512, rel):
    """An absolute bound on the full field (every element range-checked on
    the device); 1e-5 of the range gives codes beyond 7 bits in most tiles."""
    eb = float(rel * (cosmo512.max() - cosmo512.min()))
    check_parity(codec, torch, cosmo512, 3, fz.EB_ABS, eb, all_cores=True)


def test_1d_64m_values(codec, torch):
    """A 1-D field of 2^26 values (256 MiB): 8192 chunks of 4 tiles."""
    rng = np.random.default_rng(26)
    x = np.cumsum(rng.standard_normal(1 << 26, dtype=np.float32), dtype=np.float64)
    x = (x / np.abs(x).max()).astype(np.float32)
    check_parity(codec, torch, x, 1, fz.EB_REL, 1e-4, all_cores=True)


# ------------------------------------------------------------ edge cases
def _tile_kinds(stream: bytes):
    """(narrow, wide, narrow with escapes) tile counts of a stream, from its
    flag bytes: a tile is narrow when the planes of magnitude bits 7..14
    (flag bytes 7..14 and 23..30 of its 32) are all absent.  A narrow tile
    whose stream has outliers in it holds sign-only escape codes; counted
    here from the outlier records' code indices."""
    nt = fz.inspect(stream[:64])["n_tiles"]
    info = fz.inspect(stream[:64])
    f = np.frombuffer(stream, np.uint8, 32 * nt, 64).reshape(nt, 32)
    narrow = (np.concatenate([f[:, 7:15], f[:, 23:31]], axis=1) == 0).all(axis=1)
    recs = np.frombuffer(stream, np.uint32, 2 * info["n_outliers"],
                         len(stream) - 8 * info["n_outliers"]).reshape(-1, 2)
    esc_tiles = np.unique(recs[:, 0] // 2048)
    return (int(narrow.sum()), int((~narrow).sum()),
            int(narrow[esc_tiles[esc_tiles < nt]].sum()))


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_narrow_and_wide_tiles_mix(codec, torch, ndim):
    """Smooth regions (codes within 7 bits: the 16-plane transposes) beside
    noisy ones (wider codes: the 32-plane transposes) and isolated spikes
    (escapes: a narrow-by-flags tile holding sign-only escape codes, which
    the decompressor's narrow path must patch)."""
    rng = np.random.default_rng(40 + ndim)
    shape = {1: (3 * 8192 + 77,), 2: (2 * 128 + 9, 3 * 64 + 5), 3: (3 * 8 + 3, 2 * 32 + 7, 3 * 32 + 1)}[ndim]
    x = fields.grf(shape, -3.0, 50 + ndim).astype(np.float32)
    flat = x.reshape(-1)
    half = flat.size // 2
    flat[half:] += rng.normal(0, 2.0, flat.size - half).astype(np.float32)    # noisy half
    spikes = rng.choice(half, 6, replace=False)
    flat[spikes] = 5000.0                                                  # escapes in the smooth half
    g, _ = check_parity(codec, torch, x, ndim, fz.EB_ABS, 1e-2)
    n_narrow, n_wide, n_narrow_esc = _tile_kinds(g)
    assert n_narrow > 0 and n_wide > 0 and n_narrow_esc > 0, (n_narrow, n_wide, n_narrow_esc)
    assert fz.inspect(g[:64])["n_outliers"] > 0


def test_all_zero_and_constant(codec, torch):
    check_parity(codec, torch, np.zeros((40, 70, 33), np.float32), 3, fz.EB_ABS, 0.1)
    check_parity(codec, torch, np.full((40, 70, 33), 7.25, np.float32), 3, fz.EB_REL, 1e-3)
    check_parity(codec, torch, np.full((1000, 3), -2.0, np.float32), 2, fz.EB_ABS, 1e-3)


@pytest.mark.parametrize("shape,ndim", [((24, 64, 64), 3), ((40, 67, 96), 3),
                                        ((300, 260), 2), ((301, 259), 2),
                                        ((40000,), 1)])
def test_outliers(codec, torch, shape, ndim):
    rng = np.random.default_rng(8)
    x = rng.normal(0, 1, shape).astype(np.float32)
    flat = x.reshape(-1)
    idx = rng.choice(flat.size, 40, replace=False)
    flat[idx] = rng.choice([-1, 1], 40) * rng.uniform(2e4, 9e4, 40)
    g, _ = check_parity(codec, torch, x, ndim, fz.EB_ABS, 0.5)
    assert fz.inspect(g[:64])["n_outliers"] >= 40


def test_many_outliers(codec, torch):
    rng = np.random.default_rng(9)
    x = (rng.normal(0, 1, (16, 96, 64)) * 3e4).astype(np.float32)
    g, _ = check_parity(codec, torch, x, 3, fz.EB_ABS, 0.5)
    assert fz.inspect(g[:64])["n_outliers"] > 10000


def test_deterministic(codec, torch):
    x = fields.grf((33, 100, 70), -2.5, 2).astype(np.float32)
    a = gpu_compress(codec, torch, x, 3, fz.EB_REL, 1e-4)
    b = gpu_compress(codec, torch, x, 3, fz.EB_REL, 1e-4)
    assert a == b


# ------------------------------------------------------------ errors
def _status(codec, torch, x, ndim, mode, eb, cap=None):
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    dims = list(x.shape[::-1])[:ndim]
    cap = cap if cap is not None else fz.compress_bound(dims, ndim)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    return codec.compress_into(xt, out, mode, eb, ndim, raise_on_error=False)


@pytest.mark.parametrize("mode", [fz.EB_ABS, fz.EB_REL])
def test_nonfinite(codec, torch, mode):
    for bad in (np.nan, np.inf, -np.inf):
        x = np.ones((20, 40, 40), np.float32)
        x[7, 3, 5] = bad
        assert _status(codec, torch, x, 3, mode, 1e-3)[0] == fz.ERR_NONFINITE
        assert oracle.compress(x, 3, mode, 1e-3)[0] == oracle.ERR_NONFINITE


def test_eb_range(codec, torch):
    x = np.ones((64, 64), np.float32)
    x[3, 3] = 1e7
    assert _status(codec, torch, x, 2, fz.EB_ABS, 1e-3)[0] == fz.ERR_EB_RANGE
    assert oracle.compress(x, 2, fz.EB_ABS, 1e-3)[0] == oracle.ERR_EB_RANGE
    # a relative bound whose absolute value underflows fp32
    assert _status(codec, torch, x, 2, fz.EB_REL, 1e-300)[0] == fz.ERR_EB_RANGE


def test_capacity_reports_size(codec, torch):
    x = fields.grf((40, 64, 64), -3.0, 3).astype(np.float32)
    ost, ostream = oracle.compress(x, 3, fz.EB_REL, 1e-4)
    st, size = _status(codec, torch, x, 3, fz.EB_REL, 1e-4, cap=len(ostream) - 16)
    assert st == fz.ERR_CAPACITY and size == len(ostream)
    st, size = _status(codec, torch, x, 3, fz.EB_REL, 1e-4, cap=100)
    assert st == fz.ERR_CAPACITY and size == fz.stream_min_bytes((64, 64, 40), 3)
    st, size = _status(codec, torch, x, 3, fz.EB_REL, 1e-4, cap=len(ostream))
    assert st == fz.OK and size == len(ostream)


def _dec_status(codec, torch, s, cap=None, nbytes=None):
    st_t = torch.from_numpy(np.frombuffer(bytes(s), np.uint8).copy()).cuda()
    out = torch.empty(cap if cap is not None else 1 << 22, dtype=torch.float32,
                      device="cuda")
    return codec.decompress_into(st_t, out, nbytes=nbytes, raise_on_error=False)


def test_corrupt_streams(codec, torch):
    x = fields.grf((40, 70), -3.0, 3).astype(np.float32)
    x[5, 5] = 3e4
    _, s = oracle.compress(x, 2, fz.EB_ABS, 0.05)
    assert _dec_status(codec, torch, s) == fz.OK
    bad = bytearray(s); bad[0] = ord("X")
    assert _dec_status(codec, torch, bad) == fz.ERR_CORRUPT
    assert _dec_status(codec, torch, s, nbytes=len(s) - 16) == fz.ERR_CORRUPT
    bad = bytearray(s); bad[64] ^= 0x01                 # a flag bit
    assert _dec_status(codec, torch, bad) == fz.ERR_CORRUPT
    assert _dec_status(codec, torch, s, cap=10) == fz.ERR_CAPACITY
    if fz.inspect(s[:64])["n_outliers"]:
        bad = bytearray(s); bad[-8] ^= 0x01              # outlier index
        assert _dec_status(codec, torch, bad) == fz.ERR_CORRUPT
        assert oracle.decompress(bytes(bad))[0] == oracle.ERR_CORRUPT


def _tile_blocks(stream, n_elems):
    """compacted 16-byte blocks per tile: the set bits of its 32 flag bytes"""
    b = np.frombuffer(stream, np.uint8)
    nt = (n_elems + 2047) // 2048
    return np.unpackbits(b[64:64 + 32 * nt].reshape(nt, 32), axis=1).sum(1)


@pytest.mark.parametrize("ndim", [3, 2])
def test_dense_tiles_stored_a_round_early(codec, torch, ndim):
    """A compute warp keeps each tile's compacted blocks in its ring until
    the tile's prefix arrives two rounds later, and stages the next tile's
    bit planes in 256 blocks at the other end; a waiting tile of more than
    184 blocks (of the ring's 440) is therefore stored a round early.  Fields
    of about 10,000 tiles (several rounds per warp on the whole GPU) with
    dense and sparse tiles alternating: byte parity with the oracle, and the
    oracle's own stream shows both kinds in numbers."""
    x = fields.dense_sparse(ndim, 96 + ndim)
    g, _ = check_parity(codec, torch, x, ndim, fz.EB_ABS, 0.05)
    nnz = _tile_blocks(g, x.size)
    assert (nnz > 184).sum() >= 2000 and (nnz <= 104).sum() >= 2000


def test_bounded_wait_times_out_and_recovers(codec, torch):
    """A unit that never publishes its look-back aggregate: the successors'
    bounded waits give up and the call reports FZ_ERR_TIMEOUT; the context
    and the GPU stay usable.  The compressor's units are 15 tiles, the
    decompressor's offsets pass takes 512 chunks per unit, so the second
    field spans two of those."""
    x = fields.grf((32, 128, 128), -3.0, 6).astype(np.float32)
    y = fields.grf((72, 256, 256), -3.0, 7).astype(np.float32)     # 576 chunks
    _, s = oracle.compress(y, 3, fz.EB_REL, 1e-3)
    codec.set_wait_limit_ns(20_000_000)
    codec.debug_skip_publish(5)
    try:
        assert _status(codec, torch, x, 3, fz.EB_REL, 1e-3)[0] == fz.ERR_TIMEOUT
        assert _dec_status(codec, torch, s, cap=y.size) == fz.ERR_TIMEOUT
    finally:
        codec.debug_skip_publish(None)
        codec.set_wait_limit_ns(2_000_000_000)
    check_parity(codec, torch, x, 3, fz.EB_REL, 1e-3)
    check_parity(codec, torch, y, 3, fz.EB_REL, 1e-3)


# ------------------------------------------------------------ host API
def test_host_buffer_calls(codec, torch):
    x = fields.climate2d(300, 500)
    _, ostream = oracle.compress(x, 2, fz.EB_REL, 1e-3)
    s = codec.compress_host(x, mode="rel", eb=1e-3)
    assert s.tobytes() == ostream
    y = codec.decompress_host(s)
    _, xr = oracle.decompress(ostream)
    np.testing.assert_array_equal(y.ravel().view(np.uint32), xr.view(np.uint32))


def _host_pipeline_cases():
    rng = np.random.default_rng(77)
    out = []
    # 3-D: 256^3 floats (64 MiB of output): four slabs of chunk planes
    out.append(("grf3d_256", fields.grf((256, 256, 256), -3.0, 71).astype(np.float32), 3,
                fz.EB_REL, 1e-3))
    # 3-D with a ragged last chunk plane and escapes in every slab
    x = fields.grf((261, 250, 260), -2.5, 72).astype(np.float32)
    x.reshape(-1)[rng.integers(0, x.size, 4000)] = 5e4
    out.append(("grf3d_ragged_escapes", x, 3, fz.EB_ABS, 1e-2))
    # 2-D: chunk rows of 128 rows, the last one ragged
    out.append(("grf2d_4100x4099", fields.grf((4100, 4099), -3.0, 73).astype(np.float32), 2,
                fz.EB_REL, 1e-4))
    # 1-D: chunks of 8192 values, the last one ragged
    out.append(("noise1d", (np.cumsum(rng.standard_normal((1 << 24) + 4321)) * 1e-2)
                .astype(np.float32), 1, fz.EB_REL, 1e-3))
    return out


@pytest.mark.parametrize("case", range(4))
def test_host_buffer_decompression_in_slabs(codec, torch, case):
    # fields of 64 MiB or more: the host-buffer decompression copies the
    # stream in and the field out in slabs, overlapped with the decoding
    name, x, nd, mode, eb = _host_pipeline_cases()[case]
    assert 4 * x.size >= 64 << 20, name
    st, ostream = oracle.compress(x, nd, mode, eb, all_cores=True)
    assert st == oracle.OK
    s = codec.compress_host(x, mode="rel" if mode == fz.EB_REL else "abs", eb=eb, ndim=nd)
    assert s.tobytes() == ostream, name
    y = codec.decompress_host(s)
    _, xr = oracle.decompress(ostream, all_cores=True)
    np.testing.assert_array_equal(y.ravel().view(np.uint32), xr.view(np.uint32), err_msg=name)
    # the device-buffer call and the host-buffer call alternate on one context
    ys = codec.decompress(torch.from_numpy(np.frombuffer(ostream, np.uint8).copy()).cuda())
    assert torch.equal(ys.reshape(-1).cpu(), torch.from_numpy(xr)), name
    y2 = codec.decompress_host(s)
    np.testing.assert_array_equal(y2.ravel().view(np.uint32), xr.view(np.uint32), err_msg=name)


@pytest.mark.parametrize("case", ["grf3d", "escapes2d", "narrow_cap"])
def test_host_buffer_compression_into_pinned_memory(codec, torch, case):
    # a pinned output buffer, as the end-to-end measurement uses, and one too
    # small for the stream
    rng = np.random.default_rng(81)
    if case == "grf3d":
        x, nd, mode, eb = fields.grf((96, 128, 160), -3.0, 82).astype(np.float32), 3, "rel", 1e-3
    else:
        x = fields.grf((700, 900), -2.5, 83).astype(np.float32)
        x.reshape(-1)[rng.integers(0, x.size, 3000)] = 4e4
        nd, mode, eb = 2, "abs", 1e-2
    st, ostream = oracle.compress(x, nd, fz.EB_REL if mode == "rel" else fz.EB_ABS, eb)
    assert st == oracle.OK
    cap = len(ostream) + 4096 if case != "narrow_cap" else len(ostream) - 1
    pinned = torch.empty(cap, dtype=torch.uint8, pin_memory=True)
    out = pinned.numpy()
    if case == "narrow_cap":
        with pytest.raises(fz.FZError) as e:
            codec.compress_host(x, mode=mode, eb=eb, ndim=nd, out=out)
        assert e.value.status == fz.ERR_CAPACITY
        return
    s = codec.compress_host(x, mode=mode, eb=eb, ndim=nd, out=out)
    assert s.tobytes() == ostream, case
    y = codec.decompress_host(s)
    _, xr = oracle.decompress(ostream)
    np.testing.assert_array_equal(y.ravel().view(np.uint32), xr.view(np.uint32))


def test_host_buffer_decompression_in_slabs_corrupt(codec, torch):
    x = fields.grf((256, 256, 256), -3.0, 74).astype(np.float32)
    s = codec.compress_host(x, mode="rel", eb=1e-3).copy()
    # a flag byte of the second slab set where its block was zero: the
    # offsets no longer add up to the header's block count
    flags = s[64:64 + 32 * (x.size // 2048)]
    zero = np.flatnonzero(flags[flags.size // 2:] != 0xFF)[0] + flags.size // 2
    s[64 + zero] |= (~s[64 + zero]) & 0xFF
    with pytest.raises(fz.FZError) as e:
        codec.decompress_host(s)
    assert e.value.status == fz.ERR_CORRUPT
    y = codec.decompress_host(codec.compress_host(x, mode="rel", eb=1e-3))
    _, ostream = oracle.compress(x, 3, fz.EB_REL, 1e-3, all_cores=True)
    _, xr = oracle.decompress(ostream, all_cores=True)
    np.testing.assert_array_equal(y.ravel().view(np.uint32), xr.view(np.uint32))


# ------------------------------------------------------------ wide quantiser
def _wide_cases():
    rng = np.random.default_rng(91)
    rough = {1: (70001,), 2: (130, 211), 3: (19, 37, 45)}
    out = []
    for nd, shape in rough.items():
        x = (rng.standard_normal(shape) * 3e4).astype(np.float32)
        out.append((f"rough{nd}d_abs", x, nd, fz.EB_ABS, 5e-4))
        out.append((f"rough{nd}d_rel", x, nd, fz.EB_REL, 2e-8))
    smooth = (fields.grf((40, 64, 96), -3.0, 92) * 1e5).astype(np.float32)
    out.append(("smooth3d_abs", smooth, 3, fz.EB_ABS, 2e-3))
    out.append(("smooth3d_rel", smooth, 3, fz.EB_REL, 1e-8))
    return out


@pytest.mark.parametrize("case", range(8))
def test_wide_quantiser_matches_the_oracle(codec, torch, case):
    """|q| past 2^22 - 1 (up to 2^28 - 1): the second launch with integer
    quantisation gives the oracle's stream (header byte 7 set) and its
    reconstruction; absolute bounds reach it through the range pass that
    classifies the first launch's range error, relative bounds through the
    range pass itself."""
    name, x, ndim, mode, eb = _wide_cases()[case]
    g, xr = check_parity(codec, torch, x, ndim, mode, eb)
    info = fz.inspect(g[:64])
    assert info["wide"], name
    # the reconstruction is within the bound
    err = np.abs(x.ravel().astype(np.float64) - xr.astype(np.float64))
    slack = 2.0 ** -22 * np.maximum(np.abs(x.ravel()), np.abs(xr)).astype(np.float64)
    assert np.all(err <= info["eb"] + slack)


def test_wide_quantiser_limits_and_other_entries(codec, torch):
    x = (np.random.default_rng(93).standard_normal((19, 37, 45)) * 3e4).astype(np.float32)
    # beyond 2^28 - 1: refused by both, in both modes
    assert _status(codec, torch, x * np.float32(1e4), 3, fz.EB_ABS, 5e-4)[0] == fz.ERR_EB_RANGE
    assert oracle.compress(x * np.float32(1e4), 3, oracle.EB_ABS, 5e-4)[0] == oracle.ERR_EB_RANGE
    assert _status(codec, torch, x, 3, fz.EB_REL, 1e-10)[0] == fz.ERR_EB_RANGE
    assert oracle.compress(x, 3, oracle.EB_REL, 1e-10)[0] == oracle.ERR_EB_RANGE
    # whole-field Lorenzo with the wide quantiser
    st, ostream = oracle.compress(x, 3, oracle.EB_ABS, 5e-4, whole=True)
    assert st == oracle.OK and ostream[7] == 1
    s = codec.compress(torch.from_numpy(x).cuda(), mode="abs", eb=5e-4, whole=True)
    assert s.cpu().numpy().tobytes() == ostream
    y = codec.decompress(s).cpu().numpy().ravel()
    st, want = oracle.decompress(ostream)
    np.testing.assert_array_equal(y.view(np.uint32), want.view(np.uint32))
    # a server decompresses a wide stream like fz_decompress
    st, stream = oracle.compress(x, 3, oracle.EB_ABS, 5e-4)
    srv = fz.Server(0, pool_bytes=256 << 20)
    try:
        got = srv.fetch(srv.submit_decompress(np.frombuffer(stream, np.uint8).copy()))
    finally:
        srv.close()
    st, want = oracle.decompress(stream)
    np.testing.assert_array_equal(got.reshape(-1).view(np.uint32), want.view(np.uint32))
    # batches keep |q| within 2^22 - 1
    xt = torch.from_numpy(x).cuda()
    out = torch.zeros(fz.compress_bound([45, 37, 19], 3), dtype=torch.uint8, device="cuda")
    b = fz.Batch(codec, [(xt, out, "rel", 2e-8, 3)])
    try:
        sizes, sts = b.compress()
        assert sts[0] == fz.ERR_EB_RANGE
    finally:
        b.close()
