"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle step to a fact the paper or mathematics fixes:
hand-worked streams (tests/golden), hand-worked Lorenzo residuals, closed
forms, invariants and brute force on tiny inputs.  A plausible slip in the
oracle (a dropped Lorenzo term, a wrong sign, a transposed operand, an
off-by-one in the compaction) fails at least one of them.
"""
import itertools
import math
import struct

import numpy as np
import pytest

import oracle
from golden_io import expected_bytes, load
from paper_2304_12557_gb300 import fields

GOLDEN = ["g1_1d_basic.txt", "g2_1d_escape.txt", "g3_2d_basic.txt",
          "g4_3d_rel.txt"]


# ------------------------------------------------------------ golden streams
@pytest.mark.parametrize("name", GOLDEN)
def test_golden_stream_bytes(name):
    rec = load(name)
    st, s = oracle.compress(rec["x"], rec["ndim"], rec["mode"], rec["eb"])
    assert st == oracle.OK
    exp = expected_bytes(rec)
    assert s == exp


@pytest.mark.parametrize("name", GOLDEN)
def test_golden_stream_decodes_to_q(name):
    # with 2eb = 1 the reconstruction is q itself, i.e. the input integers
    rec = load(name)
    st, xr = oracle.decompress(expected_bytes(rec))
    assert st == oracle.OK
    np.testing.assert_array_equal(xr, rec["x"].ravel())


# ------------------------------------------------------------ Lorenzo
def test_lorenzo_1d_hand():
    q = np.array([3, 5, 4, 4], np.int32)
    np.testing.assert_array_equal(oracle.lorenzo(q, 1), [3, 2, -1, 0])


def test_lorenzo_2d_hand():
    q = np.array([[1, 2], [3, 5]], np.int32)      # rows are y
    np.testing.assert_array_equal(oracle.lorenzo(q, 2), [[1, 1], [2, 1]])


def test_lorenzo_3d_hand():
    q = np.array([[[0, 1], [2, 4]], [[1, 3], [3, 4]]], np.int32)
    exp = np.array([[[0, 1], [2, 1]], [[1, 1], [0, -2]]], np.int32)
    np.testing.assert_array_equal(oracle.lorenzo(q, 3), exp)


@pytest.mark.parametrize("ndim,shape", [(1, (20000,)), (2, (150, 140)),
                                        (3, (20, 40, 40))])
def test_lorenzo_annihilates_lower_dim_sums(ndim, shape):
    # The d-D first-order Lorenzo residual is the mixed difference
    # D_x D_y D_z q; it vanishes for any sum of functions that each miss one
    # coordinate, at every point not on a chunk's first line/plane.
    rng = np.random.default_rng(7)
    ch = oracle.chunk_shape(ndim)
    if ndim == 1:
        q = np.full(shape, int(rng.integers(-1000, 1000)), np.int32)
        d = oracle.lorenzo(q, 1)
        x = np.arange(shape[0])
        interior = x % ch[0] != 0
        assert np.all(d[interior] == 0)
        assert np.all(d[~interior] == q[~interior])
        return
    if ndim == 2:
        ny, nx = shape
        f = rng.integers(-1000, 1000, ny)
        g = rng.integers(-1000, 1000, nx)
        q = (f[:, None] + g[None, :]).astype(np.int32)
        d = oracle.lorenzo(q, 2)
        yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        interior = (xx % ch[0] != 0) & (yy % ch[1] != 0)
        assert np.all(d[interior] == 0)
        assert np.any(d[~interior] != 0)
        return
    nz, ny, nx = shape
    f = rng.integers(-500, 500, (nz, ny))
    g = rng.integers(-500, 500, (nz, nx))
    h = rng.integers(-500, 500, (ny, nx))
    q = (f[:, :, None] + g[:, None, :] + h[None, :, :]).astype(np.int32)
    d = oracle.lorenzo(q, 3)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                             indexing="ij")
    interior = (xx % ch[0] != 0) & (yy % ch[1] != 0) & (zz % ch[2] != 0)
    assert np.all(d[interior] == 0)
    assert np.any(d[~interior] != 0)


def test_lorenzo_matches_mixed_difference_inside_chunk():
    # brute force on a tiny block inside one chunk: residual = sum over the
    # 2^d corners of (-1)^(#offsets) q[p - offsets]
    rng = np.random.default_rng(3)
    q = rng.integers(-5000, 5000, (8, 32, 32)).astype(np.int32)
    d = oracle.lorenzo(q, 3)
    for z, y, x in [(1, 1, 1), (7, 31, 31), (3, 17, 5)]:
        s = 0
        for a, b, c in itertools.product((0, 1), repeat=3):
            s += (-1) ** (a + b + c) * int(q[z - c, y - b, x - a])
        assert d[z, y, x] == s


def test_lorenzo_chunk_independence():
    rng = np.random.default_rng(11)
    q = rng.integers(-3000, 3000, (16, 64, 64)).astype(np.int32)
    d0 = oracle.lorenzo(q, 3)
    q2 = q.copy()
    q2[8:16, 32:64, 0:32] += 77            # one whole chunk (z 8.., y 32.., x 0..)
    d1 = oracle.lorenzo(q2, 3)
    changed = d0 != d1
    assert changed[8:16, 32:64, 0:32].any()
    changed[8:16, 32:64, 0:32] = False
    assert not changed.any()
    # adding a constant to a chunk changes only its origin corner residual
    diff = (d1 - d0)[8:16, 32:64, 0:32]
    assert diff[0, 0, 0] == 77 and np.count_nonzero(diff) == 1


@pytest.mark.parametrize("ndim,shape", [(1, (20001,)), (2, (131, 200)),
                                        (3, (17, 45, 33))])
def test_lorenzo_inverse_identity(ndim, shape):
    rng = np.random.default_rng(5)
    q = rng.integers(-(2 ** 22) + 1, 2 ** 22, shape).astype(np.int32)
    d = oracle.lorenzo(q, ndim)
    np.testing.assert_array_equal(oracle.lorenzo_inverse(d, ndim), q)


# ------------------------------------------------------------ codes
def test_sign_magnitude_exhaustive():
    for v in range(-32767, 32768):
        c = oracle.encode(v)
        assert (c & 0x7FFF) == abs(v)
        assert (c >> 15) == (1 if v < 0 else 0)
        assert oracle.decode(c) == v
    assert oracle.encode(0) == 0          # never negative zero


@pytest.mark.parametrize("v", [32768, -32768, 40000, -(2 ** 25), 2 ** 25])
def test_escape_code(v):
    assert oracle.encode(v) == 0x8000


# ------------------------------------------------------------ bitshuffle
def test_bitshuffle_constant_codes():
    # every code = 1 -> each group's planes 0 and 16 are all ones
    w = np.full(1024, 0x00010001, np.uint32)
    out = oracle.bitshuffle(w)
    exp = np.zeros(1024, np.uint32)
    exp[0:32] = 0xFFFFFFFF
    exp[512:544] = 0xFFFFFFFF
    np.testing.assert_array_equal(out, exp)
    f = oracle.block_flags(out)
    np.testing.assert_array_equal(f, [0xFF, 0, 0, 0, 0xFF, 0, 0, 0])


@pytest.mark.parametrize("g,t,b", [(3, 5, 31), (0, 0, 0), (31, 31, 31),
                                   (17, 2, 9), (8, 30, 16)])
def test_bitshuffle_single_bit(g, t, b):
    w = np.zeros(1024, np.uint32)
    w[32 * g + t] = np.uint32(1) << np.uint32(b)
    out = oracle.bitshuffle(w)
    nz = np.flatnonzero(out)
    assert list(nz) == [32 * b + g]
    assert out[32 * b + g] == (1 << t)
    f = oracle.block_flags(out)
    k = (32 * b + g) // 4
    exp = np.zeros(8, np.uint32)
    exp[k // 32] = 1 << (k % 32)
    np.testing.assert_array_equal(f, exp)


def test_bitshuffle_inverse_and_popcount():
    rng = np.random.default_rng(2)
    for _ in range(5):
        w = rng.integers(0, 2 ** 32, 1024, dtype=np.uint64).astype(np.uint32)
        out = oracle.bitshuffle(w)
        np.testing.assert_array_equal(oracle.bitunshuffle(out), w)
        pc = lambda a: int(np.unpackbits(a.view(np.uint8)).sum())
        assert pc(out) == pc(w)
        # each group's 32x32 bit matrix is transposed: compare with numpy bits
        bits = np.unpackbits(w.view(np.uint8), bitorder="little").reshape(32, 32, 32)
        obits = np.unpackbits(out.view(np.uint8), bitorder="little").reshape(32, 32, 32)
        # bits[g, t, b] == obits[b, g, t]
        np.testing.assert_array_equal(bits.transpose(2, 0, 1), obits)


def test_block_flags_naive():
    rng = np.random.default_rng(9)
    out = np.zeros(1024, np.uint32)
    ks = rng.choice(256, 40, replace=False)
    for k in ks:
        out[4 * k + rng.integers(0, 4)] = rng.integers(1, 2 ** 32, dtype=np.uint64)
    f = oracle.block_flags(out)
    got = {32 * j + t for j in range(8) for t in range(32) if (f[j] >> t) & 1}
    assert got == set(int(k) for k in ks)


# ------------------------------------------------------------ tile geometry
@pytest.mark.parametrize("ndim,dims", [(1, (20000,)), (2, (130, 300)),
                                       (3, (40, 70, 17))])
def test_tile_coords_cover_field_once(ndim, dims):
    nt = oracle.num_tiles(ndim, dims)
    seen = set()
    inside = 0
    for t in range(nt):
        for p in range(0, 2048, 7 if nt > 50 else 1):
            ok, c = oracle.tile_coord(ndim, dims, t, p)
            if ok:
                inside += 1
                assert c not in seen
                seen.add(c)
                assert all(c[i] < dims[i] for i in range(ndim))
    if nt <= 50:
        assert inside == int(np.prod(dims))


def test_tile_coords_brick_order_3d():
    # group g = bx + 4*by holds an 8x4x2 brick, codes x-fastest
    dims = (64, 64, 16)
    ok, c = oracle.tile_coord(3, dims, 0, 64 * 5 + 8 * 2 + 3 + 32)
    # g=5 -> bx=1, by=1 ; l = 3 + 8*2 + 32*1 -> ix=3, iy=2, iz=1
    assert ok and c == (8 + 3, 4 + 2, 1)
    ok, c = oracle.tile_coord(3, dims, 4 * 1 + 2, 0)   # chunk 1 (cx=1), tile 2
    assert ok and c == (32, 0, 4)


# ------------------------------------------------------------ prequant / eb
def test_prequant_ties_to_even():
    # 2eb = 1: x = k + 0.5 is exactly representable, round half to even
    for x, q in [(2.5, 2), (3.5, 4), (-2.5, -2), (-3.5, -4), (0.5, 0),
                 (-0.5, 0), (1.5, 2), (2.4999998, 2), (4194302.5, 4194302)]:
        st, got = oracle.prequant1(x, 1.0)
        assert st == 0 and got == q, (x, got)


def test_prequant_range_guard():
    # |q| <= 2^28 - 1: every 3-D residual (a signed sum of eight q) fits the
    # outlier record's i32.  Floats near 2^28 are 16 apart.
    assert oracle.QMAX == 2 ** 28 - 1
    assert oracle.prequant1(4194304.0, 1.0) == (0, 4194304)
    assert oracle.prequant1(-4194303.5, 1.0) == (0, -4194304)
    assert oracle.prequant1(268435440.0, 1.0) == (0, 268435440)
    assert oracle.prequant1(-268435440.0, 1.0) == (0, -268435440)
    assert oracle.prequant1(268435456.0, 1.0)[0] == oracle.ERR_EB_RANGE
    assert oracle.prequant1(-268435456.0, 1.0)[0] == oracle.ERR_EB_RANGE
    assert oracle.prequant1(float("inf"), 1.0)[0] == oracle.ERR_EB_RANGE


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_wide_quantiser_flag_and_round_trip(ndim):
    # a field whose |q| passes 2^22 - 1 sets header byte 7 and still round
    # trips to the closed form fl(float(q) * 2eb); the 3-D stencil's residuals
    # then need outlier records beyond 2^22
    rng = np.random.default_rng(31 + ndim)
    shape = {1: (70001,), 2: (130, 211), 3: (19, 37, 45)}[ndim]
    x = (rng.standard_normal(shape) * 3e4).astype(np.float32)
    st, s = oracle.compress(x, ndim, oracle.EB_ABS, 5e-4)
    assert st == oracle.OK
    assert s[7] == 1
    ebx2, ebx2_r = struct.unpack("<2f", s[36:44])
    q = np.rint(x.astype(np.float32) * np.float32(ebx2_r)).astype(np.int64)
    assert np.abs(q).max() > 2 ** 22
    st, xr = oracle.decompress(s)
    assert st == oracle.OK
    exp = (q.astype(np.float32) * np.float32(ebx2)).astype(np.float32).ravel()
    np.testing.assert_array_equal(xr.view(np.uint32), exp.view(np.uint32))
    # the same field a little smaller stays narrow: byte 7 = 0
    st, s2 = oracle.compress((x / 64).astype(np.float32), ndim, oracle.EB_ABS, 5e-4)
    assert st == oracle.OK and s2[7] == 0
    # and beyond 2^28 - 1 it is refused
    assert oracle.compress(x * np.float32(1e4), ndim, oracle.EB_ABS, 5e-4)[0] == oracle.ERR_EB_RANGE


def test_derive_eb_rounds_down_and_reciprocal():
    for rel, lo, hi in [(1e-3, -1.0, 3.0), (1e-4, 265.0, 301.5),
                        (1e-2, 0.06, 15.6), (0.3, 0.0, 1e-30)]:
        st, e, e2, r = oracle.derive_eb(oracle.EB_REL, rel, lo, hi)
        assert st == 0
        eb_d = rel * (float(np.float32(hi)) - float(np.float32(lo)))
        assert float(e) <= eb_d < float(np.nextafter(e, np.float32(np.inf)))
        assert e2 == np.float32(2) * e
        assert r == np.float32(1.0 / float(e2))


def test_derive_eb_constant_field_and_errors():
    st, e, _, _ = oracle.derive_eb(oracle.EB_REL, 1e-3, 5.0, 5.0)
    assert st == 0 and e <= 5e-3 and np.nextafter(e, np.float32(1)) > 5e-3
    st, e, _, _ = oracle.derive_eb(oracle.EB_REL, 1e-3, 0.0, 0.0)
    assert st == 0 and e <= 1e-3
    assert oracle.derive_eb(oracle.EB_ABS, 1e-46)[0] == oracle.ERR_EB_RANGE
    assert oracle.derive_eb(oracle.EB_ABS, 3e38)[0] == oracle.ERR_EB_RANGE


# ------------------------------------------------------------ pipeline
def _field(shape, seed):
    return fields.grf(shape, -3.0, seed).astype(np.float32) * 10 + 3


@pytest.mark.parametrize("shape,ndim", fields.small_cases())
@pytest.mark.parametrize("mode,eb", [(oracle.EB_REL, 1e-2), (oracle.EB_REL, 1e-4),
                                     (oracle.EB_ABS, 0.37)])
def test_round_trip_equals_closed_form(shape, ndim, mode, eb):
    # all stages after pre-quantisation are lossless (Sec. 2.3, 4.3), so the
    # reconstruction is the elementwise closed form fl(q * 2eb)
    x = _field(shape, 13) if min(shape) > 1 else \
        np.random.default_rng(1).standard_normal(shape).astype(np.float32)
    st, s = oracle.compress(x, ndim, mode, eb)
    assert st == oracle.OK
    hdr = s[:64]
    eb_f, ebx2, ebx2_r = struct.unpack("<3f", hdr[32:44])
    st, xr = oracle.decompress(s)
    assert st == oracle.OK
    # closed form in numpy: independent of the C code
    # q is an integer (Sec. 2.3), so q = 0 reconstructs to +0.0
    q = np.rint(x.astype(np.float32) * np.float32(ebx2_r)).astype(np.int32)
    exp = (q.astype(np.float32) * np.float32(ebx2)).astype(np.float32).ravel()
    np.testing.assert_array_equal(xr.view(np.uint32), exp.view(np.uint32))
    # pointwise bound |x - x'| <= eb + 2^-22 max(|x|,|x'|)  (fp32 slack)
    xd = x.astype(np.float64).ravel()
    err = np.abs(xd - xr.astype(np.float64))
    slack = 2.0 ** -22 * np.maximum(np.abs(xd), np.abs(xr.astype(np.float64)))
    assert np.all(err <= eb_f + slack)
    # size closed form
    nt = struct.unpack("<I", hdr[20:24])[0]
    nnz, nout = struct.unpack("<2I", hdr[44:52])
    assert len(s) == 64 + 32 * nt + 16 * nnz + 8 * nout


def test_size_all_zero_field():
    x = np.zeros((40, 70, 33), np.float32)
    st, s = oracle.compress(x, 3, oracle.EB_ABS, 0.1)
    nt = oracle.num_tiles(3, (33, 70, 40))
    assert st == 0 and len(s) == 64 + 32 * nt


@pytest.mark.parametrize("k", [1, 500, 32767, 12345])
def test_size_constant_field(k):
    # constant q = k: the only non-zero residual of a chunk is its origin
    # corner (= k), so each chunk holds popcount(k) non-zero 16-byte blocks
    x = np.full((20, 50, 40), float(k), np.float32)
    st, s = oracle.compress(x, 3, oracle.EB_ABS, 0.5)
    nt = oracle.num_tiles(3, (40, 50, 20))
    nchunks = nt // 4
    assert st == 0
    assert len(s) == 64 + 32 * nt + 16 * bin(k).count("1") * nchunks


def test_outlier_path_round_trip():
    rng = np.random.default_rng(8)
    x = rng.normal(0, 1, (20, 40, 40)).astype(np.float32)
    x[3, 5, 7] = 5e4
    x[10, 33, 1] = -7e4
    x[19, 39, 39] = 4e4
    st, s = oracle.compress(x, 3, oracle.EB_ABS, 0.5)
    assert st == 0
    nout = struct.unpack("<I", s[48:52])[0]
    assert nout >= 3
    st, xr = oracle.decompress(s)
    q = np.rint(x * np.float32(1.0)).astype(np.int32).astype(np.float32)
    np.testing.assert_array_equal(xr.view(np.uint32), q.ravel().view(np.uint32))


def test_errors():
    x = np.ones((10, 10), np.float32)
    x[3, 3] = np.nan
    assert oracle.compress(x, 2, oracle.EB_REL, 1e-3)[0] == oracle.ERR_NONFINITE
    x[3, 3] = np.inf
    assert oracle.compress(x, 2, oracle.EB_ABS, 1e-3)[0] == oracle.ERR_NONFINITE
    x[3, 3] = 1e7
    assert oracle.compress(x, 2, oracle.EB_ABS, 1e-3)[0] == oracle.ERR_EB_RANGE
    assert oracle.compress(x, 2, oracle.EB_ABS, -1.0)[0] == oracle.ERR_ARG
    assert oracle.compress(x, 4, oracle.EB_ABS, 1.0)[0] == oracle.ERR_ARG


def test_corrupt_streams():
    x = _field((40, 70), 3)
    st, s = oracle.compress(x, 2, oracle.EB_REL, 1e-3)
    assert oracle.decompress(s)[0] == oracle.OK
    bad = bytearray(s); bad[0] = ord("X")
    assert oracle.decompress(bytes(bad))[0] == oracle.ERR_CORRUPT
    assert oracle.decompress(s[:-1])[0] == oracle.ERR_CORRUPT
    bad = bytearray(s); bad[64] ^= 0x80          # flip a flag bit
    assert oracle.decompress(bytes(bad))[0] == oracle.ERR_CORRUPT


def test_psnr_matches_uniform_error_model():
    # a rough field's quantisation error is ~uniform on [-eb, eb]: MSE = eb^2/3
    x = fields.grf((64, 128, 128), -2.0, 21).astype(np.float32)
    st, s = oracle.compress(x, 3, oracle.EB_REL, 1e-3)
    st, xr = oracle.decompress(s)
    rng_ = float(x.max()) - float(x.min())
    mse = float(np.mean((x.ravel().astype(np.float64) - xr) ** 2))
    psnr = 20 * math.log10(rng_) - 10 * math.log10(mse)
    assert abs(psnr - (20 * math.log10(1 / 1e-3) + 4.77)) < 0.2
