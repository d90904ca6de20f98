"""CPU: the whole-field Lorenzo variant of the oracle (the paper's chunks
make each chunk independent, Sec. 2.3; the variant takes every neighbour
inside the field, so there is no residual spike at chunk faces).  Pinned
against a brute-force stencil, the closed form for linear fields, the
chunked residuals where a field fits one chunk, exact round trips, and
reconstructions identical to the chunked stream's (both are lossless on
the quantised values).  The GPU library does not decode this variant yet
and must refuse its streams."""
import numpy as np
import pytest

import oracle
import paper_2304_12557_gb300 as fz
from paper_2304_12557_gb300 import fields


def _brute(q, ndim):
    """sum over the 2^ndim stencil corners, zero outside the field"""
    q = q.astype(np.int64)
    p = np.pad(q, [(1, 0)] * q.ndim)           # a zero layer below every axis
    out = np.zeros_like(q)
    for corner in range(1 << ndim):
        sl, sign = [], 1
        for ax in range(q.ndim):                # numpy axes: z, y, x (last = x)
            bit = (corner >> (q.ndim - 1 - ax)) & 1 if ax >= q.ndim - ndim else 0
            sl.append(slice(1 - bit, p.shape[ax] - bit))
            sign = -sign if bit else sign
        out += sign * p[tuple(sl)]
    return out


@pytest.mark.parametrize("shape,ndim", [((7,), 1), ((9000,), 1), ((5, 6), 2), ((130, 70), 2),
                                        ((3, 4, 5), 3), ((10, 40, 33), 3)])
def test_matches_brute_force_and_inverts(shape, ndim):
    rng = np.random.default_rng(sum(shape))
    q = rng.integers(-1000, 1000, shape).astype(np.int32)
    d = oracle.lorenzo_whole(q, ndim)
    np.testing.assert_array_equal(d.astype(np.int64), _brute(q, ndim))
    np.testing.assert_array_equal(oracle.lorenzo_whole_inverse(d, ndim), q.astype(np.int64))


def test_equals_chunked_inside_one_chunk():
    rng = np.random.default_rng(1)
    for shape, ndim in (((8192,), 1), ((128, 64), 2), ((8, 32, 32), 3)):
        q = rng.integers(-500, 500, shape).astype(np.int32)
        np.testing.assert_array_equal(oracle.lorenzo_whole(q, ndim), oracle.lorenzo(q, ndim))


def test_linear_field_closed_form():
    """q = a x + b y + c z + e: the residual is e at the origin, a, b, c on
    the three axes through it and 0 everywhere else -- in the chunked form
    every chunk repeats that pattern at its own origin."""
    a, b, c, e = 3, -5, 7, 11
    z, y, x = np.meshgrid(np.arange(20), np.arange(70), np.arange(40), indexing="ij")
    q = (a * x + b * y + c * z + e).astype(np.int32)
    d = oracle.lorenzo_whole(q, 3)
    want = np.zeros_like(d)
    want[0, 0, 1:] = a
    want[0, 1:, 0] = b
    want[1:, 0, 0] = c
    want[0, 0, 0] = e
    np.testing.assert_array_equal(d, want)
    assert np.count_nonzero(oracle.lorenzo(q, 3)) > np.count_nonzero(d)


def test_stream_round_trip_and_same_reconstruction():
    x = fields.bumps3d(64)                      # 2 x 2 x 8 chunks
    for eb in (1e-2, 1e-3):
        st, sw = oracle.compress(x, 3, oracle.EB_REL, eb, whole=True)
        assert st == oracle.OK and sw[4] == 2
        st, sc = oracle.compress(x, 3, oracle.EB_REL, eb)
        assert st == oracle.OK and sc[4] == 1
        stw, xw = oracle.decompress(sw)
        stc, xc = oracle.decompress(sc)
        assert stw == stc == oracle.OK
        np.testing.assert_array_equal(xw.view(np.uint32), xc.view(np.uint32))


def test_outliers_in_the_whole_field_form():
    x = fields.grf((40, 64, 96), -3.0, 9).astype(np.float32)
    x[5, 6, 7] = 5e4
    st, s = oracle.compress(x, 3, oracle.EB_ABS, 0.01, whole=True)
    assert st == oracle.OK
    st, xr = oracle.decompress(s)
    assert st == oracle.OK
    assert np.max(np.abs(xr - x.reshape(-1))) <= 0.01 * (1 + 1e-5) + 2 ** -22 * 5e4


def test_library_header_reads_the_variant():
    _, s = oracle.compress(fields.bumps3d(64), 3, oracle.EB_REL, 1e-3, whole=True)
    assert fz.inspect(s[:64])["version"] == 2
