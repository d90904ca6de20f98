"""CPU: the log transform for point-wise relative bounds (Sec. 4.1: the
particle dataset is compressed log-transformed with the absolute bound a
point-wise relative bound implies), pinned against the closed forms
(math.log2, 2**y), exact values at powers of two and integers, the bound's
formula, and the end-to-end bound |x' - x| <= eps |x| through the oracle
compressor."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_12557_gb300 import fields


def _rand_floats(n, seed, lo=-149.0, hi=127.9):
    """Positive floats with log2 spread uniformly over [lo, hi)."""
    rng = np.random.default_rng(seed)
    return np.exp2(rng.uniform(lo, hi, n)).astype(np.float32)


def test_log2_exact_at_powers_of_two():
    for k in range(-149, 128):
        a = np.float32(2.0 ** k)
        assert oracle.pw_log2(a) == np.float32(k), k


def test_log2_matches_closed_form():
    a = _rand_floats(20000, 1)
    a = a[a > 0]
    y = np.array([oracle.pw_log2(v) for v in a], np.float64)
    ref = np.log2(a.astype(np.float64))
    tol = 3e-7 + np.abs(ref) * 2.0 ** -23        # formula error + one rounding of e + log2 m
    assert np.all(np.abs(y - ref) <= tol), np.max(np.abs(y - ref) - tol)


def test_exp2_exact_at_integers():
    for k in range(-149, 128):
        assert oracle.pw_exp2(np.float32(k)) == np.float32(2.0 ** k), k


def test_exp2_matches_closed_form():
    rng = np.random.default_rng(2)
    y = rng.uniform(-126.0, 127.99, 20000).astype(np.float32)
    e = np.array([oracle.pw_exp2(v) for v in y], np.float64)
    ref = np.exp2(y.astype(np.float64))
    assert np.all(np.abs(e / ref - 1.0) <= 1e-6)
    assert oracle.pw_exp2(np.float32(128.0)) == np.float32(np.finfo(np.float32).max)
    assert oracle.pw_exp2(np.float32(-151.0)) == 0.0


def test_bound_formula_and_domain():
    for eps in (1e-4, 1e-3, 0.01, 0.1, 0.5):
        st, eb = oracle.pwrel_bound(eps)
        assert st == oracle.OK and eb == math.log2(1.0 + eps) - 2.0 ** -14
    for eps in (9e-5, 0.51, float("nan"), -1e-3):
        assert oracle.pwrel_bound(eps)[0] == oracle.ERR_ARG


def test_forward_inverse_special_values():
    fmin = np.finfo(np.float32).tiny
    x = np.array([0.0, -0.0, 1.0, -1.0, 2.5, -1e-30, fmin, -fmin, 1e-45, -3e38, 7.0],
                 np.float32)
    st, y, signs = oracle.pwrel_forward(x)
    assert st == oracle.OK
    assert y[0] == -160.0 and y[1] == -160.0 and y[2] == 0.0 and y[3] == 0.0
    assert y[8] == -149.0                          # the smallest subnormal
    neg = [(int(signs[0]) >> i) & 1 for i in range(x.size)]
    assert neg == [0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0]
    xr = oracle.pwrel_inverse(y, signs)
    np.testing.assert_array_equal(xr[[0, 2, 3, 8]], x[[0, 2, 3, 8]])   # exact at 0 and powers
    assert np.signbit(xr[1]) and xr[1] == 0.0
    bad = x.copy()
    bad[4] = np.inf
    assert oracle.pwrel_forward(bad)[0] == oracle.ERR_NONFINITE
    bad[4] = np.nan
    assert oracle.pwrel_forward(bad)[0] == oracle.ERR_NONFINITE


def _check_bound(x, xr, eps):
    x = x.astype(np.float64)
    xr = xr.astype(np.float64)
    err = np.abs(xr - x)
    sub = np.abs(x) < np.finfo(np.float32).tiny
    assert np.all(err[~sub] <= eps * np.abs(x[~sub])), np.max(err[~sub] / np.abs(x[~sub]))
    assert np.all(err[sub] <= np.maximum(eps * np.abs(x[sub]), 2.0 ** -149))
    assert np.all(xr[x == 0] == 0)


@pytest.mark.parametrize("eps", [1e-4, 1e-3, 1e-2, 0.1])
def test_bound_through_the_compressor(eps):
    x = fields.particles1d(1 << 16, seed=7)
    x[:50] = np.exp2(np.random.default_rng(3).uniform(-149, -127, 50)).astype(np.float32)
    x[50:60] = [3.0e38, -3.0e38, 1e-38, 0.0, -0.0, 1.0, -1.0, 2.0, 1e-20, -1e20]
    st, y, signs = oracle.pwrel_forward(x)
    assert st == oracle.OK
    _, eb = oracle.pwrel_bound(eps)
    st, s = oracle.compress(y, 1, oracle.EB_ABS, eb)
    assert st == oracle.OK
    st, yr = oracle.decompress(s)
    assert st == oracle.OK
    _check_bound(x, oracle.pwrel_inverse(yr, signs), eps)


def test_bound_is_tight_enough_to_matter():
    """A bound without the margin would be exceeded somewhere (so the margin
    is doing work), and the relative errors use most of eps."""
    eps = 1e-3
    x = fields.particles1d(1 << 16, seed=8)
    _, y, signs = oracle.pwrel_forward(x)
    _, eb = oracle.pwrel_bound(eps)
    st, s = oracle.compress(y, 1, oracle.EB_ABS, eb)
    _, yr = oracle.decompress(s)
    xr = oracle.pwrel_inverse(yr, signs).astype(np.float64)
    nz = x != 0
    rel = np.abs(xr[nz] - x[nz]) / np.abs(x[nz].astype(np.float64))
    assert rel.max() > 0.9 * (2.0 ** eb - 1.0)
