"""The oracle's all-cores variant (the paper's multi-threaded CPU version,
Sec. 4.4) must give the one-thread oracle's streams and reconstructions bit
for bit: it runs the same per-point, per-tile and per-chunk steps, only
spread over OpenMP threads."""
import numpy as np
import pytest

import oracle
from paper_2304_12557_gb300 import fields


def _cases():
    rng = np.random.default_rng(31)
    a = fields.grf((21, 70, 45), -3.0, 3).astype(np.float32)
    b = a.copy()
    b.reshape(-1)[rng.choice(b.size, 50, replace=False)] = 3e4      # escapes
    c = fields.climate2d(300, 333)
    d = np.cumsum(rng.normal(0, 1, 50_001)).astype(np.float32)
    e = np.zeros((9, 40, 33), np.float32)
    return [(a, 3, oracle.EB_REL, 1e-3), (a, 3, oracle.EB_ABS, 0.05), (b, 3, oracle.EB_ABS, 0.25),
            (c, 2, oracle.EB_REL, 1e-4), (d, 1, oracle.EB_REL, 1e-2), (e, 3, oracle.EB_REL, 1e-3)]


@pytest.mark.parametrize("case", range(6))
def test_all_cores_stream_and_reconstruction_equal_one_thread(case):
    x, ndim, mode, eb = _cases()[case]
    st1, s1 = oracle.compress(x, ndim, mode, eb)
    st2, s2 = oracle.compress(x, ndim, mode, eb, all_cores=True)
    assert st1 == st2 == oracle.OK
    assert s1 == s2
    r1 = oracle.decompress(s1)
    r2 = oracle.decompress(s1, all_cores=True)
    assert r1[0] == r2[0] == oracle.OK
    assert np.array_equal(r1[1].view(np.uint32), r2[1].view(np.uint32))


def test_all_cores_errors_match_one_thread():
    x = fields.grf((8, 40, 40), -3.0, 4).astype(np.float32)
    y = x.copy()
    y[2, 3, 4] = np.nan
    assert oracle.compress(y, 3, oracle.EB_REL, 1e-3, all_cores=True)[0] == oracle.ERR_NONFINITE
    assert oracle.compress(x, 3, oracle.EB_ABS, 1e-9, all_cores=True)[0] == oracle.ERR_EB_RANGE
    st, s = oracle.compress(x, 3, oracle.EB_REL, 1e-3)
    bad = bytearray(s)
    bad[64] ^= 1                                      # a flag bit without its block
    assert oracle.decompress(bytes(bad), all_cores=True)[0] == oracle.ERR_CORRUPT
    assert oracle.decompress(bytes(bad))[0] == oracle.ERR_CORRUPT


def test_threads_reported():
    assert oracle.threads() >= 1
