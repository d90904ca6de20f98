"""GPU: the log transform for point-wise relative bounds (Sec. 4.1).  The
transform kernels are bit-exact with the oracle's evaluation of the same
formulas (log values and sign words; reconstructions), and the whole chain
-- transform, compression of the log field with the derived absolute
bound, decompression, inverse -- gives the oracle's stream byte for byte
and |x' - x| <= eps |x| everywhere."""
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


def _mixed(n, seed):
    """Every kind of float32 the transform meets: spread magnitudes
    (subnormal to near FLT_MAX), both signs, zeros of both signs."""
    rng = np.random.default_rng(seed)
    x = np.exp2(rng.uniform(-149.0, 127.9, n)).astype(np.float32)
    x *= rng.choice(np.array([-1, 1], np.float32), n)
    z = rng.random(n) < 0.01
    x[z] = np.where(rng.random(z.sum()) < 0.5, 0.0, -0.0).astype(np.float32)
    return x


def _u32(a):
    return np.ascontiguousarray(a).view(np.uint32)


@pytest.mark.parametrize("n", [1, 31, 33, 4097, 5_000_003])
def test_forward_matches_oracle(codec, torch, n):
    x = _mixed(n, 11 + n % 97)
    y, signs = codec.pwrel_forward(torch.from_numpy(x).cuda())
    st, yo, so = oracle.pwrel_forward(x)
    assert st == oracle.OK
    np.testing.assert_array_equal(_u32(y.cpu().numpy()), _u32(yo))
    np.testing.assert_array_equal(signs.cpu().numpy().view(np.uint32), so)


@pytest.mark.parametrize("n", [1, 33, 1_000_001])
def test_inverse_matches_oracle(codec, torch, n):
    rng = np.random.default_rng(n)
    y = rng.uniform(-170.0, 130.0, n).astype(np.float32)
    y[: min(n, 8)] = np.array([-160, -154, -154.0001, -150, -149, 0, 127.99, 128],
                              np.float32)[: min(n, 8)]
    signs = rng.integers(0, 2 ** 32, (n + 31) // 32, dtype=np.uint64).astype(np.uint32)
    xg = codec.pwrel_inverse(torch.from_numpy(y).cuda(),
                             torch.from_numpy(signs.view(np.int32)).cuda())
    xo = oracle.pwrel_inverse(y, signs)
    np.testing.assert_array_equal(_u32(xg.cpu().numpy()), _u32(xo))


def test_forward_flags_nonfinite(codec, torch):
    x = _mixed(1000, 3)
    x[500] = np.nan
    with pytest.raises(fz.FZError) as e:
        codec.pwrel_forward(torch.from_numpy(x).cuda())
    assert e.value.status == fz.ERR_NONFINITE
    x[500] = 1.0                                   # the context is still usable
    codec.pwrel_forward(torch.from_numpy(x).cuda())


@pytest.mark.parametrize("eps", [1e-4, 1e-3, 1e-2])
def test_chain_bound_and_stream(codec, torch, eps):
    x = fields.particles1d(1 << 20, seed=21)
    x[:64] = _mixed(64, 5)
    xt = torch.from_numpy(x).cuda()
    y, signs = codec.pwrel_forward(xt)
    eb = fz.pwrel_bound(eps)
    s = codec.compress(y, mode="abs", eb=eb, ndim=1)
    yr = codec.decompress(s)
    xr = codec.pwrel_inverse(yr, signs).cpu().numpy().astype(np.float64)
    # the oracle's chain gives the same stream
    _, yo, _ = oracle.pwrel_forward(x)
    st, so = oracle.compress(yo, 1, oracle.EB_ABS, eb)
    assert st == oracle.OK and s.cpu().numpy().tobytes() == so
    xd = x.astype(np.float64)
    err = np.abs(xr - xd)
    sub = np.abs(xd) < np.finfo(np.float32).tiny
    assert np.all(err[~sub] <= eps * np.abs(xd[~sub]))
    assert np.all(err[sub] <= np.maximum(eps * np.abs(xd[sub]), 2.0 ** -149))
    assert np.all(xr[xd == 0] == 0)
