"""GPU: the request server.  Compress and decompress requests of mixed sizes
submitted all at once (so that later ones join batches while earlier ones
run) and one at a time must give the same results, and the same as the
single-field calls; admission waits for pool room; errors are per request."""
import numpy as np
import pytest

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


def _many_escapes():
    rng = np.random.default_rng(9)
    return (rng.normal(0, 1, (16, 96, 64)) * 3e4).astype(np.float32)   # > 10000 escapes


def _workload():
    comp = [
        (fields.climate2d(300, 500), "rel", 1e-3),
        (fields.bumps3d(64), "rel", 1e-4),
        (fields.grf((33, 70, 41), -3.0, 41).astype(np.float32), "rel", 1e-3),
        (fields.grf((257, 301), -2.5, 42).astype(np.float32), "abs", 0.01),
        (fields.grf((30001,), -2.0, 43).astype(np.float32), "rel", 1e-3),
        (_many_escapes(), "abs", 0.5),
    ]
    for i, (shape, ndim, beta, eb) in enumerate(fields.batch_shapes(count=40, seed=44)):
        if np.prod(shape) * 4 <= (4 << 20):
            comp.append((fields.grf(shape, beta, 200 + i).astype(np.float32), "rel", eb))
        if len(comp) >= 20:
            break
    dec_src = [
        (fields.grf((40, 64, 96), -3.0, 45).astype(np.float32), "rel", 1e-3),
        (fields.climate2d(260, 77), "rel", 1e-2),
        (fields.grf((8193,), -2.0, 46).astype(np.float32), "abs", 1e-3),
        (fields.bumps3d(64), "rel", 1e-3),
    ]
    return comp, dec_src


def _expected(codec, torch, comp, dec_src):
    want_c = [codec.compress(torch.from_numpy(x).cuda(), mode=m, eb=e, ndim=x.ndim)
              .cpu().numpy() for x, m, e in comp]
    streams = [codec.compress(torch.from_numpy(x).cuda(), mode=m, eb=e, ndim=x.ndim)
               .cpu().numpy() for x, m, e in dec_src]
    want_d = [codec.decompress(torch.from_numpy(s).cuda()).cpu().numpy() for s in streams]
    return want_c, streams, want_d


def _submit_all(srv, comp, streams):
    ids = []
    for i in range(max(len(comp), len(streams))):
        if i < len(comp):
            x, m, e = comp[i]
            ids.append(("c", i, srv.submit_compress(x, m, e)))
        if i < len(streams):
            ids.append(("d", i, srv.submit_decompress(streams[i])))
    return ids


def test_server_same_results_alone_and_in_the_mix(codec, torch):
    comp, dec_src = _workload()
    want_c, streams, want_d = _expected(codec, torch, comp, dec_src)
    srv = fz.Server(0, pool_bytes=1 << 30, max_batch=64)
    try:
        # in the mix: everything submitted before anything is fetched
        ids = _submit_all(srv, comp, streams)
        mix = {(k, i): srv.fetch(rid) for k, i, rid in ids}
        # alone: each request by itself
        alone = {}
        for k, i, _ in ids:
            if k == "c":
                x, m, e = comp[i]
                alone[(k, i)] = srv.fetch(srv.submit_compress(x, m, e))
            else:
                alone[(k, i)] = srv.fetch(srv.submit_decompress(streams[i]))
        for (k, i), got in mix.items():
            want = want_c[i] if k == "c" else want_d[i]
            assert got.tobytes() == want.tobytes(), (k, i)
            assert alone[(k, i)].tobytes() == got.tobytes(), (k, i)
        assert fz.inspect(mix[("c", 5)][:64].tobytes())["n_outliers"] > 10000
        st = srv.stats()
        assert st["completed"] == 2 * len(ids) and st["failed"] == 0
        assert st["p99_ms"] >= st["p50_ms"] > 0 and st["queued"] == 0
    finally:
        srv.close()


def test_server_admission_waits_for_pool_room(codec, torch):
    xs = [fields.grf((64, 128, 128), -3.0, 60 + i).astype(np.float32) for i in range(10)]
    want = [codec.compress(torch.from_numpy(x).cuda(), mode="rel", eb=1e-3).cpu().numpy()
            for x in xs]
    # each request holds ~4 MiB in and up to ~6.5 MiB out: a few at a time fit
    srv = fz.Server(0, pool_bytes=24 << 20, max_batch=8)
    try:
        ids = [srv.submit_compress(x, "rel", 1e-3) for x in xs]
        assert srv.stats()["queued"] > 0 or srv.stats()["in_flight"] < len(xs)
        for rid, w in zip(ids, want):
            assert srv.fetch(rid).tobytes() == w.tobytes()
        big = np.zeros((64, 512, 512), np.float32)              # 64 MiB > the pool
        with pytest.raises(fz.FZError) as e:
            srv.submit_compress(big, "rel", 1e-3)
        assert e.value.status == fz.ERR_CAPACITY
    finally:
        srv.close()


def test_server_errors_are_per_request(codec, torch):
    good = fields.bumps3d(64)
    bad = good.copy()
    bad[1, 2, 3] = np.inf
    s = codec.compress(torch.from_numpy(good).cuda(), mode="rel", eb=1e-3).cpu().numpy()
    corrupt = s.copy()
    corrupt[64] ^= 0x01                                          # a flag bit: counts mismatch
    srv = fz.Server(0, pool_bytes=256 << 20)
    try:
        ids = [srv.submit_compress(bad, "rel", 1e-3), srv.submit_decompress(corrupt),
               srv.submit_compress(good, "rel", 1e-3)]
        assert srv.wait(ids[0])[0] == fz.ERR_NONFINITE
        assert srv.wait(ids[1])[0] == fz.ERR_CORRUPT
        assert srv.fetch(ids[2]).tobytes() == s.tobytes()
        for rid in ids[:2]:
            with pytest.raises(fz.FZError):
                srv.fetch(rid)
        with pytest.raises(fz.FZError) as e:                     # not a stream at all
            srv.submit_decompress(np.zeros(100, np.uint8))
        assert e.value.status == fz.ERR_CORRUPT
    finally:
        srv.close()
