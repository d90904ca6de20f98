"""GPU: the request server.  Compress and decompress requests of mixed sizes
submitted all at once (so that later ones join batches while earlier ones
run) and one at a time must give the same results, equal to the oracle's;
requests that arrive while a batch runs join a later batch and are in
flight on the device beside it; admission waits for pool room; errors are
per request."""
import time

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


def _oracle_stream(x, mode, eb):
    st, s = oracle.compress(x, x.ndim, oracle.EB_ABS if mode == "abs" else oracle.EB_REL, eb,
                            all_cores=True)
    assert st == oracle.OK
    return np.frombuffer(s, np.uint8)


def _expected(codec, torch, comp, dec_src):
    """Every expected result from the oracle: the compress requests' streams,
    the decompress requests' input streams and their reconstructions."""
    want_c = [_oracle_stream(x, m, e) for x, m, e in comp]
    streams = [_oracle_stream(x, m, e) for x, m, e in dec_src]
    want_d = []
    for s in streams:
        st, r = oracle.decompress(s.tobytes(), all_cores=True)
        assert st == oracle.OK
        want_d.append(r)
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


def _smooth_on_device(torch, shape, seed):
    """A smooth synthetic field made on the GPU (running sums of noise along
    x and y), copied to pinned host memory."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(shape, generator=g, device="cuda").cumsum(-1).cumsum(-2)
    x = (x / x.abs().max()).float()
    h = torch.empty(shape, dtype=torch.float32).pin_memory()
    h.copy_(x)
    return h


def test_late_requests_join_a_later_batch_in_flight_beside_the_first(codec, torch):
    """Wave 1 (2 GiB of fields) forms one batch; as soon as the server has
    launched it, wave 2 (small compress and decompress requests) arrives.
    Wave 2 must run in later batches, be launched before wave 1 is done, and
    be in flight on the device while wave 1's batch is (its GPU interval,
    from CUDA events on its stream, starts before the batch's ends); every
    result must equal the single calls' (and, for wave 2, the oracle's)."""
    wave1 = [_smooth_on_device(torch, (32, 1024, 1024), 500 + i) for i in range(16)]
    small = [fields.bumps3d(64), fields.climate2d(300, 500),
             fields.grf((33, 70, 41), -3.0, 47).astype(np.float32)]
    want_small = [_oracle_stream(x, "rel", 1e-3) for x in small]
    dec_want = []
    for s in want_small:
        st, r = oracle.decompress(s.tobytes())
        assert st == oracle.OK
        dec_want.append(r)
    srv = fz.Server(0, pool_bytes=8 << 30, max_batch=64)
    try:
        ids1 = [srv.submit_compress(x, "rel", 1e-3) for x in wave1]
        t0 = time.monotonic()
        while srv.info(ids1[-1])["launch_ms"] < 0:        # wave 1's batch launched
            assert time.monotonic() - t0 < 30
            time.sleep(20e-6)
        ids2c = [srv.submit_compress(x, "rel", 1e-3) for x in small]
        ids2d = [srv.submit_decompress(s) for s in want_small]
        for rid in ids1 + ids2c + ids2d:
            srv.wait(rid)
        inf1 = [srv.info(r) for r in ids1]
        inf2c = [srv.info(r) for r in ids2c]
        inf2d = [srv.info(r) for r in ids2d]
        got1 = [srv.fetch(r) for r in ids1]
        got2c = [srv.fetch(r) for r in ids2c]
        got2d = [srv.fetch(r) for r in ids2d]
    finally:
        srv.close()
    # wave 1 may have been split over batches while it was being submitted;
    # wave 2 came after all of them had been launched
    b1 = max(i["batch"] for i in inf1)
    assert min(i["batch"] for i in inf1) >= 1
    assert all(i["batch"] > b1 for i in inf2c)
    wave1_done = max(i["done_ms"] for i in inf1)
    wave1_gpu_end = max(i["gpu_end_ms"] for i in inf1)
    wave2 = inf2c + inf2d
    assert all(i["submit_ms"] >= 0 and i["gpu_end_ms"] >= i["gpu_start_ms"] >= 0 for i in wave2)
    assert min(i["launch_ms"] for i in wave2) < wave1_done
    assert min(i["gpu_start_ms"] for i in wave2) < wave1_gpu_end
    assert min(i["launch_seq"] for i in wave2) > max(i["launch_seq"] for i in inf1)
    for x, g in zip(wave1[:3], got1[:3]):
        want = codec.compress(x.cuda(), mode="rel", eb=1e-3).cpu().numpy()
        assert g.tobytes() == want.tobytes()
    for g, w in zip(got2c, want_small):
        assert g.tobytes() == w.tobytes()
    for g, w in zip(got2d, dec_want):
        assert np.array_equal(g.reshape(-1).view(np.uint32), w.view(np.uint32))


def test_server_admission_waits_for_pool_room(codec, torch):
    xs = [fields.grf((64, 128, 128), -3.0, 60 + i).astype(np.float32) for i in range(10)]
    want = [_oracle_stream(x, "rel", 1e-3) for x in xs]
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
    s = _oracle_stream(good, "rel", 1e-3)
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
