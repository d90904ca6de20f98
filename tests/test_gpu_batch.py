"""GPU: many fields through one planned batch (one persistent launch per
dimensionality, replayed from a CUDA graph).  Every field's stream must be
byte for byte the oracle's and the single-field call's on the same data,
across graph replays, in-place changes of the inputs, graph-off runs,
autotuning and per-field errors."""
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


def _outliers(shape, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, shape).astype(np.float32)
    flat = x.reshape(-1)
    idx = rng.choice(flat.size, n, replace=False)
    flat[idx] = rng.choice([-1, 1], n) * rng.uniform(2e4, 9e4, n)
    return x


def _specs():
    """(array, ndim, mode, eb): aligned rows (TMA), unaligned rows (direct
    loads), 1-D, absolute and relative bounds, escapes, degenerate fields,
    and a run of small uneven fields shaped like the batched workload."""
    s = [
        (fields.climate2d(300, 500), 2, "rel", 1e-3),
        (fields.grf((257, 301), -3.0, 21).astype(np.float32), 2, "rel", 1e-2),
        (_outliers((40, 64, 96), 60, 22), 3, "abs", 0.5),
        (fields.grf((33, 70, 41), -3.0, 23).astype(np.float32), 3, "rel", 1e-4),
        (fields.bumps3d(64), 3, "rel", 1e-3),
        (fields.grf((30001,), -2.0, 24).astype(np.float32), 1, "rel", 1e-3),
        (fields.grf((8192,), -2.0, 25).astype(np.float32), 1, "abs", 1e-3),
        (fields.grf((129, 65), -2.5, 26).astype(np.float32), 2, "abs", 0.01),
        (np.zeros((16, 32, 32), np.float32), 3, "rel", 1e-3),
        (np.full((20, 40), 3.5, np.float32), 2, "rel", 1e-3),
    ]
    for i, (shape, ndim, beta, eb) in enumerate(fields.batch_shapes(count=60, seed=27)):
        if np.prod(shape) * 4 > (2 << 20):
            continue
        s.append((fields.grf(shape, beta, 100 + i).astype(np.float32), ndim, "rel", eb))
        if len(s) >= 30:
            break
    return s


def _single(codec, xt, ndim, mode, eb):
    return codec.compress(xt, mode=mode, eb=eb, ndim=ndim).cpu().numpy().tobytes()


def _make_batch(codec, torch, specs, cap_override=None):
    xs, outs, spec = [], [], []
    for i, (x, ndim, mode, eb) in enumerate(specs):
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        dims = list(xt.shape[::-1])[:ndim]
        cap = fz.compress_bound(dims, ndim)
        if cap_override and i in cap_override:
            cap = cap_override[i]
        out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        xs.append(xt)
        outs.append(out)
        spec.append((xt, out, mode, eb, ndim))
    return xs, outs, fz.Batch(codec, spec)


def _check(codec, specs, xs, outs, sizes, sts):
    for i, (x, ndim, mode, eb) in enumerate(specs):
        assert sts[i] == fz.OK, (i, sts[i])
        got = outs[i][: sizes[i]].cpu().numpy().tobytes()
        assert got == _single(codec, xs[i], ndim, mode, eb), i


def test_batch_equals_single_field_streams(codec, torch):
    specs = _specs()
    assert len(specs) >= 25
    xs, outs, b = _make_batch(codec, torch, specs)
    try:
        sizes, sts = b.compress()
        _check(codec, specs, xs, outs, sizes, sts)
        # every field against the oracle, and the escapes really happened
        for i, (x, ndim, mode, eb) in enumerate(specs):
            st, o = oracle.compress(x, ndim, oracle.EB_ABS if mode == "abs" else oracle.EB_REL,
                                    eb)
            assert st == oracle.OK and outs[i][: sizes[i]].cpu().numpy().tobytes() == o, i
        assert fz.inspect(outs[2][:64].cpu().numpy().tobytes())["n_outliers"] >= 60
        # a replay of the captured graph gives the same streams
        for o_ in outs:
            o_.zero_()
        sizes2, sts2 = b.compress()
        assert sizes2 == sizes and sts2 == sts
        _check(codec, specs, xs, outs, sizes2, sts2)
        # new contents in place: the replay compresses the new data
        for x in xs:
            x.mul_(1.7).add_(0.25)
        sizes3, sts3 = b.compress()
        _check(codec, specs, xs, outs, sizes3, sts3)
        # without the graph
        b.set_graph(False)
        sizes4, sts4 = b.compress()
        assert sizes4 == sizes3
        _check(codec, specs, xs, outs, sizes4, sts4)
    finally:
        b.close()


def test_batch_dense_tiles_stored_a_round_early(codec, torch):
    """A batch warp's ring has 360 blocks, so a waiting tile of more than
    104 blocks is stored a round early, before the next tile is staged.
    Large fields whose dense and sparse tiles alternate (both launches,
    several rounds per warp) beside small fields of the usual mix: every
    stream equals the oracle's."""
    specs = [(fields.dense_sparse(3, 98), 3, "abs", 0.05),
             (fields.dense_sparse(2, 99), 2, "abs", 0.05)] + _specs()[:6]
    xs, outs, b = _make_batch(codec, torch, specs)
    try:
        sizes, sts = b.compress()
        for i, (x, ndim, mode, eb) in enumerate(specs):
            assert sts[i] == fz.OK, (i, sts[i])
            st, o = oracle.compress(x, ndim, oracle.EB_ABS if mode == "abs" else oracle.EB_REL,
                                    eb)
            assert st == oracle.OK and outs[i][: sizes[i]].cpu().numpy().tobytes() == o, i
    finally:
        b.close()


def test_batch_escapes_in_consecutive_rounds(codec, torch):
    """Fields with escapes in nearly every tile and several rounds of work
    per block: a warp repacks an escaped tile while its previous tile's
    blocks are still waiting to be stored (the batch keeps one plane buffer
    per warp), in 2-D and 3-D, and in a relative-bound field."""
    specs = [
        (_outliers((96, 256, 256), 12000, 31), 3, "abs", 0.5),
        (_outliers((1024, 1536), 4000, 32), 2, "abs", 0.5),
        (_outliers((64, 128, 256), 6000, 33), 3, "rel", 1e-6),
        (fields.bumps3d(64), 3, "rel", 1e-3),
    ]
    xs, outs, b = _make_batch(codec, torch, specs)
    try:
        sizes, sts = b.compress()
        _check(codec, specs, xs, outs, sizes, sts)
        for i in range(3):
            assert fz.inspect(outs[i][:64].cpu().numpy().tobytes())["n_outliers"] >= 3000
    finally:
        b.close()


def test_batch_relative_only(codec, torch):
    """A batch of relative bounds only: its kernels skip the per-element
    quantiser check (the range pass has bounded every element)."""
    specs = [s for s in _specs() if s[2] == "rel"]
    assert len(specs) >= 20
    xs, outs, b = _make_batch(codec, torch, specs)
    try:
        sizes, sts = b.compress()
        _check(codec, specs, xs, outs, sizes, sts)
    finally:
        b.close()


def test_batch_row_class_boxes_edges(codec, torch):
    """Row-class TMA boxes (load path tma 2) on the shapes where the classes
    shift: every row width mod 4, field starts 4, 8 and 12 bytes past a
    16-byte boundary, planes whose row count is not a multiple of 4 (the
    class of a plane's first row moves from plane to plane), tiles reaching
    past y, z and x, a 2-D field of exactly 4 rows and one of 3 (which keeps
    direct loads), and escapes."""
    rng = np.random.default_rng(61)
    shapes = [((13, 5, 37), 3, 1), ((9, 7, 66), 3, 2), ((21, 33, 99), 3, 3), ((4, 301), 2, 1),
              ((3, 150), 2, 2), ((129, 67), 2, 3), ((17, 40, 70), 3, 0), ((2, 45, 41), 3, 1)]
    xs, outs, spec, want = [], [], [], []
    for i, (shape, ndim, lead) in enumerate(shapes):
        x = fields.grf(shape, -2.5, 62 + i).astype(np.float32)
        mode, eb = ("abs", 1e-2) if i % 2 else ("rel", 1e-3)
        if i == 2:
            x.reshape(-1)[rng.integers(0, x.size, 300)] = 3e4
        buf = torch.zeros(x.size + 4, dtype=torch.float32, device="cuda")
        xt = buf[lead: lead + x.size].view(*shape)
        xt.copy_(torch.from_numpy(x))
        out = torch.zeros(fz.compress_bound(list(shape[::-1])[:ndim], ndim), dtype=torch.uint8,
                          device="cuda")
        xs.append((buf, xt))
        outs.append(out)
        spec.append((xt, out, mode, eb, ndim))
        st, o = oracle.compress(x, ndim, oracle.EB_ABS if mode == "abs" else oracle.EB_REL, eb)
        assert st == oracle.OK
        want.append(o)
    b = fz.Batch(codec, spec)
    try:
        for tma in (2, 1, 2):
            b.set_load_path(tma, False)
            for o in outs:
                o.zero_()
            sizes, sts = b.compress()
            for i in range(len(spec)):
                assert sts[i] == fz.OK, (tma, i, sts[i])
                assert outs[i][: sizes[i]].cpu().numpy().tobytes() == want[i], (tma, i)
    finally:
        b.close()


def test_batch_autotune_keeps_streams(codec, torch):
    specs = _specs()[:14]
    xs, outs, b = _make_batch(codec, torch, specs)
    try:
        t = b.autotune(reps=2)
        assert t["ms_direct"] > 0 and t["ms_tma"] > 0 and t["ms_tma_staged"] > 0
        sizes, sts = b.compress()
        _check(codec, specs, xs, outs, sizes, sts)
    finally:
        b.close()


def test_batch_per_field_errors(codec, torch):
    good = fields.bumps3d(64)
    bad = good.copy()
    bad[5, 6, 7] = np.nan
    small = fields.climate2d(300, 500)
    specs = [(good, 3, "rel", 1e-3), (bad, 3, "rel", 1e-3), (small, 2, "rel", 1e-4),
             (bad, 3, "abs", 1e-3), (good, 3, "abs", 1e-9)]
    need = len(_single(codec, torch.from_numpy(small).cuda(), 2, "rel", 1e-4))
    min_bytes = fz.stream_min_bytes((500, 300), 2)
    xs, outs, b = _make_batch(codec, torch, specs, cap_override={2: min_bytes + 16})
    try:
        sizes, sts = b.compress()
        assert sts[0] == fz.OK
        assert sts[1] == fz.ERR_NONFINITE and sizes[1] == 0
        assert sts[2] == fz.ERR_CAPACITY and sizes[2] == need
        assert sts[3] == fz.ERR_NONFINITE
        assert sts[4] == fz.ERR_EB_RANGE
        assert outs[0][: sizes[0]].cpu().numpy().tobytes() == _single(codec, xs[0], 3, "rel",
                                                                         1e-3)
    finally:
        b.close()


def test_batch_rejects_bad_fields(codec, torch):
    x = torch.zeros((8, 8), device="cuda")
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")       # below header + flags
    with pytest.raises(fz.FZError) as e:
        fz.Batch(codec, [(x, out, "rel", 1e-3)])
    assert e.value.status == fz.ERR_CAPACITY
    out = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(fz.FZError) as e:
        fz.Batch(codec, [(x, out, "rel", -1.0)])
    assert e.value.status == fz.ERR_ARG


def test_batch_every_load_path(codec, torch):
    """The four load paths give the same streams: direct loads, TMA for the
    aligned fields only, TMA for all through row-aligned staging copies, TMA
    for all with row-class boxes for the unaligned fields.
    The fields cover every row misalignment (dims[0] % 4 = 1, 2, 3), a field
    that starts off a 16-byte boundary, absolute and relative bounds, escapes
    in a staged field, and ragged edges."""
    base = torch.from_numpy(fields.grf((40, 130), -2.5, 41).astype(np.float32).ravel()).cuda()
    off = torch.empty(base.numel() + 1, dtype=torch.float32, device="cuda")
    off[1:] = base
    specs = [
        (fields.grf((37, 45, 33), -3.0, 42).astype(np.float32), 3, "rel", 1e-3),
        (fields.grf((19, 70, 66), -3.0, 43).astype(np.float32), 3, "abs", 1e-3),
        (fields.grf((301, 259), -2.5, 44).astype(np.float32), 2, "rel", 1e-4),
        (_outliers((24, 50, 71), 200, 45), 3, "abs", 0.5),
        (fields.grf((64, 96, 128), -3.0, 46).astype(np.float32), 3, "rel", 1e-3),
        (fields.grf((517, 203), -2.5, 47).astype(np.float32), 2, "abs", 1e-2),
    ]
    xs, outs, spec = [], [], []
    for x, ndim, mode, eb in specs:
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        out = torch.zeros(fz.compress_bound(list(xt.shape[::-1])[:ndim], ndim),
                          dtype=torch.uint8, device="cuda")
        xs.append(xt)
        outs.append(out)
        spec.append((xt, out, mode, eb, ndim))
    xo = off[1:].view(40, 130)                      # 4-byte aligned only
    xs.append(xo)
    outs.append(torch.zeros(fz.compress_bound([130, 40], 2), dtype=torch.uint8, device="cuda"))
    spec.append((xo, outs[-1], "rel", 1e-3, 2))
    specs.append((xo.cpu().numpy(), 2, "rel", 1e-3))
    want = []
    for x, ndim, mode, eb in specs:
        st, o = oracle.compress(np.ascontiguousarray(x), ndim,
                                oracle.EB_ABS if mode == "abs" else oracle.EB_REL, eb)
        assert st == oracle.OK
        want.append(o)
    b = fz.Batch(codec, spec)
    try:
        for tma, staged in [(1, True), (0, False), (2, False), (1, False), (1, True), (2, False)]:
            b.set_load_path(tma, staged)
            t = b.tuning()
            assert t["tma"] == tma and t["staged"] == (tma == 1 and staged)
            for o in outs:
                o.zero_()
            sizes, sts = b.compress()
            for i in range(len(specs)):
                assert sts[i] == fz.OK, (tma, staged, i, sts[i])
                assert outs[i][: sizes[i]].cpu().numpy().tobytes() == want[i], (tma, staged, i)
        assert fz.inspect(outs[3][:64].cpu().numpy().tobytes())["n_outliers"] >= 200
        t = b.autotune(reps=2)
        assert t["ms_direct"] > 0 and t["ms_tma"] > 0 and t["ms_tma_staged"] > 0
        assert t["ms_tma_classes"] > 0
        sizes, sts = b.compress()
        for i in range(len(specs)):
            assert outs[i][: sizes[i]].cpu().numpy().tobytes() == want[i], i
    finally:
        b.close()
