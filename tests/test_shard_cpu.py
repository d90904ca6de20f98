"""A field split into slabs (one per rank): the slab plan, the concatenation
of slab streams into the whole field's stream, and the multi-rank protocol
over torch.distributed with gloo ranks on CPU.  The slabs are compressed by
the oracle here (no GPU); the expected stream is the oracle's stream of the
whole field."""
import os
import socket

import numpy as np
import pytest

import oracle
import paper_2304_12557_gb300 as fz
from paper_2304_12557_gb300 import fields

ALIGN = {1: 8192, 2: 128, 3: 8}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2304_12557_gb300 import build
    build.build()
    fz.load_library()


@pytest.mark.parametrize("dims,ndim", [((64, 64, 64), 3), ((33, 70, 9), 3),
                                       ((50, 40, 300), 3), ((3600, 1800), 2),
                                       ((70, 129), 2), ((100000,), 1),
                                       ((5,), 1)])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
def test_shard_extent_partitions_chunk_rows(dims, ndim, world):
    L = dims[ndim - 1]
    A = ALIGN[ndim]
    rows = -(-L // A)
    ext = [fz.shard_extent(dims, ndim, world, r) for r in range(world)]
    assert ext[0][0] == 0 and ext[-1][1] == L
    for (b0, e0), (b1, e1) in zip(ext, ext[1:]):
        assert e0 == b1                                  # contiguous, in order
    counts = []
    for b, e in ext:
        assert b <= e and b % A == 0 and (e % A == 0 or e == L)
        counts.append(-(-(e - b) // A))
    assert sum(counts) == rows and max(counts) - min(counts) <= 1


def test_shard_extent_rejects():
    with pytest.raises(fz.FZError):
        fz.shard_extent((64, 64, 64), 3, 2, 2)
    with pytest.raises(fz.FZError):
        fz.shard_extent((0, 64), 2, 1, 0)


def _with_outliers(x, n, seed):
    rng = np.random.default_rng(seed)
    flat = x.reshape(-1)
    idx = rng.choice(flat.size, n, replace=False)
    flat[idx] = rng.choice([-1, 1], n) * rng.uniform(2e4, 9e4, n)
    return x


def _slab_parts(x, ndim, mode, eb, world):
    dims = x.shape[::-1][:ndim]
    lo, hi = float(x.min()) + 0.0, float(x.max()) + 0.0
    parts = []
    for r in range(world):
        b, e = fz.shard_extent(dims, ndim, world, r)
        if b == e:
            continue
        slab = np.ascontiguousarray(x[b:e])
        if mode == fz.EB_REL:
            st, p = oracle.compress_ranged(slab, ndim, eb, lo, hi)
        else:
            st, p = oracle.compress(slab, ndim, mode, eb)
        assert st == 0
        parts.append(p)
    return parts


CASES = [
    (lambda: fields.bumps3d(64), 3, fz.EB_REL, 1e-3),
    (lambda: fields.grf((33, 70, 41), -3.0, 5).astype(np.float32), 3, fz.EB_REL, 1e-4),
    (lambda: fields.climate2d(300, 500), 2, fz.EB_REL, 1e-3),
    (lambda: fields.climate2d(260, 77), 2, fz.EB_ABS, 0.01),
    (lambda: fields.grf((70001,), -2.0, 6).astype(np.float32), 1, fz.EB_REL, 1e-3),
    # escaped residuals in every slab: their code indices must move
    (lambda: _with_outliers(np.random.default_rng(8).normal(0, 1, (40, 67, 96))
                            .astype(np.float32), 60, 8), 3, fz.EB_ABS, 0.5),
    (lambda: _with_outliers(np.random.default_rng(9).normal(0, 1, (520, 130))
                            .astype(np.float32), 60, 9), 2, fz.EB_ABS, 0.5),
    (lambda: _with_outliers(np.random.default_rng(10).normal(0, 1, (40000,))
                            .astype(np.float32), 30, 10), 1, fz.EB_REL, 1e-6),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("world", [2, 3, 5])
def test_concat_equals_single_stream(case, world):
    make, ndim, mode, eb = CASES[case]
    x = np.ascontiguousarray(make(), dtype=np.float32)
    st, whole = oracle.compress(x, ndim, mode, eb)
    assert st == 0
    parts = _slab_parts(x, ndim, mode, eb, world)
    got = fz.concat_streams_host(parts)
    assert got == whole
    if case >= 5:
        outs = [fz.inspect(p[:64])["n_outliers"] for p in parts]
        assert sum(1 for n in outs if n) >= 2           # several slabs rebased


def test_concat_rejects_inconsistent_parts():
    x = fields.bumps3d(64)
    p = _slab_parts(x, 3, fz.EB_ABS, 1e-3, 2)
    with pytest.raises(fz.FZError) as e:                # another bound
        q = _slab_parts(x, 3, fz.EB_ABS, 2e-3, 2)
        fz.concat_streams_host([p[0], q[1]])
    assert e.value.status == fz.ERR_CORRUPT
    y = np.ascontiguousarray(x[:, :, :40])              # another cross-section
    _, r = oracle.compress(np.ascontiguousarray(y[32:]), 3, fz.EB_ABS, 1e-3)
    with pytest.raises(fz.FZError) as e:
        fz.concat_streams_host([p[0], r])
    assert e.value.status == fz.ERR_CORRUPT
    _, a = oracle.compress(np.ascontiguousarray(x[:20]), 3, fz.EB_ABS, 1e-3)
    _, b = oracle.compress(np.ascontiguousarray(x[20:]), 3, fz.EB_ABS, 1e-3)
    with pytest.raises(fz.FZError) as e:                # not on a chunk boundary
        fz.concat_streams_host([a, b])
    assert e.value.status == fz.ERR_CORRUPT
    with pytest.raises(fz.FZError) as e:                # truncated part
        fz.concat_streams_host([p[0][:-1], p[1]])
    assert e.value.status == fz.ERR_CORRUPT
    _, rel = oracle.compress(np.ascontiguousarray(x[32:]), 3, fz.EB_REL, 1e-3)
    with pytest.raises(fz.FZError) as e:                # another mode
        fz.concat_streams_host([p[0], rel])
    assert e.value.status == fz.ERR_CORRUPT
    # whole-field residuals cross slab faces: version-2 parts are refused
    _, w0 = oracle.compress(np.ascontiguousarray(x[:32]), 3, fz.EB_ABS, 1e-3, whole=True)
    _, w1 = oracle.compress(np.ascontiguousarray(x[32:]), 3, fz.EB_ABS, 1e-3, whole=True)
    with pytest.raises(fz.FZError) as e:
        fz.concat_streams_host([w0, w1])
    assert e.value.status == fz.ERR_VERSION


def test_oracle_ranged_reduces_to_rel_and_abs():
    """The oracle's supplied-range entry: with the field's own range it is
    the relative mode; with any range its codes are those of the absolute
    mode at the bound that range gives."""
    x = fields.grf((40, 50, 60), -3.0, 11).astype(np.float32)
    lo, hi = float(x.min()), float(x.max())
    assert oracle.compress_ranged(x, 3, 1e-3, lo, hi) == oracle.compress(x, 3, fz.EB_REL, 1e-3)
    st, s = oracle.compress_ranged(x, 3, 1e-3, lo - 1.0, hi + 3.0)
    info = fz.inspect(s[:64])
    assert st == 0 and info["mode"] == fz.EB_REL
    assert info["range_min"] == np.float32(lo - 1.0) and info["range_max"] == np.float32(hi + 3.0)
    st, a = oracle.compress(x, 3, fz.EB_ABS, 1e-3 * (float(np.float32(hi + 3.0))
                                                     - float(np.float32(lo - 1.0))))
    assert st == 0 and a[64:] == s[64:] and fz.inspect(a[:64])["eb"] == info["eb"]
    assert oracle.compress_ranged(x, 3, 1e-3, hi, lo)[0] == oracle.ERR_ARG
    assert oracle.compress_ranged(x, 3, 1e-3, lo, float("inf"))[0] == oracle.ERR_ARG


# ------------------------------------------------------------ gloo ranks
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, mode, eb, path):
    import torch
    import torch.distributed as dist

    import oracle as orc
    import paper_2304_12557_gb300 as lib
    from paper_2304_12557_gb300 import fields as fl, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x = fl.grf((40, 64, 48), -3.0, 12).astype(np.float32)   # every rank builds it
        slab = np.ascontiguousarray(shard.slab_of(x, 3, world, rank))

        def value_range(s):
            return float(s.min()), float(s.max()), bool(~np.isfinite(s).all())

        def compress(s, m, e, rng):
            if rng is None:
                st, b = orc.compress(s, 3, lib.EB_ABS, e)
            else:
                st, b = orc.compress_ranged(s, 3, e, rng[0], rng[1])
            assert st == 0
            return torch.from_numpy(np.frombuffer(b, np.uint8).copy())

        def concat(parts):
            return lib.concat_streams_host([p.numpy().tobytes() for p in parts])

        out = shard.compress_distributed(slab, mode, eb, value_range=value_range,
                                         compress=compress, concat=concat)
        if rank == 0:
            with open(path, "wb") as f:
                f.write(out)
        else:
            assert out is None
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode,eb", [(fz.EB_REL, 1e-3), (fz.EB_ABS, 0.02)])
def test_gloo_two_ranks_make_the_single_stream(tmp_path, mode, eb):
    import torch.multiprocessing as mp
    path = str(tmp_path / "stream.bin")
    mp.start_processes(_rank_main, args=(2, _free_port(), mode, eb, path), nprocs=2,
                       join=True, start_method="spawn")
    x = fields.grf((40, 64, 48), -3.0, 12).astype(np.float32)
    st, whole = oracle.compress(x, 3, mode, eb)
    assert st == 0 and open(path, "rb").read() == whole
