"""One field split into slabs across ranks, compressed into the single stream
of the whole field.

Chunks are independent (Sec. 2.3: the chunk-local Lorenzo residual never
reaches across a chunk), so slabs of whole chunk rows along the slowest axis
compress on their own, and their streams concatenate into the stream a single
GPU makes of the field, byte for byte.  The one exchange the method needs is
the value range of a relative bound (Sec. 4.1): an all-reduce of each slab's
(min, max, non-finite) before quantisation.  The slab streams are then
gathered in rank order and concatenated (the library's fz_concat_streams).

The protocol is written against torch.distributed and takes the per-rank
steps as callables, so the same code drives the library on GPUs and any
stand-in on CPU ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import EB_ABS, EB_REL, shard_extent


def slab_bounds(dims, ndim: int, world: int, rank: int):
    """[begin, end) of this rank's slab along the slowest axis."""
    return shard_extent(dims, ndim, world, rank)


def slab_of(x, ndim: int, world: int, rank: int):
    """This rank's slab of a field indexed [z, y, x] (x fastest): a view
    along the tensor's first axis, which is the slowest one."""
    dims = list(x.shape[::-1])[:ndim]
    b, e = slab_bounds(dims, ndim, world, rank)
    return x[b:e]


def global_range(lo: float, hi: float, nonfinite: bool, device=None, group=None):
    """All-reduce of the slabs' ranges: (min, max, any non-finite)."""
    t = torch.tensor([-float(lo), float(hi), 1.0 if nonfinite else 0.0],
                     dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    v = t.cpu().tolist()
    return -v[0] + 0.0, v[1] + 0.0, v[2] > 0


def gather_parts(part, group=None):
    """Every rank's uint8 stream (1-D tensor, same device kind on every
    rank), in rank order, on every rank."""
    world = dist.get_world_size(group)
    n = torch.tensor([part.numel()], dtype=torch.int64, device=part.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes)
    buf = torch.zeros(m, dtype=torch.uint8, device=part.device)
    buf[: part.numel()] = part
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    return [b[:s] for b, s in zip(bufs, sizes)]


def compress_distributed(x_slab, mode, eb, *, value_range, compress, concat,
                         device=None, group=None, root: int = 0):
    """The sharded compression of one field.

    x_slab       this rank's slab (a non-empty one on every rank)
    value_range  x_slab -> (min, max, nonfinite): the range pass
    compress     (x_slab, mode, eb, rng) -> 1-D uint8 tensor, the slab's
                 stream; rng is the field's (min, max) for a relative bound,
                 None for an absolute one
    concat       list of the slabs' streams -> the field's stream
    Returns the field's stream on `root`, None elsewhere.  A non-finite
    element anywhere raises ValueError on every rank.
    """
    rng = None
    if mode in (EB_REL, "rel"):
        lo, hi, bad = value_range(x_slab)
        lo, hi, bad = global_range(lo, hi, bad, device=device, group=group)
        if bad:
            raise ValueError("the field holds NaN or Inf")
        rng = (lo, hi)
    elif mode not in (EB_ABS, "abs"):
        raise ValueError(f"mode must be 'abs' or 'rel', got {mode!r}")
    part = compress(x_slab, mode, eb, rng)
    parts = gather_parts(part, group=group)
    if dist.get_rank(group) != root:
        return None
    return concat(parts)


def codec_compress_distributed(codec, x_slab, ndim: int, mode, eb, group=None, root=0):
    """compress_distributed with this library's kernels on each rank's GPU
    (x_slab a float32 CUDA tensor indexed [z, y, x])."""
    def value_range(x):
        return codec.value_range(x)

    def compress(x, m, e, rng):
        dims = list(x.shape[::-1])[:ndim]
        from . import compress_bound
        out = torch.empty(compress_bound(dims, ndim), dtype=torch.uint8, device=x.device)
        if rng is None:
            _, size = codec.compress_into(x, out, "abs", e, ndim)
        else:
            _, size = codec.compress_ranged_into(x, out, e, rng[0], rng[1], ndim)
        return out[:size]

    def concat(parts):
        total = sum(p.numel() for p in parts)
        out = torch.empty(total, dtype=torch.uint8, device=parts[0].device)
        _, size = codec.concat_into(parts, out)
        return out[:size]

    return compress_distributed(x_slab, mode, eb, value_range=value_range,
                                compress=compress, concat=concat,
                                device=x_slab.device, group=group, root=root)
