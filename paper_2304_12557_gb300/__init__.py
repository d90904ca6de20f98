"""GB300 (sm_103a) implementation of the FZ-GPU compression path
(Zhang, Tian et al., HPDC'23, arXiv 2304.12557).

This module is a thin ctypes binding over the C ABI in ``include/fz.h``
(``_build/libfz_gb300.so``).  It only marshals arguments: every step of
compression and decompression runs in the library's CUDA kernels.  PyTorch
is used for device memory and streams.  There is no CPU fallback: if the
library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = ["Codec", "FZError", "load_library", "library_path", "EB_ABS",
           "EB_REL", "OK", "ERR_ARG", "ERR_CAPACITY", "ERR_NONFINITE",
           "ERR_EB_RANGE", "ERR_CORRUPT", "ERR_TIMEOUT", "ERR_CUDA", "ERR_VERSION",
           "compress_bound", "stream_min_bytes", "inspect", "shard_extent",
           "concat_streams_host", "Batch", "Server", "PENDING", "C_API"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libfz_gb300.so")

OK = 0
ERR_ARG = -1
ERR_CAPACITY = -2
ERR_NONFINITE = -3
ERR_EB_RANGE = -4
ERR_CORRUPT = -6
ERR_TIMEOUT = -7
ERR_CUDA = -8
ERR_VERSION = -9
PENDING = 1
EB_ABS = 0
EB_REL = 1

# every entry point declared in include/fz.h
C_API = ["fz_create", "fz_destroy", "fz_compress_bound", "fz_stream_min_bytes",
         "fz_compress", "fz_compress_whole", "fz_decompress", "fz_compress_host",
         "fz_decompress_host", "fz_inspect", "fz_strerror",
         "fz_set_wait_limit_ns", "fz_debug_skip_publish",
         "fz_set_profiling", "fz_get_kernel_times", "fz_set_call_timing",
         "fz_get_call_times", "fz_range",
         "fz_compress_ranged", "fz_shard_extent", "fz_concat_streams",
         "fz_concat_streams_host", "fz_batch_create", "fz_batch_destroy",
         "fz_batch_compress", "fz_batch_set_graph", "fz_batch_autotune",
         "fz_batch_tuning", "fz_batch_set_load_path", "fz_server_create", "fz_server_destroy",
         "fz_server_submit", "fz_server_poll", "fz_server_fetch",
         "fz_server_get_stats", "fz_server_request_info", "fz_compress_staged", "fz_set_staged_shuffle",
         "fz_compress_noalloc",
         "fz_pwrel_bound", "fz_pwrel_forward", "fz_pwrel_inverse"]

_lib = None
_lock = threading.Lock()
_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p


class FZError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = load_library().fz_strerror(status).decode()
        super().__init__(f"{what}: {msg} ({status})" if what else msg)


class _Info(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("dims", _u64 * 3), ("eb_requested", ctypes.c_double),
                ("eb", ctypes.c_float), ("ebx2", ctypes.c_float),
                ("ebx2_r", ctypes.c_float), ("range_min", ctypes.c_float),
                ("range_max", ctypes.c_float), ("n_tiles", _u64),
                ("nnz_blocks", _u64), ("n_outliers", _u64),
                ("stream_bytes", _u64), ("version", ctypes.c_uint32),
                ("wide", ctypes.c_uint32)]


class _Field(ctypes.Structure):
    _fields_ = [("d_in", _vp), ("dims", _u64 * 3), ("ndim", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("eb", ctypes.c_double),
                ("d_out", _vp), ("out_capacity", _u64)]


class _Request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("ndim", ctypes.c_int32),
                ("dims", _u64 * 3), ("mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("eb", ctypes.c_double),
                ("h_in", _vp), ("in_bytes", _u64)]


class _RequestInfo(ctypes.Structure):
    _fields_ = [("batch", _u64), ("launch_seq", _u64), ("submit_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("launch_ms", ctypes.c_double),
                ("done_ms", ctypes.c_double), ("gpu_start_ms", ctypes.c_double),
                ("gpu_end_ms", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("completed", _u64), ("failed", _u64), ("queued", _u64),
                ("in_flight", _u64), ("pool_used", _u64), ("pool_bytes", _u64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("seconds", ctypes.c_double)]


def library_path() -> str:
    return _LIB_PATH


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library not built ({p}); run __graft_entry__.build() "
                "or python -m paper_2304_12557_gb300.build")
        L = ctypes.CDLL(p)
        dims_t = ctypes.POINTER(_u64)
        L.fz_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
        L.fz_destroy.argtypes = [_vp]
        L.fz_destroy.restype = None
        L.fz_compress_bound.argtypes = [dims_t, ctypes.c_int]
        L.fz_compress_bound.restype = _u64
        L.fz_stream_min_bytes.argtypes = [dims_t, ctypes.c_int]
        L.fz_stream_min_bytes.restype = _u64
        L.fz_compress.argtypes = [_vp, _vp, dims_t, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, _vp, _u64,
                                  ctypes.POINTER(_u64), _vp]
        L.fz_compress_whole.argtypes = L.fz_compress.argtypes
        L.fz_decompress.argtypes = [_vp, _vp, _u64, _vp, _u64, _vp]
        L.fz_compress_host.argtypes = L.fz_compress.argtypes
        L.fz_decompress_host.argtypes = L.fz_decompress.argtypes
        L.fz_inspect.argtypes = [_vp, _u64, ctypes.POINTER(_Info)]
        L.fz_strerror.argtypes = [ctypes.c_int]
        L.fz_strerror.restype = ctypes.c_char_p
        L.fz_set_wait_limit_ns.argtypes = [_vp, _u64]
        L.fz_debug_skip_publish.argtypes = [_vp, _u64]
        L.fz_set_profiling.argtypes = [_vp, ctypes.c_int]
        L.fz_get_kernel_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
        L.fz_set_call_timing.argtypes = [_vp, ctypes.c_int]
        L.fz_get_call_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
        L.fz_compress_noalloc.argtypes = [_vp, dims_t, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, _vp, _u64,
                                          ctypes.POINTER(_u64), _vp]
        L.fz_pwrel_bound.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        L.fz_pwrel_forward.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp]
        L.fz_pwrel_inverse.argtypes = [_vp, _vp, _u64, _vp, _vp, _vp]
        L.fz_range.argtypes = [_vp, _vp, _u64, ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(ctypes.c_int), _vp]
        L.fz_compress_ranged.argtypes = [_vp, _vp, dims_t, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_float,
                                         ctypes.c_float, _vp, _u64,
                                         ctypes.POINTER(_u64), _vp]
        L.fz_shard_extent.argtypes = [dims_t, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.POINTER(_u64),
                                      ctypes.POINTER(_u64)]
        L.fz_concat_streams.argtypes = [_vp, ctypes.POINTER(_vp), dims_t,
                                        ctypes.c_int, _vp, _u64,
                                        ctypes.POINTER(_u64), _vp]
        L.fz_concat_streams_host.argtypes = [ctypes.POINTER(_vp), dims_t,
                                             ctypes.c_int, _vp, _u64,
                                             ctypes.POINTER(_u64)]
        L.fz_batch_create.argtypes = [_vp, ctypes.POINTER(_Field), ctypes.c_int,
                                      ctypes.POINTER(_vp)]
        L.fz_batch_destroy.argtypes = [_vp]
        L.fz_batch_destroy.restype = None
        L.fz_batch_compress.argtypes = [_vp, ctypes.POINTER(_u64),
                                        ctypes.POINTER(ctypes.c_int), _vp]
        L.fz_batch_set_graph.argtypes = [_vp, ctypes.c_int]
        L.fz_batch_autotune.argtypes = [_vp, ctypes.c_int, _vp]
        L.fz_batch_tuning.argtypes = [_vp, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_double)]
        L.fz_batch_set_load_path.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
        L.fz_server_create.argtypes = [ctypes.c_int, _u64, ctypes.c_int,
                                       ctypes.POINTER(_vp)]
        L.fz_server_destroy.argtypes = [_vp]
        L.fz_server_destroy.restype = None
        L.fz_server_submit.argtypes = [_vp, ctypes.POINTER(_Request),
                                       ctypes.POINTER(_u64)]
        L.fz_server_poll.argtypes = [_vp, _u64, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(_u64)]
        L.fz_server_fetch.argtypes = [_vp, _u64, _vp, _u64]
        L.fz_server_get_stats.argtypes = [_vp, ctypes.POINTER(_ServerStats),
                                          ctypes.c_int]
        L.fz_server_request_info.argtypes = [_vp, _u64, ctypes.POINTER(_RequestInfo)]
        L.fz_set_staged_shuffle.argtypes = [_vp, ctypes.c_int]
        L.fz_compress_staged.argtypes = [_vp, _vp, dims_t, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, _vp, _u64,
                                         ctypes.POINTER(_u64),
                                         ctypes.POINTER(ctypes.c_double), _vp]
        _lib = L
        return L


def _dims(dims):
    d = [int(v) for v in dims] + [1] * (3 - len(dims))
    return (_u64 * 3)(*d)


def compress_bound(dims, ndim: int | None = None) -> int:
    ndim = ndim or len(dims)
    return int(load_library().fz_compress_bound(_dims(dims), ndim))


def stream_min_bytes(dims, ndim: int | None = None) -> int:
    ndim = ndim or len(dims)
    return int(load_library().fz_stream_min_bytes(_dims(dims), ndim))


def inspect(header: bytes) -> dict:
    info = _Info()
    buf = ctypes.create_string_buffer(bytes(header[:64]), 64)
    st = load_library().fz_inspect(buf, len(header[:64]), ctypes.byref(info))
    if st != OK:
        raise FZError(st, "fz_inspect")
    return {"ndim": info.ndim, "mode": info.mode,
            "dims": tuple(int(v) for v in info.dims),
            "eb_requested": info.eb_requested, "eb": info.eb,
            "ebx2": info.ebx2, "ebx2_r": info.ebx2_r,
            "range_min": info.range_min, "range_max": info.range_max,
            "n_tiles": info.n_tiles, "nnz_blocks": info.nnz_blocks,
            "n_outliers": info.n_outliers, "stream_bytes": info.stream_bytes,
            "version": info.version, "wide": bool(info.wide)}


def pwrel_bound(eps: float) -> float:
    """Absolute bound on the log values that gives the point-wise relative
    bound eps (Sec. 4.1's log-transformed particle data)."""
    e = ctypes.c_double()
    st = load_library().fz_pwrel_bound(float(eps), ctypes.byref(e))
    if st != OK:
        raise FZError(st, "fz_pwrel_bound")
    return e.value


def shard_extent(dims, ndim: int, n_shards: int, shard: int):
    """Slab `shard` of `n_shards` of a field: (begin, end) along its slowest
    axis (z for 3-D, y for 2-D, x for 1-D), whole chunk rows."""
    b, e = _u64(0), _u64(0)
    st = load_library().fz_shard_extent(_dims(dims), ndim, n_shards, shard,
                                        ctypes.byref(b), ctypes.byref(e))
    if st != OK:
        raise FZError(st, "fz_shard_extent")
    return int(b.value), int(e.value)


def concat_streams_host(parts) -> bytes:
    """Stream of a whole field from the streams (bytes) of its consecutive
    slabs, on the host."""
    bufs = [ctypes.create_string_buffer(bytes(p), len(p)) for p in parts]
    ptrs = (_vp * len(bufs))(*[ctypes.cast(b, _vp) for b in bufs])
    sizes = (_u64 * len(bufs))(*[len(p) for p in parts])
    total = _u64(0)
    L = load_library()
    st = L.fz_concat_streams_host(ptrs, sizes, len(bufs), None, 0,
                                  ctypes.byref(total))
    if st == ERR_CAPACITY:
        out = ctypes.create_string_buffer(int(total.value))
        st = L.fz_concat_streams_host(ptrs, sizes, len(bufs), out,
                                      total.value, ctypes.byref(total))
    if st != OK:
        raise FZError(st, "fz_concat_streams_host")
    return out.raw[: int(total.value)]


class Batch:
    """A planned batch: many fields compressed by one persistent launch per
    dimensionality (see fz_batch_create).  `fields` is a list of
    (x, out, mode, eb[, ndim]) with x a contiguous float32 CUDA tensor
    indexed [z, y, x] and out a uint8 CUDA tensor for its stream.  The tensors
    must stay alive (and in place) while the batch is used."""

    def __init__(self, codec, fields):
        self._L = load_library()
        self._codec = codec
        self._keep = []
        arr = (_Field * len(fields))()
        for i, spec in enumerate(fields):
            x, out, mode, eb = spec[:4]
            ndim = spec[4] if len(spec) > 4 else x.dim()
            assert x.is_cuda and x.is_contiguous() and out.is_cuda
            dims = list(x.shape[::-1])[:ndim] + [1] * (3 - ndim)
            arr[i].d_in = x.data_ptr()
            arr[i].dims = (_u64 * 3)(*[int(d) for d in dims])
            arr[i].ndim = ndim
            arr[i].mode = _mode(mode)
            arr[i].eb = float(eb)
            arr[i].d_out = out.data_ptr()
            arr[i].out_capacity = out.numel() * out.element_size()
            self._keep.append((x, out))
        self.n = len(fields)
        self._h = _vp()
        st = self._L.fz_batch_create(codec._ctx, arr, self.n, ctypes.byref(self._h))
        if st != OK:
            raise FZError(st, "fz_batch_create")
        self._sizes = (_u64 * self.n)()
        self._st = (ctypes.c_int * self.n)()

    def compress(self, stream=None):
        """Run the batch; returns (sizes, statuses) lists."""
        st = self._L.fz_batch_compress(self._h, self._sizes, self._st,
                                       Codec._stream(stream))
        if st == ERR_CUDA:
            raise FZError(st, "fz_batch_compress")
        return list(self._sizes), list(self._st)

    def set_graph(self, on: bool):
        st = self._L.fz_batch_set_graph(self._h, int(bool(on)))
        if st != OK:
            raise FZError(st, "fz_batch_set_graph")

    def autotune(self, reps: int = 3, stream=None):
        st = self._L.fz_batch_autotune(self._h, int(reps), Codec._stream(stream))
        if st != OK:
            raise FZError(st, "fz_batch_autotune")
        return self.tuning()

    def set_load_path(self, tma, staged: bool):
        """tma 0/False: direct loads; 1/True: TMA for aligned rows; 2: also
        row-class TMA boxes for the other 2-D/3-D fields."""
        st = self._L.fz_batch_set_load_path(self._h, int(tma), int(bool(staged)))
        if st != OK:
            raise FZError(st, "fz_batch_set_load_path")

    def tuning(self):
        """The load path in use (tma 0/1/2, staged) and the tuning runs'
        median times: direct loads, TMA for aligned rows, TMA with staging
        copies, TMA with row-class boxes."""
        on, staged = ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_double * 4)()
        st = self._L.fz_batch_tuning(self._h, ctypes.byref(on), ctypes.byref(staged), ms)
        if st != OK:
            raise FZError(st, "fz_batch_tuning")
        return {"tma": on.value, "staged": bool(staged.value), "ms_direct": ms[0],
                "ms_tma": ms[1], "ms_tma_staged": ms[2], "ms_tma_classes": ms[3]}

    def close(self):
        if self._h:
            self._L.fz_batch_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A request server with continuous batching (see fz_server_create).
    Inputs are host arrays (numpy, or CPU torch tensors; pinned memory lets
    the server copy them without blocking); each is kept alive here until
    its result is fetched."""

    def __init__(self, device: int = 0, pool_bytes: int = 8 << 30,
                 max_batch: int = 256):
        self._L = load_library()
        self._h = _vp()
        st = self._L.fz_server_create(device, int(pool_bytes), int(max_batch),
                                      ctypes.byref(self._h))
        if st != OK:
            raise FZError(st, "fz_server_create")
        self._meta = {}

    @staticmethod
    def _host_ptr(a):
        if hasattr(a, "data_ptr"):                   # torch CPU tensor
            assert not a.is_cuda and a.is_contiguous()
            return a.data_ptr(), a.numel() * a.element_size()
        return a.ctypes.data, a.nbytes

    def submit_compress(self, x, mode="rel", eb=1e-3, ndim=None):
        """x: float32 host array indexed [z, y, x].  Returns the request id."""
        shape = tuple(x.shape)
        ndim = ndim or len(shape)
        q = _Request()
        q.op = 0
        q.ndim = ndim
        q.dims = (_u64 * 3)(*([int(d) for d in shape[::-1][:ndim]] + [1] * (3 - ndim)))
        q.mode = _mode(mode)
        q.eb = float(eb)
        q.h_in, q.in_bytes = self._host_ptr(x)
        rid = _u64(0)
        st = self._L.fz_server_submit(self._h, ctypes.byref(q), ctypes.byref(rid))
        if st != OK:
            raise FZError(st, "fz_server_submit")
        self._meta[rid.value] = ("c", x, None)
        return rid.value

    def submit_decompress(self, stream):
        """stream: uint8 host array holding a whole stream.  Returns the id."""
        info = inspect(bytes(memoryview(stream)[:64]) if not hasattr(stream, "data_ptr")
                       else stream[:64].numpy().tobytes())
        q = _Request()
        q.op = 1
        q.h_in, q.in_bytes = self._host_ptr(stream)
        rid = _u64(0)
        st = self._L.fz_server_submit(self._h, ctypes.byref(q), ctypes.byref(rid))
        if st != OK:
            raise FZError(st, "fz_server_submit")
        d = info["dims"][: info["ndim"]]
        self._meta[rid.value] = ("d", stream, tuple(d[::-1]))
        return rid.value

    def poll(self, rid):
        """None while the request runs, else (status, size)."""
        st, size = ctypes.c_int(), _u64()
        r = self._L.fz_server_poll(self._h, rid, ctypes.byref(st), ctypes.byref(size))
        if r == PENDING:
            return None
        if r != OK:
            raise FZError(r, "fz_server_poll")
        return st.value, size.value

    def wait(self, rid, timeout: float = 60.0):
        import time
        t0 = time.monotonic()
        while True:
            r = self.poll(rid)
            if r is not None:
                return r
            if time.monotonic() - t0 > timeout:
                raise TimeoutError(f"request {rid} still running")
            time.sleep(50e-6)

    def fetch(self, rid, out=None):
        """The result as a numpy array (the stream, or the field shaped
        [z, y, x]); releases the request.  A failed request raises."""
        import numpy as np
        st, size = self.wait(rid)
        kind, _, shape = self._meta.pop(rid)
        if st != OK:
            self._L.fz_server_fetch(self._h, rid, None, 0)
            raise FZError(st, "request")
        if out is None:
            out = np.empty(size, np.uint8) if kind == "c" else np.empty(shape, np.float32)
        r = self._L.fz_server_fetch(self._h, rid, _vp(out.ctypes.data), out.nbytes)
        if r != OK:
            raise FZError(r, "fz_server_fetch")
        return out

    def discard(self, rid):
        """Release a done request without copying its output."""
        self.wait(rid)
        self._meta.pop(rid, None)
        self._L.fz_server_fetch(self._h, rid, None, 0)

    def info(self, rid):
        """Where the request's time went (see fz_server_request_info): a dict
        of batch, launch_seq and host/GPU times in ms; call before fetch."""
        i = _RequestInfo()
        st = self._L.fz_server_request_info(self._h, rid, ctypes.byref(i))
        if st != OK:
            raise FZError(st, "fz_server_request_info")
        return {k: getattr(i, k) for k, _ in _RequestInfo._fields_}

    def stats(self, reset: bool = False):
        s = _ServerStats()
        st = self._L.fz_server_get_stats(self._h, ctypes.byref(s), int(bool(reset)))
        if st != OK:
            raise FZError(st, "fz_server_get_stats")
        return {k: getattr(s, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if self._h:
            self._L.fz_server_destroy(self._h)
            self._h = _vp()
        self._meta.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _mode(mode) -> int:
    if mode in ("abs", EB_ABS):
        return EB_ABS
    if mode in ("rel", EB_REL):
        return EB_REL
    raise ValueError(f"mode must be 'abs' or 'rel', got {mode!r}")


class Codec:
    """A library context bound to one CUDA device.

    Fields are torch tensors (float32, contiguous) indexed [z, y, x] with x
    fastest; their dims go to the library fastest-first.  One Codec serves one
    stream at a time.
    """

    def __init__(self, device: int = 0):
        self._L = load_library()
        self._ctx = _vp()
        self.device = device
        st = self._L.fz_create(ctypes.byref(self._ctx), device)
        if st != OK:
            raise FZError(st, "fz_create")

    def close(self):
        if self._ctx:
            self._L.fz_destroy(self._ctx)
            self._ctx = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ options
    def set_wait_limit_ns(self, ns: int):
        st = self._L.fz_set_wait_limit_ns(self._ctx, int(ns))
        if st != OK:
            raise FZError(st, "fz_set_wait_limit_ns")

    def debug_skip_publish(self, chunk: int | None):
        v = (1 << 64) - 1 if chunk is None else int(chunk)
        st = self._L.fz_debug_skip_publish(self._ctx, v)
        if st != OK:
            raise FZError(st, "fz_debug_skip_publish")

    def set_profiling(self, on: bool):
        st = self._L.fz_set_profiling(self._ctx, int(bool(on)))
        if st != OK:
            raise FZError(st, "fz_set_profiling")

    def kernel_times_ms(self):
        """[range, compress, outliers, decompress, decompression offsets] of
        the last call (ms)."""
        ms = (ctypes.c_double * 5)()
        st = self._L.fz_get_kernel_times(self._ctx, ms)
        if st != OK:
            raise FZError(st, "fz_get_kernel_times")
        return list(ms)

    def set_call_timing(self, on: bool):
        st = self._L.fz_set_call_timing(self._ctx, int(bool(on)))
        if st != OK:
            raise FZError(st, "fz_set_call_timing")

    def call_times_ms(self):
        """[last fz_compress, last fz_decompress] call time (ms), from the
        library's own events at the call's entry and after its read-back."""
        ms = (ctypes.c_double * 2)()
        st = self._L.fz_get_call_times(self._ctx, ms)
        if st != OK:
            raise FZError(st, "fz_get_call_times")
        return list(ms)

    # ------------------------------------------------------------ device
    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return _vp(s.cuda_stream)

    def compress_into(self, x, out, mode="rel", eb=1e-3, ndim=None,
                      stream=None, raise_on_error=True, whole=False):
        """Compress device tensor x into the uint8 device tensor out.
        Returns (status, size).  whole: the whole-field Lorenzo variant
        (fz_compress_whole, stream version 2)."""
        ndim = ndim or x.dim()
        dims = list(x.shape[::-1])[:ndim]
        assert x.is_cuda and x.is_contiguous(), "x must be a contiguous CUDA tensor"
        size = _u64(0)
        fn = self._L.fz_compress_whole if whole else self._L.fz_compress
        st = fn(self._ctx, _vp(x.data_ptr()), _dims(dims), ndim,
                _mode(mode), float(eb), _vp(out.data_ptr()),
                out.numel() * out.element_size(),
                ctypes.byref(size), self._stream(stream))
        if st != OK and raise_on_error:
            raise FZError(st, "fz_compress_whole" if whole else "fz_compress")
        return st, int(size.value)

    def compress(self, x, mode="rel", eb=1e-3, ndim=None, stream=None, whole=False):
        """Compress a float32 CUDA tensor; returns the stream as a uint8 CUDA
        tensor (a view of a buffer sized for the worst case)."""
        import torch
        ndim = ndim or x.dim()
        dims = list(x.shape[::-1])[:ndim]
        cap = stream_min_bytes(dims, ndim) + 16 * 256 * (x.numel() // 2048 + 4)
        out = torch.empty(cap, dtype=torch.uint8, device=x.device)
        st, size = self.compress_into(x, out, mode, eb, ndim, stream, False, whole)
        if st == ERR_CAPACITY:
            out = torch.empty(size, dtype=torch.uint8, device=x.device)
            st, size = self.compress_into(x, out, mode, eb, ndim, stream, False, whole)
        if st != OK:
            raise FZError(st, "fz_compress_whole" if whole else "fz_compress")
        return out[:size]

    def compress_staged_into(self, x, out, mode="rel", eb=1e-3, ndim=None,
                             stream=None, raise_on_error=True):
        """The same stream through the unfused kernel sequence (codes and
        shuffled words in HBM).  Returns (status, size, stage_ms) with
        stage_ms = [range, quantise, shuffle+mark, scan, encode]."""
        ndim = ndim or x.dim()
        dims = list(x.shape[::-1])[:ndim]
        assert x.is_cuda and x.is_contiguous(), "x must be a contiguous CUDA tensor"
        size = _u64(0)
        ms = (ctypes.c_double * 5)()
        st = self._L.fz_compress_staged(self._ctx, _vp(x.data_ptr()), _dims(dims), ndim,
                                        _mode(mode), float(eb), _vp(out.data_ptr()),
                                        out.numel() * out.element_size(),
                                        ctypes.byref(size), ms, self._stream(stream))
        if st != OK and raise_on_error:
            raise FZError(st, "fz_compress_staged")
        return st, int(size.value), list(ms)

    def set_staged_shuffle(self, kind: str):
        """The unfused path's bitshuffle: 'register' (default) or 'ballot'
        (Listing 1's warp ballots); the stream is the same."""
        k = {"register": 0, "ballot": 1}[kind]
        st = self._L.fz_set_staged_shuffle(self._ctx, k)
        if st != OK:
            raise FZError(st, "fz_set_staged_shuffle")

    def value_range(self, x, stream=None):
        """(min, max, nonfinite) of a float32 CUDA tensor (the range pass)."""
        lo, hi, bad = ctypes.c_float(), ctypes.c_float(), ctypes.c_int()
        st = self._L.fz_range(self._ctx, _vp(x.data_ptr()), x.numel(),
                              ctypes.byref(lo), ctypes.byref(hi),
                              ctypes.byref(bad), self._stream(stream))
        if st != OK:
            raise FZError(st, "fz_range")
        return lo.value, hi.value, bool(bad.value)

    def pwrel_forward(self, x, stream=None):
        """(y, signs) for a float32 CUDA tensor x: y = log2|x| (-160 for
        zeros), signs one int32 word per 32 elements (bit set: negative)."""
        import torch
        assert x.is_cuda and x.is_contiguous() and x.dtype == torch.float32
        y = torch.empty_like(x)
        signs = torch.empty((x.numel() + 31) // 32, dtype=torch.int32, device=x.device)
        st = self._L.fz_pwrel_forward(self._ctx, _vp(x.data_ptr()), x.numel(),
                                      _vp(y.data_ptr()), _vp(signs.data_ptr()),
                                      self._stream(stream))
        if st != OK:
            raise FZError(st, "fz_pwrel_forward")
        return y, signs

    def pwrel_inverse(self, y, signs, stream=None):
        """x' = +-2^y (0 below -154) for float32 CUDA y and the forward's signs."""
        import torch
        assert y.is_cuda and y.is_contiguous() and y.dtype == torch.float32
        assert signs.is_cuda and signs.numel() >= (y.numel() + 31) // 32
        x = torch.empty_like(y)
        st = self._L.fz_pwrel_inverse(self._ctx, _vp(y.data_ptr()), y.numel(),
                                      _vp(signs.data_ptr()), _vp(x.data_ptr()),
                                      self._stream(stream))
        if st != OK:
            raise FZError(st, "fz_pwrel_inverse")
        return x

    def compress_ranged_into(self, x, out, eb, range_min, range_max, ndim=None,
                             stream=None, raise_on_error=True):
        """Relative bound eb against the supplied value range (x a slab of a
        field with that range).  Returns (status, size)."""
        ndim = ndim or x.dim()
        dims = list(x.shape[::-1])[:ndim]
        assert x.is_cuda and x.is_contiguous(), "x must be a contiguous CUDA tensor"
        size = _u64(0)
        st = self._L.fz_compress_ranged(self._ctx, _vp(x.data_ptr()), _dims(dims),
                                        ndim, float(eb), float(range_min),
                                        float(range_max), _vp(out.data_ptr()),
                                        out.numel() * out.element_size(),
                                        ctypes.byref(size), self._stream(stream))
        if st != OK and raise_on_error:
            raise FZError(st, "fz_compress_ranged")
        return st, int(size.value)

    def concat_into(self, parts, out, stream=None, raise_on_error=True):
        """Concatenate slab streams (uint8 CUDA tensors, in slab order) into
        the whole field's stream in `out`.  Returns (status, size)."""
        ptrs = (_vp * len(parts))(*[p.data_ptr() for p in parts])
        sizes = (_u64 * len(parts))(*[p.numel() for p in parts])
        size = _u64(0)
        st = self._L.fz_concat_streams(self._ctx, ptrs, sizes, len(parts),
                                       _vp(out.data_ptr()), out.numel(),
                                       ctypes.byref(size), self._stream(stream))
        if st != OK and raise_on_error:
            raise FZError(st, "fz_concat_streams")
        return st, int(size.value)

    def decompress_into(self, stream_t, out, nbytes=None, stream=None,
                        raise_on_error=True):
        n = int(nbytes if nbytes is not None else stream_t.numel())
        st = self._L.fz_decompress(self._ctx, _vp(stream_t.data_ptr()), n,
                                   _vp(out.data_ptr()), out.numel(),
                                   self._stream(stream))
        if st != OK and raise_on_error:
            raise FZError(st, "fz_decompress")
        return st

    def decompress(self, stream_t, stream=None):
        """Decompress a uint8 CUDA tensor; returns a float32 CUDA tensor
        shaped [z, y, x] (trailing unit dims dropped per the stream's ndim)."""
        import torch
        info = inspect(stream_t[:64].cpu().numpy().tobytes())
        d = info["dims"][: info["ndim"]]
        out = torch.empty(tuple(d[::-1]), dtype=torch.float32,
                          device=stream_t.device)
        self.decompress_into(stream_t, out, stream=stream)
        return out

    # ------------------------------------------------------------ host
    def compress_host(self, x_np, mode="rel", eb=1e-3, ndim=None,
                      capacity=None, stream=None, out=None):
        """Host-buffer form (copies in and out inside the library).  x_np is a
        C-contiguous float32 numpy array; returns the stream as bytes."""
        import numpy as np
        ndim = ndim or x_np.ndim
        dims = list(x_np.shape[::-1])[:ndim]
        cap = capacity or (stream_min_bytes(dims, ndim) +
                           16 * 256 * (x_np.size // 2048 + 4))
        buf = out if out is not None else np.empty(cap, np.uint8)
        size = _u64(0)
        st = self._L.fz_compress_host(self._ctx, _vp(x_np.ctypes.data),
                                      _dims(dims), ndim, _mode(mode), float(eb),
                                      _vp(buf.ctypes.data), buf.size,
                                      ctypes.byref(size), self._stream(stream))
        if st != OK:
            raise FZError(st, "fz_compress_host")
        return buf[: size.value]

    def decompress_host(self, stream_np, out=None, stream=None):
        import numpy as np
        info = inspect(bytes(stream_np[:64]))
        d = info["dims"][: info["ndim"]]
        res = out if out is not None else np.empty(tuple(d[::-1]), np.float32)
        st = self._L.fz_decompress_host(self._ctx, _vp(stream_np.ctypes.data),
                                        stream_np.size, _vp(res.ctypes.data),
                                        res.size, self._stream(stream))
        if st != OK:
            raise FZError(st, "fz_decompress_host")
        return res
