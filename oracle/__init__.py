"""CPU oracle of the FZ-GPU compression path (arXiv 2304.12557).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library never calls it and it never calls the product library; the two share
no source.

The arithmetic lives in ``fz_oracle.c`` (plain C, fp32 without contraction);
this module only compiles it with gcc and marshals numpy arrays through
ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fz_oracle.c")
_HDR = os.path.join(_HERE, "fz_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfzoracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = -1
ERR_CAPACITY = -2
ERR_NONFINITE = -3
ERR_EB_RANGE = -4
ERR_CORRUPT = -6
EB_ABS = 0
EB_REL = 1
HEADER_BYTES = 64
QMAX = 268435455          # 2^28 - 1: largest |q| the quantiser takes
QNARROW = 4194303        # 2^22 - 1: beyond it a stream sets header byte 7

_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libfzoracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(
            ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-Wall", "-pthread", "-o", tmp, _SRC, "-lm"],
            check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.fzo_derive_eb.argtypes = [ctypes.c_int, ctypes.c_double,
                                        ctypes.c_float, ctypes.c_float,
                                        _f32p, _f32p, _f32p]
            L.fzo_prequant1.argtypes = [ctypes.c_float, ctypes.c_float, _i32p]
            L.fzo_chunk_shape.argtypes = [ctypes.c_int, _u32p]
            L.fzo_chunk_shape.restype = None
            L.fzo_lorenzo.argtypes = [_i32p, _u32p, ctypes.c_int, _i32p]
            L.fzo_lorenzo.restype = None
            L.fzo_lorenzo_inverse.argtypes = [_i32p, _u32p, ctypes.c_int, _i64p]
            L.fzo_lorenzo_inverse.restype = None
            L.fzo_encode.argtypes = [ctypes.c_int32]
            L.fzo_encode.restype = ctypes.c_uint16
            L.fzo_decode.argtypes = [ctypes.c_uint16]
            L.fzo_decode.restype = ctypes.c_int32
            L.fzo_tile_coord.argtypes = [ctypes.c_int, _u32p, ctypes.c_uint64,
                                         ctypes.c_uint32, _u32p]
            L.fzo_num_tiles.argtypes = [ctypes.c_int, _u32p]
            L.fzo_num_tiles.restype = ctypes.c_uint64
            L.fzo_bitshuffle.argtypes = [_u32p, _u32p]
            L.fzo_bitshuffle.restype = None
            L.fzo_bitunshuffle.argtypes = [_u32p, _u32p]
            L.fzo_bitunshuffle.restype = None
            L.fzo_block_flags.argtypes = [_u32p, _u32p]
            L.fzo_block_flags.restype = None
            L.fzo_compress_bound.argtypes = [ctypes.c_int, _u32p]
            L.fzo_compress_bound.restype = ctypes.c_uint64
            L.fzo_compress.argtypes = [_f32p, _u32p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, _u8p, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_uint64)]
            L.fzo_compress_ranged.argtypes = [_f32p, _u32p, ctypes.c_int,
                                              ctypes.c_double, ctypes.c_float,
                                              ctypes.c_float, _u8p, ctypes.c_uint64,
                                              ctypes.POINTER(ctypes.c_uint64)]
            L.fzo_decompress.argtypes = [_u8p, ctypes.c_uint64, _f32p,
                                         ctypes.c_uint64]
            L.fzo_reconstruct_closed_form.argtypes = [_f32p, ctypes.c_uint64,
                                                      ctypes.c_float,
                                                      ctypes.c_float, _f32p]
            L.fzo_lorenzo_whole.argtypes = [_i32p, _u32p, ctypes.c_int, _i32p]
            L.fzo_lorenzo_whole.restype = None
            L.fzo_lorenzo_whole_inverse.argtypes = [_i32p, _u32p, ctypes.c_int, _i64p]
            L.fzo_lorenzo_whole_inverse.restype = None
            L.fzo_compress_whole.argtypes = [_f32p, _u32p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, _u8p, ctypes.c_uint64,
                                             ctypes.POINTER(ctypes.c_uint64)]
            L.fzo_pwrel_bound.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
            L.fzo_pw_log2.argtypes = [ctypes.c_float]
            L.fzo_pw_log2.restype = ctypes.c_float
            L.fzo_pw_exp2.argtypes = [ctypes.c_float]
            L.fzo_pw_exp2.restype = ctypes.c_float
            L.fzo_pwrel_forward.argtypes = [_f32p, ctypes.c_uint64, _f32p, _u32p]
            L.fzo_pwrel_inverse.argtypes = [_f32p, ctypes.c_uint64, _u32p, _f32p]
            L.fzo_pwrel_inverse.restype = None
            L.fzo_threads.argtypes = []
            L.fzo_compress_mt.argtypes = L.fzo_compress.argtypes
            L.fzo_decompress_mt.argtypes = L.fzo_decompress.argtypes
            _lib = L
    return _lib


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _dims3(dims) -> np.ndarray:
    d = list(int(v) for v in dims) + [1] * (3 - len(dims))
    return np.asarray(d, dtype=np.uint32)


# ---------------------------------------------------------------- steps
def derive_eb(mode: int, eb: float, fmin: float = 0.0, fmax: float = 0.0):
    """Returns (status, eb_f, ebx2, ebx2_r) as numpy float32 scalars."""
    a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    st = lib().fzo_derive_eb(mode, eb, fmin, fmax, ctypes.byref(a),
                             ctypes.byref(b), ctypes.byref(c))
    return st, np.float32(a.value), np.float32(b.value), np.float32(c.value)


def prequant1(x: float, ebx2_r: float):
    q = ctypes.c_int32()
    st = lib().fzo_prequant1(x, ebx2_r, ctypes.byref(q))
    return st, q.value


def chunk_shape(ndim: int):
    c = np.zeros(3, np.uint32)
    lib().fzo_chunk_shape(ndim, _ptr(c, _u32p))
    return tuple(int(v) for v in c)


def lorenzo(q: np.ndarray, ndim: int) -> np.ndarray:
    """q indexed [z, y, x] (numpy C order, x fastest)."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    dims = _dims3(q.shape[::-1])
    out = np.empty_like(q)
    lib().fzo_lorenzo(_ptr(q, _i32p), _ptr(dims, _u32p), ndim, _ptr(out, _i32p))
    return out


def lorenzo_inverse(delta: np.ndarray, ndim: int) -> np.ndarray:
    delta = np.ascontiguousarray(delta, dtype=np.int32)
    dims = _dims3(delta.shape[::-1])
    out = np.empty(delta.shape, np.int64)
    lib().fzo_lorenzo_inverse(_ptr(delta, _i32p), _ptr(dims, _u32p), ndim,
                              _ptr(out, _i64p))
    return out


def lorenzo_whole(q: np.ndarray, ndim: int) -> np.ndarray:
    """Whole-field Lorenzo residuals (zero only outside the field)."""
    q = np.ascontiguousarray(q, dtype=np.int32)
    dims = _dims3(q.shape[::-1])
    out = np.empty_like(q)
    lib().fzo_lorenzo_whole(_ptr(q, _i32p), _ptr(dims, _u32p), ndim, _ptr(out, _i32p))
    return out


def lorenzo_whole_inverse(delta: np.ndarray, ndim: int) -> np.ndarray:
    delta = np.ascontiguousarray(delta, dtype=np.int32)
    dims = _dims3(delta.shape[::-1])
    out = np.empty(delta.shape, np.int64)
    lib().fzo_lorenzo_whole_inverse(_ptr(delta, _i32p), _ptr(dims, _u32p), ndim,
                                    _ptr(out, _i64p))
    return out


def encode(d: int) -> int:
    return int(lib().fzo_encode(d))


def decode(c: int) -> int:
    return int(lib().fzo_decode(c))


def tile_coord(ndim: int, dims, tile: int, p: int):
    d = _dims3(dims)
    c = np.zeros(3, np.uint32)
    inside = lib().fzo_tile_coord(ndim, _ptr(d, _u32p), tile, p, _ptr(c, _u32p))
    return bool(inside), tuple(int(v) for v in c)


def num_tiles(ndim: int, dims) -> int:
    d = _dims3(dims)
    return int(lib().fzo_num_tiles(ndim, _ptr(d, _u32p)))


def bitshuffle(words: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    assert w.size == 1024
    out = np.empty(1024, np.uint32)
    lib().fzo_bitshuffle(_ptr(w, _u32p), _ptr(out, _u32p))
    return out


def bitunshuffle(out: np.ndarray) -> np.ndarray:
    o = np.ascontiguousarray(out, dtype=np.uint32)
    assert o.size == 1024
    w = np.empty(1024, np.uint32)
    lib().fzo_bitunshuffle(_ptr(o, _u32p), _ptr(w, _u32p))
    return w


def block_flags(out: np.ndarray) -> np.ndarray:
    o = np.ascontiguousarray(out, dtype=np.uint32)
    f = np.empty(8, np.uint32)
    lib().fzo_block_flags(_ptr(o, _u32p), _ptr(f, _u32p))
    return f


# ---------------------------------------------------------------- pipeline
def compress_bound(ndim: int, dims) -> int:
    d = _dims3(dims)
    return int(lib().fzo_compress_bound(ndim, _ptr(d, _u32p)))


def threads() -> int:
    """Threads the all-cores calls use (one per online host core)."""
    return int(lib().fzo_threads())


def compress(x: np.ndarray, ndim: int, mode: int, eb: float, whole: bool = False,
             all_cores: bool = False):
    """x indexed [z, y, x] (x fastest).  Returns (status, bytes).  whole:
    the whole-field Lorenzo variant (stream version 2).  all_cores: the
    same stream computed over all host cores (Sec. 4.4's FZ-OMP)."""
    assert not (whole and all_cores)
    fn = (lib().fzo_compress_whole if whole else
          lib().fzo_compress_mt if all_cores else lib().fzo_compress)
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = _dims3(x.shape[::-1][:ndim])
    cap = compress_bound(ndim, dims)
    cap = min(cap, 64 + 32 * num_tiles(ndim, dims) * 129 + 8 * x.size)
    out = np.empty(cap, np.uint8)
    size = ctypes.c_uint64()
    st = fn(_ptr(x, _f32p), _ptr(dims, _u32p), ndim, mode, eb,
            _ptr(out, _u8p), cap, ctypes.byref(size))
    if st == ERR_CAPACITY:
        out = np.empty(size.value, np.uint8)
        st = fn(_ptr(x, _f32p), _ptr(dims, _u32p), ndim, mode,
                eb, _ptr(out, _u8p), size.value, ctypes.byref(size))
    if st != OK:
        return st, b""
    return st, out[: size.value].tobytes()


def compress_ranged(x: np.ndarray, ndim: int, eb: float, range_min: float,
                    range_max: float):
    """Relative bound against a supplied value range (x one slab of a field
    whose range that is).  Returns (status, bytes)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = _dims3(x.shape[::-1][:ndim])
    cap = compress_bound(ndim, dims)
    cap = min(cap, 64 + 32 * num_tiles(ndim, dims) * 129 + 8 * x.size)
    out = np.empty(cap, np.uint8)
    size = ctypes.c_uint64()
    args = (ctypes.c_float(range_min), ctypes.c_float(range_max))
    st = lib().fzo_compress_ranged(_ptr(x, _f32p), _ptr(dims, _u32p), ndim, eb,
                                   *args, _ptr(out, _u8p), cap, ctypes.byref(size))
    if st == ERR_CAPACITY:
        out = np.empty(size.value, np.uint8)
        st = lib().fzo_compress_ranged(_ptr(x, _f32p), _ptr(dims, _u32p), ndim,
                                       eb, *args, _ptr(out, _u8p), size.value,
                                       ctypes.byref(size))
    if st != OK:
        return st, b""
    return st, out[: size.value].tobytes()


def decompress(stream: bytes, n_elems: int | None = None, all_cores: bool = False):
    """Returns (status, float32 array of the field's element count).
    all_cores: the same reconstruction over all host cores."""
    buf = np.frombuffer(stream, dtype=np.uint8).copy()
    if n_elems is None:
        if len(stream) < 20:
            return ERR_CORRUPT, None
        d = np.frombuffer(stream[8:20], dtype="<u4").astype(np.int64)
        n_elems = int(max(1, d[0]) * max(1, d[1]) * max(1, d[2]))
    out = np.empty(max(n_elems, 1), np.float32)
    fn = lib().fzo_decompress_mt if all_cores else lib().fzo_decompress
    st = fn(_ptr(buf, _u8p), len(stream), _ptr(out, _f32p), n_elems)
    return st, (out[:n_elems] if st == OK else None)


def reconstruct_closed_form(x: np.ndarray, ebx2_r, ebx2):
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    out = np.empty_like(x)
    st = lib().fzo_reconstruct_closed_form(_ptr(x, _f32p), x.size,
                                           float(ebx2_r), float(ebx2),
                                           _ptr(out, _f32p))
    return st, out


# ------------------------------------------- point-wise relative bounds
def pwrel_bound(eps: float):
    """(status, eb_abs): the absolute bound for the log values (Sec. 4.1)."""
    e = ctypes.c_double()
    st = lib().fzo_pwrel_bound(eps, ctypes.byref(e))
    return st, e.value


def pw_log2(a: float) -> np.float32:
    return np.float32(lib().fzo_pw_log2(a))


def pw_exp2(y: float) -> np.float32:
    return np.float32(lib().fzo_pw_exp2(y))


def pwrel_forward(x: np.ndarray):
    """(status, y, signs): y = log2|x| (-160 for zeros), sign bits packed
    32 per uint32 word."""
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    y = np.empty_like(x)
    signs = np.zeros((x.size + 31) // 32, np.uint32)
    st = lib().fzo_pwrel_forward(_ptr(x, _f32p), x.size, _ptr(y, _f32p), _ptr(signs, _u32p))
    return st, y, signs


def pwrel_inverse(y: np.ndarray, signs: np.ndarray) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
    signs = np.ascontiguousarray(signs, dtype=np.uint32)
    x = np.empty_like(y)
    lib().fzo_pwrel_inverse(_ptr(y, _f32p), y.size, _ptr(signs, _u32p), _ptr(x, _f32p))
    return x
