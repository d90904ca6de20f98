"""CPU-side checks of the CUDA library: it builds, loads, exports every entry
point include/fz.h declares, and its host-only calls behave.  No kernel runs
here (no GPU on this machine)."""
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import paper_2304_12557_gb300 as fz
from golden_io import expected_bytes, load

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2304_12557_gb300 import build
    build.build()
    return fz.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fz_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_binding_api():
    assert declared_functions() == sorted(fz.C_API)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", fz.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fz_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_strerror_and_bounds(lib):
    import oracle
    assert lib.fz_strerror(0) == b"success"
    assert b"corrupt" in lib.fz_strerror(fz.ERR_CORRUPT)
    for ndim, dims in [(1, (5,)), (2, (3600, 1800)), (3, (512, 512, 512)),
                       (3, (33, 70, 9))]:
        assert fz.compress_bound(dims, ndim) == oracle.compress_bound(ndim, dims)
        nt = oracle.num_tiles(ndim, dims)
        assert fz.stream_min_bytes(dims, ndim) == 64 + 32 * nt
    assert fz.compress_bound((0, 4), 2) == 0
    assert fz.compress_bound((1 << 20, 1 << 20), 2) == 0      # too many codes


@pytest.mark.parametrize("name", ["g1_1d_basic.txt", "g2_1d_escape.txt",
                                  "g3_2d_basic.txt", "g4_3d_rel.txt"])
def test_inspect_golden(lib, name):
    rec = load(name)
    info = fz.inspect(expected_bytes(rec))
    assert info["ndim"] == rec["ndim"] and info["mode"] == rec["mode"]
    assert info["dims"] == tuple(rec["dims"])
    assert info["stream_bytes"] == rec["size"]
    assert info["nnz_blocks"] == int(rec["header"]["nnz"])
    assert info["eb"] == float(rec["header"]["eb_f"])
    assert info["version"] == 1


def test_inspect_reads_version_2(lib):
    import oracle
    from paper_2304_12557_gb300 import fields
    x = fields.bumps3d(32)
    st, s = oracle.compress(x, 3, oracle.EB_REL, 1e-3, whole=True)
    assert st == oracle.OK
    info = fz.inspect(s[:64])
    assert info["version"] == 2 and info["stream_bytes"] == len(s)
    bad = bytearray(s[:64])
    bad[4] = 3                                           # no version 3
    with pytest.raises(fz.FZError) as e:
        fz.inspect(bytes(bad))
    assert e.value.status == fz.ERR_CORRUPT


def test_inspect_rejects_corrupt(lib):
    s = bytearray(expected_bytes(load("g1_1d_basic.txt")))
    s[0] = ord("Q")
    with pytest.raises(fz.FZError) as e:
        fz.inspect(bytes(s))
    assert e.value.status == fz.ERR_CORRUPT


def test_create_without_gpu_fails_cleanly(lib):
    import ctypes
    ctx = ctypes.c_void_p()
    st = lib.fz_create(ctypes.byref(ctx), 0)
    if st == fz.OK:                       # a GPU is present after all
        lib.fz_destroy(ctx)
        pytest.skip("a CUDA device is visible")
    assert st == fz.ERR_CUDA


def test_transpose32_host_build():
    """The kernels' in-register 32x32 bit transpose, compiled as host code,
    against the bitshuffle definition (bit t of out[b] = bit b of in[t])."""
    src = r'''
#include <cstdio>
#include "fz_device.cuh"
int main() {
  unsigned s = 12345u;
  for (int rep = 0; rep < 64; ++rep) {
    uint32_t a[32];
    for (int i = 0; i < 32; ++i) { s = s * 1664525u + 1013904223u; a[i] = s ^ (s >> 7) * (rep & 1); }
    if (rep == 0) for (int i = 0; i < 32; ++i) a[i] = 1u << i;
    for (int i = 0; i < 32; ++i) printf("%u ", a[i]);
    fz::transpose32(a);
    for (int i = 0; i < 32; ++i) printf("%u ", a[i]);
    printf("\n");
  }
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "t.cu")
        exe = os.path.join(d, "t")
        open(cpp, "w").write(src)
        inc = os.path.join(ROOT, "paper_2304_12557_gb300", "csrc")
        subprocess.run(["nvcc", "-std=c++17", "-I", inc, "-o", exe, cpp],
                       check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    for line in out.strip().splitlines():
        v = np.array([int(t) for t in line.split()], dtype=np.uint64).astype(np.uint32)
        a, b = v[:32], v[32:]
        bits_in = np.unpackbits(a.view(np.uint8), bitorder="little").reshape(32, 32)
        bits_out = np.unpackbits(b.view(np.uint8), bitorder="little").reshape(32, 32)
        np.testing.assert_array_equal(bits_out, bits_in.T)


def test_fastdiv_host_build():
    """The kernels' division by a runtime constant (multiply-high), compiled
    as host code, against exact integer division for numerators < 2^31."""
    src = r'''
#include <cstdio>
#include <cstdint>
#include "fz_device.cuh"
int main() {
  uint32_t ds[] = {1, 2, 3, 5, 7, 16, 17, 57, 64, 100, 127, 128, 129, 1000, 4095, 4096,
                   65535, 65536, 524287, 524288, 1u << 30, (1u << 31) - 1};
  uint64_t s = 88172645463325252ull, bad = 0, n_checked = 0;
  for (uint32_t d : ds) {
    fz::FastDiv f(d);
    uint32_t edges[] = {0, 1, d - 1, d, d + 1, 2 * d - 1, 2 * d, 0x7FFFFFFFu, 0x7FFFFFFEu,
                        (0x7FFFFFFFu / d) * d, (0x7FFFFFFFu / d) * d - 1};
    for (uint32_t n : edges) {
      if (n > 0x7FFFFFFFu) continue;
      bad += f.div(n) != n / d; ++n_checked;
    }
    for (int i = 0; i < 200000; ++i) {
      s ^= s << 13; s ^= s >> 7; s ^= s << 17;
      uint32_t n = (uint32_t)(s & 0x7FFFFFFFu);
      if (i & 1) n &= 0xFFFFF;
      bad += f.div(n) != n / d; ++n_checked;
    }
  }
  printf("%llu %llu\n", (unsigned long long)bad, (unsigned long long)n_checked);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "t.cu")
        exe = os.path.join(d, "t")
        open(cpp, "w").write(src)
        inc = os.path.join(ROOT, "paper_2304_12557_gb300", "csrc")
        subprocess.run(["nvcc", "-std=c++17", "-I", inc, "-o", exe, cpp],
                       check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    bad, checked = (int(v) for v in out.split())
    assert checked > 4_000_000 and bad == 0


def test_narrow_transpose_host_build():
    """The narrow tiles' transpose (16 byte-code words, 16-word transpose),
    compiled as host code, against the 32x32 transpose: for code pairs whose
    magnitudes fit in 7 bits, word k is row narrow_row(k) of transpose32 and
    the other 16 rows are zero -- the identity both kernels rely on."""
    src = r'''
#include <cstdio>
#include <cstdint>
#include "fz_device.cuh"
int main() {
  uint64_t s = 0x9E3779B97F4A7C15ull, bad = 0, cases = 0;
  for (int rep = 0; rep < 100000; ++rep) {
    const int m = rep % 8;                       // magnitude bits of this case
    uint32_t w[32];
    for (int i = 0; i < 32; ++i) {
      uint32_t c[2];
      for (int h = 0; h < 2; ++h) {
        s ^= s << 13; s ^= s >> 7; s ^= s << 17;
        uint32_t mag = m ? (uint32_t)(s & ((1u << m) - 1u)) : 0u;
        uint32_t sgn = ((s >> 20) & 1u) ? 0x8000u : 0u;   // includes sign-only (escape) codes
        if (((s >> 24) & 3u) == 0) { mag = 0; sgn = 0; }
        c[h] = mag | sgn;
      }
      w[i] = c[0] | c[1] << 16;
    }
    uint32_t a[32];
    for (int i = 0; i < 32; ++i) a[i] = w[i];
    fz::transpose32(a);
    uint32_t u[16];
    fz::squeeze_narrow(w, u);
    fz::transpose16(u);
    bool live[32] = {};
    for (int k = 0; k < 16; ++k) {
      live[fz::narrow_row(k)] = true;
      bad += u[k] != a[fz::narrow_row(k)];
    }
    for (int b = 0; b < 32; ++b) bad += !live[b] && a[b] != 0u;
    ++cases;
  }
  printf("%llu %llu\n", (unsigned long long)bad, (unsigned long long)cases);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "t.cu")
        exe = os.path.join(d, "t")
        open(cpp, "w").write(src)
        inc = os.path.join(ROOT, "paper_2304_12557_gb300", "csrc")
        subprocess.run(["nvcc", "-std=c++17", "-I", inc, "-o", exe, cpp],
                       check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    bad, cases = (int(t) for t in out.split())
    assert cases == 100000 and bad == 0


def test_pwrel_bound_through_the_library(lib):
    """The library's bound for the log transform equals the oracle's
    formula, and the domain is enforced (host-only call, no GPU)."""
    import math
    assert fz.pwrel_bound(1e-3) == math.log2(1.001) - 2.0 ** -14
    for eps in (9e-5, 0.6, float("nan")):
        with pytest.raises(fz.FZError) as e:
            fz.pwrel_bound(eps)
        assert e.value.status == fz.ERR_ARG
