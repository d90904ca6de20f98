// fz_compress.cu -- GB300 compression kernels.
//
//  range_kernel     value range + non-finite scan (relative bounds, Sec. 4.1)
//  compress_kernel  one CTA per chunk (4 tiles, 8192 codes), single pass:
//                   TMA tile load -> pre-quantisation (Sec. 2.3) -> chunk-local
//                   Lorenzo residual (Sec. 2.3, 3.1) -> sign-magnitude codes
//                   (Sec. 3.2) -> 32x32 bitshuffle (Sec. 3.3) -> zero-block
//                   flags and compaction (Sec. 3.4) -> decoupled look-back for
//                   the payload offset -> one bulk store per tile.
//  outlier_kernel   rare path: rewrites the escaped residuals of the chunks
//                   that had any, at offsets found by compress_kernel.
//
// The paper splits this work into a quantisation kernel, a fused
// bitshuffle+mark kernel, a CUB scan and an encode kernel with the codes,
// shuffled words and byte flags passing through global memory; here one
// kernel does all of it and global memory sees only the input and the stream.
#include <cuda.h>
#include <cuda_runtime.h>

#include "fz_device.cuh"
#include "fz_kernels.h"

namespace fz {

// ====================================================================
// value range (min, max, non-finite) of a float field
// ====================================================================
__global__ void __launch_bounds__(256) range_kernel(const float *__restrict__ x,
                                                    uint64_t n, float2 *partial,
                                                    RangeResult *res) {
  float lo = INFINITY, hi = -INFINITY;
  uint32_t bad = 0;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  const bool vec = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
  uint64_t done = 0;
  if (vec) {
    const uint64_t n4 = n / 4;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    for (uint64_t i = tid; i < n4; i += nth) {
      float4 v = __ldcs(&x4[i]);
      float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bad |= (__float_as_uint(a[k]) & 0x7F800000u) == 0x7F800000u;
        lo = fminf(lo, a[k]);
        hi = fmaxf(hi, a[k]);
      }
    }
    done = n4 * 4;
  }
  for (uint64_t i = done + tid; i < n; i += nth) {
    float a = x[i];
    bad |= (__float_as_uint(a) & 0x7F800000u) == 0x7F800000u;
    lo = fminf(lo, a);
    hi = fmaxf(hi, a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  __shared__ float slo[8], shi[8];
  __shared__ uint32_t sbad[8];
  __shared__ bool last;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { slo[w] = lo; shi[w] = hi; sbad[w] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      lo = fminf(lo, slo[k]);
      hi = fmaxf(hi, shi[k]);
      bad |= sbad[k];
    }
    partial[blockIdx.x] = make_float2(lo, bad ? __int_as_float(-1) : hi);
    if (bad) partial[blockIdx.x].x = __int_as_float(-1);
    __threadfence();
    uint32_t prev = atomicAdd(&res->counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // the last block reduces the partials (NaN payload marks a non-finite)
  __threadfence();
  lo = INFINITY; hi = -INFINITY; bad = 0;
  for (uint32_t i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
    float2 p = __ldcg(&partial[i]);
    if (__float_as_int(p.x) == -1 || __float_as_int(p.y) == -1) bad = 1;
    else { lo = fminf(lo, p.x); hi = fmaxf(hi, p.y); }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  if (l == 0) { slo[w] = lo; shi[w] = hi; sbad[w] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      lo = fminf(lo, slo[k]);
      hi = fmaxf(hi, shi[k]);
      bad |= sbad[k];
    }
    res->fmin = __fadd_rn(lo, 0.0f);   // +0 for a zero of either sign
    res->fmax = __fadd_rn(hi, 0.0f);
    res->nonfinite = bad;
    res->counter = 0;                  // ready for the next call
  }
}

// ====================================================================
// compression
// ====================================================================
template <int NDIM>
struct Brick {
  using G = Geo<NDIM>;
  static constexpr int N = 64;
};

// byte offset inside the chunk box (swizzled rows of 32 floats) of the
// chunk-local element (lx, ly, lz)
template <int NDIM>
__device__ __forceinline__ uint32_t box_offset(uint32_t lx, uint32_t ly,
                                               uint32_t lz) {
  if constexpr (NDIM == 3) {
    uint32_t r = ly + 32u * lz;
    return swz(r, lx >> 2) + ((lx & 3u) << 2);
  } else if constexpr (NDIM == 2) {
    uint32_t half = lx >> 5, col = lx & 31u;
    return half * 16384u + swz(ly, col >> 2) + ((col & 3u) << 2);
  } else {
    uint32_t r = lx >> 5, col = lx & 31u;
    return swz(r, col >> 2) + ((col & 3u) << 2);
  }
}

// Fill the chunk box with plain loads (fields whose rows are not 16-byte
// aligned, and every 1-D field).  Out-of-field elements read as 0.
template <int NDIM>
__device__ __forceinline__ void fill_box_generic(const CompressArgs &a,
                                                 uint8_t *box, uint32_t cx,
                                                 uint32_t cy, uint32_t cz) {
  using G = Geo<NDIM>;
  const uint64_t X = a.dims[0], Y = a.dims[1];
  for (uint32_t e0 = 0; e0 < (uint32_t)kChunkCodes; e0 += kThreads * 8) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t e = e0 + k * kThreads + threadIdx.x;
      uint32_t lx = e % G::CX, ly = (e / G::CX) % G::CY, lz = e / (G::CX * G::CY);
      uint64_t gx = (uint64_t)cx * G::CX + lx, gy = (uint64_t)cy * G::CY + ly,
               gz = (uint64_t)cz * G::CZ + lz;
      bool in = gx < X && gy < a.dims[1] && gz < a.dims[2];
      v[k] = in ? __ldcs(&a.x[gx + X * (gy + Y * gz)]) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t e = e0 + k * kThreads + threadIdx.x;
      uint32_t lx = e % G::CX, ly = (e / G::CX) % G::CY, lz = e / (G::CX * G::CY);
      *reinterpret_cast<float *>(box + box_offset<NDIM>(lx, ly, lz)) = v[k];
    }
  }
}

// Load a thread's brick from the box (warp t = tile t of the chunk, lane g =
// brick g) and pre-quantise it: returns biased q (q + 2^22 - 1) and folds the
// unsigned maximum into qmax (> kBiasedMax means out of range / non-finite).
template <int NDIM>
__device__ __forceinline__ void load_quant(const uint8_t *box, int t, int g,
                                           float r, int32_t (&tq)[64],
                                           uint32_t &qmax) {
  using G = Geo<NDIM>;
  const int bx = g % G::NBX, by = g / G::NBX;
#pragma unroll
  for (int iz = 0; iz < G::BZ; ++iz) {
#pragma unroll
    for (int iy = 0; iy < G::BY; ++iy) {
#pragma unroll
      for (int h = 0; h < G::BX / 4; ++h) {
        uint32_t off;
        if constexpr (NDIM == 3) {
          uint32_t row = (uint32_t)(4 * by + iy + 32 * (2 * t + iz));
          off = swz(row, (uint32_t)(2 * bx + h));
        } else if constexpr (NDIM == 2) {
          uint32_t row = (uint32_t)(32 * t + 8 * by + iy);
          off = (uint32_t)(bx >> 2) * 16384u + swz(row, (uint32_t)(2 * (bx & 3) + h));
        } else {
          uint32_t row = (uint32_t)(64 * t + 2 * g + (h >> 3));
          off = swz(row, (uint32_t)(h & 7));
        }
        float4 v = *reinterpret_cast<const float4 *>(box + off);
        float f[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = 4 * h + k + G::BX * (iy + G::BY * iz);
          float s = __fadd_rn(__fmul_rn(f[k], r), kRoundMagic);
          uint32_t b = __float_as_uint(s) - kBiasBits;
          qmax = max(qmax, b);
          tq[e] = (int32_t)b;
        }
      }
    }
  }
}

// Chunk-local Lorenzo residual of the thread's brick, in place on tq (biased
// q in, residual out).  `halo` carries the neighbour values across the warp
// boundary (previous tile of the chunk), already in biased form:
//   3-D: the previous z plane of this brick (32 values), 2-D: the previous
//   y row (8 values, used by by == 0 lanes), 1-D: the previous element.
// Neighbours outside the chunk are q = 0 (biased kPadBiased) for the first
// difference and 0 for the later ones.
template <int NDIM>
__device__ __forceinline__ void lorenzo(int32_t (&v)[64], const int32_t *halo,
                                        int g) {
  using G = Geo<NDIM>;
  const int bx = g % G::NBX, by = g / G::NBX;
  const unsigned full = 0xffffffffu;
  if constexpr (NDIM == 3) {
    // D_z (biased values; previous plane from halo)
#pragma unroll
    for (int e = 63; e >= 32; --e) v[e] -= v[e - 32];
#pragma unroll
    for (int e = 0; e < 32; ++e) v[e] -= halo[e];
    // D_y: row iy-1 of the brick, or row iy = 3 of the brick below (lane-4)
#pragma unroll
    for (int iz = 0; iz < 2; ++iz) {
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) {
        int32_t up = __shfl_up_sync(full, v[ix + 24 + 32 * iz], 4);
        if (by == 0) up = 0;
#pragma unroll
        for (int iy = 3; iy >= 1; --iy) v[ix + 8 * iy + 32 * iz] -= v[ix + 8 * (iy - 1) + 32 * iz];
        v[ix + 32 * iz] -= up;
      }
    }
    // D_x: element ix-1, or ix = 7 of the brick to the left (lane-1)
#pragma unroll
    for (int row = 0; row < 8; ++row) {
      int32_t left = __shfl_up_sync(full, v[7 + 8 * row], 1);
      if (bx == 0) left = 0;
#pragma unroll
      for (int ix = 7; ix >= 1; --ix) v[ix + 8 * row] -= v[ix - 1 + 8 * row];
      v[8 * row] -= left;
    }
  } else if constexpr (NDIM == 2) {
    // D_y on biased values: row iy-1, or row 7 of the brick below (lane-8),
    // or for by == 0 the last row of the previous tile (halo)
#pragma unroll
    for (int ix = 0; ix < 8; ++ix) {
      int32_t up = __shfl_up_sync(full, v[ix + 56], 8);
      if (by == 0) up = halo[ix];
#pragma unroll
      for (int iy = 7; iy >= 1; --iy) v[ix + 8 * iy] -= v[ix + 8 * (iy - 1)];
      v[ix] -= up;
    }
    // D_x
#pragma unroll
    for (int row = 0; row < 8; ++row) {
      int32_t left = __shfl_up_sync(full, v[7 + 8 * row], 1);
      if (bx == 0) left = 0;
#pragma unroll
      for (int ix = 7; ix >= 1; --ix) v[ix + 8 * row] -= v[ix - 1 + 8 * row];
      v[8 * row] -= left;
    }
  } else {
    int32_t left = __shfl_up_sync(full, v[63], 1);
    if (g == 0) left = halo[0];
#pragma unroll
    for (int e = 63; e >= 1; --e) v[e] -= v[e - 1];
    v[0] -= left;
  }
}

// zero the residuals of brick elements that lie outside the field
template <int NDIM>
__device__ __forceinline__ void mask_outside(int32_t (&v)[64], const CompressArgs &a,
                                             uint32_t cx, uint32_t cy, uint32_t cz,
                                             int t, int g) {
  using G = Geo<NDIM>;
  const int bx = g % G::NBX, by = g / G::NBX;
#pragma unroll
  for (int e = 0; e < 64; ++e) {
    const int ix = e % G::BX, iy = (e / G::BX) % G::BY, iz = e / (G::BX * G::BY);
    uint64_t gx, gy = 0, gz = 0;
    if constexpr (NDIM == 3) {
      gx = (uint64_t)cx * 32 + 8 * bx + ix;
      gy = (uint64_t)cy * 32 + 4 * by + iy;
      gz = (uint64_t)cz * 8 + 2 * t + iz;
    } else if constexpr (NDIM == 2) {
      gx = (uint64_t)cx * 64 + 8 * bx + ix;
      gy = (uint64_t)cy * 128 + 32 * t + 8 * by + iy;
    } else {
      gx = (uint64_t)cx * 8192 + 2048 * t + 64 * g + e;
    }
    if (!(gx < a.dims[0] && gy < a.dims[1] && gz < a.dims[2])) v[e] = 0;
  }
}

// byte offset of warp t's k-th 4 KB piece of the box: the rows its tile
// occupies (3-D: planes 2t..2t+1; 2-D: rows 32t.. of both x halves; 1-D:
// elements 2048t..)
template <int NDIM>
__device__ __forceinline__ uint32_t piece_offset(int t, int k) {
  if constexpr (NDIM == 2) return (uint32_t)(k * 16384 + t * 4096);
  return (uint32_t)(t * 8192 + k * 4096);
}

template <int NDIM>
__device__ __forceinline__ bool chunk_is_edge(const CompressArgs &a, uint32_t cx,
                                              uint32_t cy, uint32_t cz) {
  using G = Geo<NDIM>;
  return (uint64_t)(cx + 1) * G::CX > a.dims[0] ||
         (uint64_t)(cy + 1) * G::CY > a.dims[1] ||
         (uint64_t)(cz + 1) * G::CZ > a.dims[2];
}

// halo written by warp t for warp t+1: the part of the thread's biased q
// that the next tile's first difference needs
template <int NDIM>
__device__ __forceinline__ void write_halo(int32_t *xch, const int32_t (&tq)[64],
                                           int g) {
  using G = Geo<NDIM>;
  if constexpr (NDIM == 3) {
    // last z plane of the brick: 32 values, row-swizzled per lane
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      int4 v = make_int4(tq[32 + 4 * c], tq[33 + 4 * c], tq[34 + 4 * c], tq[35 + 4 * c]);
      *reinterpret_cast<int4 *>(xch + 32 * g + 4 * (c ^ (g & 7))) = v;
    }
  } else if constexpr (NDIM == 2) {
    if (g / G::NBX == G::NBY - 1) {
      const int bx = g % G::NBX;
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) xch[8 * bx + ix] = tq[56 + ix];
    }
  } else {
    if (g == 31) xch[0] = tq[63];
  }
}

template <int NDIM>
__device__ __forceinline__ void read_halo(int32_t (&halo)[32], const int32_t *xch,
                                          int t, int g) {
  using G = Geo<NDIM>;
  if constexpr (NDIM == 3) {
    if (t == 0) {
#pragma unroll
      for (int e = 0; e < 32; ++e) halo[e] = kPadBiased;
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        int4 v = *reinterpret_cast<const int4 *>(xch + 32 * g + 4 * (c ^ (g & 7)));
        halo[4 * c] = v.x; halo[4 * c + 1] = v.y; halo[4 * c + 2] = v.z; halo[4 * c + 3] = v.w;
      }
    }
  } else if constexpr (NDIM == 2) {
    const int bx = g % G::NBX;
#pragma unroll
    for (int ix = 0; ix < 8; ++ix) halo[ix] = t == 0 ? kPadBiased : xch[8 * bx + ix];
  } else {
    halo[0] = t == 0 ? kPadBiased : xch[0];
  }
}

// residual -> 16-bit sign-magnitude code pairs (Sec. 3.2); |r| >= 2^15 gets
// the escape code 0x8000.  Returns the OR of |r| over the brick.
__device__ __forceinline__ uint32_t pack_codes(const int32_t (&v)[64],
                                               uint32_t (&w)[32], bool escapes) {
  uint32_t orabs = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    int32_t d0 = v[2 * i], d1 = v[2 * i + 1];
    uint32_t a0 = (uint32_t)abs(d0), a1 = (uint32_t)abs(d1);
    orabs |= a0 | a1;
    uint32_t c0 = a0 | ((uint32_t)(d0 >> 16) & 0x8000u);
    uint32_t c1 = a1 | ((uint32_t)(d1 >> 16) & 0x8000u);
    if (escapes) {
      c0 = a0 > 32767u ? 0x8000u : c0;
      c1 = a1 > 32767u ? 0x8000u : c1;
    }
    w[i] = __byte_perm(c0, c1, 0x5410);
  }
  return orabs;
}

// one warp: everything from the box to the compacted tile in shared memory.
// Returns this tile's block count; writes the flag bytes to global memory.
struct TileOut {
  uint32_t nnz;
  uint32_t nout;
};

template <int NDIM>
__device__ __forceinline__ void compute_residuals(const CompressArgs &a, const uint8_t *box,
                                                  const int32_t *xch_prev, int32_t *xch_own,
                                                  float r, uint32_t cx, uint32_t cy,
                                                  uint32_t cz, int t, int g,
                                                  int32_t (&v)[64], uint32_t &qmax,
                                                  bool edge, bool sync_between) {
  load_quant<NDIM>(box, t, g, r, v, qmax);
  write_halo<NDIM>(xch_own, v, g);
  if (sync_between) __syncthreads();
  int32_t halo[32];
  read_halo<NDIM>(halo, xch_prev, t, g);
  lorenzo<NDIM>(v, halo, g);
  if (edge) mask_outside<NDIM>(v, a, cx, cy, cz, t, g);
}

template <int NDIM, bool TMA>
__global__ void __launch_bounds__(kThreads, 4)
    compress_kernel(const CompressArgs a, const __grid_constant__ CUtensorMap tmap) {
  using G = Geo<NDIM>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *box = smem;                                   // 32 KB, per warp 8 KB
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kBoxBytes);
  uint32_t *sh = reinterpret_cast<uint32_t *>(smem + kBoxBytes + 16);
  // sh[0] ticket, sh[1..4] tile nnz, sh[5..8] tile nout, sh[9] flags,
  // sh[10..11] base (u64), sh[12] eb ok, sh[13] r bits
  const int tid = threadIdx.x, t = tid >> 5, g = tid & 31;
  SetScratch *cur = a.set_cur;

  if (tid == 0) {
    uint32_t c = atomicAdd(&cur->ticket, 1u);
    sh[0] = c;
    // zero the other set's status word for this chunk (used by the next call)
    a.status_next[c] = 0;
    if (c == 0) {
      SetScratch *nx = a.set_next;
      nx->ticket = 0; nx->err = 0; nx->nnz = 0; nx->nout = 0;
      nx->n_chunks = 0; nx->hdr_nout = 0;
    }
    float fmin = 0.f, fmax = 0.f;
    bool nonfinite = false;
    if (a.mode == 1) {
      fmin = a.range->fmin; fmax = a.range->fmax;
      nonfinite = a.range->nonfinite != 0;
    }
    EbParams p = derive_eb(a.mode, a.eb_req, fmin, fmax);
    sh[12] = (p.ok && !nonfinite) ? 1u : 0u;
    sh[13] = __float_as_uint(p.ebx2_r);
    if (c == a.n_chunks - 1) {
      // the header's static fields; the totals follow after the look-back
      StreamHeader *h = reinterpret_cast<StreamHeader *>(a.out);
      h->magic[0] = 'F'; h->magic[1] = 'Z'; h->magic[2] = 'G'; h->magic[3] = '1';
      h->version = 1; h->ndim = (uint8_t)NDIM; h->mode = (uint8_t)a.mode;
      h->reserved0 = 0;
      h->dims[0] = (uint32_t)a.dims[0]; h->dims[1] = (uint32_t)a.dims[1];
      h->dims[2] = (uint32_t)a.dims[2];
      h->n_tiles = (uint32_t)(a.n_chunks * kTilesPerChunk);
      h->eb_requested = a.eb_req;
      h->eb = p.eb; h->ebx2 = p.ebx2; h->ebx2_r = p.ebx2_r;
      h->range_min = fmin; h->range_max = fmax;
      h->reserved1 = 0;
      if (!p.ok) atomicOr(&cur->err, kErrEbParam);
      if (nonfinite) atomicOr(&cur->err, kErrNonFinite);
    }
    if (TMA) mbar_init(bar, 1);
  }
  __syncthreads();
  const uint64_t c = sh[0];
  if (sh[12] == 0) return;                 // the same decision in every CTA
  const float r = __uint_as_float(sh[13]);
  const uint32_t cx = (uint32_t)(c % a.ncx);
  const uint32_t cy = (uint32_t)((c / a.ncx) % a.ncy);
  const uint32_t cz = (uint32_t)(c / ((uint64_t)a.ncx * a.ncy));

  // ---- stage the chunk in shared memory
  bool load_ok = true;
  if constexpr (TMA) {
    if (tid == 0) {
      mbar_expect_tx(bar, kBoxBytes);
      if constexpr (NDIM == 3) {
        tma_load_3d(box, &tmap, bar, (int)(cx * 32), (int)(cy * 32), (int)(cz * 8));
      } else {
        tma_load_2d(box, &tmap, bar, (int)(cx * 64), (int)(cy * 128));
        tma_load_2d(box + 16384, &tmap, bar, (int)(cx * 64 + 32), (int)(cy * 128));
      }
    }
    load_ok = mbar_wait_bounded(bar, 0, a.wait_limit_ns);
    if (!load_ok && g == 0) atomicOr(&cur->err, kErrTimeout);
  } else {
    fill_box_generic<NDIM>(a, box, cx, cy, cz);
    __syncthreads();
  }

  // ---- per warp: tile t of the chunk.  Each warp reads only its own two
  // 4 KB pieces of the box, which it reuses afterwards as scratch.
  uint8_t *piece_a = box + piece_offset<NDIM>(t, 0);
  uint8_t *piece_b = box + piece_offset<NDIM>(t, 1);
  int32_t *xch_own = reinterpret_cast<int32_t *>(
      smem + kBoxBytes + 1024 + t * 4096); // halo handed to warp t+1
  const int32_t *xch_prev = reinterpret_cast<const int32_t *>(
      smem + kBoxBytes + 1024 + (t > 0 ? t - 1 : 0) * 4096);
  const bool edge = chunk_is_edge<NDIM>(a, cx, cy, cz);
  int32_t v[64];
  uint32_t qmax = 0;
  compute_residuals<NDIM>(a, box, xch_prev, xch_own, r, cx, cy, cz, t, g, v, qmax,
                          edge, true);
  if (__any_sync(0xffffffffu, qmax > kBiasedMax) && g == 0)
    atomicOr(&cur->err, kErrRange);

  uint32_t w[32];
  uint32_t orabs = pack_codes(v, w, false);
  const bool esc = (orabs >> 15) != 0;
  uint32_t nout_lane = 0;
  if (__any_sync(0xffffffffu, esc)) {       // rare: some |residual| >= 2^15
#pragma unroll
    for (int e = 0; e < 64; ++e) nout_lane += (uint32_t)abs(v[e]) > 32767u;
    pack_codes(v, w, true);
  }
  __syncwarp();                             // every lane is done with the box
  transpose32(w);                           // lane g now holds out[32b+g]

  // ---- plane buffer: word (b, g) -> lane b gets plane b's 32 words
  uint32_t *pb = reinterpret_cast<uint32_t *>(piece_a);       // 4 KB
#pragma unroll
  for (int b = 0; b < 32; ++b) pb[32 * b + 4 * ((g >> 2) ^ (b & 7)) + (g & 3)] = w[b];
  __syncwarp();
  uint4 blk[8];
  uint32_t F = 0;                           // lane b: flag byte of plane b
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    blk[i] = *reinterpret_cast<const uint4 *>(pb + 32 * g + 4 * (i ^ (g & 7)));
    F |= ((blk[i].x | blk[i].y | blk[i].z | blk[i].w) != 0u ? 1u : 0u) << i;
  }
  const uint32_t pc = __popc(F);
  uint32_t P = pc;                          // inclusive scan over lanes
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, P, o);
    if (g >= o) P += y;
  }
  const uint32_t tile_nnz = __shfl_sync(0xffffffffu, P, 31);
  P -= pc;                                  // exclusive
  const uint64_t tile = c * kTilesPerChunk + t;
  a.out[64 + tile * 32 + g] = (uint8_t)F;   // flag byte b = plane b (Listing 1)
  const uint32_t tile_nout = __reduce_add_sync(0xffffffffu, nout_lane);
  if (g == 0) { sh[1 + t] = tile_nnz; sh[5 + t] = tile_nout; }
  __syncthreads();                          // (B) all halos read, counts known

  // ---- compaction into this warp's second piece (Listing 2:
  // block k goes to PreSum[k] when it is non-zero)
  uint4 *cb = reinterpret_cast<uint4 *>(piece_b);
  {
    uint32_t rank = P;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if ((F >> i) & 1u) { cb[rank] = blk[i]; ++rank; }
    }
  }

  // ---- chunk totals, look-back (warp 0), offsets
  uint32_t off_t = 0;
  uint64_t agg = 0;
#pragma unroll
  for (int k = 0; k < kTilesPerChunk; ++k) {
    if (k < t) off_t += sh[1 + k];
    agg += ((uint64_t)sh[1 + k] << 32) | sh[5 + k];
  }
  if (t == 0) {
    const bool publish = c != a.skip_publish_chunk;
    uint64_t excl = lookback(a.status_cur, c, agg, publish, &cur->err,
                             a.wait_limit_ns);
    if (g == 0) {
      sh[10] = (uint32_t)excl;
      sh[11] = (uint32_t)(excl >> 32);
      a.chunk_out_prefix[c] = (uint32_t)excl;           // outlier prefix
      a.chunk_out_count[c] = (uint32_t)agg;
      if (c == a.n_chunks - 1) {
        uint64_t inc = excl + agg;
        StreamHeader *h = reinterpret_cast<StreamHeader *>(a.out);
        h->nnz_blocks = (uint32_t)(inc >> 32);
        h->n_outliers = (uint32_t)inc;
        cur->nnz = inc >> 32;
        cur->nout = inc & 0xffffffffull;
      }
    }
  }
  __syncthreads();                          // (C)
  const uint64_t base_blocks = sh[11];     // block part of the prefix
  const uint64_t first = base_blocks + off_t;
  const uint64_t pay = 64 + 32 * a.n_chunks * kTilesPerChunk;
  if (tile_nnz > 0) {
    const uint64_t end = pay + 16 * (first + tile_nnz);
    if (end <= a.out_capacity) {
      if (g == 0) {
        fence_proxy_async_smem();
        bulk_store(a.out + pay + 16 * first, cb, tile_nnz * 16);
        bulk_commit();
        bulk_wait_read_all();
      }
    } else if (g == 0) {
      atomicOr(&cur->err, kErrCapacity);
    }
  }
  (void)load_ok;
}

// ====================================================================
// outlier pass (only for chunks that escaped some residual)
// ====================================================================
template <int NDIM, bool TMA>
__global__ void __launch_bounds__(kThreads, 4)
    outlier_kernel(const CompressArgs a, const __grid_constant__ CUtensorMap tmap,
                   uint64_t out_section) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *box = smem;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kBoxBytes);
  uint32_t *sh = reinterpret_cast<uint32_t *>(smem + kBoxBytes + 16);
  const int tid = threadIdx.x, t = tid >> 5, g = tid & 31;
  const uint64_t c = blockIdx.x;
  if (a.chunk_out_count[c] == 0) return;
  if (tid == 0) {
    float fmin = 0.f, fmax = 0.f;
    if (a.mode == 1) { fmin = a.range->fmin; fmax = a.range->fmax; }
    EbParams p = derive_eb(a.mode, a.eb_req, fmin, fmax);
    sh[13] = __float_as_uint(p.ebx2_r);
    if (TMA) mbar_init(bar, 1);
  }
  __syncthreads();
  const float r = __uint_as_float(sh[13]);
  const uint32_t cx = (uint32_t)(c % a.ncx);
  const uint32_t cy = (uint32_t)((c / a.ncx) % a.ncy);
  const uint32_t cz = (uint32_t)(c / ((uint64_t)a.ncx * a.ncy));
  if constexpr (TMA) {
    if (tid == 0) {
      mbar_expect_tx(bar, kBoxBytes);
      if constexpr (NDIM == 3) {
        tma_load_3d(box, &tmap, bar, (int)(cx * 32), (int)(cy * 32), (int)(cz * 8));
      } else {
        tma_load_2d(box, &tmap, bar, (int)(cx * 64), (int)(cy * 128));
        tma_load_2d(box + 16384, &tmap, bar, (int)(cx * 64 + 32), (int)(cy * 128));
      }
    }
    if (!mbar_wait_bounded(bar, 0, a.wait_limit_ns) && g == 0)
      atomicOr(&a.set_cur->err, kErrTimeout);
  } else {
    fill_box_generic<NDIM>(a, box, cx, cy, cz);
    __syncthreads();
  }
  int32_t *xch_own = reinterpret_cast<int32_t *>(smem + kBoxBytes + 1024 + t * 4096);
  const int32_t *xch_prev = reinterpret_cast<const int32_t *>(
      smem + kBoxBytes + 1024 + (t > 0 ? t - 1 : 0) * 4096);
  int32_t v[64];
  uint32_t qmax = 0;
  compute_residuals<NDIM>(a, box, xch_prev, xch_own, r, cx, cy, cz, t, g, v, qmax,
                          chunk_is_edge<NDIM>(a, cx, cy, cz), true);
  uint32_t cnt = 0;
#pragma unroll
  for (int e = 0; e < 64; ++e) cnt += (uint32_t)abs(v[e]) > 32767u;
  // exclusive scan of the counts in (tile, lane) = stream order
  uint32_t inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (g >= o) inc += y;
  }
  if (g == 31) sh[1 + t] = inc;
  __syncthreads();
  uint32_t before = inc - cnt;
  for (int k = 0; k < t; ++k) before += sh[1 + k];
  uint64_t pos = (uint64_t)a.chunk_out_prefix[c] + before;
  const uint64_t tile = c * kTilesPerChunk + t;
#pragma unroll
  for (int e = 0; e < 64; ++e) {
    if ((uint32_t)abs(v[e]) > 32767u) {
      const uint64_t at = out_section + 8 * pos;
      if (at + 8 <= a.out_capacity) {
        uint2 rec = make_uint2((uint32_t)(tile * kTileCodes + 64 * g + e), (uint32_t)v[e]);
        *reinterpret_cast<uint2 *>(a.out + at) = rec;
      } else {
        atomicOr(&a.set_cur->err, kErrCapacity);
      }
      ++pos;
    }
  }
}

// ====================================================================
// launchers
// ====================================================================
void launch_range(const float *x, uint64_t n, float2 *partial, int nblocks,
                  RangeResult *res, cudaStream_t s) {
  range_kernel<<<nblocks, 256, 0, s>>>(x, n, partial, res);
}

size_t compress_smem_bytes() { return kBoxBytes + 1024 + 4 * 4096 + 1024; }

template <int NDIM, bool TMA>
static cudaError_t launch_c(const CompressArgs &a, const CUtensorMap &tm,
                            cudaStream_t s, bool outliers, uint64_t out_section) {
  const size_t smem = compress_smem_bytes();
  if (!outliers) {
    auto k = compress_kernel<NDIM, TMA>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)a.n_chunks, kThreads, smem, s>>>(a, tm);
  } else {
    auto k = outlier_kernel<NDIM, TMA>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)a.n_chunks, kThreads, smem, s>>>(a, tm, out_section);
  }
  return cudaGetLastError();
}

cudaError_t launch_compress(int ndim, bool tma, const CompressArgs &a,
                            const CUtensorMap &tm, cudaStream_t s) {
  if (ndim == 3) return tma ? launch_c<3, true>(a, tm, s, false, 0) : launch_c<3, false>(a, tm, s, false, 0);
  if (ndim == 2) return tma ? launch_c<2, true>(a, tm, s, false, 0) : launch_c<2, false>(a, tm, s, false, 0);
  return launch_c<1, false>(a, tm, s, false, 0);
}

cudaError_t launch_outliers(int ndim, bool tma, const CompressArgs &a,
                            const CUtensorMap &tm, uint64_t out_section,
                            cudaStream_t s) {
  if (ndim == 3) return tma ? launch_c<3, true>(a, tm, s, true, out_section) : launch_c<3, false>(a, tm, s, true, out_section);
  if (ndim == 2) return tma ? launch_c<2, true>(a, tm, s, true, out_section) : launch_c<2, false>(a, tm, s, true, out_section);
  return launch_c<1, false>(a, tm, s, true, out_section);
}

}  // namespace fz
