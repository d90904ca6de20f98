// fz_decompress.cu -- GB300 decompression kernel (Sec. 4.4: the compression
// pipeline run backwards).
//
// Persistent warps; each warp takes chunks from a ticket counter in stream
// order and for each chunk:
//   flags -> popcounts -> warp-level decoupled look-back (payload offset)
//   per tile: gather the non-zero 16-byte blocks (Listing 2 backwards),
//   inverse bitshuffle (the same register transpose), sign-magnitude decode,
//   outlier patch (rare), chunk-local inverse Lorenzo as prefix sums along
//   x and y (in-register + warp scans) and z/y across tiles (a carried
//   plane/row), q * 2eb, stores.
// The header is validated on the device, so the call needs no host read of
// the stream before the launch.
#include <cuda_runtime.h>

#include "fz_device.cuh"
#include "fz_kernels.h"

namespace fz {

struct Hdr {
  int ndim, mode;
  uint32_t dims[3];
  uint64_t n_tiles, nnz, nout, n_chunks, ncx, ncy, n_elems;
  float ebx2;
  bool ok;
};

__device__ __forceinline__ uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

__device__ Hdr read_header(const DecompressArgs &a) {
  Hdr h{};
  h.ok = false;
  if (a.in_size < 64) return h;
  const StreamHeader *s = reinterpret_cast<const StreamHeader *>(a.in);
  if (s->magic[0] != 'F' || s->magic[1] != 'Z' || s->magic[2] != 'G' || s->magic[3] != '1')
    return h;
  if (s->version != 1 || s->reserved0 != 0 || s->mode > 1) return h;
  h.ndim = s->ndim;
  h.mode = s->mode;
  if (h.ndim < 1 || h.ndim > 3) return h;
  for (int i = 0; i < 3; ++i) h.dims[i] = s->dims[i];
  for (int i = 0; i < 3; ++i) {
    if (i < h.ndim && h.dims[i] == 0) return h;
    if (i >= h.ndim && h.dims[i] != 1) return h;
  }
  uint64_t cx = h.ndim == 1 ? 8192 : (h.ndim == 2 ? 64 : 32);
  uint64_t cy = h.ndim == 1 ? 1 : (h.ndim == 2 ? 128 : 32);
  uint64_t cz = h.ndim == 3 ? 8 : 1;
  h.ncx = cdiv(h.dims[0], cx);
  h.ncy = cdiv(h.dims[1], cy);
  h.n_chunks = h.ncx * h.ncy * cdiv(h.dims[2], cz);
  h.n_tiles = h.n_chunks * kTilesPerChunk;
  if (h.n_tiles * kTileCodes > 0xFFFFFFFFull) return h;
  if (s->n_tiles != h.n_tiles) return h;
  h.nnz = s->nnz_blocks;
  h.nout = s->n_outliers;
  if (64 + 32 * h.n_tiles + 16 * h.nnz + 8 * h.nout != a.in_size) return h;
  h.n_elems = (uint64_t)h.dims[0] * h.dims[1] * h.dims[2];
  h.ebx2 = s->ebx2;
  h.ok = true;
  return h;
}

// first record index in [0, n) whose stream index is >= key (records sorted)
__device__ __forceinline__ uint64_t lower_bound_rec(const uint2 *rec, uint64_t n,
                                                    uint32_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (__ldg(&rec[mid].x) < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// residual of the escaped code with stream index `key`, searched among the
// chunk's records [lo, hi); false when absent or not a real outlier
__device__ __noinline__ bool find_outlier(const uint2 *rec, uint64_t lo, uint64_t hi,
                                          uint32_t key, int32_t *val) {
  uint64_t k = lo + lower_bound_rec(rec + lo, hi - lo, key);
  if (k >= hi) return false;
  uint2 r = __ldg(&rec[k]);
  if (r.x != key) return false;
  int32_t v = (int32_t)r.y;
  if (v >= -32767 && v <= 32767) return false;
  *val = v;
  return true;
}

// decode 32 packed code pairs to residuals; escapes (0x8000) decode to 0 and
// set the returned flag
__device__ __forceinline__ bool decode_codes(const uint32_t (&w)[32], int32_t (&v)[64]) {
  uint32_t esc = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    uint32_t c0 = w[i] & 0xFFFFu, c1 = w[i] >> 16;
    esc |= (c0 == 0x8000u) | (c1 == 0x8000u);
    int32_t s0 = -(int32_t)(c0 >> 15), s1 = -(int32_t)(c1 >> 15);
    v[2 * i] = ((int32_t)(c0 & 0x7FFFu) ^ s0) - s0;
    v[2 * i + 1] = ((int32_t)(c1 & 0x7FFFu) ^ s1) - s1;
  }
  return esc != 0;
}

// position of brick element e of lane g in tile t of chunk (cx,cy,cz)
template <int NDIM>
__device__ __forceinline__ void elem_coord(uint64_t cx, uint64_t cy, uint64_t cz, int t,
                                           int g, int e, uint64_t &x, uint64_t &y,
                                           uint64_t &z) {
  using G = Geo<NDIM>;
  const int bx = g % G::NBX, by = g / G::NBX;
  const int ix = e % G::BX, iy = (e / G::BX) % G::BY, iz = e / (G::BX * G::BY);
  if constexpr (NDIM == 3) {
    x = cx * 32 + 8 * bx + ix; y = cy * 32 + 4 * by + iy; z = cz * 8 + 2 * t + iz;
  } else if constexpr (NDIM == 2) {
    x = cx * 64 + 8 * bx + ix; y = cy * 128 + 32 * t + 8 * by + iy; z = 0;
  } else {
    x = cx * 8192 + 2048 * t + 64 * g + e; y = 0; z = 0;
  }
}

// inverse Lorenzo inside the tile: v holds residuals in, q out.  `carry`
// holds the previous tile's boundary values of q (3-D: this brick's last
// plane, 2-D: the last row, 1-D: the last element) and is updated.
template <int NDIM>
__device__ __forceinline__ void inverse_lorenzo(int32_t (&v)[64], int32_t (&carry)[32], int g) {
  using G = Geo<NDIM>;
  const unsigned full = 0xffffffffu;
  const int bx = g % G::NBX, by = g / G::NBX;
  if constexpr (NDIM == 3) {
    // S_x: rows of 8, then an exclusive scan of row totals over the 4 bx lanes
#pragma unroll
    for (int row = 0; row < 8; ++row) {
#pragma unroll
      for (int ix = 1; ix < 8; ++ix) v[ix + 8 * row] += v[ix - 1 + 8 * row];
      const int32_t tot = v[7 + 8 * row];
      int32_t inc = tot;
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        int32_t y = __shfl_up_sync(full, inc, o);
        if (bx >= o) inc += y;
      }
      const int32_t ex = inc - tot;
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) v[ix + 8 * row] += ex;
    }
    // S_y: columns of 4, then over the 8 by lanes (lane stride 4)
#pragma unroll
    for (int iz = 0; iz < 2; ++iz) {
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) {
#pragma unroll
        for (int iy = 1; iy < 4; ++iy) v[ix + 8 * iy + 32 * iz] += v[ix + 8 * (iy - 1) + 32 * iz];
        const int32_t tot = v[ix + 24 + 32 * iz];
        int32_t inc = tot;
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
          int32_t y = __shfl_up_sync(full, inc, o);
          if (g >= o) inc += y;
        }
        const int32_t ex = inc - tot;
#pragma unroll
        for (int iy = 0; iy < 4; ++iy) v[ix + 8 * iy + 32 * iz] += ex;
      }
    }
    // S_z: the two planes of the tile plus the carried plane
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      v[e] += carry[e];
      v[e + 32] += v[e];
      carry[e] = v[e + 32];
    }
  } else if constexpr (NDIM == 2) {
    // S_x over 8 bx lanes
#pragma unroll
    for (int row = 0; row < 8; ++row) {
#pragma unroll
      for (int ix = 1; ix < 8; ++ix) v[ix + 8 * row] += v[ix - 1 + 8 * row];
      const int32_t tot = v[7 + 8 * row];
      int32_t inc = tot;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        int32_t y = __shfl_up_sync(full, inc, o);
        if (bx >= o) inc += y;
      }
      const int32_t ex = inc - tot;
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) v[ix + 8 * row] += ex;
    }
    // S_y over 4 by lanes (lane stride 8), plus the previous tile's last row
#pragma unroll
    for (int ix = 0; ix < 8; ++ix) {
#pragma unroll
      for (int iy = 1; iy < 8; ++iy) v[ix + 8 * iy] += v[ix + 8 * (iy - 1)];
      const int32_t tot = v[ix + 56];
      int32_t inc = tot;
#pragma unroll
      for (int o = 8; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(full, inc, o);
        if (g >= o) inc += y;
      }
      const int32_t ex = inc - tot + carry[ix];
#pragma unroll
      for (int iy = 0; iy < 8; ++iy) v[ix + 8 * iy] += ex;
      carry[ix] = __shfl_sync(full, v[ix + 56], bx + 8 * (G::NBY - 1));
    }
  } else {
#pragma unroll
    for (int e = 1; e < 64; ++e) v[e] += v[e - 1];
    const int32_t tot = v[63];
    int32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(full, inc, o);
      if (g >= o) inc += y;
    }
    const int32_t ex = inc - tot + carry[0];
#pragma unroll
    for (int e = 0; e < 64; ++e) v[e] += ex;
    carry[0] = __shfl_sync(full, v[63], 31);
  }
}

template <int NDIM>
__device__ __forceinline__ void store_brick(const DecompressArgs &a, const Hdr &h,
                                            const int32_t (&q)[64], uint64_t cx,
                                            uint64_t cy, uint64_t cz, int t, int g,
                                            bool edge, bool vec) {
  using G = Geo<NDIM>;
  const float e2 = h.ebx2;
  const uint64_t X = h.dims[0], Y = h.dims[1];
  float f[64];
#pragma unroll
  for (int e = 0; e < 64; ++e) {
    // (float)q exactly for |q| < 2^22, then the stream's one multiply
    float qf = __fsub_rn(__int_as_float(q[e] + (int32_t)kMagicBits), kRoundMagic);
    f[e] = __fmul_rn(qf, e2);
  }
#pragma unroll
  for (int row = 0; row < 64 / G::BX; ++row) {
    uint64_t x0, y, z;
    elem_coord<NDIM>(cx, cy, cz, t, g, row * G::BX, x0, y, z);
    float *dst = a.out + x0 + X * (y + Y * z);
    const bool full_row = !edge || (x0 + G::BX <= X && y < Y && z < h.dims[2]);
    if (vec && full_row) {
#pragma unroll
      for (int k = 0; k < G::BX / 4; ++k)
        __stcs(reinterpret_cast<float4 *>(dst) + k,
               make_float4(f[row * G::BX + 4 * k], f[row * G::BX + 4 * k + 1],
                           f[row * G::BX + 4 * k + 2], f[row * G::BX + 4 * k + 3]));
    } else if (full_row) {
#pragma unroll
      for (int k = 0; k < G::BX; ++k) __stcs(dst + k, f[row * G::BX + k]);
    } else if (y < Y && z < h.dims[2]) {
#pragma unroll
      for (int k = 0; k < G::BX; ++k)
        if (x0 + k < X) __stcs(dst + k, f[row * G::BX + k]);
    }
  }
}

template <int NDIM>
__device__ void decompress_chunks(const DecompressArgs &a, const Hdr &h, uint32_t *pb,
                                  SetScratch *cur) {
  using G = Geo<NDIM>;
  const unsigned full = 0xffffffffu;
  const int g = threadIdx.x & 31;
  const uint8_t *flags = a.in + 64;
  const uint8_t *payload = flags + 32 * h.n_tiles;
  const uint2 *recs = reinterpret_cast<const uint2 *>(payload + 16 * h.nnz);
  const bool vec = ((h.dims[0] & 3u) == 0) && ((reinterpret_cast<uintptr_t>(a.out) & 15u) == 0);
  while (true) {
    uint64_t c = 0;
    if (g == 0) c = atomicAdd(&cur->ticket, 1u);
    c = __shfl_sync(full, c, 0);
    if (c >= h.n_chunks) break;
    if (g == 0) a.status_next[c] = 0;
    const uint64_t cx = c % h.ncx, cy = (c / h.ncx) % h.ncy, cz = c / (h.ncx * h.ncy);
    // flags of the chunk's 4 tiles: lane l holds word l
    const uint32_t fw = __ldg(reinterpret_cast<const uint32_t *>(flags + 128 * c) + g);
    const uint32_t pcw = __popc(fw);
    const uint32_t chunk_cnt = __reduce_add_sync(full, pcw);
    const bool publish = c != a.skip_publish_chunk;
    const uint64_t excl = lookback(a.status_cur, c, (uint64_t)chunk_cnt << 32, publish,
                                   &cur->err, a.wait_limit_ns) >> 32;
    if (c == h.n_chunks - 1 && g == 0 && excl + chunk_cnt != h.nnz)
      atomicOr(&cur->err, kErrCorrupt);
    // outliers of this chunk (rare path)
    uint64_t o_lo = 0, o_hi = 0;
    if (h.nout) {
      if (g == 0) {
        o_lo = lower_bound_rec(recs, h.nout, (uint32_t)(c * kChunkCodes));
        o_hi = lower_bound_rec(recs, h.nout, (uint32_t)((c + 1) * kChunkCodes));
      }
      o_lo = __shfl_sync(full, o_lo, 0);
      o_hi = __shfl_sync(full, o_hi, 0);
    }
    uint32_t matched = 0;
    const bool edge = (cx + 1) * G::CX > h.dims[0] || (cy + 1) * G::CY > h.dims[1] ||
                      (cz + 1) * G::CZ > h.dims[2];
    int32_t carry[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) carry[e] = 0;
    uint64_t tile_base = excl;
#pragma unroll 1
    for (int t = 0; t < kTilesPerChunk; ++t) {
      // lane b: flag byte of plane b
      const uint32_t F = (__shfl_sync(full, fw, 8 * t + (g >> 2)) >> (8 * (g & 3))) & 0xFFu;
      const uint32_t pc = __popc(F);
      uint32_t P = pc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(full, P, o);
        if (g >= o) P += y;
      }
      P -= pc;
      // gather plane b's blocks into the plane buffer
      uint32_t rank = P;
      bool oob = false;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        uint4 val = make_uint4(0, 0, 0, 0);
        if ((F >> i) & 1u) {
          const uint64_t bi = tile_base + rank;
          if (bi < h.nnz) val = __ldcs(reinterpret_cast<const uint4 *>(payload) + bi);
          else oob = true;
          ++rank;
        }
        *reinterpret_cast<uint4 *>(pb + 32 * g + 4 * (i ^ (g & 7))) = val;
      }
      if (oob) atomicOr(&cur->err, kErrCorrupt);
      __syncwarp();
      uint32_t w[32];
#pragma unroll
      for (int b = 0; b < 32; ++b) w[b] = pb[32 * b + 4 * ((g >> 2) ^ (b & 7)) + (g & 3)];
      __syncwarp();
      tile_base += __reduce_add_sync(full, (g >> 3) == t ? pcw : 0u);
      transpose32(w);                    // lane g: the 32 code words of brick g
      int32_t v[64];
      const bool esc = decode_codes(w, v);
      if (__any_sync(full, esc || edge)) {
        // rare path: patch escapes from the outlier list; padding must be 0.
        // Fully unrolled so that v and w stay in registers.
        const uint64_t tile = c * kTilesPerChunk + t;
        uint32_t bad = 0;
#pragma unroll
        for (int e = 0; e < 64; ++e) {
          const uint32_t code = (w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
          uint64_t x, y, z;
          elem_coord<NDIM>(cx, cy, cz, t, g, e, x, y, z);
          const bool inside = x < h.dims[0] && y < h.dims[1] && z < h.dims[2];
          bad |= (!inside && code != 0);
          if (inside && code == 0x8000u) {
            int32_t val;
            if (find_outlier(recs, o_lo, o_hi, (uint32_t)(tile * kTileCodes + 64 * g + e), &val)) {
              v[e] = val;
              ++matched;
            } else {
              bad = 1;
            }
          }
        }
        if (bad) atomicOr(&cur->err, kErrCorrupt);
      }
      inverse_lorenzo<NDIM>(v, carry, g);
      store_brick<NDIM>(a, h, v, cx, cy, cz, t, g, edge, vec);
    }
    if (h.nout) {
      const uint32_t m = __reduce_add_sync(full, matched);
      if (g == 0) {
        if (m != o_hi - o_lo) atomicOr(&cur->err, kErrCorrupt);
        atomicAdd(reinterpret_cast<unsigned long long *>(&cur->nout), (unsigned long long)m);
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads, 3) decompress_kernel(const DecompressArgs a) {
  __shared__ __align__(16) uint32_t plane_buf[kThreads / 32][1024];
  SetScratch *cur = a.set_cur;
  const int w = threadIdx.x >> 5, g = threadIdx.x & 31;
  const Hdr h = read_header(a);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    SetScratch *nx = a.set_next;
    nx->ticket = 0; nx->err = 0; nx->nnz = 0; nx->nout = 0; nx->n_chunks = 0; nx->hdr_nout = 0;
    if (!h.ok) atomicOr(&cur->err, kErrCorrupt);
    else if (a.out_cap_elems < h.n_elems) atomicOr(&cur->err, kErrCapacity);
    else if (h.n_chunks > a.status_cap) atomicOr(&cur->err, kErrCorrupt);
    cur->n_chunks = h.ok ? h.n_chunks : 0;
    cur->nnz = h.ok ? h.nnz : 0;
    cur->hdr_nout = h.ok ? (uint32_t)h.nout : 0;
  }
  if (!h.ok || a.out_cap_elems < h.n_elems || h.n_chunks > a.status_cap) return;
  uint32_t *pb = plane_buf[w];
  if (h.ndim == 3) decompress_chunks<3>(a, h, pb, cur);
  else if (h.ndim == 2) decompress_chunks<2>(a, h, pb, cur);
  else decompress_chunks<1>(a, h, pb, cur);
  (void)g;
}

cudaError_t launch_decompress(const DecompressArgs &a, int grid, cudaStream_t s) {
  decompress_kernel<<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

int decompress_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decompress_kernel, kThreads, 0) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace fz
