// fz_decompress.cu -- GB300 decompression kernel (Sec. 4.4: the compression
// pipeline run backwards).
//
// Persistent warps; each warp takes chunks from a ticket counter in stream
// order and for each chunk:
//   flags -> popcounts -> warp-level decoupled look-back (payload offset);
//   all four tiles' non-zero 16-byte blocks are copied at once with
//   asynchronous zero-filling copies into per-warp plane buffers (Listing 2
//   backwards), then per tile: escape detection on the bit planes, inverse
//   bitshuffle (the register transpose), sign-magnitude decode, outlier
//   patch (rare), chunk-local inverse Lorenzo as prefix sums (in-register and
//   warp scans, a carried plane/row across tiles), q * 2eb, 32-byte stores.
// The header is validated on the device, so the call needs no host read of
// the stream before the launch.
#include <cuda_runtime.h>

#include "fz_device.cuh"
#include "fz_kernels.h"

namespace fz {

constexpr int kDecWarps = 4;
constexpr int kDecSmemBytes = kDecWarps * kTilesPerChunk * 4096;

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

// 16-byte asynchronous copy global -> shared; with `bytes` = 0 nothing is
// read and the destination is zero-filled
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)),
               "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// PRMT with sign-replicating selectors (a selector nibble with its msb set
// copies the sign bit of the chosen byte into all 8 bits); the CUDA
// intrinsic __byte_perm masks that bit off, hence the inline PTX.
__device__ __forceinline__ uint32_t prmt_sign(uint32_t x, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(0u), "r"(sel));
  return r;
}

// decode 32 packed sign-magnitude pairs to residuals (an escape, 0x8000,
// decodes to 0 and is patched later)
__device__ __forceinline__ void decode_codes(const uint32_t (&w)[32], int32_t (&v)[64]) {
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const uint32_t s0 = prmt_sign(w[i], 0x9999);   // sign of the low code, replicated
    const uint32_t s1 = prmt_sign(w[i], 0xBBBB);   // sign of the high code
    v[2 * i] = (int32_t)(((w[i] & 0x7FFFu) ^ s0) - s0);
    v[2 * i + 1] = (int32_t)((((w[i] >> 16) & 0x7FFFu) ^ s1) - s1);
  }
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
  const int bx = g % G::NBX;
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
        const int32_t y = __shfl_up_sync(full, inc, o);
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
          const int32_t y = __shfl_up_sync(full, inc, o);
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
#pragma unroll
    for (int row = 0; row < 8; ++row) {                 // S_x over 8 bx lanes
#pragma unroll
      for (int ix = 1; ix < 8; ++ix) v[ix + 8 * row] += v[ix - 1 + 8 * row];
      const int32_t tot = v[7 + 8 * row];
      int32_t inc = tot;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int32_t y = __shfl_up_sync(full, inc, o);
        if (bx >= o) inc += y;
      }
      const int32_t ex = inc - tot;
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) v[ix + 8 * row] += ex;
    }
#pragma unroll
    for (int ix = 0; ix < 8; ++ix) {                    // S_y over 4 by lanes
#pragma unroll
      for (int iy = 1; iy < 8; ++iy) v[ix + 8 * iy] += v[ix + 8 * (iy - 1)];
      const int32_t tot = v[ix + 56];
      int32_t inc = tot;
#pragma unroll
      for (int o = 8; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(full, inc, o);
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
      const int32_t y = __shfl_up_sync(full, inc, o);
      if (g >= o) inc += y;
    }
    const int32_t ex = inc - tot + carry[0];
#pragma unroll
    for (int e = 0; e < 64; ++e) v[e] += ex;
    carry[0] = __shfl_sync(full, v[63], 31);
  }
}

// q (biased by the float bits of 1.5*2^23, which the chunk origin carries)
// -> fl(float(q) * 2eb), stored row by row (8 floats per row)
template <int NDIM>
__device__ __forceinline__ void store_brick(const DecompressArgs &a, const Hdr &h,
                                            const int32_t (&q)[64], uint64_t cx, uint64_t cy,
                                            uint64_t cz, int t, int g, bool edge, int vw) {
  const float e2 = h.ebx2;
  const uint64_t X = h.dims[0], Y = h.dims[1];
#pragma unroll
  for (int row = 0; row < 8; ++row) {
    float f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      f[k] = __fmul_rn(__fsub_rn(__int_as_float(q[8 * row + k]), kRoundMagic), e2);
    uint64_t x0, y, z;
    elem_coord<NDIM>(cx, cy, cz, t, g, 8 * row, x0, y, z);
    float *dst = a.out + x0 + X * (y + Y * z);
    const bool full_row = !edge || (x0 + 8 <= X && y < Y && z < h.dims[2]);
    if (full_row && vw == 8) {
      asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(dst),
                   "f"(f[0]), "f"(f[1]), "f"(f[2]), "f"(f[3]), "f"(f[4]), "f"(f[5]),
                   "f"(f[6]), "f"(f[7])
                   : "memory");
    } else if (full_row && vw == 4) {
      __stcs(reinterpret_cast<float4 *>(dst), make_float4(f[0], f[1], f[2], f[3]));
      __stcs(reinterpret_cast<float4 *>(dst) + 1, make_float4(f[4], f[5], f[6], f[7]));
    } else if (full_row) {
#pragma unroll
      for (int k = 0; k < 8; ++k) __stcs(dst + k, f[k]);
    } else if (y < Y && z < h.dims[2]) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (x0 + k < X) __stcs(dst + k, f[k]);
    }
  }
}

template <int NDIM>
__device__ void decompress_chunks(const DecompressArgs &a, const Hdr &h, uint32_t *pbuf,
                                  SetScratch *cur) {
  using G = Geo<NDIM>;
  const unsigned full = 0xffffffffu;
  const int g = threadIdx.x & 31;
  const uint8_t *flags = a.in + 64;
  const uint8_t *payload = flags + 32 * h.n_tiles;
  const uint2 *recs = reinterpret_cast<const uint2 *>(payload + 16 * h.nnz);
  const uintptr_t op = reinterpret_cast<uintptr_t>(a.out);
  const int vw = (h.dims[0] % 8 == 0 && op % 32 == 0) ? 8
                 : (h.dims[0] % 4 == 0 && op % 16 == 0) ? 4 : 1;
  const FastDiv dx((uint32_t)h.ncx), dy((uint32_t)h.ncy);
  while (true) {
    uint64_t c = 0;
    if (g == 0) c = atomicAdd(&cur->ticket, 1u);
    c = __shfl_sync(full, c, 0);
    if (c >= h.n_chunks) break;
    if (g == 0) a.status_next[c * kStatusStride] = 0;
    const uint32_t cr = dx.div((uint32_t)c);
    const uint64_t cx = (uint32_t)c - cr * dx.d, cz = dy.div(cr), cy = cr - (uint32_t)cz * dy.d;
    // flags of the chunk's 4 tiles: lane l holds word l
    const uint32_t fw = __ldg(reinterpret_cast<const uint32_t *>(flags + 128 * c) + g);
    const uint32_t chunk_cnt = __reduce_add_sync(full, (uint32_t)__popc(fw));
    const bool publish = c != a.skip_publish_chunk;
    const uint64_t excl = lookback(a.status_cur, c, (uint64_t)chunk_cnt << 32, publish,
                                   &cur->err, a.wait_limit_ns) >> 32;
    if (c == h.n_chunks - 1 && g == 0 && excl + chunk_cnt != h.nnz)
      atomicOr(&cur->err, kErrCorrupt);

    // gather all four tiles: lane b copies plane b's present blocks (Listing
    // 2 backwards: block k of the tile comes from payload[PreSum[k]])
    uint64_t base = excl;
    bool oob = false;
#pragma unroll
    for (int t = 0; t < kTilesPerChunk; ++t) {
      const uint32_t F = (__shfl_sync(full, fw, 8 * t + (g >> 2)) >> (8 * (g & 3))) & 0xFFu;
      const uint32_t pc = __popc(F);
      uint32_t P = pc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, P, o);
        if (g >= o) P += y;
      }
      const uint32_t tile_cnt = __shfl_sync(full, P, 31);
      uint64_t rank = base + P - pc;
      uint32_t *dst = pbuf + 1024 * t + 32 * g;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const bool present = (F >> i) & 1u;
        const bool valid = present && rank < h.nnz;
        oob |= present && !valid;
        cp_async16(dst + 4 * (i ^ (g & 7)), payload + 16 * (valid ? rank : 0), valid ? 16u : 0u);
        rank += present;
      }
      cp_async_commit();
      base += tile_cnt;
    }
    if (oob) atomicOr(&cur->err, kErrCorrupt);

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
#pragma unroll 1
    for (int t = 0; t < kTilesPerChunk; ++t) {
      switch (t) {
        case 0: cp_async_wait<3>(); break;
        case 1: cp_async_wait<2>(); break;
        case 2: cp_async_wait<1>(); break;
        default: cp_async_wait<0>(); break;
      }
      __syncwarp();
      const uint32_t *pb = pbuf + 1024 * t;
      uint32_t w[32];
#pragma unroll
      for (int b = 0; b < 32; ++b) w[b] = pb[32 * b + 4 * ((g >> 2) ^ (b & 7)) + (g & 3)];
      // an escape (0x8000) has its sign plane set and every magnitude plane
      // clear: find them on the planes, before the transpose
      uint32_t lo_or = 0, hi_or = 0;
#pragma unroll
      for (int b = 0; b < 15; ++b) { lo_or |= w[b]; hi_or |= w[b + 16]; }
      const uint32_t esc_even = w[15] & ~lo_or, esc_odd = w[31] & ~hi_or;
      transpose32(w);                    // lane g: the 32 code words of brick g
      int32_t v[64];
      decode_codes(w, v);
      if (__any_sync(full, (esc_even | esc_odd) != 0 || edge)) {
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
      // the chunk origin carries the float bias of 1.5*2^23 into every q
      if (t == 0 && g == 0) v[0] += (int32_t)kMagicBits;
      inverse_lorenzo<NDIM>(v, carry, g);
      store_brick<NDIM>(a, h, v, cx, cy, cz, t, g, edge, vw);
    }
    __syncwarp();                        // plane buffers free for the next chunk
    if (h.nout) {
      const uint32_t m = __reduce_add_sync(full, matched);
      if (g == 0) {
        if (m != o_hi - o_lo) atomicOr(&cur->err, kErrCorrupt);
        atomicAdd(reinterpret_cast<unsigned long long *>(&cur->nout), (unsigned long long)m);
      }
    }
  }
}

__global__ void __launch_bounds__(kDecWarps * 32, 3) decompress_kernel(const DecompressArgs a) {
  extern __shared__ __align__(16) uint32_t dsmem[];
  SetScratch *cur = a.set_cur;
  const int w = threadIdx.x >> 5;
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
  uint32_t *pbuf = dsmem + w * kTilesPerChunk * 1024;
  if (h.ndim == 3) decompress_chunks<3>(a, h, pbuf, cur);
  else if (h.ndim == 2) decompress_chunks<2>(a, h, pbuf, cur);
  else decompress_chunks<1>(a, h, pbuf, cur);
}

cudaError_t launch_decompress(const DecompressArgs &a, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(decompress_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kDecSmemBytes);
  if (e != cudaSuccess) return e;
  decompress_kernel<<<grid, kDecWarps * 32, kDecSmemBytes, s>>>(a);
  return cudaGetLastError();
}

int decompress_blocks_per_sm() {
  int n = 0;
  cudaFuncSetAttribute(decompress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kDecSmemBytes);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decompress_kernel, kDecWarps * 32,
                                                    kDecSmemBytes) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace fz
