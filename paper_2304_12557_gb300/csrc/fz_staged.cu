// fz_staged.cu -- the compression path as the paper's sequence of separate
// kernels with the intermediate data in HBM, for measuring what fusing them
// saves on this GPU.  The stream is byte for byte the fused kernel's.
//
//  staged_quant_kernel    pre-quantisation and chunk-local Lorenzo residual
//                         (Sec. 2.3, 3.1) -> 16-bit sign-magnitude codes
//                         (Sec. 3.2), written to HBM (4 KiB per tile)
//  staged_shuffle_kernel  reads the codes, bitshuffles (Sec. 3.3) and marks
//                         (Sec. 3.4, Listing 1): shuffled words to HBM, the
//                         stream's flag bytes, each tile's block count; the
//                         transpose is either the in-register one or, as in
//                         Listing 1, 32 warp ballots per 32-word group
//  staged_scan_kernel     exclusive scan of the tiles' (blocks, escapes)
//                         counts (the paper's prefix sum)
//  staged_encode_kernel   copies every tile's non-zero blocks to their place
//                         in the payload (Listing 2) and writes the header
// The escapes are written by the usual outlier pass afterwards.
#include <cuda_runtime.h>

#include "fz_compress_impl.cuh"
#include "fz_device.cuh"
#include "fz_kernels.h"

namespace fz {

namespace {

constexpr int kStagedWarps = 4;        // warps per block, one tile per warp at a time
constexpr int kScanTiles = 1024;       // tiles per scan block

}  // namespace

template <int NDIM, int V, bool CHECK>
__global__ void __launch_bounds__(kStagedWarps * 32)
    staged_quant_kernel(const CompressArgs a, uint32_t *codes) {
  const unsigned full = 0xffffffffu;
  const int g = threadIdx.x & 31;
  const uint64_t n_tiles = a.n_chunks * kTilesPerChunk;
  uint32_t err = 0;
  const FieldRt rt = derive_field(a, err);
  if (blockIdx.x == 0 && threadIdx.x == 0 && err) atomicOr(&a.set_cur->err, err);
  if (!rt.ok) return;
  const ChunkGrid cg(rt.dx, rt.dy);
  const uint64_t n_warps = (uint64_t)gridDim.x * kStagedWarps;
  for (uint64_t T = blockIdx.x * (uint64_t)kStagedWarps + (threadIdx.x >> 5); T < n_tiles;
       T += n_warps) {
    const TileGeo q = tile_geo<NDIM>(a, cg, T, g);
    float hf[32];
    load_halo<NDIM, V>(a, q, hf);
    int32_t v[64];
    uint32_t qmax = 0;
    residuals_first<NDIM, CHECK>(GlobalRows<NDIM, V>{a, q}, q, g, rt.p.ebx2_r, hf, v, qmax);
    residuals_rest<NDIM>(a, q, g, rt.p.ebx2_r, v);
    if (CHECK && __any_sync(full, qmax > kBiasedMax) && g == 0) atomicOr(&a.set_cur->err, kErrRange);
    uint32_t w[32];
    uint32_t orabs = 0;
#pragma unroll
    for (int e = 0; e < 64; ++e) orabs |= (uint32_t)abs(v[e]);
    uint32_t nout = 0;
    if (__any_sync(full, (orabs >> 15) != 0)) nout = pack_codes_escaped(v, w);
    else pack_codes(v, w);
    uint4 *dst = reinterpret_cast<uint4 *>(codes + T * 1024 + 32 * g);
#pragma unroll
    for (int i = 0; i < 8; ++i)
      __stcg(dst + i, make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]));
    const uint32_t tile_nout = __reduce_add_sync(full, nout);
    if (g == 0) a.tile_out_count[T] = tile_nout;
  }
}

__global__ void __launch_bounds__(kStagedWarps * 32)
    staged_shuffle_kernel(const uint32_t *codes, uint32_t *shuf, uint8_t *out,
                          uint32_t *tile_nnz, uint64_t n_tiles) {
  const unsigned full = 0xffffffffu;
  const int g = threadIdx.x & 31;
  const uint64_t n_warps = (uint64_t)gridDim.x * kStagedWarps;
  for (uint64_t T = blockIdx.x * (uint64_t)kStagedWarps + (threadIdx.x >> 5); T < n_tiles;
       T += n_warps) {
    uint32_t w[32];
    const uint4 *src = reinterpret_cast<const uint4 *>(codes + T * 1024 + 32 * g);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint4 u = __ldcg(src + i);
      w[4 * i] = u.x; w[4 * i + 1] = u.y; w[4 * i + 2] = u.z; w[4 * i + 3] = u.w;
    }
    transpose32(w);                      // lane g: shuffled words 32b + g
    uint32_t mine = 0;                   // lane b: which words of plane b are non-zero
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      __stcg(shuf + T * 1024 + 32 * b + g, w[b]);
      const uint32_t m = __ballot_sync(full, w[b] != 0u);
      if (g == b) mine = m;
    }
    uint32_t F = 0;                      // lane b: plane b's flag byte (blocks of 4 words)
#pragma unroll
    for (int i = 0; i < 8; ++i) F |= (((mine >> (4 * i)) & 0xFu) != 0u ? 1u : 0u) << i;
    out[64 + T * 32 + g] = (uint8_t)F;   // Listing 1's flags
    const uint32_t cnt = __reduce_add_sync(full, (uint32_t)__popc(F));
    if (g == 0) tile_nnz[T] = cnt;
  }
}

// The same step with Listing 1's bitshuffle.  A warp takes a tile's 32
// groups one at a time, lane t holding word t of the group (one coalesced
// 128-byte load); the ballot of bit b over the lanes is the group's plane-b
// word, and lane b keeps it (plane b of group g is word 32b + g, the
// columns-written reading of Listing 1).  After the 32 groups lane b holds
// plane b's 32 words: it stores them (128 contiguous bytes) and takes its
// flag byte from them (block j of the plane: words 4j..4j+3).  That is 32
// ballots per group, about one warp instruction per code for the transpose
// alone, against about four per 32 codes for transpose32.
__global__ void __launch_bounds__(kStagedWarps * 32)
    staged_shuffle_ballot_kernel(const uint32_t *codes, uint32_t *shuf, uint8_t *out,
                                 uint32_t *tile_nnz, uint64_t n_tiles) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const uint64_t n_warps = (uint64_t)gridDim.x * kStagedWarps;
  for (uint64_t T = blockIdx.x * (uint64_t)kStagedWarps + (threadIdx.x >> 5); T < n_tiles;
       T += n_warps) {
    uint32_t row[32];                    // lane b: plane b's word of every group
#pragma unroll
    for (int g = 0; g < 32; ++g) {
      const uint32_t wd = __ldcg(codes + T * 1024 + 32 * g + lane);
#pragma unroll
      for (int b = 0; b < 32; ++b) {
        const uint32_t m = __ballot_sync(full, (wd >> b) & 1u);
        if (lane == b) row[g] = m;
      }
    }
    uint4 *dst = reinterpret_cast<uint4 *>(shuf + T * 1024 + 32 * lane);
    uint32_t F = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      __stcg(dst + j, make_uint4(row[4 * j], row[4 * j + 1], row[4 * j + 2], row[4 * j + 3]));
      F |= ((row[4 * j] | row[4 * j + 1] | row[4 * j + 2] | row[4 * j + 3]) != 0u ? 1u : 0u) << j;
    }
    out[64 + T * 32 + lane] = (uint8_t)F;   // Listing 1's flags
    const uint32_t cnt = __reduce_add_sync(full, (uint32_t)__popc(F));
    if (lane == 0) tile_nnz[T] = cnt;
  }
}

// Exclusive scan of (blocks << 32 | escapes) over tiles: a block of
// kScanTiles threads per unit of tiles, ticketed in order, decoupled
// look-back across units.  Writes each tile's prefix and, from the last
// unit, the stream's totals.
__global__ void __launch_bounds__(kScanTiles)
    staged_scan_kernel(const CompressArgs a, const uint32_t *tile_nnz, uint64_t *tile_excl,
                       uint64_t *status) {
  const unsigned full = 0xffffffffu;
  __shared__ uint64_t warp_tot[kScanTiles / 32];
  __shared__ uint64_t s_unit, s_excl;
  const int g = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t n_tiles = a.n_chunks * kTilesPerChunk;
  const uint64_t n_units = (n_tiles + kScanTiles - 1) / kScanTiles;
  if (threadIdx.x == 0) s_unit = atomicAdd(&a.set_cur->ticket, 1u);
  __syncthreads();
  const uint64_t u = s_unit;
  if (u >= n_units) return;
  const uint64_t T = u * kScanTiles + threadIdx.x;
  const uint64_t val = T < n_tiles ? ((uint64_t)tile_nnz[T] << 32) | a.tile_out_count[T] : 0;
  uint64_t inc = val;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(full, inc, o);
    if (g >= o) inc += y;
  }
  if (g == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint64_t t = warp_tot[g];
    uint64_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(full, ti, o);
      if (g >= o) ti += y;
    }
    const uint64_t total = __shfl_sync(full, ti, 31);
    const uint64_t excl = lookback(status, u, total, true, &a.set_cur->err, a.wait_limit_ns);
    warp_tot[g] = ti - t;
    if (g == 0) {
      s_excl = excl;
      if (u == n_units - 1) {
        a.set_cur->nnz = (excl + total) >> 32;
        a.set_cur->nout = (excl + total) & 0xffffffffull;
      }
    }
  }
  __syncthreads();
  if (T < n_tiles) tile_excl[T] = s_excl + warp_tot[w] + inc - val;
}

__global__ void __launch_bounds__(kStagedWarps * 32)
    staged_encode_kernel(const CompressArgs a, const uint32_t *shuf, const uint64_t *tile_excl,
                         int ndim) {
  const unsigned full = 0xffffffffu;
  const int g = threadIdx.x & 31;
  const uint64_t n_tiles = a.n_chunks * kTilesPerChunk;
  const uint64_t pay = 64 + 32 * n_tiles;
  uint32_t err = 0;
  const FieldRt rt = derive_field(a, err);
  if (!rt.ok) return;
  const uint64_t n_warps = (uint64_t)gridDim.x * kStagedWarps;
  for (uint64_t T = blockIdx.x * (uint64_t)kStagedWarps + (threadIdx.x >> 5); T < n_tiles;
       T += n_warps) {
    const uint32_t F = a.out[64 + T * 32 + g];
    const uint32_t pc = __popc(F);
    uint32_t P = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(full, P, o);
      if (g >= o) P += y;
    }
    const uint32_t tile_nnz = __shfl_sync(full, P, 31);
    P -= pc;
    const uint64_t excl = tile_excl[T];
    if (g == 0) {
      a.tile_out_prefix[T] = (uint32_t)excl;
      if (T == n_tiles - 1) {
        const uint64_t inc = excl + (((uint64_t)tile_nnz << 32) | a.tile_out_count[T]);
        StreamHeader *h = reinterpret_cast<StreamHeader *>(a.out);
        h->magic[0] = 'F'; h->magic[1] = 'Z'; h->magic[2] = 'G'; h->magic[3] = '1';
        h->version = 1; h->ndim = (uint8_t)ndim; h->mode = (uint8_t)a.mode;
        h->reserved0 = 0;
        h->dims[0] = (uint32_t)a.dims[0]; h->dims[1] = (uint32_t)a.dims[1];
        h->dims[2] = (uint32_t)a.dims[2];
        h->n_tiles = (uint32_t)n_tiles;
        h->eb_requested = a.eb_req;
        h->eb = rt.p.eb; h->ebx2 = rt.p.ebx2; h->ebx2_r = rt.p.ebx2_r;
        h->nnz_blocks = (uint32_t)(inc >> 32);
        h->n_outliers = (uint32_t)inc;
        h->range_min = rt.fmin; h->range_max = rt.fmax;
        h->reserved1 = 0;
      }
    }
    uint64_t dst = pay + 16 * ((excl >> 32) + P);
    if (pay + 16 * ((excl >> 32) + tile_nnz) <= a.out_capacity) {
      const uint4 *src = reinterpret_cast<const uint4 *>(shuf + T * 1024 + 32 * g);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if ((F >> i) & 1u) {
          __stcs(reinterpret_cast<uint4 *>(a.out + dst), __ldcs(src + i));
          dst += 16;
        }
      }
    } else if (g == 0) {
      atomicOr(&a.set_cur->err, kErrCapacity);
    }
  }
}

// ====================================================================
// launch: the four kernels, each bracketed by events when ev != NULL
// ====================================================================
namespace {

template <int NDIM, int V, bool CHECK>
cudaError_t launch_quant(const CompressArgs &a, uint32_t *codes, int blocks, cudaStream_t s) {
  staged_quant_kernel<NDIM, V, CHECK><<<blocks, kStagedWarps * 32, 0, s>>>(a, codes);
  return cudaGetLastError();
}

template <int NDIM>
cudaError_t launch_quant_v(const CompressArgs &a, uint32_t *codes, int blocks, int v,
                           cudaStream_t s) {
  const bool check = a.mode == 0 || a.range_given;
  if (v == 8) return check ? launch_quant<NDIM, 8, true>(a, codes, blocks, s)
                           : launch_quant<NDIM, 8, false>(a, codes, blocks, s);
  if (v == 4) return check ? launch_quant<NDIM, 4, true>(a, codes, blocks, s)
                           : launch_quant<NDIM, 4, false>(a, codes, blocks, s);
  return check ? launch_quant<NDIM, 1, true>(a, codes, blocks, s)
               : launch_quant<NDIM, 1, false>(a, codes, blocks, s);
}

}  // namespace

cudaError_t launch_staged(int ndim, const CompressArgs &a, const StagedScratch &w, int sms,
                          bool ballot, cudaEvent_t *ev, cudaStream_t s) {
  const uint64_t n_tiles = a.n_chunks * kTilesPerChunk;
  const uintptr_t p = reinterpret_cast<uintptr_t>(a.x);
  const int v = (a.dims[0] % 8 == 0 && p % 32 == 0) ? 8 : (a.dims[0] % 4 == 0 && p % 16 == 0) ? 4 : 1;
  const int blocks = sms * 8;
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], s);
  e = ndim == 3   ? launch_quant_v<3>(a, w.codes, blocks, v, s)
      : ndim == 2 ? launch_quant_v<2>(a, w.codes, blocks, v, s)
                  : launch_quant_v<1>(a, w.codes, blocks, v, s);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], s);
  if (ballot)
    staged_shuffle_ballot_kernel<<<blocks, kStagedWarps * 32, 0, s>>>(w.codes, w.shuf, a.out,
                                                                       w.tile_nnz, n_tiles);
  else
    staged_shuffle_kernel<<<blocks, kStagedWarps * 32, 0, s>>>(w.codes, w.shuf, a.out,
                                                                w.tile_nnz, n_tiles);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], s);
  const uint64_t units = (n_tiles + kScanTiles - 1) / kScanTiles;
  staged_scan_kernel<<<(unsigned)units, kScanTiles, 0, s>>>(a, w.tile_nnz, w.tile_excl, w.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[3], s);
  staged_encode_kernel<<<blocks, kStagedWarps * 32, 0, s>>>(a, w.shuf, w.tile_excl, ndim);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[4], s);
  return cudaSuccess;
}

uint64_t staged_status_words(uint64_t n_tiles) { return (n_tiles + kScanTiles - 1) / kScanTiles; }

}  // namespace fz
