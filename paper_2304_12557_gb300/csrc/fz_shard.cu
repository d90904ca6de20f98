// fz_shard.cu -- one field split into slabs across ranks: the slab plan, the
// concatenation of the slabs' streams into the whole field's stream (host
// form, and the plan and outlier-index kernel behind the device form in
// fz_api.cu).
//
// Chunks are independent (Sec. 2.3), and the stream lists tiles chunk by
// chunk with the chunk grid x fastest, so the chunks of a slab of whole chunk
// rows along the slowest axis are a contiguous run of the field's chunk
// order.  A slab's stream is therefore a contiguous run of the field's flag
// words, of its payload blocks (Listing 2 keeps them in tile order) and of
// its outlier list, with code indices counted from the slab's first tile.
#include <cuda_runtime.h>

#include <cstring>

#include "fz.h"
#include "fz_device.cuh"
#include "fz_kernels.h"

namespace fz {

namespace {

uint32_t get32(const uint8_t *p) {
  uint32_t v;
  std::memcpy(&v, p, 4);
  return v;
}
void put32(uint8_t *p, uint32_t v) { std::memcpy(p, &v, 4); }

// extent of one chunk along the slowest axis (3-D z: 8, 2-D y: 128, 1-D x: 8192)
uint64_t slab_align(int ndim) { return ndim == 3 ? 8 : (ndim == 2 ? 128 : 8192); }

}  // namespace

int concat_plan(const uint8_t (*hdrs)[64], const uint64_t *sizes, int n, ConcatPart *parts,
                ConcatPlan *plan) {
  if (!hdrs || !sizes || !parts || !plan || n < 1) return FZ_ERR_ARG;
  fz_info first{};
  uint64_t slow = 0, tiles = 0, nnz = 0, nout = 0;
  for (int i = 0; i < n; ++i) {
    fz_info f{};
    if (sizes[i] < 64 || fz_inspect(hdrs[i], 64, &f) != FZ_OK) return FZ_ERR_CORRUPT;
    if (f.stream_bytes != sizes[i]) return FZ_ERR_CORRUPT;
    // whole-field residuals cross slab faces: such slabs do not concatenate
    if (f.version != 1) return FZ_ERR_VERSION;
    const int ax = f.ndim - 1;
    if (i == 0) {
      first = f;
    } else {
      // same quantiser: ndim, mode, requested and derived bound, range
      // (header bytes 24..43 and 52..59) and the same cross-section
      if (f.ndim != first.ndim || f.mode != first.mode ||
          std::memcmp(hdrs[i] + 24, hdrs[0] + 24, 20) != 0 ||
          std::memcmp(hdrs[i] + 52, hdrs[0] + 52, 8) != 0)
        return FZ_ERR_CORRUPT;
      for (int k = 0; k < ax; ++k)
        if (f.dims[k] != first.dims[k]) return FZ_ERR_CORRUPT;
    }
    // every slab but the last ends on a chunk boundary
    if (i + 1 < n && f.dims[ax] % slab_align(f.ndim) != 0) return FZ_ERR_CORRUPT;
    parts[i].tiles = f.n_tiles;
    parts[i].nnz = f.nnz_blocks;
    parts[i].nout = f.n_outliers;
    parts[i].tile_off = tiles;
    parts[i].nnz_off = nnz;
    parts[i].out_off = nout;
    slow += f.dims[ax];
    tiles += f.n_tiles;
    nnz += f.nnz_blocks;
    nout += f.n_outliers;
  }
  const int ax = first.ndim - 1;
  if (slow > 0xFFFFFFFFull || nnz > 0xFFFFFFFFull || nout > 0xFFFFFFFFull) return FZ_ERR_CORRUPT;
  uint64_t dims[3] = {first.dims[0], first.dims[1], first.dims[2]};
  dims[ax] = slow;
  const uint64_t min_bytes = fz_stream_min_bytes(dims, first.ndim);
  if (min_bytes == 0 || min_bytes != 64 + 32 * tiles) return FZ_ERR_CORRUPT;
  std::memcpy(plan->hdr, hdrs[0], 64);
  // the wide quantiser's flag: set when any slab needed it (the codes and
  // outlier records are the same either way)
  for (int i = 0; i < n; ++i) plan->hdr[7] |= hdrs[i][7];
  put32(plan->hdr + 8 + 4 * ax, (uint32_t)slow);
  put32(plan->hdr + 20, (uint32_t)tiles);
  put32(plan->hdr + 44, (uint32_t)nnz);
  put32(plan->hdr + 48, (uint32_t)nout);
  plan->n_tiles = tiles;
  plan->nnz = nnz;
  plan->nout = nout;
  plan->total = 64 + 32 * tiles + 16 * nnz + 8 * nout;
  return FZ_OK;
}

// outlier records (u32 code index, i32 residual) of one slab, moved to the
// field's code numbering
__global__ void __launch_bounds__(256) rebase_outliers_kernel(const uint2 *__restrict__ src,
                                                              uint2 *__restrict__ dst,
                                                              uint64_t n, uint32_t add) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    uint2 r = src[i];
    r.x += add;
    dst[i] = r;
  }
}

cudaError_t launch_rebase_outliers(const void *src, void *dst, uint64_t n, uint32_t add,
                                   cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want < 4096 ? want : 4096);
  rebase_outliers_kernel<<<blocks, 256, 0, s>>>(static_cast<const uint2 *>(src),
                                                static_cast<uint2 *>(dst), n, add);
  return cudaGetLastError();
}

}  // namespace fz

extern "C" {

int fz_shard_extent(const uint64_t dims[3], int ndim, int n_shards, int shard, uint64_t *begin,
                    uint64_t *end) {
  if (!begin || !end || n_shards < 1 || shard < 0 || shard >= n_shards) return FZ_ERR_ARG;
  if (fz_stream_min_bytes(dims, ndim) == 0) return FZ_ERR_ARG;
  const uint64_t L = dims[ndim - 1], A = fz::slab_align(ndim);
  const uint64_t rows = (L + A - 1) / A;           // chunk rows, < 2^32
  const uint64_t r0 = rows * (uint64_t)shard / (uint64_t)n_shards;
  const uint64_t r1 = rows * (uint64_t)(shard + 1) / (uint64_t)n_shards;
  *begin = r0 * A < L ? r0 * A : L;
  *end = r1 * A < L ? r1 * A : L;
  return FZ_OK;
}

int fz_concat_streams_host(const void *const *h_parts, const uint64_t *part_sizes, int n_parts,
                           void *h_out, uint64_t cap, uint64_t *out_size) {
  if (out_size) *out_size = 0;
  if (!h_parts || !part_sizes || !out_size || n_parts < 1 || (!h_out && cap > 0))
    return FZ_ERR_ARG;
  for (int i = 0; i < n_parts; ++i)
    if (!h_parts[i]) return FZ_ERR_ARG;
  uint8_t(*hdrs)[64] = new uint8_t[n_parts][64];
  fz::ConcatPart *parts = new fz::ConcatPart[n_parts];
  for (int i = 0; i < n_parts; ++i)
    std::memcpy(hdrs[i], h_parts[i], part_sizes[i] < 64 ? part_sizes[i] : 64);
  fz::ConcatPlan plan;
  int st = fz::concat_plan(hdrs, part_sizes, n_parts, parts, &plan);
  if (st == FZ_OK && plan.total > cap) {
    *out_size = plan.total;
    st = FZ_ERR_CAPACITY;
  }
  if (st == FZ_OK) {
    uint8_t *o = static_cast<uint8_t *>(h_out);
    const uint64_t pay = 64 + 32 * plan.n_tiles, outs = pay + 16 * plan.nnz;
    std::memcpy(o, plan.hdr, 64);
    for (int i = 0; i < n_parts; ++i) {
      const uint8_t *p = static_cast<const uint8_t *>(h_parts[i]);
      const fz::ConcatPart &q = parts[i];
      std::memcpy(o + 64 + 32 * q.tile_off, p + 64, 32 * q.tiles);
      std::memcpy(o + pay + 16 * q.nnz_off, p + 64 + 32 * q.tiles, 16 * q.nnz);
      const uint8_t *src = p + 64 + 32 * q.tiles + 16 * q.nnz;
      uint8_t *dst = o + outs + 8 * q.out_off;
      const uint32_t add = (uint32_t)(q.tile_off * fz::kTileCodes);
      for (uint64_t k = 0; k < q.nout; ++k) {
        fz::put32(dst + 8 * k, fz::get32(src + 8 * k) + add);
        std::memcpy(dst + 8 * k + 4, src + 8 * k + 4, 4);
      }
    }
    *out_size = plan.total;
  }
  delete[] hdrs;
  delete[] parts;
  return st;
}

}  // extern "C"
