// fz_noalloc.cu -- fz_compress_noalloc: compression for callers that cannot
// allocate device memory.
//
// Some callers must not allocate GPU memory while they run:
//  * applications whose memory pool (a framework's caching allocator, or
//    an arena sized at start-up) has already reserved the free HBM, so that
//    a cudaMalloc inside the library would fail or fragment the pool;
//  * latency-critical loops that cannot afford the device-wide
//    synchronisation and driver round trips of cudaMalloc/cudaFree;
//  * deployments with a fixed memory plan decided before the work starts.
// fz_compress needs a context whose scratch is allocated by fz_create.  This
// entry point instead keeps the same scratch in one statically sized device
// array that is part of the library image, so it allocates nothing.  The
// caller still passes the input and output buffers.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>

#include "fz.h"
#include "fz_device.cuh"
#include "fz_kernels.h"

namespace {

constexpr uint64_t kMaxTiles = FZ_NOALLOC_MAX_CODES / fz::kTileCodes;
// look-back words per set: one per unit of consecutive tiles
constexpr uint64_t kMaxUnits = fz::compress_status_words(kMaxTiles);
constexpr int kRangeBlocks = 1216;
constexpr int kMaxDevices = 64;

// Layout of the static scratch (every array 64-byte aligned).
struct NoAllocScratch {
  fz::SetScratch sets[2];                 // result blocks (64 B each)
  fz::RangeResult range;                  // min/max/non-finite + counter
  uint32_t pad[12];
  float2 partial[kRangeBlocks];           // per-block range partials
  uint64_t status[2][kMaxUnits * fz::kStatusStride];  // look-back words (set 1 is only
                                          // ever written with zeros)
  uint32_t out_prefix[kMaxTiles];
  uint32_t out_count[kMaxTiles];
};
static_assert(offsetof(NoAllocScratch, partial) % 64 == 0, "alignment");
static_assert(offsetof(NoAllocScratch, status) % 64 == 0, "alignment");
// the size the public header states (FZ_NOALLOC_SCRATCH_BYTES)
static_assert(sizeof(NoAllocScratch) <= FZ_NOALLOC_SCRATCH_BYTES, "scratch size as documented");

}  // namespace

// The scratch itself: one array per device that loads the library, held
// until the process exits.  In host code this name is only a host-side
// stand-in; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

namespace {

std::mutex g_mu;
NoAllocScratch *g_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (the current device),
// looked up once per device.
NoAllocScratch *scratch_on(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return nullptr;
    g_addr[dev] = static_cast<NoAllocScratch *>(p);
  }
  return g_addr[dev];
}

bool shape_of(const uint64_t dims[3], int ndim, uint64_t d[3], uint64_t *n_chunks,
              uint64_t *n_elems, uint32_t *ncx, uint32_t *ncy) {
  if (!dims || ndim < 1 || ndim > 3) return false;
  for (int i = 0; i < 3; ++i) {
    d[i] = i < ndim ? dims[i] : 1;
    if (d[i] == 0 || d[i] > 0xFFFFFFFFull) return false;
  }
  const uint64_t cx = ndim == 1 ? 8192 : (ndim == 2 ? 64 : 32);
  const uint64_t cy = ndim == 1 ? 1 : (ndim == 2 ? 128 : 32);
  const uint64_t cz = ndim == 3 ? 8 : 1;
  const uint64_t a = (d[0] + cx - 1) / cx, b = (d[1] + cy - 1) / cy, c = (d[2] + cz - 1) / cz;
  const unsigned __int128 nc = (unsigned __int128)a * b * c;
  if (nc * fz::kChunkCodes > 0xFFFFFFFFull) return false;
  *n_chunks = (uint64_t)nc;
  *n_elems = d[0] * d[1] * d[2];
  *ncx = (uint32_t)a;
  *ncy = (uint32_t)b;
  return true;
}

int read_result(const fz::SetScratch *dev_res, fz::SetScratch *host, cudaStream_t s) {
  if (cudaMemcpyAsync(host, dev_res, sizeof(*host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

}  // namespace

extern "C" int fz_compress_noalloc(const float *d_in, const uint64_t dims[3], int ndim,
                                   int mode, double eb, void *d_out, uint64_t cap,
                                   uint64_t *out_size, void *stream) {
  if (out_size) *out_size = 0;
  uint64_t d[3], n_chunks = 0, n_elems = 0;
  uint32_t ncx = 0, ncy = 0;
  if (!d_in || !d_out || !out_size || !shape_of(dims, ndim, d, &n_chunks, &n_elems, &ncx, &ncy))
    return FZ_ERR_ARG;
  if (n_chunks * fz::kTilesPerChunk > kMaxTiles) return FZ_ERR_ARG;  // beyond the scratch
  if (mode != FZ_EB_ABS && mode != FZ_EB_REL) return FZ_ERR_ARG;
  if (!(eb > 0.0) || !std::isfinite(eb)) return FZ_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(d_out) & 15u) || (reinterpret_cast<uintptr_t>(d_in) & 3u))
    return FZ_ERR_ARG;
  const uint64_t n_tiles = n_chunks * fz::kTilesPerChunk;
  const uint64_t min_bytes = 64 + 32 * n_tiles;
  if (cap < min_bytes) {
    *out_size = min_bytes;
    return FZ_ERR_CAPACITY;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return FZ_ERR_CUDA;
  NoAllocScratch *sc = scratch_on(dev);
  if (!sc) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // the array keeps the previous call's contents: clear what must start at 0
  // (both result blocks, the range counter, this field's look-back words)
  const uint64_t units = fz::compress_status_words(n_tiles);
  if (cudaMemsetAsync(sc, 0, offsetof(NoAllocScratch, partial), s) != cudaSuccess ||
      cudaMemsetAsync(sc->status[0], 0, units * fz::kStatusStride * sizeof(uint64_t), s) !=
          cudaSuccess)
    return FZ_ERR_CUDA;
  if (mode == FZ_EB_REL) {
    const uint64_t want = (n_elems / 4 + 255) / 256;
    const int nb = (int)(want < (uint64_t)kRangeBlocks ? (want ? want : 1) : kRangeBlocks);
    fz::launch_range(d_in, n_elems, sc->partial, nb, &sc->range, s);
    if (cudaGetLastError() != cudaSuccess) return FZ_ERR_CUDA;
  }
  fz::CompressArgs a{};
  a.x = d_in;
  a.allow_wide = 0;                   // |q| up to 2^22 - 1 (no second launch)
  for (int i = 0; i < 3; ++i) a.dims[i] = d[i];
  a.pitch = d[0];
  a.ncx = ncx;
  a.ncy = ncy;
  a.n_chunks = n_chunks;
  a.mode = mode;
  a.eb_req = eb;
  a.range = &sc->range;
  a.set_cur = &sc->sets[0];
  a.set_next = &sc->sets[1];
  a.status_cur = sc->status[0];
  a.status_next = sc->status[1];
  a.tile_out_prefix = sc->out_prefix;
  a.tile_out_count = sc->out_count;
  a.out = static_cast<uint8_t *>(d_out);
  a.out_capacity = cap;
  a.wait_limit_ns = 2000000000ull;
  a.skip_publish_chunk = ~0ull;
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  const bool tma = fz::compress_uses_tma(ndim, a) && fz::encode_field_tmap(ndim, d, d_in, &tm);
  if (fz::launch_compress(ndim, a, tma ? &tm : nullptr, sms, s, mode == FZ_EB_REL) !=
      cudaSuccess)
    return FZ_ERR_CUDA;
  fz::SetScratch r;
  int st = read_result(&sc->sets[0], &r, s);
  if (st) return st;
  if (r.err & fz::kErrNonFinite) return FZ_ERR_NONFINITE;
  if (r.err & (fz::kErrEbParam | fz::kErrRange)) {
    if (mode == FZ_EB_REL) return FZ_ERR_EB_RANGE;
    // an absolute bound: the input's finiteness decides the status
    fz::launch_range(d_in, n_elems, sc->partial, kRangeBlocks, &sc->range, s);
    fz::RangeResult rr;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&rr, &sc->range, sizeof(rr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return FZ_ERR_CUDA;
    return rr.nonfinite ? FZ_ERR_NONFINITE : FZ_ERR_EB_RANGE;
  }
  if (r.err & fz::kErrTimeout) return FZ_ERR_TIMEOUT;
  const uint64_t total = min_bytes + 16 * r.nnz + 8 * r.nout;
  if ((r.err & fz::kErrCapacity) || total > cap) {
    *out_size = total;
    return FZ_ERR_CAPACITY;
  }
  if (r.nout > 0) {
    // escaped residuals: the rare second pass, reporting into result block 1
    // (zeroed above; the compression kernel only ever writes zeros to it)
    a.set_cur = &sc->sets[1];
    if (cudaMemsetAsync(&sc->sets[1], 0, sizeof(fz::SetScratch), s) != cudaSuccess ||
        fz::launch_outliers(ndim, a, min_bytes + 16 * r.nnz, s) != cudaSuccess)
      return FZ_ERR_CUDA;
    if ((st = read_result(&sc->sets[1], &r, s))) return st;
    if (r.err & fz::kErrTimeout) return FZ_ERR_TIMEOUT;
    if (r.err & fz::kErrCapacity) {
      *out_size = total;
      return FZ_ERR_CAPACITY;
    }
  }
  *out_size = total;
  return FZ_OK;
}
