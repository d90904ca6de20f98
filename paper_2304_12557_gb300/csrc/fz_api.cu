// fz_api.cu -- the C ABI declared in include/fz.h: context and scratch
// management, argument checks, launches and status mapping.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "fz.h"
#include "fz_device.cuh"
#include "fz_kernels.h"
#include "fz_pwrel.h"

using fz::RangeResult;
using fz::SetScratch;

struct fz_ctx {
  int device = 0;
  int num_sms = 1;
  int dec_blocks_per_sm = 1;
  // scratch: two alternating sets (see SetScratch)
  SetScratch *sets = nullptr;          // [2]
  uint64_t *status = nullptr;          // [2][cap]
  uint32_t *out_prefix = nullptr;      // [cap]
  uint32_t *out_count = nullptr;       // [cap]
  uint64_t cap = 0;
  RangeResult *range = nullptr;
  float2 *partial = nullptr;
  int range_blocks = 0;
  SetScratch *h_res = nullptr;         // pinned, mapped
  SetScratch *h_res_dev = nullptr;     // h_res as the device addresses it
  // the pipelined host-buffer decompression: copy streams, events and the
  // slab boundaries' payload offsets (mapped pinned memory)
  cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
  cudaEvent_t pipe_ev[24] = {};
  uint32_t *h_slab = nullptr, *h_slab_dev = nullptr;
  RangeResult *h_range = nullptr;      // pinned
  int cur = 0;
  uint64_t dirty_hi[2] = {0, 0};
  bool hdr_dirty[2] = {false, false};
  uint64_t wait_limit_ns = 2000000000ull;
  uint64_t skip_publish = ~0ull;
  // host-call staging
  void *stage_in = nullptr;
  uint64_t stage_in_cap = 0;
  void *stage_out = nullptr;
  uint64_t stage_out_cap = 0;
  // version-2 decompression: faces and scan work space, grown on demand
  void *whole = nullptr;
  uint64_t whole_bytes = 0;
  // the unfused path's scratch (fz_compress_staged), grown on demand
  void *staged = nullptr;
  uint64_t staged_tiles = 0;
  cudaEvent_t staged_ev[6] = {};
  int staged_shuffle = FZ_SHUFFLE_REGISTER;
  // profiling: events around each kernel of the last call
  bool profiling = false;
  cudaEvent_t ev[2 * fz::kProfSlots] = {};
  bool ev_used[fz::kProfSlots] = {};
  // whole-call timing: [0] compress, [1] decompress (start, end)
  bool call_timing = false;
  cudaEvent_t call_ev[4] = {};
  bool call_used[2] = {};
};

namespace fz {
int context_device(const fz_ctx *c) { return c ? c->device : -1; }
}  // namespace fz

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

constexpr uint64_t kMaxCodes = 0xFFFFFFFFull;

struct Shape {
  int ndim;
  uint64_t d[3];
  uint64_t ncx, ncy, ncz, n_chunks, n_tiles, n_elems;
};

bool make_shape(const uint64_t dims[3], int ndim, Shape *s) {
  if (!dims || ndim < 1 || ndim > 3) return false;
  s->ndim = ndim;
  for (int i = 0; i < 3; ++i) {
    s->d[i] = i < ndim ? dims[i] : 1;
    if (s->d[i] == 0 || s->d[i] > 0xFFFFFFFFull) return false;
  }
  const uint64_t cx = ndim == 1 ? 8192 : (ndim == 2 ? 64 : 32);
  const uint64_t cy = ndim == 1 ? 1 : (ndim == 2 ? 128 : 32);
  const uint64_t cz = ndim == 3 ? 8 : 1;
  s->ncx = (s->d[0] + cx - 1) / cx;
  s->ncy = (s->d[1] + cy - 1) / cy;
  s->ncz = (s->d[2] + cz - 1) / cz;
  // guard the products against overflow before the code-count limit
  if (s->ncx > kMaxCodes || s->ncy > kMaxCodes || s->ncz > kMaxCodes) return false;
  const unsigned __int128 nc = (unsigned __int128)s->ncx * s->ncy * s->ncz;
  if (nc * fz::kChunkCodes > kMaxCodes) return false;
  s->n_chunks = (uint64_t)nc;
  s->n_tiles = s->n_chunks * fz::kTilesPerChunk;
  s->n_elems = s->d[0] * s->d[1] * s->d[2];
  return true;
}

void free_scratch(fz_ctx *c) {
  cudaFree(c->sets); cudaFree(c->status); cudaFree(c->out_prefix);
  cudaFree(c->out_count);
  c->sets = nullptr; c->status = nullptr; c->out_prefix = nullptr;
  c->out_count = nullptr; c->cap = 0;
}

int ensure_cap(fz_ctx *c, uint64_t n) {
  if (n <= c->cap && c->sets) return FZ_OK;
  uint64_t cap = c->cap ? c->cap : 4096;
  while (cap < n) cap *= 2;
  free_scratch(c);
  if (cudaMalloc(&c->sets, 2 * sizeof(SetScratch)) != cudaSuccess ||
      cudaMalloc(&c->status, 2 * cap * fz::kStatusStride * sizeof(uint64_t)) != cudaSuccess ||
      cudaMalloc(&c->out_prefix, cap * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&c->out_count, cap * sizeof(uint32_t)) != cudaSuccess) {
    free_scratch(c);
    return FZ_ERR_CUDA;
  }
  if (cudaMemset(c->sets, 0, 2 * sizeof(SetScratch)) != cudaSuccess ||
      cudaMemset(c->status, 0, 2 * cap * fz::kStatusStride * sizeof(uint64_t)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    free_scratch(c);
    return FZ_ERR_CUDA;
  }
  c->cap = cap;
  c->dirty_hi[0] = c->dirty_hi[1] = 0;
  c->hdr_dirty[0] = c->hdr_dirty[1] = false;
  return FZ_OK;
}

// make the current set clean before a launch
int prepare_set(fz_ctx *c, cudaStream_t s) {
  const int A = c->cur;
  if (c->dirty_hi[A] > 0) {
    if (cudaMemsetAsync(c->status + A * c->cap * fz::kStatusStride, 0,
                        c->dirty_hi[A] * fz::kStatusStride * sizeof(uint64_t), s) !=
        cudaSuccess)
      return FZ_ERR_CUDA;
    c->dirty_hi[A] = 0;
  }
  if (c->hdr_dirty[A]) {
    if (cudaMemsetAsync(c->sets + A, 0, sizeof(SetScratch), s) != cudaSuccess)
      return FZ_ERR_CUDA;
    c->hdr_dirty[A] = false;
  }
  return FZ_OK;
}

// after a launch that used `used` status entries of the current set and
// zeroed the first `zeroed` entries (and the header) of the other set
void retire_set(fz_ctx *c, uint64_t used, uint64_t zeroed) {
  const int A = c->cur, B = 1 - A;
  c->dirty_hi[A] = used;
  c->hdr_dirty[A] = true;
  if (c->dirty_hi[B] <= zeroed) c->dirty_hi[B] = 0;
  c->hdr_dirty[B] = false;
  c->cur = B;
}

void mark_all_dirty(fz_ctx *c) {
  c->dirty_hi[0] = c->dirty_hi[1] = c->cap;
  c->hdr_dirty[0] = c->hdr_dirty[1] = true;
}

int range_pass(fz_ctx *c, const float *x, uint64_t n, cudaStream_t s) {
  const uint64_t want = (n / 4 + 255) / 256;
  int nb = (int)(want < (uint64_t)c->range_blocks ? (want ? want : 1) : c->range_blocks);
  fz::launch_range(x, n, c->partial, nb, c->range, s);
  return cudaGetLastError() == cudaSuccess ? FZ_OK : FZ_ERR_CUDA;
}

// The result block of `set` to the host; `done` (may be NULL) is recorded
// after it, before the wait.  One warp stores the 64 bytes into the mapped
// pinned block, launched as a programmatic dependent of the kernel before it
// (its launch overlaps that kernel; it reads the block once that grid has
// finished): a device-to-host copy at the end of the stream adds about 6 us
// to a call, this about 1.
int read_set(fz_ctx *c, int set, cudaStream_t s, cudaEvent_t done = nullptr) {
  if (fz::launch_copy_result(c->sets + set, c->h_res_dev, s) != cudaSuccess ||
      (done && cudaEventRecord(done, s) != cudaSuccess) ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

// the input's finiteness decides between NONFINITE and EB_RANGE
int classify_range_error(fz_ctx *c, const float *x, uint64_t n, cudaStream_t s) {
  if (range_pass(c, x, n, s) != FZ_OK) return FZ_ERR_CUDA;
  if (cudaMemcpyAsync(c->h_range, c->range, sizeof(RangeResult), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FZ_ERR_CUDA;
  return c->h_range->nonfinite ? FZ_ERR_NONFINITE : FZ_ERR_EB_RANGE;
}

// events k (start) / k+kProfSlots (end) bracket kernel k when profiling is on
void prof_begin(fz_ctx *c, int k, cudaStream_t s) {
  if (c->profiling) cudaEventRecord(c->ev[k], s);
}
void prof_end(fz_ctx *c, int k, cudaStream_t s) {
  if (c->profiling) {
    cudaEventRecord(c->ev[k + fz::kProfSlots], s);
    c->ev_used[k] = true;
  }
}
void prof_reset(fz_ctx *c) {
  for (bool &u : c->ev_used) u = false;
}

uint32_t rd32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
         ((uint32_t)p[3] << 24);
}

}  // namespace

extern "C" {

const char *fz_strerror(int st) {
  switch (st) {
    case FZ_OK: return "success";
    case FZ_ERR_ARG: return "invalid argument";
    case FZ_ERR_CAPACITY: return "output buffer too small";
    case FZ_ERR_NONFINITE: return "input contains NaN or Inf";
    case FZ_ERR_EB_RANGE: return "error bound too small for the data range";
    case FZ_ERR_CORRUPT: return "corrupt or inconsistent stream";
    case FZ_ERR_TIMEOUT: return "a bounded device wait timed out";
    case FZ_ERR_CUDA: return "CUDA runtime error";
    case FZ_ERR_VERSION: return "stream version not read by this call";
    default: return "unknown status";
  }
}

int fz_create(fz_ctx **out, int device) {
  if (!out) return FZ_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return FZ_ERR_CUDA;
  DeviceGuard guard(device);
  if (!guard.ok) return FZ_ERR_CUDA;
  fz_ctx *c = new (std::nothrow) fz_ctx();
  if (!c) return FZ_ERR_CUDA;
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (c->num_sms < 1) c->num_sms = 1;
  c->dec_blocks_per_sm = fz::decompress_blocks_per_sm();
  c->range_blocks = c->num_sms * 8;
  if (cudaMalloc(&c->range, sizeof(RangeResult)) != cudaSuccess ||
      cudaMemset(c->range, 0, sizeof(RangeResult)) != cudaSuccess ||
      cudaMalloc(&c->partial, c->range_blocks * sizeof(float2)) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void **>(&c->h_res), sizeof(SetScratch),
                    cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->h_res_dev), c->h_res, 0) !=
          cudaSuccess ||
      cudaMallocHost(&c->h_range, sizeof(RangeResult)) != cudaSuccess ||
      ensure_cap(c, 4096) != FZ_OK) {
    fz_destroy(c);
    return FZ_ERR_CUDA;
  }
  for (cudaEvent_t &e : c->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      fz_destroy(c);
      return FZ_ERR_CUDA;
    }
  }
  for (cudaEvent_t &e : c->call_ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      fz_destroy(c);
      return FZ_ERR_CUDA;
    }
  }
  *out = c;
  return FZ_OK;
}

void fz_destroy(fz_ctx *c) {
  if (!c) return;
  DeviceGuard guard(c->device);
  free_scratch(c);
  cudaFree(c->whole);
  cudaFree(c->staged);
  for (cudaEvent_t e : c->staged_ev)
    if (e) cudaEventDestroy(e);
  cudaFree(c->range);
  cudaFree(c->partial);
  cudaFree(c->stage_in);
  cudaFree(c->stage_out);
  if (c->h_res) cudaFreeHost(c->h_res);
  if (c->h_slab) cudaFreeHost(c->h_slab);
  for (cudaEvent_t e : c->pipe_ev)
    if (e) cudaEventDestroy(e);
  if (c->pipe_in) cudaStreamDestroy(c->pipe_in);
  if (c->pipe_out) cudaStreamDestroy(c->pipe_out);
  if (c->h_range) cudaFreeHost(c->h_range);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->call_ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

uint64_t fz_stream_min_bytes(const uint64_t dims[3], int ndim) {
  Shape sh;
  if (!make_shape(dims, ndim, &sh)) return 0;
  return 64 + 32 * sh.n_tiles;
}

uint64_t fz_compress_bound(const uint64_t dims[3], int ndim) {
  Shape sh;
  if (!make_shape(dims, ndim, &sh)) return 0;
  return 64 + 32 * sh.n_tiles + 16 * 256 * sh.n_tiles + 8 * (uint64_t)fz::kTileCodes * sh.n_tiles;
}

int fz_set_wait_limit_ns(fz_ctx *c, uint64_t ns) {
  if (!c || ns == 0) return FZ_ERR_ARG;
  c->wait_limit_ns = ns;
  return FZ_OK;
}

int fz_set_profiling(fz_ctx *c, int on) {
  if (!c) return FZ_ERR_ARG;
  c->profiling = on != 0;
  prof_reset(c);
  return FZ_OK;
}

int fz_get_kernel_times(fz_ctx *c, double ms[5]) {
  if (!c || !ms) return FZ_ERR_ARG;
  DeviceGuard guard(c->device);
  for (int k = 0; k < fz::kProfSlots; ++k) {
    ms[k] = 0.0;
    if (!c->ev_used[k]) continue;
    float t = 0.f;
    if (cudaEventSynchronize(c->ev[k + fz::kProfSlots]) != cudaSuccess ||
        cudaEventElapsedTime(&t, c->ev[k], c->ev[k + fz::kProfSlots]) != cudaSuccess)
      return FZ_ERR_CUDA;
    ms[k] = t;
  }
  return FZ_OK;
}

int fz_set_staged_shuffle(fz_ctx *c, int kind) {
  if (!c || (kind != FZ_SHUFFLE_REGISTER && kind != FZ_SHUFFLE_BALLOT)) return FZ_ERR_ARG;
  c->staged_shuffle = kind;
  return FZ_OK;
}

int fz_set_call_timing(fz_ctx *c, int on) {
  if (!c) return FZ_ERR_ARG;
  c->call_timing = on != 0;
  c->call_used[0] = c->call_used[1] = false;
  return FZ_OK;
}

int fz_get_call_times(fz_ctx *c, double ms[2]) {
  if (!c || !ms) return FZ_ERR_ARG;
  DeviceGuard guard(c->device);
  for (int k = 0; k < 2; ++k) {
    ms[k] = 0.0;
    if (!c->call_used[k]) continue;
    float t = 0.f;
    if (cudaEventSynchronize(c->call_ev[2 * k + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, c->call_ev[2 * k], c->call_ev[2 * k + 1]) != cudaSuccess)
      return FZ_ERR_CUDA;
    ms[k] = t;
  }
  return FZ_OK;
}

int fz_debug_skip_publish(fz_ctx *c, uint64_t chunk) {
  if (!c) return FZ_ERR_ARG;
  c->skip_publish = chunk;
  return FZ_OK;
}

// fz_compress and fz_compress_ranged: rng = NULL takes a relative bound's
// range from a range pass over d_in, else rng[0..1] is the range
static int compress_impl(fz_ctx *c, const float *d_in, const uint64_t dims[3], int ndim,
                         int mode, double eb, const float *rng, void *d_out, uint64_t cap,
                         uint64_t *out_size, void *stream, bool whole = false,
                         bool force_wide = false) {
  if (out_size) *out_size = 0;
  Shape sh;
  if (!c || !d_in || !d_out || !out_size || !make_shape(dims, ndim, &sh)) return FZ_ERR_ARG;
  if (mode != FZ_EB_ABS && mode != FZ_EB_REL) return FZ_ERR_ARG;
  if (!(eb > 0.0) || !std::isfinite(eb)) return FZ_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(d_out) & 15u) || (reinterpret_cast<uintptr_t>(d_in) & 3u))
    return FZ_ERR_ARG;
  const uint64_t min_bytes = 64 + 32 * sh.n_tiles;
  if (cap < min_bytes) {
    *out_size = min_bytes;
    return FZ_ERR_CAPACITY;
  }
  DeviceGuard guard(c->device);
  if (!guard.ok) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool timed = c->call_timing;
  if (timed) cudaEventRecord(c->call_ev[0], s);
  int st = ensure_cap(c, sh.n_tiles);             // at least one look-back word per unit
  if (st) return st;
  if ((st = prepare_set(c, s))) return st;
  prof_reset(c);
  if (mode == FZ_EB_REL && !rng) {
    prof_begin(c, 0, s);
    if ((st = range_pass(c, d_in, sh.n_elems, s))) return st;
    prof_end(c, 0, s);
  }

  const int A = c->cur;
  fz::CompressArgs a{};
  a.x = d_in;
  for (int i = 0; i < 3; ++i) a.dims[i] = sh.d[i];
  a.pitch = sh.d[0];
  a.ncx = (uint32_t)sh.ncx;
  a.ncy = (uint32_t)sh.ncy;
  a.n_chunks = sh.n_chunks;
  a.mode = mode;
  a.eb_req = eb;
  a.range = c->range;
  a.range_given = rng != nullptr;
  a.range_lo = rng ? rng[0] : 0.f;
  a.range_hi = rng ? rng[1] : 0.f;
  a.set_cur = c->sets + A;
  a.set_next = c->sets + (1 - A);
  a.status_cur = c->status + A * c->cap * fz::kStatusStride;
  a.status_next = c->status + (1 - A) * c->cap * fz::kStatusStride;
  a.tile_out_prefix = c->out_prefix;
  a.tile_out_count = c->out_count;
  a.out = static_cast<uint8_t *>(d_out);
  a.out_capacity = cap;
  a.wait_limit_ns = c->wait_limit_ns;
  a.skip_publish_chunk = c->skip_publish;
  a.whole = whole;
  a.allow_wide = 1;
  a.wide = force_wide;
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  const bool tma = !force_wide && fz::compress_uses_tma(sh.ndim, a) &&
                   fz::encode_field_tmap(sh.ndim, sh.d, d_in, &tm);
  prof_begin(c, 1, s);
  if (fz::launch_compress(sh.ndim, a, tma ? &tm : nullptr, c->num_sms, s,
                          mode == FZ_EB_REL && !rng && !force_wide) != cudaSuccess) {
    mark_all_dirty(c);
    return FZ_ERR_CUDA;
  }
  prof_end(c, 1, s);
  const uint64_t words = fz::compress_status_words(sh.n_tiles);
  retire_set(c, words, words);
  if ((st = read_set(c, A, s, timed ? c->call_ev[1] : nullptr))) {
    mark_all_dirty(c);
    return st;
  }
  c->call_used[0] = timed;
  const SetScratch r = *c->h_res;
  if (r.err & (fz::kErrNonFinite | fz::kErrEbParam | fz::kErrRange | fz::kErrTimeout |
               fz::kErrWide)) {
    // the kernel may have stopped before zeroing the next call's look-back
    // words: clear every set before the next launch
    mark_all_dirty(c);
  }
  if (r.err & fz::kErrNonFinite) return FZ_ERR_NONFINITE;
  if ((r.err & fz::kErrWide) && !force_wide)       // the range passes |q| = 2^22 - 1
    return compress_impl(c, d_in, dims, ndim, mode, eb, rng, d_out, cap, out_size, stream,
                         whole, true);
  if (r.err & (fz::kErrEbParam | fz::kErrRange)) {
    // elements checked one by one: NaN/Inf fail the same check.  A finite
    // field that passes |q| = 2^22 - 1 gets one more launch with the wide
    // quantiser, which checks |q| <= 2^28 - 1 against the range pass that
    // classify_range_error has just run (its result stays in c->range).
    if (mode == FZ_EB_ABS || rng) {
      const int cls = classify_range_error(c, d_in, sh.n_elems, s);
      if (cls == FZ_ERR_EB_RANGE && !force_wide && !(r.err & fz::kErrEbParam))
        return compress_impl(c, d_in, dims, ndim, mode, eb, rng, d_out, cap, out_size, stream,
                             whole, true);
      return cls;
    }
    return FZ_ERR_EB_RANGE;
  }
  if (r.err & fz::kErrTimeout) return FZ_ERR_TIMEOUT;
  const uint64_t total = min_bytes + 16 * r.nnz + 8 * r.nout;
  if ((r.err & fz::kErrCapacity) || total > cap) {
    *out_size = total;
    return FZ_ERR_CAPACITY;
  }
  if (r.nout > 0) {
    // rare path: write the escaped residuals behind the payload
    if ((st = prepare_set(c, s))) return st;
    a.set_cur = c->sets + c->cur;
    prof_begin(c, 2, s);
    if (fz::launch_outliers(sh.ndim, a, min_bytes + 16 * r.nnz, s) != cudaSuccess) {
      mark_all_dirty(c);
      return FZ_ERR_CUDA;
    }
    prof_end(c, 2, s);
    const int B = c->cur;
    c->hdr_dirty[B] = true;
    if ((st = read_set(c, B, s, timed ? c->call_ev[1] : nullptr))) return st;
    if (c->h_res->err & fz::kErrTimeout) return FZ_ERR_TIMEOUT;
    if (c->h_res->err & fz::kErrCapacity) {
      *out_size = total;
      return FZ_ERR_CAPACITY;
    }
  }
  *out_size = total;
  return FZ_OK;
}

int fz_compress(fz_ctx *c, const float *d_in, const uint64_t dims[3], int ndim, int mode,
                double eb, void *d_out, uint64_t cap, uint64_t *out_size, void *stream) {
  return compress_impl(c, d_in, dims, ndim, mode, eb, nullptr, d_out, cap, out_size, stream);
}

int fz_compress_whole(fz_ctx *c, const float *d_in, const uint64_t dims[3], int ndim, int mode,
                      double eb, void *d_out, uint64_t cap, uint64_t *out_size, void *stream) {
  return compress_impl(c, d_in, dims, ndim, mode, eb, nullptr, d_out, cap, out_size, stream,
                       true);
}

int fz_compress_ranged(fz_ctx *c, const float *d_in, const uint64_t dims[3], int ndim,
                       double eb, float range_min, float range_max, void *d_out, uint64_t cap,
                       uint64_t *out_size, void *stream) {
  if (out_size) *out_size = 0;
  if (!std::isfinite(range_min) || !std::isfinite(range_max) || range_min > range_max)
    return FZ_ERR_ARG;
  const float rng[2] = {range_min + 0.0f, range_max + 0.0f};   // +0 for a zero of either sign
  return compress_impl(c, d_in, dims, ndim, FZ_EB_REL, eb, rng, d_out, cap, out_size, stream);
}

int fz_range(fz_ctx *c, const float *d_in, uint64_t n, float *h_min, float *h_max,
             int *h_nonfinite, void *stream) {
  if (!c || !d_in || !h_min || !h_max || !h_nonfinite || n == 0 ||
      (reinterpret_cast<uintptr_t>(d_in) & 3u))
    return FZ_ERR_ARG;
  DeviceGuard guard(c->device);
  if (!guard.ok) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (range_pass(c, d_in, n, s) != FZ_OK ||
      cudaMemcpyAsync(c->h_range, c->range, sizeof(RangeResult), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FZ_ERR_CUDA;
  *h_min = c->h_range->fmin;
  *h_max = c->h_range->fmax;
  *h_nonfinite = c->h_range->nonfinite ? 1 : 0;
  return FZ_OK;
}

// ---------------------------------------------------------------- pwrel
int fz_pwrel_bound(double eps, double *eb_abs) {
  if (!eb_abs || !(eps >= 1e-4 && eps <= 0.5)) return FZ_ERR_ARG;
  *eb_abs = std::log2(1.0 + eps) - std::ldexp(1.0, -14);
  return FZ_OK;
}

int fz_pwrel_forward(fz_ctx *c, const float *d_x, uint64_t n, float *d_y, uint32_t *d_signs,
                     void *stream) {
  if (!c || !d_x || !d_y || !d_signs || n == 0 || (reinterpret_cast<uintptr_t>(d_x) & 3u) ||
      (reinterpret_cast<uintptr_t>(d_y) & 3u) || (reinterpret_cast<uintptr_t>(d_signs) & 3u))
    return FZ_ERR_ARG;
  DeviceGuard guard(c->device);
  if (!guard.ok) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the range block's non-finite word serves as this call's flag
  uint32_t *flag = &c->range->nonfinite;
  if (cudaMemsetAsync(flag, 0, sizeof(uint32_t), s) != cudaSuccess ||
      fz::launch_pwrel_forward(d_x, n, d_y, d_signs, flag, s) != cudaSuccess ||
      cudaMemcpyAsync(c->h_range, c->range, sizeof(RangeResult), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FZ_ERR_CUDA;
  return c->h_range->nonfinite ? FZ_ERR_NONFINITE : FZ_OK;
}

int fz_pwrel_inverse(fz_ctx *c, const float *d_y, uint64_t n, const uint32_t *d_signs,
                     float *d_x, void *stream) {
  if (!c || !d_y || !d_x || !d_signs || n == 0 || (reinterpret_cast<uintptr_t>(d_x) & 3u) ||
      (reinterpret_cast<uintptr_t>(d_y) & 3u) || (reinterpret_cast<uintptr_t>(d_signs) & 3u))
    return FZ_ERR_ARG;
  DeviceGuard guard(c->device);
  if (!guard.ok) return FZ_ERR_CUDA;
  return fz::launch_pwrel_inverse(d_y, n, d_signs, d_x, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? FZ_OK
             : FZ_ERR_CUDA;
}

// scratch of the unfused path for n_tiles tiles: codes, shuffled words,
// counts, prefixes and the scan's status words
static int ensure_staged(fz_ctx *c, uint64_t n_tiles, fz::StagedScratch *w) {
  const uint64_t units = fz::staged_status_words(n_tiles);
  auto layout = [&](uint64_t tiles, uint8_t *base, fz::StagedScratch *o) {
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
      const uint64_t at = off;
      off = (off + bytes + 255) / 256 * 256;
      return base + at;
    };
    o->codes = reinterpret_cast<uint32_t *>(take(tiles * 4096));
    o->shuf = reinterpret_cast<uint32_t *>(take(tiles * 4096));
    o->tile_nnz = reinterpret_cast<uint32_t *>(take(tiles * 4));
    o->tile_excl = reinterpret_cast<uint64_t *>(take(tiles * 8));
    o->status = reinterpret_cast<uint64_t *>(take(fz::staged_status_words(tiles) *
                                                  fz::kStatusStride * 8));
    return off;
  };
  if (n_tiles > c->staged_tiles || !c->staged) {
    cudaFree(c->staged);
    c->staged = nullptr;
    c->staged_tiles = 0;
    fz::StagedScratch tmp;
    const uint64_t bytes = layout(n_tiles, nullptr, &tmp);
    if (cudaMalloc(&c->staged, bytes) != cudaSuccess) return FZ_ERR_CUDA;
    c->staged_tiles = n_tiles;
    for (cudaEvent_t &e : c->staged_ev)
      if (!e && cudaEventCreate(&e) != cudaSuccess) return FZ_ERR_CUDA;
  }
  layout(c->staged_tiles, static_cast<uint8_t *>(c->staged), w);
  (void)units;
  return FZ_OK;
}

int fz_compress_staged(fz_ctx *c, const float *d_in, const uint64_t dims[3], int ndim, int mode,
                       double eb, void *d_out, uint64_t cap, uint64_t *out_size, double ms[5],
                       void *stream) {
  if (out_size) *out_size = 0;
  Shape sh;
  if (!c || !d_in || !d_out || !out_size || !make_shape(dims, ndim, &sh)) return FZ_ERR_ARG;
  if (mode != FZ_EB_ABS && mode != FZ_EB_REL) return FZ_ERR_ARG;
  if (!(eb > 0.0) || !std::isfinite(eb)) return FZ_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(d_out) & 15u) || (reinterpret_cast<uintptr_t>(d_in) & 3u))
    return FZ_ERR_ARG;
  const uint64_t min_bytes = 64 + 32 * sh.n_tiles;
  if (cap < min_bytes) {
    *out_size = min_bytes;
    return FZ_ERR_CAPACITY;
  }
  DeviceGuard guard(c->device);
  if (!guard.ok) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fz::StagedScratch w;
  int st = ensure_cap(c, sh.n_tiles);
  if (st || (st = ensure_staged(c, sh.n_tiles, &w)) || (st = prepare_set(c, s))) return st;
  if (cudaMemsetAsync(w.status, 0,
                      fz::staged_status_words(sh.n_tiles) * fz::kStatusStride * 8, s) !=
      cudaSuccess)
    return FZ_ERR_CUDA;
  cudaEvent_t *ev = ms ? c->staged_ev : nullptr;
  if (ev) cudaEventRecord(ev[5], s);
  if (mode == FZ_EB_REL && (st = range_pass(c, d_in, sh.n_elems, s))) return st;
  const int A = c->cur;
  fz::CompressArgs a{};
  a.x = d_in;
  for (int i = 0; i < 3; ++i) a.dims[i] = sh.d[i];
  a.pitch = sh.d[0];
  a.ncx = (uint32_t)sh.ncx;
  a.ncy = (uint32_t)sh.ncy;
  a.n_chunks = sh.n_chunks;
  a.mode = mode;
  a.eb_req = eb;
  a.range = c->range;
  a.set_cur = c->sets + A;
  a.tile_out_prefix = c->out_prefix;
  a.tile_out_count = c->out_count;
  a.out = static_cast<uint8_t *>(d_out);
  a.out_capacity = cap;
  a.wait_limit_ns = c->wait_limit_ns;
  a.skip_publish_chunk = ~0ull;
  if (fz::launch_staged(sh.ndim, a, w, c->num_sms, c->staged_shuffle == FZ_SHUFFLE_BALLOT, ev,
                        s) != cudaSuccess) {
    mark_all_dirty(c);
    return FZ_ERR_CUDA;
  }
  c->hdr_dirty[A] = true;                         // this set's block is used; cleared next call
  if ((st = read_set(c, A, s))) return st;
  SetScratch r = *c->h_res;
  if (ms) {
    float t[5] = {0, 0, 0, 0, 0};
    cudaEventElapsedTime(&t[0], ev[5], ev[0]);
    for (int k = 0; k < 4; ++k) cudaEventElapsedTime(&t[k + 1], ev[k], ev[k + 1]);
    for (int k = 0; k < 5; ++k) ms[k] = t[k];
  }
  if (r.err & fz::kErrNonFinite) return FZ_ERR_NONFINITE;
  if (r.err & (fz::kErrEbParam | fz::kErrRange)) {
    if (mode == FZ_EB_ABS) return classify_range_error(c, d_in, sh.n_elems, s);
    return FZ_ERR_EB_RANGE;
  }
  if (r.err & fz::kErrTimeout) return FZ_ERR_TIMEOUT;
  const uint64_t total = min_bytes + 16 * r.nnz + 8 * r.nout;
  if ((r.err & fz::kErrCapacity) || total > cap) {
    *out_size = total;
    return FZ_ERR_CAPACITY;
  }
  if (r.nout > 0) {
    if (fz::launch_outliers(sh.ndim, a, min_bytes + 16 * r.nnz, s) != cudaSuccess) {
      mark_all_dirty(c);
      return FZ_ERR_CUDA;
    }
    if ((st = read_set(c, A, s))) return st;
    if (c->h_res->err & fz::kErrCapacity) {
      *out_size = total;
      return FZ_ERR_CAPACITY;
    }
  }
  *out_size = total;
  return FZ_OK;
}

int fz_concat_streams(fz_ctx *c, const void *const *d_parts, const uint64_t *part_sizes,
                      int n_parts, void *d_out, uint64_t cap, uint64_t *out_size, void *stream) {
  if (out_size) *out_size = 0;
  if (!c || !d_parts || !part_sizes || !d_out || !out_size || n_parts < 1) return FZ_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_out) & 15u) return FZ_ERR_ARG;
  for (int i = 0; i < n_parts; ++i)
    if (!d_parts[i] || (reinterpret_cast<uintptr_t>(d_parts[i]) & 7u)) return FZ_ERR_ARG;
  DeviceGuard guard(c->device);
  if (!guard.ok) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t(*hdrs)[64] = new (std::nothrow) uint8_t[n_parts][64];
  fz::ConcatPart *parts = new (std::nothrow) fz::ConcatPart[n_parts];
  int st = (hdrs && parts) ? FZ_OK : FZ_ERR_CUDA;
  // the parts' headers, after whatever wrote them on the stream
  for (int i = 0; st == FZ_OK && i < n_parts; ++i) {
    std::memset(hdrs[i], 0, 64);
    const uint64_t nb = part_sizes[i] < 64 ? part_sizes[i] : 64;
    if (nb && cudaMemcpyAsync(hdrs[i], d_parts[i], nb, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = FZ_ERR_CUDA;
  }
  if (st == FZ_OK && cudaStreamSynchronize(s) != cudaSuccess) st = FZ_ERR_CUDA;
  fz::ConcatPlan plan;
  if (st == FZ_OK) st = fz::concat_plan(hdrs, part_sizes, n_parts, parts, &plan);
  if (st == FZ_OK && plan.total > cap) {
    *out_size = plan.total;
    st = FZ_ERR_CAPACITY;
  }
  if (st == FZ_OK) {
    uint8_t *o = static_cast<uint8_t *>(d_out);
    const uint64_t pay = 64 + 32 * plan.n_tiles, outs = pay + 16 * plan.nnz;
    bool ok = cudaMemcpyAsync(o, plan.hdr, 64, cudaMemcpyHostToDevice, s) == cudaSuccess;
    for (int i = 0; ok && i < n_parts; ++i) {
      const uint8_t *p = static_cast<const uint8_t *>(d_parts[i]);
      const fz::ConcatPart &q = parts[i];
      const uint8_t *src_out = p + 64 + 32 * q.tiles + 16 * q.nnz;
      ok = cudaMemcpyAsync(o + 64 + 32 * q.tile_off, p + 64, 32 * q.tiles,
                           cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
           (q.nnz == 0 || cudaMemcpyAsync(o + pay + 16 * q.nnz_off, p + 64 + 32 * q.tiles,
                                          16 * q.nnz, cudaMemcpyDeviceToDevice,
                                          s) == cudaSuccess) &&
           fz::launch_rebase_outliers(src_out, o + outs + 8 * q.out_off, q.nout,
                                      (uint32_t)(q.tile_off * fz::kTileCodes), s) == cudaSuccess;
    }
    // the header copy reads plan.hdr (host memory) until the stream reaches it
    if (!ok || cudaStreamSynchronize(s) != cudaSuccess) st = FZ_ERR_CUDA;
    else *out_size = plan.total;
  }
  delete[] hdrs;
  delete[] parts;
  return st;
}

// A version-2 stream (whole-field Lorenzo), after the offsets pass: phase 1
// (chunk-local prefix sums on the chunks' faces), the cross-chunk scans of
// the faces, phase 2 (the field).  Both phases count the matched outliers.
static int decompress_whole(fz_ctx *c, fz::DecompressArgs a, const SetScratch &r, int grid,
                            cudaStream_t s, bool timed) {
  // the chunk grid and dimensionality of the header the offsets pass checked
  const uint64_t nch = r.n_chunks;
  const int nd = (int)r.ndim;
  if (nd < 1 || nd > 3 || r.ncx == 0 || r.ncy == 0) return FZ_ERR_CORRUPT;
  const uint32_t nc[3] = {r.ncx, r.ncy, (uint32_t)(nch / ((uint64_t)r.ncx * r.ncy))};
  uint64_t words[3], total = 0;
  for (int k = 0; k < 3; ++k) {
    words[k] = nch * (uint64_t)fz::whole_face_elems(nd, k);
    total += 2 * words[k];
  }
  const uint64_t bytes = 4 * total;
  if (bytes > c->whole_bytes) {
    cudaFree(c->whole);
    c->whole = nullptr;
    c->whole_bytes = 0;
    if (cudaMalloc(&c->whole, bytes) != cudaSuccess) return FZ_ERR_CUDA;
    c->whole_bytes = bytes;
  }
  int32_t *p = static_cast<int32_t *>(c->whole);
  int32_t *face[3], *work[3];
  for (int k = 0; k < 3; ++k) {
    face[k] = p;
    p += words[k];
    work[k] = p;
    p += words[k];
  }
  int st = prepare_set(c, s);
  if (st) return st;
  const int B = c->cur;
  a.set_cur = c->sets + B;
  a.wide = r.wide ? 1 : 0;
  for (int k = 0; k < 3; ++k) a.face[k] = face[k];
  a.phase = 1;
  prof_begin(c, 3, s);
  if (fz::launch_decompress(a, grid, s) != cudaSuccess) {
    mark_all_dirty(c);
    return FZ_ERR_CUDA;
  }
  const int32_t *corr[3];
  if (fz::launch_whole_scans(nd, nc, face, work, corr, s) != cudaSuccess) {
    mark_all_dirty(c);
    return FZ_ERR_CUDA;
  }
  a.phase = 2;
  for (int k = 0; k < 3; ++k) a.corr[k] = corr[k];
  if (fz::launch_decompress(a, grid, s) != cudaSuccess) {
    mark_all_dirty(c);
    return FZ_ERR_CUDA;
  }
  prof_end(c, 3, s);
  c->hdr_dirty[B] = true;
  if ((st = read_set(c, B, s, timed ? c->call_ev[3] : nullptr))) {
    mark_all_dirty(c);
    return st;
  }
  const SetScratch q = *c->h_res;
  if (q.err & fz::kErrCorrupt) return FZ_ERR_CORRUPT;
  if (q.nout != 2ull * r.hdr_nout) return FZ_ERR_CORRUPT;
  return FZ_OK;
}

// A version-1 stream of the wide quantiser (header byte 7), after the
// offsets pass: the kernel that converts q as integers.
static int decompress_wide(fz_ctx *c, fz::DecompressArgs a, const SetScratch &r, int grid,
                           cudaStream_t s, bool timed) {
  int st = prepare_set(c, s);
  if (st) return st;
  const int B = c->cur;
  a.set_cur = c->sets + B;
  a.wide = 1;
  a.phase = 0;
  prof_begin(c, 3, s);
  if (fz::launch_decompress(a, grid, s) != cudaSuccess) {
    mark_all_dirty(c);
    return FZ_ERR_CUDA;
  }
  prof_end(c, 3, s);
  c->hdr_dirty[B] = true;
  if ((st = read_set(c, B, s, timed ? c->call_ev[3] : nullptr))) {
    mark_all_dirty(c);
    return st;
  }
  const SetScratch q = *c->h_res;
  if (q.err & fz::kErrCorrupt) return FZ_ERR_CORRUPT;
  if (q.nout != r.hdr_nout) return FZ_ERR_CORRUPT;
  return FZ_OK;
}

// The decompression call up to its first decoding launch: argument checks,
// scratch, and the offsets pass (every chunk's first payload block and first
// outlier record) on stream s.
static int decompress_begin(fz_ctx *c, const void *d_in, uint64_t in_size, float *d_out,
                            uint64_t cap_elems, cudaStream_t s, fz::DecompressArgs *out_a,
                            int *out_grid, int *out_set) {
  // every chunk carries 128 bytes of flags, which bounds the chunk count
  uint64_t bound = (in_size - 64) / 128;
  const uint64_t max_chunks = kMaxCodes / fz::kChunkCodes + 1;
  if (bound > max_chunks) bound = max_chunks;
  int st = ensure_cap(c, bound ? bound : 1);
  if (st) return st;
  if ((st = prepare_set(c, s))) return st;
  const int A = c->cur;
  fz::DecompressArgs a{};
  a.in = static_cast<const uint8_t *>(d_in);
  a.in_size = in_size;
  a.out = d_out;
  a.out_cap_elems = cap_elems;
  a.set_cur = c->sets + A;
  a.set_next = c->sets + (1 - A);
  a.status_cur = c->status + A * c->cap * fz::kStatusStride;
  a.status_next = c->status + (1 - A) * c->cap * fz::kStatusStride;
  a.status_cap = c->cap;
  a.chunk_off = c->out_prefix;
  a.chunk_olo = c->out_count;
  a.wait_limit_ns = c->wait_limit_ns;
  a.skip_publish_chunk = c->skip_publish;
  a.accept_whole = 1;
  a.chunk_lo = 0;
  a.chunk_hi = 0;                                  // every chunk
  prof_reset(c);
  prof_begin(c, 4, s);
  if (fz::launch_dec_offsets(a, bound, c->num_sms, s) != cudaSuccess) {
    mark_all_dirty(c);
    return FZ_ERR_CUDA;
  }
  prof_end(c, 4, s);
  *out_a = a;
  *out_grid = c->num_sms * c->dec_blocks_per_sm;
  *out_set = A;
  return FZ_OK;
}

// The rest of the call after its decoding launches: the result block, the
// set's bookkeeping, the error mapping, and the passes of version-2 and wide
// streams (which the version-1 kernel leaves alone).
static int decompress_end(fz_ctx *c, const fz::DecompressArgs &a, int grid, int A,
                          cudaStream_t s, bool timed) {
  int st;
  if ((st = read_set(c, A, s, timed ? c->call_ev[3] : nullptr))) {
    mark_all_dirty(c);
    return st;
  }
  c->call_used[1] = timed;
  const SetScratch r = *c->h_res;
  const uint64_t words = fz::decompress_status_words(r.n_chunks);
  retire_set(c, r.n_chunks ? words : c->cap, words);
  if (r.err & fz::kErrTimeout) mark_all_dirty(c);
  // a timed-out wait leaves later offsets unreliable, so it takes precedence
  if (r.err & fz::kErrTimeout) return FZ_ERR_TIMEOUT;
  if (r.err & fz::kErrCorrupt) return FZ_ERR_CORRUPT;
  if (r.err & fz::kErrCapacity) return FZ_ERR_CAPACITY;
  if (r.version == 2) return decompress_whole(c, a, r, grid, s, timed);
  if (r.wide) return decompress_wide(c, a, r, grid, s, timed);
  if (r.nout != r.hdr_nout) return FZ_ERR_CORRUPT;
  return FZ_OK;
}

int fz_decompress(fz_ctx *c, const void *d_in, uint64_t in_size, float *d_out,
                  uint64_t cap_elems, void *stream) {
  if (!c || !d_in || !d_out) return FZ_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) & 15u) || (reinterpret_cast<uintptr_t>(d_out) & 3u))
    return FZ_ERR_ARG;
  if (in_size < 64) return FZ_ERR_CORRUPT;
  DeviceGuard guard(c->device);
  if (!guard.ok) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool timed = c->call_timing;
  if (timed) cudaEventRecord(c->call_ev[2], s);
  fz::DecompressArgs a;
  int grid, A;
  int st = decompress_begin(c, d_in, in_size, d_out, cap_elems, s, &a, &grid, &A);
  if (st) return st;
  prof_begin(c, 3, s);
  if (fz::launch_decompress(a, grid, s) != cudaSuccess) {
    mark_all_dirty(c);
    return FZ_ERR_CUDA;
  }
  prof_end(c, 3, s);
  return decompress_end(c, a, grid, A, s, timed);
}

// host-buffer decompressions of this many output bytes or more are pipelined
constexpr uint64_t kPipelineBytes = 64ull << 20;

static int grow(void **p, uint64_t *cap, uint64_t need) {
  if (need <= *cap && *p) return FZ_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, need ? need : 16) != cudaSuccess) return FZ_ERR_CUDA;
  *cap = need;
  return FZ_OK;
}

int fz_compress_host(fz_ctx *c, const float *h_in, const uint64_t dims[3], int ndim, int mode,
                     double eb, void *h_out, uint64_t cap, uint64_t *out_size, void *stream) {
  if (out_size) *out_size = 0;
  Shape sh;
  if (!c || !h_in || !h_out || !out_size || !make_shape(dims, ndim, &sh)) return FZ_ERR_ARG;
  DeviceGuard guard(c->device);
  if (!guard.ok) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st;
  if ((st = grow(&c->stage_in, &c->stage_in_cap, sh.n_elems * 4))) return st;
  uint64_t dcap = cap;
  const uint64_t bound = fz_compress_bound(dims, ndim);
  if (dcap > bound) dcap = bound;
  if ((st = grow(&c->stage_out, &c->stage_out_cap, dcap))) return st;
  if (cudaMemcpyAsync(c->stage_in, h_in, sh.n_elems * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return FZ_ERR_CUDA;
  uint64_t size = 0;
  st = fz_compress(c, static_cast<const float *>(c->stage_in), dims, ndim, mode, eb, c->stage_out,
                   dcap, &size, stream);
  *out_size = size;
  if (st) return st;
  if (cudaMemcpyAsync(h_out, c->stage_out, size, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

// Streams and events of the pipelined host-buffer decompression, made on
// first use.
static int ensure_pipe(fz_ctx *c) {
  if (c->pipe_in) return FZ_OK;
  if (cudaStreamCreateWithFlags(&c->pipe_in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->pipe_out, cudaStreamNonBlocking) != cudaSuccess)
    return FZ_ERR_CUDA;
  for (cudaEvent_t &e : c->pipe_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return FZ_ERR_CUDA;
  if (cudaHostAlloc(reinterpret_cast<void **>(&c->h_slab), 8 * sizeof(uint32_t),
                    cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->h_slab_dev), c->h_slab, 0) !=
          cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

// A version-1 stream decompressed from host memory into host memory in
// slabs of whole chunk planes (3-D), chunk rows (2-D) or chunks (1-D), whose
// outputs are contiguous.  Copies in run on one stream (header, flags and
// outlier records first, then the payload in kPieces pieces), the offsets
// pass and one decoding launch per slab on the call's stream, each slab's
// output copied out on a third stream as soon as it is decoded: the stream
// comes in while earlier slabs' fields go out (the link carries both
// directions at once), and the kernels hide behind the copies.
static int decompress_host_pipelined(fz_ctx *c, const uint8_t *h_in, uint64_t in_size,
                                     const fz_info &info, const Shape &sh, float *h_out,
                                     cudaStream_t s) {
  constexpr int kSlabs = 4, kPieces = 8;
  int st;
  if ((st = ensure_pipe(c))) return st;
  const uint64_t n = sh.n_elems;
  uint8_t *d_in = static_cast<uint8_t *>(c->stage_in);
  float *d_out = static_cast<float *>(c->stage_out);
  const uint64_t flags_end = 64 + 32 * sh.n_tiles;
  const uint64_t pay_end = flags_end + 16 * (uint64_t)info.nnz_blocks;
  // slabs: "lines" of chunks whose elements are contiguous
  const int nd = info.ndim;
  const uint64_t per_line = nd == 3 ? sh.ncx * sh.ncy : nd == 2 ? sh.ncx : 1;
  const uint64_t lines = sh.n_chunks / per_line;
  const uint64_t line_elems = nd == 3 ? 8 * sh.d[0] * sh.d[1] : nd == 2 ? 128 * sh.d[0] : 8192;
  const int K = (int)(lines < (uint64_t)kSlabs ? lines : kSlabs);
  uint64_t lo[kSlabs + 1];
  for (int k = 0; k <= K; ++k) lo[k] = lines * k / K * per_line;
  cudaEvent_t *ev = c->pipe_ev;   // 0 start, 1 header, 2..9 pieces, 10 offsets, 11.. slabs, 23 out
  cudaStream_t si = c->pipe_in, so = c->pipe_out;
  if (cudaEventRecord(ev[0], s) != cudaSuccess || cudaStreamWaitEvent(si, ev[0], 0) != cudaSuccess ||
      cudaStreamWaitEvent(so, ev[0], 0) != cudaSuccess)
    return FZ_ERR_CUDA;
  // header and flags, the outlier records, then the payload in pieces
  if (cudaMemcpyAsync(d_in, h_in, flags_end, cudaMemcpyHostToDevice, si) != cudaSuccess ||
      (in_size > pay_end && cudaMemcpyAsync(d_in + pay_end, h_in + pay_end, in_size - pay_end,
                                            cudaMemcpyHostToDevice, si) != cudaSuccess) ||
      cudaEventRecord(ev[1], si) != cudaSuccess)
    return FZ_ERR_CUDA;
  const uint64_t pay = pay_end - flags_end;
  const uint64_t piece = ((pay + kPieces - 1) / kPieces + 15) / 16 * 16;
  int pieces = 0;
  for (uint64_t off = 0; off < pay; off += piece, ++pieces) {
    const uint64_t nb = pay - off < piece ? pay - off : piece;
    if (cudaMemcpyAsync(d_in + flags_end + off, h_in + flags_end + off, nb,
                        cudaMemcpyHostToDevice, si) != cudaSuccess ||
        cudaEventRecord(ev[2 + pieces], si) != cudaSuccess)
      return FZ_ERR_CUDA;
  }
  // the offsets pass once the flags are in
  if (cudaStreamWaitEvent(s, ev[1], 0) != cudaSuccess) return FZ_ERR_CUDA;
  fz::DecompressArgs a;
  int grid, A;
  if ((st = decompress_begin(c, d_in, in_size, d_out, n, s, &a, &grid, &A))) return st;
  // each slab boundary's first payload block, read back through mapped memory
  fz::GatherIdx gi{};
  for (int k = 1; k < K; ++k) gi.idx[k - 1] = lo[k];
  if (K > 1 && (fz::launch_gather_u32(c->out_prefix, gi, K - 1, c->h_slab_dev, s) != cudaSuccess ||
                cudaEventRecord(ev[10], s) != cudaSuccess ||
                cudaEventSynchronize(ev[10]) != cudaSuccess)) {
    mark_all_dirty(c);
    return FZ_ERR_CUDA;
  }
  for (int k = 0; k < K; ++k) {
    // the payload up to the slab's end (offsets from a corrupt stream are
    // clamped; the offsets pass has flagged it)
    uint64_t end_blk = k + 1 < K ? c->h_slab[k] : info.nnz_blocks;
    if (end_blk > info.nnz_blocks) end_blk = info.nnz_blocks;
    const uint64_t need = 16 * end_blk;
    const int last = need == 0 ? -1 : (int)((need - 1) / piece);
    if (last >= 0 && cudaStreamWaitEvent(s, ev[2 + (last < pieces ? last : pieces - 1)], 0) !=
                         cudaSuccess)
      return FZ_ERR_CUDA;
    a.chunk_lo = lo[k];
    a.chunk_hi = lo[k + 1];
    const uint64_t slab_chunks = lo[k + 1] - lo[k];
    const uint64_t want = (slab_chunks + 3) / 4;                 // a warp per chunk
    const int g = (int)(want < (uint64_t)grid ? (want ? want : 1) : grid);
    if (fz::launch_decompress(a, g, s) != cudaSuccess || cudaEventRecord(ev[11 + k], s) != cudaSuccess ||
        cudaStreamWaitEvent(so, ev[11 + k], 0) != cudaSuccess) {
      mark_all_dirty(c);
      return FZ_ERR_CUDA;
    }
    const uint64_t e0 = lo[k] / per_line * line_elems;
    uint64_t e1 = lo[k + 1] / per_line * line_elems;
    if (e1 > n) e1 = n;
    if (e1 > e0 && cudaMemcpyAsync(h_out + e0, d_out + e0, 4 * (e1 - e0), cudaMemcpyDeviceToHost,
                                   so) != cudaSuccess)
      return FZ_ERR_CUDA;
  }
  if (cudaEventRecord(ev[23], so) != cudaSuccess || cudaStreamWaitEvent(s, ev[23], 0) != cudaSuccess)
    return FZ_ERR_CUDA;
  a.chunk_lo = 0;                                    // any further pass covers every chunk
  a.chunk_hi = 0;
  return decompress_end(c, a, grid, A, s, false);
}

int fz_decompress_host(fz_ctx *c, const void *h_in, uint64_t in_size, float *h_out,
                       uint64_t cap_elems, void *stream) {
  if (!c || !h_in || !h_out) return FZ_ERR_ARG;
  fz_info info;
  int st = fz_inspect(h_in, in_size, &info);
  if (st) return st;
  if (info.stream_bytes != in_size) return FZ_ERR_CORRUPT;
  const uint64_t n = info.dims[0] * info.dims[1] * info.dims[2];
  if (cap_elems < n) return FZ_ERR_CAPACITY;
  DeviceGuard guard(c->device);
  if (!guard.ok) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = grow(&c->stage_in, &c->stage_in_cap, in_size))) return st;
  if ((st = grow(&c->stage_out, &c->stage_out_cap, n * 4))) return st;
  Shape sh;
  if (info.version == 1 && !info.wide && make_shape(info.dims, info.ndim, &sh) &&
      n * 4 >= kPipelineBytes)
    return decompress_host_pipelined(c, static_cast<const uint8_t *>(h_in), in_size, info, sh,
                                     h_out, s);
  if (cudaMemcpyAsync(c->stage_in, h_in, in_size, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return FZ_ERR_CUDA;
  st = fz_decompress(c, c->stage_in, in_size, static_cast<float *>(c->stage_out), n, stream);
  if (st) return st;
  if (cudaMemcpyAsync(h_out, c->stage_out, n * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

int fz_inspect(const void *hdr, uint64_t n, fz_info *out) {
  if (!hdr || !out) return FZ_ERR_ARG;
  if (n < 64) return FZ_ERR_CORRUPT;
  const uint8_t *p = static_cast<const uint8_t *>(hdr);
  if (p[0] != 'F' || p[1] != 'Z' || p[2] != 'G' || p[3] != '1' || p[4] < 1 || p[4] > 2 ||
      p[7] > 1)
    return FZ_ERR_CORRUPT;
  const int ndim = p[5], mode = p[6];
  if (ndim < 1 || ndim > 3 || mode > 1) return FZ_ERR_CORRUPT;
  uint64_t dims[3] = {rd32(p + 8), rd32(p + 12), rd32(p + 16)};
  for (int i = ndim; i < 3; ++i)
    if (dims[i] != 1) return FZ_ERR_CORRUPT;
  Shape sh;
  if (!make_shape(dims, ndim, &sh)) return FZ_ERR_CORRUPT;
  if (rd32(p + 20) != sh.n_tiles) return FZ_ERR_CORRUPT;
  out->ndim = ndim;
  out->mode = mode;
  for (int i = 0; i < 3; ++i) out->dims[i] = dims[i];
  std::memcpy(&out->eb_requested, p + 24, 8);
  std::memcpy(&out->eb, p + 32, 4);
  std::memcpy(&out->ebx2, p + 36, 4);
  std::memcpy(&out->ebx2_r, p + 40, 4);
  out->nnz_blocks = rd32(p + 44);
  out->n_outliers = rd32(p + 48);
  std::memcpy(&out->range_min, p + 52, 4);
  std::memcpy(&out->range_max, p + 56, 4);
  out->n_tiles = sh.n_tiles;
  out->stream_bytes = 64 + 32 * sh.n_tiles + 16 * out->nnz_blocks + 8 * out->n_outliers;
  out->version = p[4];
  out->wide = p[7];
  return FZ_OK;
}

}  // extern "C"
