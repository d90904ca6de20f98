// fz_batch.cu -- many fields in one persistent launch per dimensionality.
//
// A batch is planned once (fz_batch_create): per-field argument blocks,
// tensor maps, the map from the launch's units to (field, unit of the field)
// and all scratch live on the device, and the whole call can be captured in
// a CUDA graph.  One run is:
//   memset of the batch's counters, status words and result blocks,
//   range_batch_kernel  value ranges of the relative-bound fields (Sec. 4.1),
//   prepare_kernel      each field's bound and quantiser check,
//   compress_kernel<NDIM, BATCH> per dimensionality present,
//   outlier_batch_kernel per dimensionality (tiles with escapes only),
//   copy of the per-field result blocks to pinned host memory.
// Every field keeps its own look-back domain and stream, so each stream is
// byte for byte the one fz_compress makes of that field alone.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fz.h"
#include "fz_compress_impl.cuh"
#include "fz_device.cuh"
#include "fz_kernels.h"

namespace fz {

// order-preserving u32 image of a non-NaN float
__device__ __forceinline__ uint32_t float_order(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float float_of_order(uint32_t o) {
  const uint32_t u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

// per relative-bound field: max of ~order(x) (the min), max of order(x),
// non-finite flag; all zero before the pass
struct RangeSlots {
  uint32_t inv_min, max, nonfinite, pad;
};

struct RangeSeg {
  const float *x;
  uint64_t n;          // elements in this segment
  uint32_t field;
  uint32_t pad;
};

constexpr int kRangeSegElems = 1 << 16;   // 256 KiB per segment

__global__ void __launch_bounds__(256) range_batch_kernel(const RangeSeg *segs, uint64_t n_segs,
                                                          RangeSlots *slots) {
  for (uint64_t sgi = blockIdx.x; sgi < n_segs; sgi += gridDim.x) {
    const RangeSeg sg = segs[sgi];
    float lo = INFINITY, hi = -INFINITY;
    uint32_t bad = 0;
    // elements before the first 16-byte boundary, then 16-byte loads
    const uint64_t head0 = ((16u - (reinterpret_cast<uintptr_t>(sg.x) & 15u)) & 15u) / 4;
    const uint64_t head = head0 < sg.n ? head0 : sg.n;
    if (threadIdx.x < head) {
      const float a = sg.x[threadIdx.x];
      bad |= (__float_as_uint(a) & 0x7F800000u) == 0x7F800000u;
      lo = fminf(lo, a);
      hi = fmaxf(hi, a);
    }
    uint64_t done = head;
    {
      const uint64_t n4 = (sg.n - head) / 4;
      const float4 *x4 = reinterpret_cast<const float4 *>(sg.x + head);
      for (uint64_t i = threadIdx.x; i < n4; i += blockDim.x) {
        const float4 v = __ldcs(&x4[i]);
        const float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          bad |= (__float_as_uint(a[k]) & 0x7F800000u) == 0x7F800000u;
          lo = fminf(lo, a[k]);
          hi = fmaxf(hi, a[k]);
        }
      }
      done = head + n4 * 4;
    }
    for (uint64_t i = done + threadIdx.x; i < sg.n; i += blockDim.x) {
      const float a = sg.x[i];
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
    if ((threadIdx.x & 31) == 0) {
      RangeSlots *s = slots + sg.field;
      if (bad) atomicOr(&s->nonfinite, 1u);
      if (lo <= hi) {                      // the warp saw finite values
        atomicMax(&s->inv_min, ~float_order(lo));
        atomicMax(&s->max, float_order(hi));
      }
    }
  }
}

// One thread per field: the relative bound's range from the slots, then the
// same derivation and quantiser check as a single field's launch.
__global__ void prepare_kernel(const CompressArgs *fields, RangeResult *ranges,
                               const RangeSlots *slots, FieldRt *rt, uint32_t n) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  const CompressArgs &a = fields[f];
  if (a.mode == 1) {
    const RangeSlots s = slots[f];
    RangeResult r;
    r.fmin = __fadd_rn(float_of_order(~s.inv_min), 0.0f);   // +0 for a zero of either sign
    r.fmax = __fadd_rn(float_of_order(s.max), 0.0f);
    r.nonfinite = s.nonfinite;
    r.counter = 0;
    ranges[f] = r;
  }
  uint32_t err = 0;
  rt[f] = derive_field(a, err);
  if (err) atomicOr(&a.set_cur->err, err);
}

// One tile's escaped residuals, written at the offsets the compression
// kernel recorded (the same work as outlier_kernel, for a batch's field).
template <int NDIM>
__device__ __forceinline__ void batch_tile_outliers(const CompressArgs &a, const FieldRt &rt,
                                                    uint64_t T, int g) {
  const uint64_t n_tiles = a.n_chunks * kTilesPerChunk;
  const uint64_t out_section = 64 + 32 * n_tiles + 16 * a.set_cur->nnz;
  int32_t v[64];
  residuals_global<NDIM, 1>(a, T, g, rt.p.ebx2_r, v);
  uint32_t cnt = 0;
#pragma unroll
  for (int e = 0; e < 64; ++e) cnt += (uint32_t)abs(v[e]) > 32767u;
  uint32_t inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (g >= o) inc += y;
  }
  uint64_t pos = (uint64_t)a.tile_out_prefix[T] + inc - cnt;
#pragma unroll
  for (int e = 0; e < 64; ++e) {
    if ((uint32_t)abs(v[e]) > 32767u) {
      const uint64_t at = out_section + 8 * pos;
      if (at + 8 <= a.out_capacity) {
        *reinterpret_cast<uint2 *>(a.out + at) =
            make_uint2((uint32_t)(T * kTileCodes + 64 * g + e), (uint32_t)v[e]);
      } else {
        atomicOr(&a.set_cur->err, kErrCapacity);
      }
      ++pos;
    }
  }
}

// Escapes of every field of a batch: a warp reads 32 tiles' outlier counts
// at once (the batch's counts are contiguous, fields in order) and works
// only on the tiles that recorded some.
__global__ void __launch_bounds__(128) outlier_batch_kernel(BatchArgs b, const uint64_t *tile_off,
                                                            uint32_t n_fields, uint64_t n_tiles,
                                                            const uint32_t *counts) {
  const int g = threadIdx.x & 31;
  const uint64_t n_warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t base = 32 * (blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5));
       base < n_tiles; base += 32 * n_warps) {
    const uint64_t gt = base + g;
    const uint32_t cnt = gt < n_tiles ? counts[gt] : 0u;
    uint32_t mask = __ballot_sync(0xffffffffu, cnt != 0);
    while (mask) {
      const uint64_t t = base + (__ffs(mask) - 1);
      mask &= mask - 1;
      // the field of batch tile t: the last offset <= t
      uint32_t lo = 0, hi = n_fields;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (tile_off[mid] <= t) lo = mid;
        else hi = mid;
      }
      const CompressArgs &a = b.fields[lo];
      const FieldRt rt = b.rt[lo];
      if (!rt.ok) continue;
      const uint64_t T = t - tile_off[lo];
      if (a.ndim == 3) batch_tile_outliers<3>(a, rt, T, g);
      else if (a.ndim == 2) batch_tile_outliers<2>(a, rt, T, g);
      else batch_tile_outliers<1>(a, rt, T, g);
    }
  }
}

}  // namespace fz

// ====================================================================
// host side: the plan
// ====================================================================
using fz::BatchArgs;
using fz::CompressArgs;
using fz::FieldRt;
using fz::RangeResult;
using fz::SetScratch;

namespace {

struct Cls {                       // the fields of one dimensionality
  int ndim = 0;
  bool check = false;              // some field needs the per-element check
  std::vector<uint32_t> fields;    // batch field indices
  uint64_t n_tiles = 0;
  uint64_t n_units = 0;
  uint64_t unit_off = 0;           // into the batch's unit map
  uint32_t *d_ticket = nullptr;    // into the batch's counters
};

bool shape_of(const uint64_t dims[3], int ndim, uint64_t *n_chunks, uint32_t *ncx,
              uint32_t *ncy, uint64_t d[3]) {
  const uint64_t cap = fz_stream_min_bytes(dims, ndim);
  if (cap == 0) return false;
  for (int i = 0; i < 3; ++i) d[i] = i < ndim ? dims[i] : 1;
  const uint64_t cx = ndim == 1 ? 8192 : (ndim == 2 ? 64 : 32);
  const uint64_t cy = ndim == 1 ? 1 : (ndim == 2 ? 128 : 32);
  const uint64_t cz = ndim == 3 ? 8 : 1;
  const uint64_t nx = (d[0] + cx - 1) / cx, ny = (d[1] + cy - 1) / cy, nz = (d[2] + cz - 1) / cz;
  *n_chunks = nx * ny * nz;
  *ncx = (uint32_t)nx;
  *ncy = (uint32_t)ny;
  return true;
}

}  // namespace

struct fz_batch {
  fz_ctx *ctx = nullptr;
  int device = 0;
  int num_sms = 1;
  uint32_t n = 0;
  std::vector<fz_field> host;
  std::vector<CompressArgs> args;
  std::vector<Cls> cls;
  // device memory: one allocation carved into the arrays below
  void *d_mem = nullptr;
  size_t d_bytes = 0;
  CompressArgs *d_args = nullptr;
  FieldRt *d_rt = nullptr;
  CUtensorMap *d_tmaps = nullptr;
  uint2 *d_unit_map = nullptr;
  SetScratch *d_sets = nullptr;        // n fields + the launch-level block
  SetScratch *d_batch_set = nullptr;
  RangeResult *d_ranges = nullptr;
  fz::RangeSlots *d_slots = nullptr;
  fz::RangeSeg *d_segs = nullptr;
  uint64_t n_segs = 0;
  uint64_t *d_status = nullptr;
  uint32_t *d_tile_out = nullptr;      // outlier prefixes, then counts (batch tile order)
  uint64_t *d_tile_off = nullptr;      // per field: first batch tile
  uint64_t total_tiles = 0;
  uint32_t *d_tickets = nullptr;
  // what a run clears: [d_sets, end of the zeroed region)
  void *d_zero = nullptr;
  size_t zero_bytes = 0;
  SetScratch *h_res = nullptr;      // pinned, n + 1
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  bool tma_on = true;               // the autotuned load path for TMA-eligible fields
  double tune_ms[2] = {0, 0};       // [tma off, tma on] when tuned
  uint64_t wait_limit_ns = 2000000000ull;
};

namespace {

// a0 carries only the launch-level error block and the wait limit.  CHECK:
// some field of the class needs the per-element quantiser check (absolute
// bounds, or a relative bound against a supplied range).
template <int NDIM, bool CHECK>
cudaError_t launch_batch_compress(const CompressArgs &a0, const BatchArgs &b, int sms,
                                  cudaStream_t s) {
  auto k = fz::compress_kernel<NDIM, 1, CHECK, NDIM >= 2, true>;
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  k<<<sms, fz::kCompThreads, fz::kCompSmemTma, s>>>(a0, none, b);
  return cudaGetLastError();
}

// the batch kernels' shared-memory limits, set once before any capture
cudaError_t batch_kernel_attrs() {
  static cudaError_t done = [] {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int sm = fz::kCompSmemTma;
    cudaError_t e = cudaFuncSetAttribute(fz::compress_kernel<3, 1, true, true, true>, at, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fz::compress_kernel<2, 1, true, true, true>, at, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fz::compress_kernel<1, 1, true, false, true>, at, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fz::compress_kernel<3, 1, false, true, true>, at, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fz::compress_kernel<2, 1, false, true, true>, at, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fz::compress_kernel<1, 1, false, false, true>, at, sm);
    return e;
  }();
  return done;
}

// everything one run puts on the stream
int enqueue_run(fz_batch *B, cudaStream_t s) {
  if (cudaMemsetAsync(B->d_zero, 0, B->zero_bytes, s) != cudaSuccess) return FZ_ERR_CUDA;
  if (B->n_segs) {
    const uint64_t want = B->n_segs;
    const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)B->num_sms * 8);
    fz::range_batch_kernel<<<blocks, 256, 0, s>>>(B->d_segs, B->n_segs, B->d_slots);
  }
  fz::prepare_kernel<<<(B->n + 127) / 128, 128, 0, s>>>(B->d_args, B->d_ranges, B->d_slots,
                                                        B->d_rt, B->n);
  if (cudaGetLastError() != cudaSuccess) return FZ_ERR_CUDA;
  for (const Cls &c : B->cls) {
    BatchArgs b{};
    b.fields = B->d_args;
    b.rt = B->d_rt;
    b.tmaps = B->d_tmaps;
    b.unit_map = B->d_unit_map + c.unit_off;
    b.n_units = c.n_units;
    b.ticket = c.d_ticket;
    CompressArgs a0{};
    a0.set_cur = B->d_batch_set;
    a0.wait_limit_ns = B->wait_limit_ns;
    cudaError_t e;
    if (c.check)
      e = c.ndim == 3   ? launch_batch_compress<3, true>(a0, b, B->num_sms, s)
          : c.ndim == 2 ? launch_batch_compress<2, true>(a0, b, B->num_sms, s)
                        : launch_batch_compress<1, true>(a0, b, B->num_sms, s);
    else
      e = c.ndim == 3   ? launch_batch_compress<3, false>(a0, b, B->num_sms, s)
          : c.ndim == 2 ? launch_batch_compress<2, false>(a0, b, B->num_sms, s)
                        : launch_batch_compress<1, false>(a0, b, B->num_sms, s);
    if (e != cudaSuccess) return FZ_ERR_CUDA;
  }
  {
    BatchArgs b{};
    b.fields = B->d_args;
    b.rt = B->d_rt;
    const uint64_t warps = (B->total_tiles + 31) / 32;
    const unsigned blocks =
        (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((warps + 3) / 4, B->num_sms * 8ull));
    fz::outlier_batch_kernel<<<blocks, 128, 0, s>>>(b, B->d_tile_off, B->n, B->total_tiles,
                                                     B->d_tile_out + B->total_tiles);
    if (cudaGetLastError() != cudaSuccess) return FZ_ERR_CUDA;
  }
  // the fields' result blocks and the launch-level one behind them
  if (cudaMemcpyAsync(B->h_res, B->d_sets, (B->n + 1) * sizeof(SetScratch),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

void drop_graph(fz_batch *B) {
  if (B->graph) cudaGraphExecDestroy(B->graph);
  B->graph = nullptr;
}

// the fields' tensor maps under the current load-path choice
int write_args(fz_batch *B) {
  std::vector<CUtensorMap> maps(B->n);
  for (uint32_t f = 0; f < B->n; ++f) {
    CompressArgs &a = B->args[f];
    std::memset(&maps[f], 0, sizeof(CUtensorMap));
    const fz_field &h = B->host[f];
    const bool eligible = h.ndim >= 2 && (h.dims[0] % 4) == 0 &&
                          (reinterpret_cast<uintptr_t>(h.d_in) & 15u) == 0;
    a.use_tma = 0;
    if (eligible && B->tma_on && fz::encode_field_tmap(h.ndim, a.dims, a.x, &maps[f]))
      a.use_tma = 1;
  }
  if (cudaMemcpy(B->d_args, B->args.data(), B->n * sizeof(CompressArgs),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(B->d_tmaps, maps.data(), B->n * sizeof(CUtensorMap), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// per-field statuses and sizes from the result blocks of the last run
int collect_results(fz_batch *B, uint64_t *out_sizes, int *statuses, cudaStream_t s) {
  const bool launch_timeout = (B->h_res[B->n].err & fz::kErrTimeout) != 0;
  int worst = FZ_OK;
  for (uint32_t f = 0; f < B->n; ++f) {
    const SetScratch r = B->h_res[f];
    const fz_field &h = B->host[f];
    const uint64_t tiles = B->args[f].n_chunks * fz::kTilesPerChunk;
    const uint64_t total = 64 + 32 * tiles + 16 * r.nnz + 8 * r.nout;
    int fs = FZ_OK;
    if (r.err & fz::kErrNonFinite) {
      fs = FZ_ERR_NONFINITE;
    } else if (r.err & (fz::kErrEbParam | fz::kErrRange)) {
      fs = FZ_ERR_EB_RANGE;
      if (h.mode == FZ_EB_ABS && !(r.err & fz::kErrEbParam)) {
        // an absolute bound checks elements one by one: NaN/Inf fail there too
        float lo, hi;
        int bad = 0;
        const uint64_t elems = B->args[f].dims[0] * B->args[f].dims[1] * B->args[f].dims[2];
        if (fz_range(B->ctx, h.d_in, elems, &lo, &hi, &bad, s) == FZ_OK && bad)
          fs = FZ_ERR_NONFINITE;
      }
    } else if ((r.err & fz::kErrTimeout) || launch_timeout) {
      fs = FZ_ERR_TIMEOUT;
    } else if ((r.err & fz::kErrCapacity) || total > h.out_capacity) {
      fs = FZ_ERR_CAPACITY;
    }
    statuses[f] = fs;
    out_sizes[f] = (fs == FZ_OK || fs == FZ_ERR_CAPACITY) ? total : 0;
    if (fs != FZ_OK && worst == FZ_OK) worst = fs;
  }
  return worst;
}

}  // namespace

extern "C" {

int fz_batch_create(fz_ctx *ctx, const fz_field *fields, int n, fz_batch **out) {
  if (!out) return FZ_ERR_ARG;
  *out = nullptr;
  if (!ctx || !fields || n < 1 || n > FZ_BATCH_MAX_FIELDS) return FZ_ERR_ARG;
  const int device = fz::context_device(ctx);
  if (device < 0) return FZ_ERR_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
    return FZ_ERR_CUDA;
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev};

  if (batch_kernel_attrs() != cudaSuccess) return FZ_ERR_CUDA;
  fz_batch *B = new (std::nothrow) fz_batch();
  if (!B) return FZ_ERR_CUDA;
  B->ctx = ctx;
  B->device = device;
  cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (B->num_sms < 1) B->num_sms = 1;
  B->n = (uint32_t)n;
  B->host.assign(fields, fields + n);
  B->args.resize(n);

  // per-field arguments, classes, units, range segments
  uint64_t total_tiles = 0;
  std::vector<uint64_t> tile_off(n), status_off(n);
  uint64_t total_status = 0;
  std::vector<fz::RangeSeg> segs;
  Cls by_ndim[4];
  for (int d = 1; d <= 3; ++d) by_ndim[d].ndim = d;
  for (int f = 0; f < n; ++f) {
    const fz_field &h = fields[f];
    CompressArgs &a = B->args[f];
    uint64_t nch = 0, d[3];
    uint32_t ncx = 0, ncy = 0;
    if (!h.d_in || !h.d_out || (h.mode != FZ_EB_ABS && h.mode != FZ_EB_REL) ||
        !(h.eb > 0.0) || !std::isfinite(h.eb) || (reinterpret_cast<uintptr_t>(h.d_out) & 15u) ||
        (reinterpret_cast<uintptr_t>(h.d_in) & 3u) ||
        !shape_of(h.dims, h.ndim, &nch, &ncx, &ncy, d)) {
      delete B;
      return FZ_ERR_ARG;
    }
    const uint64_t tiles = nch * fz::kTilesPerChunk;
    if (h.out_capacity < 64 + 32 * tiles) {
      delete B;
      return FZ_ERR_CAPACITY;
    }
    a.x = h.d_in;
    a.ndim = h.ndim;
    for (int i = 0; i < 3; ++i) a.dims[i] = d[i];
    a.ncx = ncx;
    a.ncy = ncy;
    a.n_chunks = nch;
    a.mode = h.mode;
    a.eb_req = h.eb;
    a.out = static_cast<uint8_t *>(h.d_out);
    a.out_capacity = h.out_capacity;
    a.wait_limit_ns = B->wait_limit_ns;
    a.skip_publish_chunk = ~0ull;
    tile_off[f] = total_tiles;
    total_tiles += tiles;
    const uint64_t units = (tiles + fz::kCompWarps - 1) / fz::kCompWarps;
    status_off[f] = total_status;
    total_status += units;
    Cls &c = by_ndim[h.ndim];
    c.fields.push_back((uint32_t)f);
    if (h.mode == FZ_EB_ABS) c.check = true;
    c.n_tiles += tiles;
    c.n_units += units;
    if (h.mode == FZ_EB_REL) {
      const uint64_t elems = d[0] * d[1] * d[2];
      for (uint64_t s0 = 0; s0 < elems; s0 += fz::kRangeSegElems)
        segs.push_back({h.d_in + s0, std::min<uint64_t>(fz::kRangeSegElems, elems - s0),
                        (uint32_t)f, 0});
    }
  }
  for (int d = 3; d >= 1; --d)
    if (!by_ndim[d].fields.empty()) B->cls.push_back(by_ndim[d]);
  uint64_t total_units = 0;
  for (Cls &c : B->cls) {
    c.unit_off = total_units;
    total_units += c.n_units;
  }
  std::vector<uint2> unit_map(total_units);
  for (const Cls &c : B->cls) {
    uint64_t u = c.unit_off;
    for (uint32_t f : c.fields) {
      const uint64_t units =
          (B->args[f].n_chunks * fz::kTilesPerChunk + fz::kCompWarps - 1) / fz::kCompWarps;
      for (uint64_t k = 0; k < units; ++k) unit_map[u++] = make_uint2(f, (uint32_t)k);
    }
  }
  B->n_segs = segs.size();

  // one device allocation; the zeroed region (results, slots, counters,
  // status words, outlier counts) is contiguous
  size_t off = 0;
  auto take = [&](size_t bytes, size_t al) {
    off = align_up(off, al);
    const size_t at = off;
    off += bytes;
    return at;
  };
  const size_t o_args = take(n * sizeof(CompressArgs), 64);
  const size_t o_rt = take(n * sizeof(FieldRt), 64);
  const size_t o_tmaps = take(n * sizeof(CUtensorMap), 128);
  const size_t o_map = take(std::max<uint64_t>(total_units, 1) * sizeof(uint2), 64);
  const size_t o_segs = take(std::max<uint64_t>(B->n_segs, 1) * sizeof(fz::RangeSeg), 64);
  const size_t o_ranges = take(n * sizeof(RangeResult), 64);
  const size_t o_toff = take(n * sizeof(uint64_t), 64);
  const size_t o_zero = align_up(off, 256);
  const size_t o_sets = take((n + 1) * sizeof(SetScratch), 256);
  const size_t o_slots = take(n * sizeof(fz::RangeSlots), 64);
  const size_t o_tick = take(8 * sizeof(uint32_t), 64);
  const size_t o_status = take(total_status * fz::kStatusStride * sizeof(uint64_t), 128);
  const size_t o_tout = take(2 * total_tiles * sizeof(uint32_t), 64);
  const size_t end = align_up(off, 256);
  B->d_bytes = end;
  if (cudaMalloc(&B->d_mem, end) != cudaSuccess ||
      cudaMallocHost(&B->h_res, (n + 1) * sizeof(SetScratch)) != cudaSuccess) {
    fz_batch_destroy(B);
    return FZ_ERR_CUDA;
  }
  uint8_t *m = static_cast<uint8_t *>(B->d_mem);
  B->d_args = reinterpret_cast<CompressArgs *>(m + o_args);
  B->d_rt = reinterpret_cast<FieldRt *>(m + o_rt);
  B->d_tmaps = reinterpret_cast<CUtensorMap *>(m + o_tmaps);
  B->d_unit_map = reinterpret_cast<uint2 *>(m + o_map);
  B->d_segs = reinterpret_cast<fz::RangeSeg *>(m + o_segs);
  B->d_ranges = reinterpret_cast<RangeResult *>(m + o_ranges);
  B->d_sets = reinterpret_cast<SetScratch *>(m + o_sets);
  B->d_batch_set = B->d_sets + n;
  B->d_slots = reinterpret_cast<fz::RangeSlots *>(m + o_slots);
  B->d_tickets = reinterpret_cast<uint32_t *>(m + o_tick);
  B->d_status = reinterpret_cast<uint64_t *>(m + o_status);
  B->d_tile_out = reinterpret_cast<uint32_t *>(m + o_tout);
  B->d_zero = m + o_zero;
  B->zero_bytes = end - o_zero;
  int ci = 0;
  for (Cls &c : B->cls) c.d_ticket = B->d_tickets + ci++;
  B->total_tiles = total_tiles;
  B->d_tile_off = reinterpret_cast<uint64_t *>(m + o_toff);
  if (cudaMemcpy(B->d_tile_off, tile_off.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    fz_batch_destroy(B);
    return FZ_ERR_CUDA;
  }
  for (int f = 0; f < n; ++f) {
    CompressArgs &a = B->args[f];
    a.range = B->d_ranges + f;
    a.set_cur = B->d_sets + f;
    a.set_next = nullptr;
    a.status_cur = B->d_status + status_off[f] * fz::kStatusStride;
    a.status_next = nullptr;
    a.tile_out_prefix = B->d_tile_out + tile_off[f];
    a.tile_out_count = B->d_tile_out + total_tiles + tile_off[f];
  }
  if (write_args(B) != FZ_OK ||
      (total_units &&
       cudaMemcpy(B->d_unit_map, unit_map.data(), total_units * sizeof(uint2),
                  cudaMemcpyHostToDevice) != cudaSuccess) ||
      (B->n_segs && cudaMemcpy(B->d_segs, segs.data(), B->n_segs * sizeof(fz::RangeSeg),
                               cudaMemcpyHostToDevice) != cudaSuccess)) {
    fz_batch_destroy(B);
    return FZ_ERR_CUDA;
  }
  *out = B;
  return FZ_OK;
}

void fz_batch_destroy(fz_batch *B) {
  if (!B) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(B->device);
  drop_graph(B);
  cudaFree(B->d_mem);
  if (B->h_res) cudaFreeHost(B->h_res);
  if (prev >= 0) cudaSetDevice(prev);
  delete B;
}

int fz_batch_set_graph(fz_batch *B, int on) {
  if (!B) return FZ_ERR_ARG;
  B->use_graph = on != 0;
  if (!B->use_graph) drop_graph(B);
  return FZ_OK;
}

int fz_batch_compress(fz_batch *B, uint64_t *out_sizes, int *statuses, void *stream) {
  if (!B || !out_sizes || !statuses) return FZ_ERR_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(B->device) != cudaSuccess)
    return FZ_ERR_CUDA;
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = FZ_OK;
  if (B->use_graph) {
    if (!B->graph) {
      drop_graph(B);
      // capture on a private stream, launch on the caller's
      cudaStream_t cs;
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return FZ_ERR_CUDA;
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return FZ_ERR_CUDA;
      }
      st = enqueue_run(B, cs);
      const cudaError_t ec = cudaStreamEndCapture(cs, &g);
      cudaStreamDestroy(cs);
      if (st != FZ_OK || ec != cudaSuccess ||
          cudaGraphInstantiate(&B->graph, g, 0) != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        B->graph = nullptr;
        return st != FZ_OK ? st : FZ_ERR_CUDA;
      }
      cudaGraphDestroy(g);
    }
    if (cudaGraphLaunch(B->graph, s) != cudaSuccess) return FZ_ERR_CUDA;
  } else {
    if ((st = enqueue_run(B, s)) != FZ_OK) return st;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return FZ_ERR_CUDA;
  return collect_results(B, out_sizes, statuses, s);
}

int fz_batch_autotune(fz_batch *B, int reps, void *stream) {
  if (!B || reps < 1) return FZ_ERR_ARG;
  std::vector<uint64_t> sizes(B->n);
  std::vector<int> sts(B->n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double best = 0.0;
  bool best_tma = B->tma_on;
  for (int choice = 0; choice < 2; ++choice) {
    B->tma_on = choice == 1;
    drop_graph(B);
    if (write_args(B) != FZ_OK) return FZ_ERR_CUDA;
    fz_batch_compress(B, sizes.data(), sts.data(), stream);       // warm-up (and graph)
    std::vector<double> t;
    for (int r = 0; r < reps; ++r) {
      const auto t0 = std::chrono::steady_clock::now();
      const int st = fz_batch_compress(B, sizes.data(), sts.data(), stream);
      const auto t1 = std::chrono::steady_clock::now();
      if (st == FZ_ERR_CUDA) return st;
      t.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
    }
    std::sort(t.begin(), t.end());
    B->tune_ms[choice] = t[t.size() / 2];
    if (choice == 0 || B->tune_ms[choice] < best) {
      best = B->tune_ms[choice];
      best_tma = B->tma_on;
    }
  }
  (void)s;
  B->tma_on = best_tma;
  drop_graph(B);
  return write_args(B);
}

int fz_batch_tuning(const fz_batch *B, int *tma_on, double ms[2]) {
  if (!B || !tma_on || !ms) return FZ_ERR_ARG;
  *tma_on = B->tma_on ? 1 : 0;
  ms[0] = B->tune_ms[0];
  ms[1] = B->tune_ms[1];
  return FZ_OK;
}

}  // extern "C"
