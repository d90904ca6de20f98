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
#include <utility>
#include <vector>

#include "fz.h"
#include "fz_compress_impl.cuh"
#include "fz_device.cuh"
#include "fz_batch_ws.h"
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


constexpr int kRangeSegElems = 1 << 16;   // 256 KiB per segment

__global__ void __launch_bounds__(256) range_batch_kernel(const RangeSeg *segs, uint64_t n_segs,
                                                          RangeSlots *slots) {
  grid_launch_dependents();              // the preparation may be scheduled now
  for (uint64_t sgi = blockIdx.x; sgi < n_segs; sgi += gridDim.x) {
    const RangeSeg sg = segs[sgi];
    if (!sg.range && !sg.dst) continue;              // the same in the whole block
    float lo = INFINITY, hi = -INFINITY;
    uint32_t bad = 0;
    // element l of the segment into the staging copy: row row0 + q, column
    // col0 + l - q X (col0 + l < 2^31: the host stages rows below 2^30 only)
    auto stage = [&](uint64_t l, float a) {
      if (sg.dst) {
        const uint32_t t = sg.col0 + (uint32_t)l;
        const uint32_t q = sg.X.div(t);
        sg.dst[(sg.row0 + q) * sg.pitch + (t - q * sg.X.d)] = a;
      }
    };
    // elements before the first 16-byte boundary, then 16-byte loads
    const uint64_t head0 = ((16u - (reinterpret_cast<uintptr_t>(sg.x) & 15u)) & 15u) / 4;
    const uint64_t head = head0 < sg.n ? head0 : sg.n;
    if (threadIdx.x < head) {
      const float a = sg.x[threadIdx.x];
      bad |= (__float_as_uint(a) & 0x7F800000u) == 0x7F800000u;
      lo = fminf(lo, a);
      hi = fmaxf(hi, a);
      stage(threadIdx.x, a);
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
          stage(head + 4 * i + k, a[k]);
        }
      }
      done = head + n4 * 4;
    }
    for (uint64_t i = done + threadIdx.x; i < sg.n; i += blockDim.x) {
      const float a = sg.x[i];
      bad |= (__float_as_uint(a) & 0x7F800000u) == 0x7F800000u;
      lo = fminf(lo, a);
      hi = fmaxf(hi, a);
      stage(i, a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && sg.range) {
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
  grid_dependency_wait();                // the first pass's ranges
  grid_launch_dependents();              // the compression may be scheduled now
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
// The run's result blocks (the fields' and the launch-level one) into
// mapped pinned memory, once the escapes pass has finished.
__global__ void __launch_bounds__(128) copy_results_kernel(const SetScratch *src, SetScratch *dst,
                                                           uint64_t count) {
  grid_dependency_wait();
  const uint64_t words = count * (sizeof(SetScratch) / 4);
  const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
  uint32_t *d = reinterpret_cast<uint32_t *>(dst);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words;
       i += (uint64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}

__global__ void __launch_bounds__(128) outlier_batch_kernel(BatchArgs b, const uint64_t *tile_off,
                                                            uint32_t n_fields, uint64_t n_tiles,
                                                            const uint32_t *counts) {
  grid_dependency_wait();                // the compressions' per-tile counts
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
// host side: the workspace and the planned batch
// ====================================================================
namespace fz {

namespace {

bool shape_of(const uint64_t dims[3], int ndim, uint64_t *n_chunks, uint32_t *ncx,
              uint32_t *ncy, uint64_t d[3]) {
  if (fz_stream_min_bytes(dims, ndim) == 0) return false;
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

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// A launch that may begin while the kernel before it on the stream drains
// (programmatic dependent launch); each of the run's kernels waits for the
// previous one's results before it reads them.
template <class... P, class... A>
cudaError_t pdl_launch(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// a0 carries only the launch-level error block and the wait limit.  CHECK:
// some field of the class needs the per-element quantiser check (absolute
// bounds, or a relative bound against a supplied range).
template <int NDIM, bool CHECK>
cudaError_t launch_batch_compress(const CompressArgs &a0, const BatchArgs &b, int sms,
                                  cudaStream_t s) {
  auto k = compress_kernel<NDIM, 1, CHECK, NDIM >= 2, true>;
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  return pdl_launch(k, dim3(sms), dim3(kCompThreads), kCompSmemBatch, s, a0, none, b);
}

bool tma_eligible(const fz_field &h) {
  return h.ndim >= 2 && (h.dims[0] % 4) == 0 && (reinterpret_cast<uintptr_t>(h.d_in) & 15u) == 0;
}

}  // namespace

cudaError_t batch_kernel_attrs() {
  static cudaError_t done = [] {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int sm = kCompSmemBatch;
    cudaError_t e = cudaFuncSetAttribute(compress_kernel<3, 1, true, true, true>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(compress_kernel<2, 1, true, true, true>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(compress_kernel<1, 1, true, false, true>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(compress_kernel<3, 1, false, true, true>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(compress_kernel<2, 1, false, true, true>, at, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(compress_kernel<1, 1, false, false, true>, at, sm);
    return e;
  }();
  return done;
}

void BatchWs::release() {
  if (d_mem_) cudaFree(d_mem_);
  if (d_stage_) cudaFree(d_stage_);
  d_stage_ = nullptr;
  stage_mem_ = 0;
  if (h_stage_) cudaFreeHost(h_stage_);
  if (h_res_) cudaFreeHost(h_res_);
  d_mem_ = nullptr;
  h_stage_ = nullptr;
  h_res_ = nullptr;
  d_cap_ = stage_cap_ = 0;
  res_cap_ = 0;
  n_ = 0;
}

int BatchWs::set(int device, const fz_field *fields, int n, cudaStream_t s) {
  if (!fields || n < 1 || n > FZ_BATCH_MAX_FIELDS) return FZ_ERR_ARG;
  if (batch_kernel_attrs() != cudaSuccess) return FZ_ERR_CUDA;
  device_ = device;
  cudaDeviceGetAttribute(&num_sms_, cudaDevAttrMultiProcessorCount, device);
  if (num_sms_ < 1) num_sms_ = 1;
  std::vector<CompressArgs> args(n);
  std::vector<uint64_t> tile_off(n), status_off(n), stage_off(n, ~0ull);
  std::vector<RangeSeg> segs;
  uint64_t stage_floats = 0;
  WsClass by_ndim[4];
  for (int d = 1; d <= 3; ++d) by_ndim[d].ndim = d;
  uint64_t total_tiles = 0, total_status = 0;
  for (int f = 0; f < n; ++f) {
    const fz_field &h = fields[f];
    CompressArgs &a = args[f];
    a = CompressArgs{};
    uint64_t nch = 0, d[3];
    uint32_t ncx = 0, ncy = 0;
    if (!h.d_in || !h.d_out || (h.mode != FZ_EB_ABS && h.mode != FZ_EB_REL) ||
        !(h.eb > 0.0) || !std::isfinite(h.eb) || (reinterpret_cast<uintptr_t>(h.d_out) & 15u) ||
        (reinterpret_cast<uintptr_t>(h.d_in) & 3u) ||
        !shape_of(h.dims, h.ndim, &nch, &ncx, &ncy, d))
      return FZ_ERR_ARG;
    const uint64_t tiles = nch * kTilesPerChunk;
    if (h.out_capacity < 64 + 32 * tiles) return FZ_ERR_CAPACITY;
    a.x = h.d_in;
    a.ndim = h.ndim;
    for (int i = 0; i < 3; ++i) a.dims[i] = d[i];
    a.pitch = d[0];
    a.ncx = ncx;
    a.ncy = ncy;
    a.n_chunks = nch;
    a.mode = h.mode;
    a.eb_req = h.eb;
    a.out = static_cast<uint8_t *>(h.d_out);
    a.out_capacity = h.out_capacity;
    a.wait_limit_ns = wait_limit_ns;
    a.skip_publish_chunk = ~0ull;
    a.allow_wide = 0;                 // |q| up to 2^22 - 1 (no second launch)
    tile_off[f] = total_tiles;
    total_tiles += tiles;
    const uint64_t units = (tiles + kCompWarps - 1) / kCompWarps;
    status_off[f] = total_status;
    total_status += units;
    WsClass &c = by_ndim[h.ndim];
    c.fields.push_back((uint32_t)f);
    if (h.mode == FZ_EB_ABS) c.check = true;
    c.n_units += units;
    // rows not 16-byte aligned (below 2^30 elements): a staging copy with
    // the row pitch rounded up to 4 elements, 256-byte aligned
    const bool stageable = h.ndim >= 2 && !tma_eligible(h) && d[0] < (1ull << 30);
    const uint64_t pitch = (d[0] + 3) / 4 * 4;
    if (stageable) {
      stage_off[f] = stage_floats;
      stage_floats += (pitch * d[1] * d[2] + 63) / 64 * 64;
    }
    if (h.mode == FZ_EB_REL || stageable) {
      const uint64_t elems = d[0] * d[1] * d[2];
      for (uint64_t s0 = 0; s0 < elems; s0 += kRangeSegElems) {
        RangeSeg sg{};
        sg.x = h.d_in + s0;
        sg.n = std::min<uint64_t>(kRangeSegElems, elems - s0);
        sg.field = (uint32_t)f;
        sg.range = h.mode == FZ_EB_REL;
        sg.row0 = s0 / d[0];
        sg.col0 = (uint32_t)(s0 % d[0]);
        sg.pitch = (uint32_t)pitch;
        sg.X = FastDiv((uint32_t)std::min<uint64_t>(d[0], 0xFFFFFFFFull));
        segs.push_back(sg);
      }
    }
  }
  std::vector<WsClass> cls;
  for (int d = 3; d >= 1; --d)
    if (!by_ndim[d].fields.empty()) cls.push_back(by_ndim[d]);
  uint64_t total_units = 0;
  for (WsClass &c : cls) {
    c.unit_off = total_units;
    total_units += c.n_units;
  }

  // layout: uploaded descriptors, then device-written arrays, then the
  // region every run clears
  size_t off = 0;
  auto take = [&](size_t bytes, size_t al) {
    off = align_up(off, al);
    const size_t at = off;
    off += bytes;
    return at;
  };
  const size_t o_args = take(n * sizeof(CompressArgs), 64);
  const size_t o_tmaps = take(n * sizeof(CUtensorMap), 128);
  const size_t o_cmaps = take(4 * n * sizeof(CUtensorMap), 128);
  const size_t o_map = take(std::max<uint64_t>(total_units, 1) * sizeof(uint2), 64);
  const size_t o_segs = take(std::max<size_t>(segs.size(), 1) * sizeof(RangeSeg), 64);
  const size_t o_toff = take(n * sizeof(uint64_t), 64);
  const size_t desc = align_up(off, 256);
  const size_t o_rt = take(n * sizeof(FieldRt), 64);
  const size_t o_ranges = take(n * sizeof(RangeResult), 64);
  const size_t o_zero = align_up(off, 256);
  off = o_zero;
  const size_t o_sets = take((n + 1) * sizeof(SetScratch), 256);
  const size_t o_slots = take(n * sizeof(RangeSlots), 64);
  const size_t o_tick = take(8 * sizeof(uint32_t), 64);
  const size_t o_status = take(total_status * kStatusStride * sizeof(uint64_t), 128);
  const size_t o_tout = take(2 * total_tiles * sizeof(uint32_t), 64);
  const size_t end = align_up(off, 256);
  if (end > d_cap_) {
    if (d_mem_) cudaFree(d_mem_);
    d_mem_ = nullptr;
    d_cap_ = 0;
    const size_t want = end + end / 4;
    if (cudaMalloc(&d_mem_, want) != cudaSuccess) return FZ_ERR_CUDA;
    d_cap_ = want;
  }
  if (desc > stage_cap_) {
    if (h_stage_) cudaFreeHost(h_stage_);
    h_stage_ = nullptr;
    stage_cap_ = 0;
    const size_t want = desc + desc / 4;
    if (cudaMallocHost(&h_stage_, want) != cudaSuccess) return FZ_ERR_CUDA;
    stage_cap_ = want;
  }
  if ((uint32_t)n + 1 > res_cap_) {
    if (h_res_) cudaFreeHost(h_res_);
    h_res_ = nullptr;
    res_cap_ = 0;
    if (cudaHostAlloc(reinterpret_cast<void **>(&h_res_), (n + 1) * 2 * sizeof(SetScratch),
                      cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&h_res_dev_), h_res_, 0) !=
            cudaSuccess)
      return FZ_ERR_CUDA;
    res_cap_ = (uint32_t)(n + 1) * 2;
  }
  uint8_t *m = static_cast<uint8_t *>(d_mem_);
  d_args_ = reinterpret_cast<CompressArgs *>(m + o_args);
  d_tmaps_ = reinterpret_cast<CUtensorMap *>(m + o_tmaps);
  d_cmaps_ = reinterpret_cast<CUtensorMap *>(m + o_cmaps);
  d_unit_map_ = reinterpret_cast<uint2 *>(m + o_map);
  d_segs_ = reinterpret_cast<RangeSeg *>(m + o_segs);
  d_tile_off_ = reinterpret_cast<uint64_t *>(m + o_toff);
  d_rt_ = reinterpret_cast<FieldRt *>(m + o_rt);
  d_ranges_ = reinterpret_cast<RangeResult *>(m + o_ranges);
  d_sets_ = reinterpret_cast<SetScratch *>(m + o_sets);
  d_slots_ = reinterpret_cast<RangeSlots *>(m + o_slots);
  d_tickets_ = reinterpret_cast<uint32_t *>(m + o_tick);
  d_tile_out_ = reinterpret_cast<uint32_t *>(m + o_tout);
  desc_bytes_ = desc;
  zero_off_ = o_zero;
  zero_bytes_ = end - o_zero;
  uint64_t *d_status = reinterpret_cast<uint64_t *>(m + o_status);
  for (int f = 0; f < n; ++f) {
    CompressArgs &a = args[f];
    a.range = d_ranges_ + f;
    a.set_cur = d_sets_ + f;
    a.status_cur = d_status + status_off[f] * kStatusStride;
    a.tile_out_prefix = d_tile_out_ + tile_off[f];
    a.tile_out_count = d_tile_out_ + total_tiles + tile_off[f];
  }
  // the descriptor image in pinned memory (units in class order)
  uint8_t *hs = static_cast<uint8_t *>(h_stage_);
  uint2 *map = reinterpret_cast<uint2 *>(hs + o_map);
  for (const WsClass &c : cls) {
    uint64_t u = c.unit_off;
    for (uint32_t f : c.fields) {
      const uint64_t units = (args[f].n_chunks * kTilesPerChunk + kCompWarps - 1) / kCompWarps;
      for (uint64_t k = 0; k < units; ++k) map[u++] = make_uint2(f, (uint32_t)k);
    }
  }
  std::memcpy(hs + o_toff, tile_off.data(), n * sizeof(uint64_t));
  host_.assign(fields, fields + n);
  args_.swap(args);
  cls_.swap(cls);
  n_ = (uint32_t)n;
  total_tiles_ = total_tiles;
  total_units_ = total_units;
  n_segs_ = segs.size();
  segs_.swap(segs);
  stage_off_.swap(stage_off);
  stage_floats_ = stage_floats;
  o_segs_ = o_segs;
  return upload(s);
}

// tensor maps under the current load-path choice, then the whole
// descriptor image to the device
int BatchWs::upload(cudaStream_t s) {
  uint8_t *hs = static_cast<uint8_t *>(h_stage_);
  const size_t o_args = reinterpret_cast<uint8_t *>(d_args_) - static_cast<uint8_t *>(d_mem_);
  const size_t o_tmaps = reinterpret_cast<uint8_t *>(d_tmaps_) - static_cast<uint8_t *>(d_mem_);
  CUtensorMap *maps = reinterpret_cast<CUtensorMap *>(hs + o_tmaps);
  const size_t o_cmaps = reinterpret_cast<uint8_t *>(d_cmaps_) - static_cast<uint8_t *>(d_mem_);
  CUtensorMap *cmaps = reinterpret_cast<CUtensorMap *>(hs + o_cmaps);
  const bool staged = tma_mode_ == 1 && stage_on_ && stage_floats_ > 0;
  if (staged && stage_mem_ < stage_floats_ * 4) {
    if (d_stage_) cudaFree(d_stage_);
    d_stage_ = nullptr;
    stage_mem_ = 0;
    if (cudaMalloc(&d_stage_, stage_floats_ * 4) != cudaSuccess) return FZ_ERR_CUDA;
    stage_mem_ = stage_floats_ * 4;
  }
  for (uint32_t f = 0; f < n_; ++f) {
    CompressArgs &a = args_[f];
    std::memset(&maps[f], 0, sizeof(CUtensorMap));
    std::memset(&cmaps[4 * f], 0, 4 * sizeof(CUtensorMap));
    a.x = host_[f].d_in;
    a.pitch = a.dims[0];
    a.use_tma = 0;
    if (staged && stage_off_[f] != ~0ull) {
      a.x = d_stage_ + stage_off_[f];
      a.pitch = (a.dims[0] + 3) / 4 * 4;
      if (!encode_field_tmap_pitch(a.ndim, a.dims, a.pitch, a.x, &maps[f])) return FZ_ERR_CUDA;
      a.use_tma = 1;
    } else if (tma_mode_ >= 1 && tma_eligible(host_[f]) &&
               encode_field_tmap(a.ndim, a.dims, a.x, &maps[f])) {
      a.use_tma = 1;
    } else if (tma_mode_ == 2 && a.ndim >= 2 &&
               encode_class_tmaps(a.ndim, a.dims, a.pitch, a.x, &cmaps[4 * f])) {
      a.use_tma = 2;
    }
  }
  for (RangeSeg &sg : segs_)
    sg.dst = staged && stage_off_[sg.field] != ~0ull ? d_stage_ + stage_off_[sg.field] : nullptr;
  if (!segs_.empty()) std::memcpy(hs + o_segs_, segs_.data(), segs_.size() * sizeof(RangeSeg));
  std::memcpy(hs + o_args, args_.data(), n_ * sizeof(CompressArgs));
  if (cudaMemcpyAsync(d_mem_, h_stage_, desc_bytes_, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

int BatchWs::set_load_path(int tma, bool staged, cudaStream_t s) {
  tma_mode_ = tma;
  stage_on_ = staged;
  return n_ ? upload(s) : FZ_OK;
}

int BatchWs::enqueue(cudaStream_t s) {
  if (!n_) return FZ_ERR_ARG;
  uint8_t *m = static_cast<uint8_t *>(d_mem_);
  if (cudaMemsetAsync(m + zero_off_, 0, zero_bytes_, s) != cudaSuccess) return FZ_ERR_CUDA;
  if (n_segs_) {
    const unsigned blocks = (unsigned)std::min<uint64_t>(n_segs_, (uint64_t)num_sms_ * 8);
    range_batch_kernel<<<blocks, 256, 0, s>>>(d_segs_, n_segs_, d_slots_);
  }
  if (pdl_launch(prepare_kernel, dim3((n_ + 127) / 128), dim3(128), 0, s,
                 static_cast<const CompressArgs *>(d_args_), d_ranges_,
                 static_cast<const RangeSlots *>(d_slots_), d_rt_, n_) != cudaSuccess)
    return FZ_ERR_CUDA;
  int ci = 0;
  for (const WsClass &c : cls_) {
    BatchArgs b{};
    b.fields = d_args_;
    b.rt = d_rt_;
    b.tmaps = d_tmaps_;
    b.cmaps = d_cmaps_;
    b.unit_map = d_unit_map_ + c.unit_off;
    b.n_units = c.n_units;
    b.ticket = d_tickets_ + ci++;
    CompressArgs a0{};
    a0.set_cur = d_sets_ + n_;
    a0.wait_limit_ns = wait_limit_ns;
    cudaError_t e;
    if (c.check)
      e = c.ndim == 3   ? launch_batch_compress<3, true>(a0, b, num_sms_, s)
          : c.ndim == 2 ? launch_batch_compress<2, true>(a0, b, num_sms_, s)
                        : launch_batch_compress<1, true>(a0, b, num_sms_, s);
    else
      e = c.ndim == 3   ? launch_batch_compress<3, false>(a0, b, num_sms_, s)
          : c.ndim == 2 ? launch_batch_compress<2, false>(a0, b, num_sms_, s)
                        : launch_batch_compress<1, false>(a0, b, num_sms_, s);
    if (e != cudaSuccess) return FZ_ERR_CUDA;
  }
  {
    BatchArgs b{};
    b.fields = d_args_;
    b.rt = d_rt_;
    const uint64_t warps = (total_tiles_ + 31) / 32;
    const unsigned blocks =
        (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((warps + 3) / 4, num_sms_ * 8ull));
    if (pdl_launch(outlier_batch_kernel, dim3(blocks), dim3(128), 0, s, b,
                   static_cast<const uint64_t *>(d_tile_off_), n_, total_tiles_,
                   static_cast<const uint32_t *>(d_tile_out_ + total_tiles_)) != cudaSuccess)
      return FZ_ERR_CUDA;
  }
  // the fields' result blocks and the launch-level one behind them
  // the fields' result blocks and the launch-level one, written into the
  // mapped pinned copy by a kernel behind the escapes pass (a device-to-host
  // copy at the end of the run would add a few microseconds)
  if (pdl_launch(copy_results_kernel, dim3((unsigned)std::min<uint64_t>((n_ + 7) / 8, 1024)),
                 dim3(128), 0, s, static_cast<const SetScratch *>(d_sets_), h_res_dev_,
                 (uint64_t)n_ + 1) != cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

int BatchWs::collect(fz_ctx *ctx, uint64_t *out_sizes, int *statuses, cudaStream_t s) const {
  const bool launch_timeout = (h_res_[n_].err & kErrTimeout) != 0;
  int worst = FZ_OK;
  for (uint32_t f = 0; f < n_; ++f) {
    const SetScratch r = h_res_[f];
    const fz_field &h = host_[f];
    const uint64_t tiles = args_[f].n_chunks * kTilesPerChunk;
    const uint64_t total = 64 + 32 * tiles + 16 * r.nnz + 8 * r.nout;
    int fs = FZ_OK;
    if (r.err & kErrNonFinite) {
      fs = FZ_ERR_NONFINITE;
    } else if (r.err & (kErrEbParam | kErrRange)) {
      fs = FZ_ERR_EB_RANGE;
      if (h.mode == FZ_EB_ABS && !(r.err & kErrEbParam) && ctx) {
        // an absolute bound checks elements one by one: NaN/Inf fail there too
        float lo, hi;
        int bad = 0;
        const uint64_t elems = args_[f].dims[0] * args_[f].dims[1] * args_[f].dims[2];
        if (fz_range(ctx, h.d_in, elems, &lo, &hi, &bad, s) == FZ_OK && bad)
          fs = FZ_ERR_NONFINITE;
      }
    } else if ((r.err & kErrTimeout) || launch_timeout) {
      fs = FZ_ERR_TIMEOUT;
    } else if ((r.err & kErrCapacity) || total > h.out_capacity) {
      fs = FZ_ERR_CAPACITY;
    }
    statuses[f] = fs;
    out_sizes[f] = (fs == FZ_OK || fs == FZ_ERR_CAPACITY) ? total : 0;
    if (fs != FZ_OK && worst == FZ_OK) worst = fs;
  }
  return worst;
}

}  // namespace fz

struct fz_batch {
  fz_ctx *ctx = nullptr;
  int device = 0;
  fz::BatchWs ws;
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  // [direct, TMA where aligned, TMA + staging, TMA + row classes] when tuned
  double tune_ms[4] = {0, 0, 0, 0};
};

namespace {

void drop_graph(fz_batch *B) {
  if (B->graph) cudaGraphExecDestroy(B->graph);
  B->graph = nullptr;
}

struct DeviceScope {
  int prev = -1;
  bool ok = false;
  explicit DeviceScope(int dev) {
    ok = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

int fz_batch_create(fz_ctx *ctx, const fz_field *fields, int n, fz_batch **out) {
  if (!out) return FZ_ERR_ARG;
  *out = nullptr;
  if (!ctx || !fields || n < 1 || n > FZ_BATCH_MAX_FIELDS) return FZ_ERR_ARG;
  const int device = fz::context_device(ctx);
  if (device < 0) return FZ_ERR_ARG;
  DeviceScope scope(device);
  if (!scope.ok) return FZ_ERR_CUDA;
  fz_batch *B = new (std::nothrow) fz_batch();
  if (!B) return FZ_ERR_CUDA;
  B->ctx = ctx;
  B->device = device;
  B->ws.set_load_path(2, false, nullptr);           // flags only: no fields yet
  int st = B->ws.set(device, fields, n, nullptr);
  if (st == FZ_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) st = FZ_ERR_CUDA;
  if (st != FZ_OK) {
    delete B;
    return st;
  }
  *out = B;
  return FZ_OK;
}

void fz_batch_destroy(fz_batch *B) {
  if (!B) return;
  DeviceScope scope(B->device);
  drop_graph(B);
  B->ws.release();
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
  DeviceScope scope(B->device);
  if (!scope.ok) return FZ_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = FZ_OK;
  if (B->use_graph) {
    if (!B->graph) {
      // capture on a private stream, launch on the caller's
      cudaStream_t cs;
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return FZ_ERR_CUDA;
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return FZ_ERR_CUDA;
      }
      st = B->ws.enqueue(cs);
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
  } else if ((st = B->ws.enqueue(s)) != FZ_OK) {
    return st;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return FZ_ERR_CUDA;
  return B->ws.collect(B->ctx, out_sizes, statuses, s);
}

int fz_batch_autotune(fz_batch *B, int reps, void *stream) {
  if (!B || reps < 1) return FZ_ERR_ARG;
  DeviceScope scope(B->device);
  if (!scope.ok) return FZ_ERR_CUDA;
  const uint32_t n = B->ws.size();
  std::vector<uint64_t> sizes(n);
  std::vector<int> sts(n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the load paths: direct loads everywhere; TMA boxes for the fields with
  // 16-byte aligned rows; TMA boxes for every 2-D/3-D field, through
  // staging copies of the others; one box per tile for the aligned fields
  // and four row-class boxes for the others
  const int tma[4] = {0, 1, 1, 2};
  const bool staged[4] = {false, false, true, false};
  double best = 0.0;
  int best_c = 3;
  for (int c = 0; c < 4; ++c) {
    drop_graph(B);
    if (B->ws.set_load_path(tma[c], staged[c], s) != FZ_OK ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return FZ_ERR_CUDA;
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
    B->tune_ms[c] = t[t.size() / 2];
    if (c == 0 || B->tune_ms[c] < best) {
      best = B->tune_ms[c];
      best_c = c;
    }
  }
  drop_graph(B);
  if (B->ws.set_load_path(tma[best_c], staged[best_c], s) != FZ_OK ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

int fz_batch_set_load_path(fz_batch *B, int tma, int staged) {
  if (!B || tma < 0 || tma > 2 || (staged != 0 && staged != 1) || (staged && tma != 1))
    return FZ_ERR_ARG;
  DeviceScope scope(B->device);
  if (!scope.ok) return FZ_ERR_CUDA;
  drop_graph(B);
  if (B->ws.set_load_path(tma, staged == 1, nullptr) != FZ_OK ||
      cudaStreamSynchronize(nullptr) != cudaSuccess)
    return FZ_ERR_CUDA;
  return FZ_OK;
}

int fz_batch_tuning(const fz_batch *B, int *tma, int *staged, double ms[4]) {
  if (!B || !tma || !staged || !ms) return FZ_ERR_ARG;
  *tma = B->ws.tma_mode();
  *staged = B->ws.staged_on() ? 1 : 0;
  for (int c = 0; c < 4; ++c) ms[c] = B->tune_ms[c];
  return FZ_OK;
}

}  // extern "C"
