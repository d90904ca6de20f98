// fz_compress.cu -- GB300 compression: the range pass and the single-field
// launches of the compression kernels (whose device code is in
// fz_compress_impl.cuh).
//
//  range_kernel     value range + non-finite scan (relative bounds, Sec. 4.1)
//  compress_kernel  one field per launch (see fz_compress_impl.cuh)
//  outlier_kernel   the rare escape pass
//
// The paper splits this work into a quantisation kernel, a fused
// bitshuffle+mark kernel, a CUB scan and an encode kernel with the codes,
// shuffled words and byte flags passing through global memory; here one
// kernel does all of it and global memory sees only the input and the stream.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

#include "fz_compress_impl.cuh"
#include "fz_device.cuh"
#include "fz_kernels.h"

namespace fz {

// ====================================================================
// value range (min, max, non-finite) of a float field
// ====================================================================
__global__ void __launch_bounds__(256) range_kernel(const float *__restrict__ x,
                                                    uint64_t n, float2 *partial,
                                                    RangeResult *res) {
  grid_launch_dependents();              // the compressor may be scheduled now
  float lo = INFINITY, hi = -INFINITY;
  uint32_t bad = 0;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  // elements before the first 16-byte boundary (x is 4-byte aligned), then
  // 16-byte loads, then the tail
  const uint64_t head0 = ((16u - (reinterpret_cast<uintptr_t>(x) & 15u)) & 15u) / 4;
  const uint64_t head = head0 < n ? head0 : n;
  if (tid < head) {
    const float a = x[tid];
    bad |= (__float_as_uint(a) & 0x7F800000u) == 0x7F800000u;
    lo = fminf(lo, a);
    hi = fmaxf(hi, a);
  }
  uint64_t done = head;
  {
    const uint64_t n4 = (n - head) / 4;
    const float4 *x4 = reinterpret_cast<const float4 *>(x + head);
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
    done = head + n4 * 4;
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
// launchers
// ====================================================================
void launch_range(const float *x, uint64_t n, float2 *partial, int nblocks,
                  RangeResult *res, cudaStream_t s) {
  range_kernel<<<nblocks, 256, 0, s>>>(x, n, partial, res);
}

// loads: 32-byte rows when every brick row starts on a 32-byte boundary,
// 16-byte when on 16, else scalar
static int vec_width(const CompressArgs &a) {
  const uintptr_t p = reinterpret_cast<uintptr_t>(a.x);
  if (a.dims[0] % 8 == 0 && p % 32 == 0) return 8;
  if (a.dims[0] % 4 == 0 && p % 16 == 0) return 4;
  return 1;
}

template <int NDIM, int V, bool CHECK, bool TMA, bool WHOLE = false, bool WIDE = false>
static cudaError_t launch_c3(const CompressArgs &a, const CUtensorMap &tm, int sms, bool pdl,
                             cudaStream_t s) {
  auto k = compress_kernel<NDIM, V, CHECK, TMA, false, WHOLE, WIDE>;
  const int smem = TMA ? kCompSmemTma : kCompSmemLdg;
  static int per_sm = 0;                    // resident blocks per SM, once
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kCompThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = n > 0 ? n : 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sms * per_sm);
  cfg.blockDim = dim3(kCompThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, a, tm, BatchArgs{});
}

template <int NDIM, int V, bool CHECK>
static cudaError_t launch_c2(const CompressArgs &a, const CUtensorMap *tm, int sms, bool pdl,
                             cudaStream_t s) {
  if constexpr (NDIM >= 2 && V >= 4) {
    if (tm) return launch_c3<NDIM, V, CHECK, true>(a, *tm, sms, pdl, s);
  }
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  return launch_c3<NDIM, V, CHECK, false>(a, none, sms, pdl, s);
}

template <int NDIM, int V>
static cudaError_t launch_c1(const CompressArgs &a, const CUtensorMap *tm, int sms, bool pdl,
                             cudaStream_t s) {
  // every element is range-checked unless a range pass has bounded them all
  return (a.mode == 0 || a.range_given) ? launch_c2<NDIM, V, true>(a, tm, sms, pdl, s)
                                        : launch_c2<NDIM, V, false>(a, tm, sms, pdl, s);
}

template <int NDIM>
static cudaError_t launch_c0(const CompressArgs &a, const CUtensorMap *tm, int sms, bool pdl,
                             cudaStream_t s) {
  switch (vec_width(a)) {
    case 8: return launch_c1<NDIM, 8>(a, tm, sms, pdl, s);
    case 4: return launch_c1<NDIM, 4>(a, tm, sms, pdl, s);
    default: return launch_c1<NDIM, 1>(a, nullptr, sms, pdl, s);
  }
}

// The field's tensor map for the per-warp TMA boxes: 3-D box {32,32,2} (a
// tile's two planes), 2-D box {32,32} (one x half of a tile's 32 rows);
// 128-byte swizzle, zero fill outside the field.  cuTensorMapEncodeTiled comes from the driver
// through the runtime's entry-point query (no link-time libcuda).
bool encode_field_tmap(int ndim, const uint64_t dims[3], const float *x, CUtensorMap *tm) {
  return encode_field_tmap_pitch(ndim, dims, dims[0], x, tm);
}

static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                         cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return enc;
}

// Class k holds the rows R = 4 j + k (R = y + Y z).  Its rows start at
// x + 4 (R pitch) bytes, all at the same offset r_k = ((x / 4) + k pitch) mod
// 4 floats past a 16-byte boundary; the map starts at that boundary (r_k
// floats before row k, inside the field's allocation, which is at least
// 16-byte aligned), takes X + r_k floats per row and the class's rows 16
// pitch bytes apart, so that it covers exactly the class's rows and nothing
// past the field's last element.
bool encode_class_tmaps(int ndim, const uint64_t dims[3], uint64_t pitch, const float *x,
                        CUtensorMap tm[4]) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
  if (!enc || ndim < 2) return false;
  const uint64_t rows = ndim == 3 ? dims[1] * dims[2] : dims[1];
  const uintptr_t xa = reinterpret_cast<uintptr_t>(x);
  if (rows < 4 || (xa & 3u) || pitch < dims[0]) return false;
  for (int k = 0; k < 4; ++k) {
    const uintptr_t start = xa + 4 * (uintptr_t)k * pitch;
    const uint64_t rk = (start >> 2) & 3u;
    cuuint64_t gdim[2] = {dims[0] + rk, (rows - (uint64_t)k + 3) / 4};
    cuuint64_t gstr[1] = {16 * pitch};
    cuuint32_t box[2] = {(cuuint32_t)(ndim == 3 ? kClassRow3 : kClassRow2), 8};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&tm[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                           reinterpret_cast<void *>(start - 4 * rk), gdim, gstr, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  return true;
}

bool encode_field_tmap_pitch(int ndim, const uint64_t dims[3], uint64_t pitch, const float *x,
                             CUtensorMap *tm) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
  if (!enc || ndim < 2) return false;
  cuuint64_t gdim[3] = {dims[0], dims[1], dims[2]};
  cuuint64_t gstr[2] = {pitch * 4, pitch * dims[1] * 4};
  cuuint32_t estr[3] = {1, 1, 1};
  cuuint32_t box3[3] = {32, 32, 2}, box2[2] = {32, 32};
  const CUresult r =
      enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ndim == 3 ? 3 : 2, const_cast<float *>(x), gdim,
          gstr, ndim == 3 ? box3 : box2, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// FZ_LOAD_PATH=ldg in the environment (read once) selects the direct-load
// variant even where TMA applies; used to compare the two load paths.
bool compress_uses_tma(int ndim, const CompressArgs &a) {
  static const bool ldg_only = [] {
    const char *e = getenv("FZ_LOAD_PATH");
    return e && strcmp(e, "ldg") == 0;
  }();
  return !ldg_only && ndim >= 2 && vec_width(a) >= 4;
}

// The whole-field variant (stream version 2): TMA boxes for 2-D/3-D fields
// whose rows are 16-byte aligned (16-byte halo and face loads), scalar loads
// otherwise; a range-checked and an unchecked kernel of each.
template <int NDIM>
static cudaError_t launch_whole(const CompressArgs &a, const CUtensorMap *tm, int sms, bool pdl,
                                cudaStream_t s) {
  const bool check = a.mode == 0 || a.range_given;
  if constexpr (NDIM >= 2) {
    if (tm && vec_width(a) >= 4)
      return check ? launch_c3<NDIM, 4, true, true, true>(a, *tm, sms, pdl, s)
                   : launch_c3<NDIM, 4, false, true, true>(a, *tm, sms, pdl, s);
  }
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  return check ? launch_c3<NDIM, 1, true, false, true>(a, none, sms, pdl, s)
               : launch_c3<NDIM, 1, false, false, true>(a, none, sms, pdl, s);
}

// The wide quantiser's launch (|q| up to 2^28 - 1): the integer path for
// every tile, scalar loads; its range was checked before (no per-element
// check).
template <int NDIM>
static cudaError_t launch_wide(const CompressArgs &a, int sms, cudaStream_t s) {
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  return a.whole ? launch_c3<NDIM, 1, false, false, true, true>(a, none, sms, false, s)
                 : launch_c3<NDIM, 1, false, false, false, true>(a, none, sms, false, s);
}

cudaError_t launch_compress(int ndim, const CompressArgs &a, const CUtensorMap *tm, int sms,
                            cudaStream_t s, bool after_range) {
  if (a.wide) {
    if (ndim == 3) return launch_wide<3>(a, sms, s);
    if (ndim == 2) return launch_wide<2>(a, sms, s);
    return launch_wide<1>(a, sms, s);
  }
  if (a.whole) {
    if (ndim == 3) return launch_whole<3>(a, tm, sms, after_range, s);
    if (ndim == 2) return launch_whole<2>(a, tm, sms, after_range, s);
    return launch_whole<1>(a, nullptr, sms, after_range, s);
  }
  if (ndim == 3) return launch_c0<3>(a, tm, sms, after_range, s);
  if (ndim == 2) return launch_c0<2>(a, tm, sms, after_range, s);
  return launch_c0<1>(a, nullptr, sms, after_range, s);
}

template <int NDIM>
static cudaError_t launch_o(const CompressArgs &a, uint64_t out_section, cudaStream_t s) {
  const uint64_t n_tiles = a.n_chunks * kTilesPerChunk;
  const unsigned blocks = (unsigned)((n_tiles + kOutWarps - 1) / kOutWarps);
  if (a.wide) {
    if (a.whole) outlier_kernel<NDIM, 1, true, true><<<blocks, kOutWarps * 32, 0, s>>>(a, out_section);
    else outlier_kernel<NDIM, 1, false, true><<<blocks, kOutWarps * 32, 0, s>>>(a, out_section);
    return cudaGetLastError();
  }
  if (a.whole) {
    outlier_kernel<NDIM, 1, true><<<blocks, kOutWarps * 32, 0, s>>>(a, out_section);
    return cudaGetLastError();
  }
  switch (vec_width(a)) {
    case 8: outlier_kernel<NDIM, 8><<<blocks, kOutWarps * 32, 0, s>>>(a, out_section); break;
    case 4: outlier_kernel<NDIM, 4><<<blocks, kOutWarps * 32, 0, s>>>(a, out_section); break;
    default: outlier_kernel<NDIM, 1><<<blocks, kOutWarps * 32, 0, s>>>(a, out_section); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_outliers(int ndim, const CompressArgs &a, uint64_t out_section,
                            cudaStream_t s) {
  if (ndim == 3) return launch_o<3>(a, out_section, s);
  if (ndim == 2) return launch_o<2>(a, out_section, s);
  return launch_o<1>(a, out_section, s);
}

}  // namespace fz
