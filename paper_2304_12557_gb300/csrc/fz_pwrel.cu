// fz_pwrel.cu -- point-wise relative error bounds by log transform.
//
// The paper compresses its particle dataset (HACC, Sec. 4.1) with a
// point-wise relative bound |x' - x| <= eps |x| by taking logarithms first
// and compressing the log field with the absolute bound that eps implies.
// These kernels are the two ends of that path around the ordinary
// compressor:
//
//   pwrel_forward_kernel  y = log2|x| (zeros -> kPwZeroLog), sign bits by
//                         warp ballot (one 32-bit word per 32 elements),
//                         non-finite inputs flagged;
//   pwrel_inverse_kernel  x' = +-2^y' (y' below kPwZeroCut -> 0).
//
// log2 and exp2 are this file's own fp32 evaluations, every step an IEEE
// round-to-nearest operation in a fixed order, so that their results are
// reproducible bit for bit (the oracle evaluates the same formulas):
//   log2 a = e + ln(m) / ln 2 for a = m 2^e, m in [1, 2), with
//     ln m = 2 atanh(s) = 2 (s + s^3/3 + ... + s^13/13), s = (m-1)/(m+1)
//     (|s| < 1/3: the omitted terms are below 1e-8);
//   2^y = 2^k * exp(f ln 2) for k = floor(y), f = y - k in [0, 1), with
//     exp(u) = sum_{n <= 10} u^n / n! (u < 0.7: the rest is below 1e-9).
#include <cfloat>
#include <cstdint>

#include "fz_device.cuh"
#include "fz_pwrel.h"

namespace fz {

__device__ __forceinline__ float pw_log2(float a) {
  uint32_t b = __float_as_uint(a);
  int e = 0;
  if (b < 0x00800000u) {                 // subnormal: scale by 2^23 (exact)
    a = __fmul_rn(a, 8388608.0f);
    b = __float_as_uint(a);
    e = -23;
  }
  e += (int)(b >> 23) - 127;
  const float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
  const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float p = 0.07692308f;                 // 1/13
  p = __fadd_rn(__fmul_rn(p, s2), 0.09090909f);
  p = __fadd_rn(__fmul_rn(p, s2), 0.11111111f);
  p = __fadd_rn(__fmul_rn(p, s2), 0.14285715f);
  p = __fadd_rn(__fmul_rn(p, s2), 0.2f);
  p = __fadd_rn(__fmul_rn(p, s2), 0.33333334f);
  p = __fadd_rn(__fmul_rn(p, s2), 1.0f);
  const float ln_m = __fmul_rn(__fmul_rn(2.0f, s), p);
  return __fadd_rn((float)e, __fmul_rn(ln_m, 1.442695f));
}

__device__ __forceinline__ float pw_exp2(float y) {
  if (!(y < 128.0f)) return FLT_MAX;
  if (y < -150.0f) return 0.0f;
  const float k = floorf(y);
  const float u = __fmul_rn(__fsub_rn(y, k), 0.6931472f);
  float p = 2.755732e-07f;               // 1/10!
  p = __fadd_rn(__fmul_rn(p, u), 2.7557319e-06f);
  p = __fadd_rn(__fmul_rn(p, u), 2.4801588e-05f);
  p = __fadd_rn(__fmul_rn(p, u), 0.0001984127f);
  p = __fadd_rn(__fmul_rn(p, u), 0.0013888889f);
  p = __fadd_rn(__fmul_rn(p, u), 0.008333334f);
  p = __fadd_rn(__fmul_rn(p, u), 0.041666668f);
  p = __fadd_rn(__fmul_rn(p, u), 0.16666667f);
  p = __fadd_rn(__fmul_rn(p, u), 0.5f);
  p = __fadd_rn(__fmul_rn(p, u), 1.0f);
  p = __fadd_rn(__fmul_rn(p, u), 1.0f);
  const int ki = (int)k;                 // -150 .. 127
  if (ki >= -126) return __fmul_rn(p, __uint_as_float((uint32_t)(ki + 127) << 23));
  // subnormal results: two exact-or-rounded steps through 2^-126
  return __fmul_rn(__fmul_rn(p, __uint_as_float((uint32_t)(ki + 126 + 127) << 23)),
                   1.17549435e-38f);
}

// Each warp takes chunks of kPwU consecutive 32-element words (one word per
// load, kPwU independent evaluations in flight per thread); chunk c covers
// elements [32 kPwU c, 32 kPwU (c + 1)) and sign words [kPwU c, kPwU (c + 1)).
constexpr int kPwU = 4;

__global__ void pwrel_forward_kernel(const float *__restrict__ x, uint64_t n,
                                     float *__restrict__ y, uint32_t *__restrict__ signs,
                                     uint32_t *flag) {
  const unsigned full = 0xffffffffu;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  for (uint64_t ch = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       ch * 32 * kPwU < n; ch += warps) {
    const uint64_t base = ch * 32 * kPwU;
    float v[kPwU];
#pragma unroll
    for (int u = 0; u < kPwU; ++u) {
      const uint64_t i = base + 32 * u + lane;
      v[u] = i < n ? x[i] : 1.0f;
    }
    uint32_t word = 0;                       // lane u keeps sign word u
#pragma unroll
    for (int u = 0; u < kPwU; ++u) {
      const uint64_t i = base + 32 * u + lane;
      const uint32_t bits = __float_as_uint(v[u]);
      const bool finite = (bits & 0x7F800000u) != 0x7F800000u;
      bad |= !finite;
      const float a = fabsf(v[u]);
      const uint32_t neg = __ballot_sync(full, (bits >> 31) != 0u);
      if (lane == (uint32_t)u) word = neg;
      if (i < n) y[i] = (a == 0.0f || !finite) ? kPwZeroLog : pw_log2(a);
    }
    if (lane < (uint32_t)kPwU && base + 32 * lane < n) signs[ch * kPwU + lane] = word;
  }
  if (__any_sync(full, bad) && lane == 0) atomicOr(flag, 1u);
}

__global__ void pwrel_inverse_kernel(const float *__restrict__ y, uint64_t n,
                                     const uint32_t *__restrict__ signs, float *__restrict__ x) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t ch = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       ch * 32 * kPwU < n; ch += warps) {
    const uint64_t base = ch * 32 * kPwU;
    float v[kPwU];
    uint32_t w[kPwU];
#pragma unroll
    for (int u = 0; u < kPwU; ++u) {
      const uint64_t i = base + 32 * u + lane;
      const bool in = i < n;
      v[u] = in ? y[i] : 0.0f;
      w[u] = in ? signs[ch * kPwU + u] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kPwU; ++u) {
      const uint64_t i = base + 32 * u + lane;
      const float a = v[u] < kPwZeroCut ? 0.0f : pw_exp2(v[u]);
      if (i < n) x[i] = ((w[u] >> lane) & 1u) ? -a : a;
    }
  }
}

static int grid_for(uint64_t n) {
  const uint64_t blocks = (n + 256 * kPwU - 1) / (256 * kPwU);
  return (int)(blocks < 152ull * 8 ? (blocks ? blocks : 1) : 152ull * 8);
}

cudaError_t launch_pwrel_forward(const float *x, uint64_t n, float *y, uint32_t *signs,
                                 uint32_t *flag, cudaStream_t s) {
  pwrel_forward_kernel<<<grid_for(n), 256, 0, s>>>(x, n, y, signs, flag);
  return cudaGetLastError();
}

cudaError_t launch_pwrel_inverse(const float *y, uint64_t n, const uint32_t *signs, float *x,
                                 cudaStream_t s) {
  pwrel_inverse_kernel<<<grid_for(n), 256, 0, s>>>(y, n, signs, x);
  return cudaGetLastError();
}

}  // namespace fz
