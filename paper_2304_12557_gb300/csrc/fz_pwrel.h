// fz_pwrel.h -- launchers of the log transform for point-wise relative
// bounds (fz_pwrel.cu), used by the C ABI in fz_api.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fz {

// the log value a zero is sent to, and the threshold below which the
// inverse gives zero (every nonzero float has log2 >= -149)
constexpr float kPwZeroLog = -160.0f;
constexpr float kPwZeroCut = -154.0f;

// y = log2|x|, sign bits (one word per 32 elements), *flag |= 1 on a
// non-finite input
cudaError_t launch_pwrel_forward(const float *x, uint64_t n, float *y, uint32_t *signs,
                                 uint32_t *flag, cudaStream_t s);
cudaError_t launch_pwrel_inverse(const float *y, uint64_t n, const uint32_t *signs, float *x,
                                 cudaStream_t s);

}  // namespace fz
