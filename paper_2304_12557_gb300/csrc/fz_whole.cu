// fz_whole.cu -- the cross-chunk sums of whole-field Lorenzo decompression
// (stream version 2).
//
// The whole-field residual is delta = D_x D_y D_z q with q = 0 outside the
// field (Sec. 2.2, Eq. 1 taken over the whole field instead of a chunk), so
// q is the whole-field prefix sum S_x S_y S_z delta.  Per axis, the whole
// prefix is the chunk-local one plus the carry from the chunks before:
// S = S^c + K, where (K f)(p) sums (S^c f) at the last coordinate of each
// earlier chunk along that axis.  Expanding
//   q = (S^c_x + K_x)(S^c_y + K_y)(S^c_z + K_z) delta
// gives the chunk-local prefix L = S^c_x S^c_y S^c_z delta (what phase 1 of
// the decompressor computes per chunk) plus terms that read only L on the
// chunks' upper faces.  Grouped by the coordinates they depend on:
//   3-D  q(x,y,z) = L + A'(y,z) + B'(x,z) + C'(x,y)
//        C' = K_z on the z-faces;
//        B' = K_y on the y-faces after their whole-field z prefix;
//        A' = K_x on the x-faces after their whole-field z, then y prefix;
//   2-D  q(x,y)   = L + A'(y) + B'(x)
//        B' = K_y on the y-faces;  A' = K_x on the x-faces after their
//        whole-field y prefix;
//   1-D  q(x)     = L + A'            A' = K_x on the chunks' last elements.
// Every step is one exclusive or inclusive scan along one axis of the chunk
// grid (face_scan_lines_kernel, face_scan_word_kernel); phase 2 of the
// decompressor adds the terms.
#include <cuda_runtime.h>

#include <cstdint>

#include "fz_kernels.h"

namespace fz {

namespace {

constexpr int kScanThreads = 256;

// out(c)(i) = [self] in(c)(i) + sum over the chunks c' before c along
// `axis` (the other two chunk coordinates equal) of in(c')(map(i)), for a
// face of U x W words per chunk (i = u + U w).  map 0: i itself; 1: w set
// to W - 1 (the face's last row); 2: u set to U - 1 (its last column).
// Unsigned arithmetic, so that a corrupt stream's sums wrap rather than
// overflow.  The chunk at step k of a line is base + k * stride.
struct Line {
  uint64_t base, stride, n;
};
__device__ __forceinline__ Line line_of(uint64_t line, uint32_t ncx, uint32_t ncy, uint32_t ncz,
                                        int axis) {
  if (axis == 0) return {(uint64_t)ncx * line, 1, ncx};
  if (axis == 1) {
    const uint64_t cx = line % ncx, cz = line / ncx;
    return {cx + (uint64_t)ncx * ncy * cz, ncx, ncy};
  }
  return {line, (uint64_t)ncx * ncy, ncz};
}
__device__ __forceinline__ uint32_t mapped(uint32_t i, uint32_t U, uint32_t W, int map) {
  const uint32_t u = i % U, w = i / U;
  return map == 1 ? u + U * (W - 1) : map == 2 ? (U - 1) + U * w : i;
}

// Faces of 32 words or more: one thread per (line, face word), consecutive
// threads on consecutive words; each thread walks its line, loading 8 steps'
// words at once before it sums them.
__global__ void __launch_bounds__(kScanThreads)
    face_scan_lines_kernel(const uint32_t *in, uint32_t *out, uint32_t ncx, uint32_t ncy,
                           uint32_t ncz, int axis, uint32_t U, uint32_t W, int map, int self,
                           uint64_t total) {
  constexpr int kStep = 8;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  const uint32_t m = U * W;
  const uint32_t i = (uint32_t)(t % m);
  const Line L = line_of(t / m, ncx, ncy, ncz, axis);
  const uint32_t mi = mapped(i, U, W, map);
  uint32_t carry = 0;
  for (uint64_t k0 = 0; k0 < L.n; k0 += kStep) {
    uint32_t mv[kStep], val[kStep];
#pragma unroll
    for (int j = 0; j < kStep; ++j) {
      mv[j] = 0;
      val[j] = 0;
      if (k0 + j < L.n) {
        const uint64_t c = L.base + (k0 + j) * L.stride;
        mv[j] = __ldg(in + c * m + mi);
        if (self) val[j] = __ldg(in + c * m + i);
      }
    }
#pragma unroll
    for (int j = 0; j < kStep; ++j) {
      if (k0 + j < L.n) out[(L.base + (k0 + j) * L.stride) * m + i] = val[j] + carry;
      carry += mv[j];
    }
  }
}

// One-word faces (1-D: the chunks' last elements): a block per line, 256
// chunks per step, a block-wide scan over the step.
__global__ void __launch_bounds__(kScanThreads)
    face_scan_word_kernel(const uint32_t *in, uint32_t *out, uint32_t ncx, uint32_t ncy,
                          uint32_t ncz, int axis, int self) {
  __shared__ uint32_t sh[kScanThreads / 32];
  const Line L = line_of(blockIdx.x, ncx, ncy, ncz, axis);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (uint64_t k0 = 0; k0 < L.n; k0 += kScanThreads) {
    const uint64_t k = k0 + threadIdx.x;
    const uint64_t c = L.base + k * L.stride;
    const uint32_t mv = k < L.n ? __ldg(in + c) : 0u;
    uint32_t inc = mv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) sh[wp] = inc;
    __syncthreads();
    uint32_t before = 0, tot = 0;
#pragma unroll
    for (int j = 0; j < kScanThreads / 32; ++j) {
      before += j < wp ? sh[j] : 0u;
      tot += sh[j];
    }
    __syncthreads();                                   // sh is reused next step
    if (k < L.n) out[c] = (self ? mv : 0u) + carry + before + inc - mv;
    carry += tot;
  }
}

cudaError_t scan(const int32_t *in, int32_t *out, const uint32_t nc[3], int axis, uint32_t U,
                 uint32_t W, int map, int self, cudaStream_t s) {
  const uint64_t lines = (uint64_t)nc[0] * nc[1] * nc[2] / nc[axis];
  const uint32_t m = U * W;
  const uint32_t *i = reinterpret_cast<const uint32_t *>(in);
  uint32_t *o = reinterpret_cast<uint32_t *>(out);
  if (m == 1) {
    face_scan_word_kernel<<<(unsigned)lines, kScanThreads, 0, s>>>(i, o, nc[0], nc[1], nc[2], axis,
                                                                   self);
  } else {
    const uint64_t total = lines * m;
    face_scan_lines_kernel<<<(unsigned)((total + kScanThreads - 1) / kScanThreads), kScanThreads, 0,
                             s>>>(i, o, nc[0], nc[1], nc[2], axis, U, W, map, self, total);
  }
  return cudaGetLastError();
}

}  // namespace

int whole_face_elems(int ndim, int k) {
  static const int e[3][3] = {{1, 0, 0}, {128, 64, 0}, {256, 256, 1024}};
  return (ndim >= 1 && ndim <= 3 && k >= 0 && k < 3) ? e[ndim - 1][k] : 0;
}

cudaError_t launch_whole_scans(int ndim, const uint32_t nc[3], int32_t *const face[3],
                               int32_t *const work[3], const int32_t *corr[3], cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  auto run = [&](const int32_t *in, int32_t *out, int axis, uint32_t U, uint32_t W, int map,
                 int self) {
    if (e == cudaSuccess) e = scan(in, out, nc, axis, U, W, map, self, s);
  };
  corr[0] = corr[1] = corr[2] = nullptr;
  if (ndim == 3) {
    // C'(x, y): the z-faces (32 x by 32 y) summed over the chunks below
    run(face[2], work[2], 2, 32, 32, 0, 0);
    corr[2] = work[2];
    // B'(x, z): y-faces (32 x by 8 z) to a whole-field z prefix, then
    // summed over the chunks before along y
    run(face[1], work[1], 2, 32, 8, 1, 1);
    run(work[1], face[1], 1, 32, 8, 0, 0);
    corr[1] = face[1];
    // A'(y, z): x-faces (32 y by 8 z) to a whole-field z, then y prefix,
    // then summed over the chunks before along x
    run(face[0], work[0], 2, 32, 8, 1, 1);
    run(work[0], face[0], 1, 32, 8, 2, 1);
    run(face[0], work[0], 0, 32, 8, 0, 0);
    corr[0] = work[0];
  } else if (ndim == 2) {
    // B'(x): y-faces (64 x) summed over the chunks before along y
    run(face[1], work[1], 1, 64, 1, 0, 0);
    corr[1] = work[1];
    // A'(y): x-faces (128 y) to a whole-field y prefix, then summed over the
    // chunks before along x
    run(face[0], work[0], 1, 128, 1, 2, 1);
    run(work[0], face[0], 0, 128, 1, 0, 0);
    corr[0] = face[0];
  } else {
    // A': the chunks' last elements summed over the chunks before
    run(face[0], work[0], 0, 1, 1, 0, 0);
    corr[0] = work[0];
  }
  return e;
}

}  // namespace fz
