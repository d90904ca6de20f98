// fz_device.cuh -- device-side building blocks shared by the GB300 kernels.
//
// Format geometry (a chunk = the Lorenzo independence unit of Sec. 2.3 =
// 4 tiles of 2048 codes; a tile = one 32x32 u32 bitshuffle unit of Sec. 3.3;
// a brick = one 64-code group of a tile, owned by one thread):
//   ndim  chunk            tile (march axis)   brick        bricks/tile
//   1     8192             2048 (x)            64           32 x 1
//   2     64 x 128         64 x 32 (y)         8 x 8        8 x 4
//   3     32 x 32 x 8      32 x 32 x 2 (z)     8 x 4 x 2    4 x 8
// group g = bx + NBX * by; codes x-fastest inside a brick.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fz {

constexpr int kTileCodes = 2048;
constexpr int kTilesPerChunk = 4;
constexpr int kChunkCodes = kTileCodes * kTilesPerChunk;
constexpr int kThreads = 128;            // 4 warps, warp t = tile t

// quantiser constants.  fl(v + 1.5*2^23) rounds v to the nearest integer
// (ties to even) in the low mantissa bits whenever |v| <= 2^22; the float's
// bit pattern minus 0x4B000001 is then q + 2^22 - 1, which lies in
// [0, 2^23 - 2] exactly when |q| <= 2^22 - 1 (the stream's limit).
constexpr float kRoundMagic = 12582912.0f;     // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;   // bits of kRoundMagic
constexpr uint32_t kBiasBits = 0x4B000001u;
constexpr int32_t kPadBiased = 0x3FFFFF;       // biased form of q = 0
constexpr uint32_t kBiasedMax = 0x7FFFFEu;     // biased form of q = 2^22-1
// The quantiser's wide range: |q| <= 2^28 - 1 (a 3-D residual, a signed
// sum of eight q, then fits an i32 outlier record).  Fields within 2^22 - 1
// use the fp32 rounding trick; the others take integer conversion (their
// streams set header byte 7 to 1).
constexpr float kWideLimit = 268435456.0f;      // 2^28: |fl(x r)| below it
constexpr uint8_t kHdrWide = 1;                 // header byte 7

// error bits gathered in device memory, mapped to FZ_ERR_* on the host
constexpr uint32_t kErrRange = 1u;     // |q| too large or non-finite input
constexpr uint32_t kErrEbParam = 2u;   // derived bound not representable
constexpr uint32_t kErrTimeout = 4u;   // bounded wait ran out
constexpr uint32_t kErrCapacity = 8u;  // payload would pass out_capacity
constexpr uint32_t kErrCorrupt = 16u;  // decompressor: inconsistent stream
constexpr uint32_t kErrNonFinite = 32u;
constexpr uint32_t kErrWide = 64u;     // the field needs the wide quantiser's launch

// look-back status word: [63:62] flag, [61:32] blocks, [31:0] outliers.
// Unit u's word lives at status[u * kStatusStride]: spacing the words out
// spreads the look-back's hot reads over more L2 lines and slices.
#ifndef FZ_STATUS_STRIDE
#define FZ_STATUS_STRIDE 16
#endif
constexpr uint64_t kStatusStride = FZ_STATUS_STRIDE;
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

template <int NDIM> struct Geo;
template <> struct Geo<1> {
  static constexpr int BX = 64, BY = 1, BZ = 1, NBX = 32, NBY = 1;
  static constexpr int CX = 8192, CY = 1, CZ = 1;
};
template <> struct Geo<2> {
  static constexpr int BX = 8, BY = 8, BZ = 1, NBX = 8, NBY = 4;
  static constexpr int CX = 64, CY = 128, CZ = 1;
};
template <> struct Geo<3> {
  static constexpr int BX = 8, BY = 4, BZ = 2, NBX = 4, NBY = 8;
  static constexpr int CX = 32, CY = 32, CZ = 8;
};

// Division by a runtime constant d >= 1 for numerators below 2^31, by a
// precomputed multiply-high: with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(n, m) + n) >> l
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994).  Replaces 64-bit division in per-tile index math.
struct FastDiv {
  uint32_t d, m, l;
  __host__ __device__ FastDiv() : d(1), m(1), l(0) {}
  __host__ __device__ explicit FastDiv(uint32_t div) : d(div) {
    l = 0;
    while ((1ull << l) < div) ++l;
    m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1);
  }
  __host__ __device__ uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(n, m);
#else
    const uint32_t t = (uint32_t)(((uint64_t)n * m) >> 32);
#endif
    return (t + n) >> l;
  }
};

// The 64-byte stream header, little-endian (matches the host's reader).
struct __align__(16) StreamHeader {
  uint8_t magic[4];        // "FZG1"
  uint8_t version, ndim, mode, reserved0;
  uint32_t dims[3];
  uint32_t n_tiles;
  double eb_requested;
  float eb, ebx2, ebx2_r;
  uint32_t nnz_blocks, n_outliers;
  float range_min, range_max;
  uint32_t reserved1;
};
static_assert(sizeof(StreamHeader) == 64, "header is 64 bytes");

// Per-call scratch that alternates between two sets so that a call can
// zero the set the next call will use (no memset launch per call).
struct SetScratch {
  uint32_t ticket;      // dynamic chunk ticket
  uint32_t err;         // error bits
  uint64_t nnz;         // compressor: total blocks; decompressor: header's
  uint64_t nout;        // compressor: total outliers; decompressor: matched
  uint64_t n_chunks;    // decompressor: chunks found in the stream header
  uint32_t hdr_nout;    // decompressor: the header's outlier count
  uint32_t version;     // decompressor: the header's stream version (0: invalid)
  uint32_t ndim;        // decompressor: the header's dimensionality
  uint32_t ncx, ncy;    // decompressor: the chunk grid's x and y extents
  uint32_t wide;        // decompressor: header byte 7 (the wide quantiser)
  uint32_t pad[2];
};
static_assert(sizeof(SetScratch) == 64, "scratch block is 64 bytes");

struct RangeResult {
  float fmin, fmax;
  uint32_t nonfinite;
  uint32_t counter;     // last-block detection, self-resetting
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The look-back's status words carry their whole message in the word
// itself (no other memory is published through them), so relaxed
// device-scope accesses suffice and no fence is needed.
__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v)
               : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];"
               : "=l"(v)
               : "l"(p)
               : "memory");
  return v;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// plain arrival (release at CTA scope: this thread's earlier shared-memory
// writes are visible to a thread whose wait on the phase succeeds)
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar,
                                                  uint32_t parity,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = global_timer();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u && global_timer() - t0 > limit_ns) return false;
  }
}

// TMA tile loads (plain, no multicast) completing on an mbarrier.
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const void *tmap,
                                            uint64_t *bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::"
      "complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(smem_dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *smem_dst, const void *tmap,
                                            uint64_t *bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::"
      "complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(smem_dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// Bulk copy shared -> global (both 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_store(void *gdst, const void *smem_src,
                                           uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::
                   "l"(gdst),
               "r"(smem_u32(smem_src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Programmatic dependent launch: a kernel that another kernel follows on
// its stream lets that grid be scheduled as soon as every one of its own
// blocks has started; the following kernel waits for this grid's completion
// (and its memory) before it reads what this grid wrote.  Without a
// programmatic dependency both are no-ops.
__device__ __forceinline__ void grid_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// 128-byte swizzle of a box row of 32 floats: 16-byte chunk c of row r sits
// at chunk position c ^ (r % 8) (the TMA SWIZZLE_128B layout for a
// 1024-byte aligned box).
__device__ __forceinline__ uint32_t swz(uint32_t row, uint32_t chunk) {
  return row * 128u + ((chunk ^ (row & 7u)) << 4);
}

// ------------------------------------------------------------ warp helpers
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Decoupled look-back (single-pass prefix sum over work units in ticket
// order), in two steps so that a caller can do other work in between:
// publish_aggregate() posts a unit's own (blocks<<32 | outliers) as soon as
// it is known, resolve_prefix() later finds the exclusive prefix over units
// < c and posts the unit's inclusive prefix.  Both are executed by one full
// warp.  Lane 0 first waits for the immediate predecessor alone; when that
// one has already posted its inclusive prefix (the common case) no other word
// is read.  Otherwise the warp scans back 32*K words per round (K per lane);
// only words nearer than the nearest inclusive prefix must have posted.  Every
// wait is bounded by limit_ns; on time-out the error bit is raised and the
// prefix found so far is used (all later writes stay bounds-checked).
__device__ __forceinline__ void publish_aggregate(uint64_t *st, uint64_t c, uint64_t agg,
                                                  bool publish) {
  if ((threadIdx.x & 31) == 0 && publish)
    st_relaxed(&st[c * kStatusStride], (c == 0 ? kFlagInc : kFlagAgg) | agg);
}

#ifndef FZ_LOOKBACK_K
#define FZ_LOOKBACK_K 1
#endif
template <int K = FZ_LOOKBACK_K>
__device__ __forceinline__ uint64_t resolve_prefix(uint64_t *st, uint64_t c, uint64_t agg,
                                                   bool publish, uint32_t *err,
                                                   uint64_t limit_ns) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  if (c == 0) return 0;                    // posted inclusive already
  uint64_t t0 = 0;
  bool timed_out = false;
  // immediate predecessor, one lane
  uint64_t pv = 0;
  if (lane == 0) {
    pv = ld_relaxed(&st[(c - 1) * kStatusStride]);
    if ((pv >> 62) == 0) {
      t0 = global_timer();
      uint32_t ns = 32;
      while ((pv >> 62) == 0) {
        __nanosleep(ns);
        if (ns < 256) ns *= 2;
        pv = ld_relaxed(&st[(c - 1) * kStatusStride]);
        if ((pv >> 62) == 0 && global_timer() - t0 > limit_ns) {
          timed_out = true;
          break;
        }
      }
    }
  }
  pv = __shfl_sync(full, pv, 0);
  timed_out = __shfl_sync(full, timed_out, 0);
  uint64_t excl = 0;
  if (!timed_out && (pv >> 62) == 2) {
    excl = pv & kValMask;
  } else if (!timed_out) {
    excl = pv & kValMask;                  // predecessor's aggregate
    int64_t j = (int64_t)c - 2;            // nearest word of the window
    while (true) {
      // entry k of lane L is word j - (L*K + k): nearest first
      uint64_t v[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int64_t idx = j - lane * K - k;
        v[k] = idx >= 0 ? ld_relaxed(&st[(uint64_t)idx * kStatusStride]) : kFlagInc;
      }
      int pl, fk;
      uint32_t it = 0;
      while (true) {
        int first = K;
#pragma unroll
        for (int k = K - 1; k >= 0; --k)
          if ((v[k] >> 62) == 2) first = k;
        const uint32_t pmask = __ballot_sync(full, first < K);
        pl = pmask ? __ffs(pmask) - 1 : 32;
        fk = __shfl_sync(full, first, pl & 31);
        bool pending = false;
#pragma unroll
        for (int k = 0; k < K; ++k)
          pending |= (lane < pl || (lane == pl && k < fk)) && (v[k] >> 62) == 0;
        if (!__any_sync(full, pending)) break;  // every exit is warp-uniform
        if (t0 == 0) t0 = global_timer();
        if (pending) {
          __nanosleep(64);
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int64_t idx = j - lane * K - k;
            if ((lane < pl || (lane == pl && k < fk)) && (v[k] >> 62) == 0)
              v[k] = ld_relaxed(&st[(uint64_t)idx * kStatusStride]);
          }
        }
        if ((++it & 15u) == 0) {
          const bool late = global_timer() - t0 > limit_ns;
          if (__any_sync(full, late)) {
            timed_out = true;
            break;
          }
        }
      }
      if (timed_out) break;
      uint64_t part = 0;
#pragma unroll
      for (int k = 0; k < K; ++k)
        part += (lane < pl || (lane == pl && k <= fk)) ? (v[k] & kValMask) : 0;
      excl += warp_sum_u64(part);
      if (pl < 32) break;
      j -= 32 * K;
    }
  }
  if (timed_out && lane == 0) atomicOr(err, kErrTimeout);
  if (lane == 0 && publish) st_relaxed(&st[c * kStatusStride], kFlagInc | (excl + agg));
  return excl;
}

// both steps at once
__device__ __forceinline__ uint64_t lookback(uint64_t *st, uint64_t c, uint64_t agg,
                                             bool publish, uint32_t *err, uint64_t limit_ns) {
  publish_aggregate(st, c, agg, publish);
  return resolve_prefix(st, c, agg, publish, err, limit_ns);
}

// ------------------------------------------------------------ bit transpose
// byte select of the pair (x, y): result byte i = byte (sel >> 4i) & 7 of
// the 8-byte value y:x (PRMT on the device; a plain loop on the host, where
// the transpose is unit-tested)
__host__ __device__ __forceinline__ uint32_t byte_perm(uint32_t x, uint32_t y,
                                                       uint32_t sel) {
#ifdef __CUDA_ARCH__
  return __byte_perm(x, y, sel);
#else
  const uint64_t v = (uint64_t)y << 32 | x;
  uint32_t r = 0;
  for (int i = 0; i < 4; ++i)
    r |= (uint32_t)((v >> (8 * ((sel >> (4 * i)) & 7u))) & 0xFFu) << (8 * i);
  return r;
#endif
}

// In-register 32x32 bit-matrix transpose (block-swap recursion, LSB-first):
// afterwards bit t of a[b] equals bit b of the input a[t].  The 16- and
// 8-bit stages move whole bytes and use byte permutes.
__host__ __device__ __forceinline__ void transpose32(uint32_t (&a)[32]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    uint32_t x = a[k], y = a[k + 16];
    a[k] = byte_perm(x, y, 0x5410);
    a[k + 16] = byte_perm(x, y, 0x7632);
  }
#pragma unroll
  for (int k0 = 0; k0 < 32; k0 += 16) {
#pragma unroll
    for (int k = k0; k < k0 + 8; ++k) {
      uint32_t x = a[k], y = a[k + 8];
      a[k] = byte_perm(x, y, 0x6240);
      a[k + 8] = byte_perm(x, y, 0x7351);
    }
  }
#pragma unroll
  for (int k0 = 0; k0 < 32; k0 += 8) {
#pragma unroll
    for (int k = k0; k < k0 + 4; ++k) {
      uint32_t x = a[k], y = a[k + 4];
      a[k] = (x & 0x0F0F0F0Fu) | ((y << 4) & 0xF0F0F0F0u);
      a[k + 4] = ((x >> 4) & 0x0F0F0F0Fu) | (y & 0xF0F0F0F0u);
    }
  }
#pragma unroll
  for (int k0 = 0; k0 < 32; k0 += 4) {
#pragma unroll
    for (int k = k0; k < k0 + 2; ++k) {
      uint32_t x = a[k], y = a[k + 2];
      a[k] = (x & 0x33333333u) | ((y << 2) & 0xCCCCCCCCu);
      a[k + 2] = ((x >> 2) & 0x33333333u) | (y & 0xCCCCCCCCu);
    }
  }
#pragma unroll
  for (int k = 0; k < 32; k += 2) {
    uint32_t x = a[k], y = a[k + 1];
    a[k] = (x & 0x55555555u) | ((y << 1) & 0xAAAAAAAAu);
    a[k + 1] = ((x >> 1) & 0x55555555u) | (y & 0xAAAAAAAAu);
  }
}

// The same transpose for a brick whose 64 codes all have magnitude < 128
// (7 magnitude bits and the sign: 16 of the 32 bit-plane rows are nonzero).
// squeeze_narrow turns the 32 code-pair words w[i] = c(2i) | c(2i+1) << 16
// into 16 words of byte codes (magnitude in bits 0..6, sign in bit 7)
//   u[j] = c(2j) | c(2j+1) << 8 | c(32+2j) << 16 | c(33+2j) << 24,
// and transpose16 swaps bit and word index within each 16-bit half of u
// (the 8-, 4-, 2- and 1-bit stages of transpose32 over 16 words).  Then
// u[r] is transpose32's row narrow_row(r) and the other rows are zero.
__host__ __device__ __forceinline__ void squeeze_narrow(const uint32_t (&w)[32],
                                                        uint32_t (&u)[16]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    // byte 0 / 2 of w | w >> 8: a code's magnitude byte with its sign bit
    const uint32_t lo = w[j] | (w[j] >> 8), hi = w[j + 16] | (w[j + 16] >> 8);
    u[j] = byte_perm(lo, hi, 0x6420);
  }
}

__host__ __device__ __forceinline__ void transpose16(uint32_t (&a)[16]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t x = a[k], y = a[k + 8];
    a[k] = byte_perm(x, y, 0x6240);
    a[k + 8] = byte_perm(x, y, 0x7351);
  }
#pragma unroll
  for (int k0 = 0; k0 < 16; k0 += 8) {
#pragma unroll
    for (int k = k0; k < k0 + 4; ++k) {
      uint32_t x = a[k], y = a[k + 4];
      a[k] = (x & 0x0F0F0F0Fu) | ((y << 4) & 0xF0F0F0F0u);
      a[k + 4] = ((x >> 4) & 0x0F0F0F0Fu) | (y & 0xF0F0F0F0u);
    }
  }
#pragma unroll
  for (int k0 = 0; k0 < 16; k0 += 4) {
#pragma unroll
    for (int k = k0; k < k0 + 2; ++k) {
      uint32_t x = a[k], y = a[k + 2];
      a[k] = (x & 0x33333333u) | ((y << 2) & 0xCCCCCCCCu);
      a[k + 2] = ((x >> 2) & 0x33333333u) | (y & 0xCCCCCCCCu);
    }
  }
#pragma unroll
  for (int k = 0; k < 16; k += 2) {
    uint32_t x = a[k], y = a[k + 1];
    a[k] = (x & 0x55555555u) | ((y << 1) & 0xAAAAAAAAu);
    a[k + 1] = ((x >> 1) & 0x55555555u) | (y & 0xAAAAAAAAu);
  }
}

// transpose32's row held by transpose16's word r: even codes' planes 0..6
// and 15 (sign), then odd codes' planes 16..22 and 31
__host__ __device__ __forceinline__ constexpr int narrow_row(int r) {
  return 16 * (r >> 3) + ((r & 7) == 7 ? 15 : (r & 7));
}

// ------------------------------------------------------------ eb derivation
// Sec. 4.1: the absolute bound from the request (relative bounds scale the
// value range).  Same rules as the stream format: double arithmetic, the
// fp32 bound rounded toward zero, 1/(2eb) rounded to fp32 from double.
struct EbParams {
  float eb, ebx2, ebx2_r;
  bool ok;
};

__device__ __forceinline__ EbParams derive_eb(int mode, double eb_req,
                                              float fmin, float fmax) {
  EbParams p{0.f, 0.f, 0.f, false};
  double eb_d = eb_req;
  if (mode == 1) {
    double range = __dsub_rn((double)fmax, (double)fmin);
    if (range == 0.0) {
      range = fabs((double)fmax);
      if (range == 0.0) range = 1.0;
    }
    eb_d = __dmul_rn(eb_req, range);
  }
  if (!(eb_d > 0.0) || !isfinite(eb_d)) return p;
  float e = __double2float_rz(eb_d);
  if (!(e >= 1.17549435e-38f)) return p;
  float e2 = __fmul_rn(2.0f, e);
  if (isinf(e2)) return p;
  p.eb = e;
  p.ebx2 = e2;
  p.ebx2_r = __double2float_rn(__ddiv_rn(1.0, (double)e2));
  p.ok = true;
  return p;
}

}  // namespace fz
