// fz_compress_impl.cuh -- the compression kernels' device code, shared by the
// single-field launch (fz_compress.cu) and the batched launch (fz_batch.cu).
//
//  compress_kernel  persistent blocks of kCompWarps compute warps and one
//                   scan warp; one 2048-code tile per compute warp and round:
//                   32-byte row loads or a TMA box -> pre-quantisation
//                   (Sec. 2.3) -> chunk-local Lorenzo residual (Sec. 2.3,
//                   3.1) -> sign-magnitude codes (Sec. 3.2) -> 32x32
//                   bitshuffle (Sec. 3.3) -> zero-block flags (Sec. 3.4,
//                   Listing 1) -> decoupled look-back on units of tiles ->
//                   compacted 16-byte block stores (Listing 2).
//  outlier_kernel   rare path: writes the escaped residuals of the tiles that
//                   had any, at offsets found by compress_kernel.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "fz_device.cuh"
#include "fz_kernels.h"

namespace fz {

// ====================================================================
// compression: persistent blocks, one 2048-code tile per warp and round
// ====================================================================
//
// One block per SM: kCompWarps compute warps and one scan warp.  Each round
// the scan warp takes a ticket for a unit of kCompWarps consecutive tiles
// (stream order); compute warp j does tile j of the unit: pre-quantisation,
// Lorenzo, codes, bitshuffle, flags, and posts the tile's aggregate (blocks,
// outliers) in shared memory.  The scan warp sums the unit, runs the
// decoupled look-back on the unit index and hands every warp its tile's
// exclusive prefix, which the warp uses one round later (a batch: midway
// through the next round) to store the compacted blocks.  The look-back
// therefore walks one status word per unit, and its latency is hidden
// behind the compute warps' next tiles.
// A compute warp's input comes either from a per-warp TMA box (its tile,
// loaded one round ahead) or, for fields whose rows are not 16-byte aligned
// and for 1-D fields, straight from global memory.

constexpr int kCompWarps = 15;                  // compute warps per block
static_assert(kCompWarps == kCompressUnitTiles, "a look-back unit is one tile per compute warp");
constexpr int kCompThreads = 32 * (kCompWarps + 1);   // + the scan warp
constexpr int kRing = 4;                        // rounds in flight per block
// A warp stores a tile's compacted blocks after computing later tiles, so
// that the scan warp has time to resolve the tile's prefix.  The blocks wait
// in the warp's ring: a shared-memory area of ring_blocks() 16-byte blocks
// whose two ends take the tiles of even and odd rounds.  A tile of round r
// is stored in round r + 2, right before round r + 2 uses that end, so its
// prefix has one and a half rounds to arrive.  Each round first transposes
// its codes into bit planes in a 256-block staging area at its own end of
// the ring (the planes are read back into registers before the compacted
// blocks are written over them), so the tile of round r + 1 waiting at the
// other end must leave 256 blocks free; a tile of more blocks than that is
// stored one round early.
template <bool BATCH>
__host__ __device__ constexpr int ring_blocks() { return BATCH ? 360 : 440; }
constexpr int kStageBlocks = 256;               // one tile's bit planes (4 KB)
static_assert(ring_blocks<true>() % 8 == 0 && ring_blocks<false>() % 8 == 0,
              "ring rows of 8 blocks (128 bytes)");
static_assert(ring_blocks<true>() >= kStageBlocks + 64, "a batch ring defers small tiles");
// per compute warp: a TMA box (TMA launches).  A single field takes one 8 KB
// box per tile; a batch has room for the row-class boxes of fields whose
// rows are not 16-byte aligned (9 KB, see issue_class_boxes).  The boxes
// come first (1024-byte aligned for the 128-byte swizzle), then the rings.
template <bool BATCH>
__host__ __device__ constexpr int box_bytes() { return BATCH ? 9216 : 8192; }
template <bool BATCH>
__host__ __device__ constexpr int ring_bytes() { return 16 * ring_blocks<BATCH>(); }
constexpr int kHalf2D = 4096;                   // second x half of a 2-D box
constexpr uint32_t kTileBoxBytes = 32 * 32 * 2 * 4;  // one tile (3-D: 2 planes; 2-D: 2 halves)
// Row-class boxes: a field's rows (index R = y + Y z) in four classes by
// R mod 4 start at one 16-byte offset each, so each class is a 2-D tensor of
// rows 16 * pitch bytes apart whose base is rounded down to 16 bytes; its
// map's x runs from that base, r_k = the class's offset in floats (0..3),
// ahead of x = 0.  Per tile: 3-D, for each of the 2 planes and 4 classes, a
// box of 8 rows of 36 floats (1152 B); 2-D, for each class, 8 rows of 68.
constexpr int kClassRow3 = 36, kClassRow2 = 68;
constexpr int kClassBox3 = 8 * kClassRow3 * 4, kClassBox2 = 8 * kClassRow2 * 4;
static_assert(8 * kClassBox3 <= 9216 && 4 * kClassBox2 <= 9216, "class boxes fit the box area");
static_assert(kClassBox3 % 128 == 0 && kClassBox2 % 128 == 0, "class boxes 128-byte aligned");

// the rounds a block has in flight, in shared memory behind the warps' areas
struct RoundSlot {
  uint64_t unit;                 // ticket: the launch's unit index
  uint32_t field, local;         // its field, and its index among the field's units:
                                 // tiles [local * kCompWarps, local * kCompWarps + kCompWarps)
  uint64_t agg[kCompWarps];      // tile aggregates, (blocks << 32) | outliers
  uint64_t excl[kCompWarps];     // their exclusive prefixes in the stream
};
struct CompShared {
  uint64_t box_bar[kCompWarps];  // per compute warp: its TMA box landed
  uint64_t ticket_bar[kRing];    // 1 arrival: the scan warp posted the unit
  uint64_t agg_bar[kRing];       // kCompWarps arrivals: every aggregate posted
  uint64_t excl_bar[kRing];      // kCompWarps arrivals: every prefix posted
  RoundSlot slot[kRing];
};
// What the kernel derives once per field: the bound (Sec. 4.1), the range it
// came from, whether the quantiser takes the field, and the chunk grid's
// divisors.
struct __align__(8) FieldRt {
  EbParams p;
  float fmin, fmax;
  uint32_t ok;
  uint32_t wide;                 // the wide quantiser (|q| up to 2^28 - 1)
  FastDiv dx, dy;
};

// A batch: several fields in one launch.  Units of kCompWarps consecutive
// tiles never straddle a field, so every field keeps its own look-back
// domain, result block and stream.
struct BatchArgs {
  const CompressArgs *fields;    // per field (device)
  const FieldRt *rt;             // per field, written by the batch's prepare pass
  const CUtensorMap *tmaps;      // per field (TMA launches), 64-byte aligned
  const CUtensorMap *cmaps;      // per field 4 row-class maps (use_tma 2), 64-byte aligned
  const uint2 *unit_map;         // per unit of the launch: (field, unit within the field)
  uint64_t n_units;
  uint32_t *ticket;              // the launch's unit counter, zero at launch
};

// a batch's compute warp keeps its current field's arguments in shared
// memory (global stores cannot alias them there, so the compiler need not
// reload them after every store)
struct __align__(16) WarpField {
  CompressArgs a;
  FieldRt rt;
};
constexpr int kWarpFieldBytes = (int)((sizeof(WarpField) + 15) / 16 * 16);

constexpr int kCompShBytes = (int)((sizeof(CompShared) + 15) / 16 * 16);
// [boxes (TMA)][rings][CompShared][WarpField per compute warp (batches)]
template <bool TMA, bool BATCH>
__host__ __device__ constexpr int comp_area_bytes() {
  return kCompWarps * ((TMA ? box_bytes<BATCH>() : 0) + ring_bytes<BATCH>());
}
constexpr int kCompSmemTma = comp_area_bytes<true, false>() + kCompShBytes + 1024;
constexpr int kCompSmemLdg = comp_area_bytes<false, false>() + kCompShBytes + 1024;
constexpr int kCompSmemBatch =
    comp_area_bytes<true, true>() + kCompShBytes + kCompWarps * kWarpFieldBytes + 1024;
static_assert(kCompSmemTma <= 227 * 1024 && kCompSmemBatch <= 227 * 1024,
              "shared memory per block");
static_assert(sizeof(CompressArgs) % 8 == 0 && sizeof(FieldRt) % 8 == 0, "copied as u64 words");

// bounded wait on an mbarrier phase by a whole warp; the result is uniform
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  const bool ok = mbar_wait_bounded(bar, parity, limit_ns);
  return __all_sync(0xffffffffu, ok);
}

// 8 consecutive floats from p.  V = 8: one 32-byte load (p 32-byte
// aligned); V = 4: two 16-byte loads; V = 1: scalar loads.
template <int V>
__device__ __forceinline__ void load8(const float *p, float (&f)[8]) {
  if constexpr (V == 8) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(f[0]), "=f"(f[1]), "=f"(f[2]), "=f"(f[3]), "=f"(f[4]), "=f"(f[5]),
          "=f"(f[6]), "=f"(f[7])
        : "l"(p));
  } else if constexpr (V == 4) {
    const float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldcs(reinterpret_cast<const float4 *>(p) + 1);
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
    f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = __ldcs(p + k);
  }
}

// The value range a relative bound is taken against (Sec. 4.1): the range
// pass's result, or the caller's range (a slab of a field split across
// ranks uses the whole field's).  Absolute bounds have none.
__device__ __forceinline__ void field_range(const CompressArgs &a, float &fmin, float &fmax,
                                            bool &nonfinite) {
  if (a.mode != 1) return;
  if (a.range_given) {
    fmin = a.range_lo; fmax = a.range_hi;
  } else {
    fmin = a.range->fmin; fmax = a.range->fmax;
    nonfinite = a.range->nonfinite != 0;
  }
}

// fl(v + 1.5*2^23) of v = fl(x * r): the integer rint(v) sits in the low
// mantissa bits; returned as raw bits (biased by kMagicBits).
// With `wide`, rint(fl(x * r)) by integer conversion (ties to even), biased
// the same way, for |q| up to 2^28 - 1.
__device__ __forceinline__ int32_t quant_bits(float x, float r, bool wide = false) {
  if (wide) return __float2int_rn(__fmul_rn(x, r)) + (int32_t)kMagicBits;
  return (int32_t)__float_as_uint(__fadd_rn(__fmul_rn(x, r), kRoundMagic));
}

// The per-field derivation: bound from the request and the range, the
// quantiser's range check for relative bounds (the element of largest
// magnitude is in the field, and fp multiply and rounding are monotone, so
// checking it checks every element), and the error bits that stop the field.
__device__ __forceinline__ FieldRt derive_field(const CompressArgs &a, uint32_t &err) {
  FieldRt rt;
  float fmin = 0.f, fmax = 0.f;
  bool nonfinite = false;
  field_range(a, fmin, fmax, nonfinite);
  rt.p = derive_eb(a.mode, a.eb_req, fmin, fmax);
  rt.fmin = fmin;
  rt.fmax = fmax;
  bool ok = rt.p.ok && !nonfinite;
  err = 0;
  rt.wide = a.wide ? 1u : 0u;
  // |fl(m r)| below 2^28 <=> |rint| <= 2^28 - 1 (floats there are 16 apart)
  auto fits_wide = [&](float m) { return fabsf(__fmul_rn(m, rt.p.ebx2_r)) < kWideLimit; };
  if (ok && !a.wide && a.mode == 1 && !a.range_given) {
    const float m = fmaxf(fabsf(fmin), fabsf(fmax));
    const uint32_t b = (uint32_t)quant_bits(m, rt.p.ebx2_r) - kBiasBits;
    if (b > kBiasedMax) {
      ok = false;
      err |= a.allow_wide && fits_wide(m) ? kErrWide : kErrRange;
    }
  }
  if (ok && a.wide) {
    // the wide quantiser's launch: the range pass over the data bounds
    // every element (relative bounds: the field's own pass; absolute bounds
    // and supplied ranges: the pass the caller ran after the first launch)
    const float m = a.mode == 1 && !a.range_given
                        ? fmaxf(fabsf(fmin), fabsf(fmax))
                        : fmaxf(fabsf(a.range->fmin), fabsf(a.range->fmax));
    if (!fits_wide(m) || a.range->nonfinite) {
      ok = false;
      err |= kErrRange;
    }
  }
  if (!rt.p.ok) err |= kErrEbParam;
  if (nonfinite) err |= kErrNonFinite;
  rt.ok = ok;
  rt.dx = FastDiv(a.ncx);
  rt.dy = FastDiv(a.ncy);
  return rt;
}

struct TileGeo {
  uint64_t x0, y0, z0;       // origin of this lane's brick
  uint64_t cx, cy, cz;       // chunk coordinates
  int t, bx, by;
  bool edge;                 // the chunk reaches past the field
};

// chunk grid divisors, built once per warp
struct ChunkGrid {
  FastDiv x, y;
  __device__ explicit ChunkGrid(const CompressArgs &a) : x(a.ncx), y(a.ncy) {}
  __device__ ChunkGrid(const FastDiv &dx, const FastDiv &dy) : x(dx), y(dy) {}
};

template <int NDIM>
__device__ __forceinline__ TileGeo tile_geo(const CompressArgs &a, const ChunkGrid &cg,
                                            uint64_t T, int g) {
  using G = Geo<NDIM>;
  TileGeo q;
  const uint32_t c = (uint32_t)(T >> 2);             // < 2^19
  q.t = (int)(T & 3);
  const uint32_t r = cg.x.div(c);
  q.cx = c - r * cg.x.d;
  q.cz = cg.y.div(r);
  q.cy = r - (uint32_t)q.cz * cg.y.d;
  q.bx = g % G::NBX;
  q.by = g / G::NBX;
  if constexpr (NDIM == 3) {
    q.x0 = q.cx * 32 + 8 * q.bx; q.y0 = q.cy * 32 + 4 * q.by; q.z0 = q.cz * 8 + 2 * q.t;
  } else if constexpr (NDIM == 2) {
    q.x0 = q.cx * 64 + 8 * q.bx; q.y0 = q.cy * 128 + 32 * q.t + 8 * q.by; q.z0 = 0;
  } else {
    q.x0 = q.cx * 8192 + 2048 * q.t + 64 * g; q.y0 = 0; q.z0 = 0;
  }
  q.edge = (q.cx + 1) * G::CX > a.dims[0] || (q.cy + 1) * G::CY > a.dims[1] ||
           (q.cz + 1) * G::CZ > a.dims[2];
  return q;
}

// ---- whole-field Lorenzo (stream version 2) ----------------------------
// The variant takes every neighbour inside the field (zero only outside it)
// instead of every neighbour inside the chunk, so a brick on a chunk's lower
// face needs values of the neighbouring chunk; they come from global memory.
// q_at: the biased quantised value Q = fl(fl(x * r) + 1.5 * 2^23) of the
// element at (x, y, z), or the biased zero outside the field (a coordinate
// of -1 wraps around and is outside too).
__device__ __forceinline__ float q_at(const CompressArgs &a, uint64_t x, uint64_t y, uint64_t z,
                                      float r) {
  const bool in = x < a.dims[0] && y < a.dims[1] && z < a.dims[2];
  const float v = in ? __ldg(a.x + x + a.pitch * (y + a.dims[1] * z)) : 0.0f;
  return __fadd_rn(__fmul_rn(v, r), kRoundMagic);
}
// the same as a biased integer, through the wide quantiser when `wide`
__device__ __forceinline__ int32_t qi_at(const CompressArgs &a, uint64_t x, uint64_t y, uint64_t z,
                                         float r, bool wide) {
  if (!wide) return __float_as_int(q_at(a, x, y, z, r));
  const bool in = x < a.dims[0] && y < a.dims[1] && z < a.dims[2];
  return quant_bits(in ? __ldg(a.x + x + a.pitch * (y + a.dims[1] * z)) : 0.0f, r, true);
}
// whether a brick's neighbours one step back along the march axis (3-D:
// the plane below, 2-D: the row above, 1-D: the element before) count:
// inside the chunk (the chunk's first tile has none) or inside the field
template <int NDIM, bool WHOLE>
__device__ __forceinline__ bool march_halo(const TileGeo &q) {
  if constexpr (WHOLE) return NDIM == 3 ? q.z0 > 0 : NDIM == 2 ? q.y0 > 0 : q.x0 > 0;
  else return q.t > 0;
}
// 3-D, a brick with by == 0: D_z Q of the row above the brick (y0 - 1) at
// x0 + ix, z0 + iz (whole-field; chunked residuals take 0 there)
__device__ __forceinline__ float face_up3(const CompressArgs &a, const TileGeo &q, int ix, int iz,
                                          float r) {
  const uint64_t x = q.x0 + ix, y = q.y0 - 1, z = q.z0 + iz;
  return __fsub_rn(q_at(a, x, y, z, r), q_at(a, x, y, z - 1, r));
}
// 3-D, a brick with bx == 0: D_y D_z Q of the column before the brick
// (x0 - 1) at y0 + iy, z0 + iz
__device__ __forceinline__ float face_left3(const CompressArgs &a, const TileGeo &q, int iy,
                                            int iz, float r) {
  const uint64_t x = q.x0 - 1, y = q.y0 + iy, z = q.z0 + iz;
  const float d1 = __fsub_rn(q_at(a, x, y, z, r), q_at(a, x, y - 1, z, r));
  const float d0 = __fsub_rn(q_at(a, x, y, z - 1, r), q_at(a, x, y - 1, z - 1, r));
  return __fsub_rn(d1, d0);
}
// 2-D, a brick with bx == 0: D_y Q of the column before the brick at y0 + iy
__device__ __forceinline__ float face_left2(const CompressArgs &a, const TileGeo &q, int iy,
                                            float r) {
  const uint64_t x = q.x0 - 1, y = q.y0 + iy;
  return __fsub_rn(q_at(a, x, y, 0, r), q_at(a, x, y - 1, 0, r));
}

// Rows of 8 floats of a lane's brick, read from global memory.  Row
// selectors: 3-D (p, iy) with p = -1 the previous plane, 0/1 the brick's
// planes; 2-D (0, iy) with iy = -1 the previous row; 1-D (0, 0, xo).
// Elements outside the field read as 0.
template <int NDIM, int V>
struct GlobalRows {
  const CompressArgs &a;
  const TileGeo &q;
  __device__ __forceinline__ void row(int p, int iy, int xo, float (&f)[8]) const {
    const uint64_t x = q.x0 + xo, y = q.y0 + iy, z = q.z0 + p;
    const float *ptr = a.x + x + a.pitch * (y + a.dims[1] * z);
    if (!q.edge) {
      load8<V>(ptr, f);
    } else {
      const bool in = y < a.dims[1] && z < a.dims[2];
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = (in && x + k < a.dims[0]) ? __ldcs(ptr + k) : 0.0f;
    }
  }
};

// The same rows from the warp's TMA box (128-byte swizzled rows of 32
// floats; the TMA unit has zero-filled everything outside the field).
// Only the brick's own rows come from the box (p = 0, 1 / iy >= 0).
template <int NDIM>
struct BoxRows {
  const uint8_t *box;
  int bx, by;
  __device__ __forceinline__ void row(int p, int iy, int, float (&f)[8]) const {
    uint32_t base, r, c0;
    if constexpr (NDIM == 3) {
      base = 0; r = (uint32_t)(4 * by + iy + 32 * p); c0 = 2 * bx;
    } else {
      base = (bx >> 2) * kHalf2D; r = (uint32_t)(8 * by + iy); c0 = 2 * (bx & 3);
    }
    const float4 u = *reinterpret_cast<const float4 *>(box + base + swz(r, c0));
    const float4 w = *reinterpret_cast<const float4 *>(box + base + swz(r, c0 + 1));
    f[0] = u.x; f[1] = u.y; f[2] = u.z; f[3] = u.w;
    f[4] = w.x; f[5] = w.y; f[6] = w.z; f[7] = w.w;
  }
};

// The same rows from the warp's row-class boxes (issue_class_boxes): brick
// row (p, iy) lies in class k = (R0 + iy) mod 4 of its plane (R0: the
// tile's first row index on it), at box row by (3-D) or 2 by + iy / 4 (2-D),
// shifted by the class's offset r[k]; k and r[k] are the same in every
// lane, so the shift is a uniform branch over three 16-byte loads.
template <int NDIM>
struct ClassBoxRows {
  const uint8_t *box;
  int bx, by;
  uint32_t r0[2];                // R0 mod 4 of the tile's planes (2-D: [0])
  uint32_t shift;                // r[k] for k = 0..3, two bits each
  __device__ __forceinline__ void row(int p, int iy, int, float (&f)[8]) const {
    const uint32_t k = (r0[NDIM == 3 ? p : 0] + (uint32_t)iy) & 3u;
    const uint32_t sh = (shift >> (2 * k)) & 3u;
    const uint8_t *rowp;
    if constexpr (NDIM == 3)
      rowp = box + (p * 4 + k) * kClassBox3 + by * (kClassRow3 * 4) + bx * 32;
    else
      rowp = box + k * kClassBox2 + (2 * by + (iy >> 2)) * (kClassRow2 * 4) + bx * 32;
    const float4 u = *reinterpret_cast<const float4 *>(rowp);
    const float4 v = *reinterpret_cast<const float4 *>(rowp + 16);
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (sh != 0) w = *reinterpret_cast<const float4 *>(rowp + 32);   // uniform
    const float e[12] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w, w.x, w.y, w.z, w.w};
    switch (sh) {
      case 0:
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] = e[j];
        break;
      case 1:
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] = e[j + 1];
        break;
      case 2:
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] = e[j + 2];
        break;
      default:
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] = e[j + 3];
        break;
    }
  }
};

// The neighbours the first Lorenzo difference needs from the previous tile
// of the chunk (3-D: the previous plane under the brick, 2-D: the row
// before the brick for by == 0 lanes), read from global memory before the
// tile's own data is waited for.  A chunk's first tile has none.
template <int NDIM, int V, bool WHOLE = false>
__device__ __forceinline__ void load_halo(const CompressArgs &a, const TileGeo &q,
                                          float (&hf)[32]) {
#pragma unroll
  for (int k = 0; k < 32; ++k) hf[k] = 0.0f;
  const GlobalRows<NDIM, V> src{a, q};
  if constexpr (NDIM == 3) {
    if (march_halo<NDIM, WHOLE>(q)) {
#pragma unroll
      for (int iy = 0; iy < 4; ++iy) {
        float h8[8];
        src.row(-1, iy, 0, h8);
#pragma unroll
        for (int k = 0; k < 8; ++k) hf[8 * iy + k] = h8[k];
      }
    }
  } else if constexpr (NDIM == 2) {
    if (march_halo<NDIM, WHOLE>(q) && q.by == 0) {
      float h8[8];
      src.row(0, -1, 0, h8);
#pragma unroll
      for (int k = 0; k < 8; ++k) hf[k] = h8[k];
    }
  }
}

// Part 1 of a brick's residuals: read the brick, pre-quantise (Sec. 2.3) and
// take the first difference against the preloaded neighbours hf (a chunk's
// first tile has none: q = 0 there).  CHECK folds the unsigned maximum of
// (bits - kBiasBits) into qmax, checking the value range per element
// (absolute bounds; with a relative bound the range pass has shown that every
// element passes).
template <int NDIM, bool CHECK, class Src, bool WIDE = false>
__device__ __forceinline__ void residuals_first(const Src &src, const TileGeo &q, int g,
                                                float r, const float (&hf)[32],
                                                int32_t (&v)[64], uint32_t &qmax) {
  constexpr bool wide = WIDE;
  const unsigned full = 0xffffffffu;
  if constexpr (NDIM == 3) {
#pragma unroll
    for (int iy = 0; iy < 4; ++iy) {                 // D_z, one row at a time
      float p0[8], p1[8];
      src.row(0, iy, 0, p0);
      src.row(1, iy, 0, p1);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int32_t q0 = quant_bits(p0[k], r, wide), q1 = quant_bits(p1[k], r, wide);
        const int32_t qh = quant_bits(hf[8 * iy + k], r, wide);   // hf = 0 when t == 0: q = 0
        if (CHECK) qmax = max(qmax, max((uint32_t)q0 - kBiasBits, (uint32_t)q1 - kBiasBits));
        v[8 * iy + k] = q0 - qh;
        v[32 + 8 * iy + k] = q1 - q0;
      }
    }
  } else if constexpr (NDIM == 2) {
#pragma unroll
    for (int row = 0; row < 8; ++row) {
      float f8[8];
      src.row(0, row, 0, f8);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        v[8 * row + k] = quant_bits(f8[k], r, wide);
        if (CHECK) qmax = max(qmax, (uint32_t)v[8 * row + k] - kBiasBits);
      }
    }
#pragma unroll
    for (int ix = 0; ix < 8; ++ix) {                 // D_y
      int32_t up = __shfl_up_sync(full, v[ix + 56], 8);
      if (q.by == 0) up = quant_bits(hf[ix], r, wide);        // hf = 0 when t == 0: q = 0
#pragma unroll
      for (int iy = 7; iy >= 1; --iy) v[ix + 8 * iy] -= v[ix + 8 * (iy - 1)];
      v[ix] -= up;
    }
  } else {
#pragma unroll
    for (int row = 0; row < 8; ++row) {
      float f8[8];
      src.row(0, 0, 8 * row, f8);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        v[8 * row + k] = quant_bits(f8[k], r, wide);
        if (CHECK) qmax = max(qmax, (uint32_t)v[8 * row + k] - kBiasBits);
      }
    }
  }
}

// ---- the compute path's residuals in fp32 ------------------------------
// The biased quantised values Q = fl(fl(x * r) + 1.5 * 2^23) are integers in
// [2^23 + 1, 2^24 - 1] (|q| <= 2^22 - 1), exact as floats, and so are their
// Lorenzo differences while a result stays within 2^24 in magnitude: a first
// difference is below 2^23, a second below 2^24.  A third (3-D) may round
// only beyond 2^24, where the residual is an escape either way (the escape
// path recomputes such a tile in integers).  Pairs of x-neighbours go through
// the packed f32x2 pipe: the multiply, the rounding add and the differences.
// The rounding add fl(p + 1.5 * 2^23) is a paired FMA with the exact factor
// 1: a paired multiply followed by a paired add is contracted into one fused
// multiply-add by this toolchain, even with explicit .rn, which rounds the
// exact product instead of fl(x * r) and changes q where fl(x * r) falls on a
// tie; an FMA whose product is already an FMA operand is left alone.
__device__ __forceinline__ float2 quant_pair(float x0, float x1, float r) {
  float p0, p1;
  asm("{\n .reg .b64 xa, ra, pa;\n mov.b64 xa, {%2, %3};\n mov.b64 ra, {%4, %4};\n"
      " mul.rn.f32x2 pa, xa, ra;\n mov.b64 {%0, %1}, pa;\n}"
      : "=f"(p0), "=f"(p1)
      : "f"(x0), "f"(x1), "f"(r));
  return __ffma2_rn(make_float2(p0, p1), make_float2(1.0f, 1.0f),
                    make_float2(kRoundMagic, kRoundMagic));
}
__device__ __forceinline__ float2 sub_pair(float2 a, float2 b) {   // a - b, one rounding
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
template <bool CHECK>
__device__ __forceinline__ void check_pair(float2 Q, uint32_t &qmax) {
  if (CHECK)
    qmax = max(qmax, max(__float_as_uint(Q.x) - kBiasBits, __float_as_uint(Q.y) - kBiasBits));
}

// Part 1 in fp32: pre-quantisation and the first difference (3-D: D_z
// against the preloaded plane hf; 2-D: D_y, with the row above the brick
// from the lane above or, for by == 0, from hf; 1-D: none).  v[i] holds
// codes 2i, 2i+1.
template <int NDIM, bool CHECK, class Src>
__device__ __forceinline__ void residuals_first_f(const Src &src, const TileGeo &q, float r,
                                                  const float (&hf)[32], float2 (&v)[32],
                                                  uint32_t &qmax) {
  const unsigned full = 0xffffffffu;
  if constexpr (NDIM == 3) {
#pragma unroll
    for (int iy = 0; iy < 4; ++iy) {
      float p0[8], p1[8];
      src.row(0, iy, 0, p0);
      src.row(1, iy, 0, p1);
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        const float2 q0 = quant_pair(p0[k], p0[k + 1], r);
        const float2 q1 = quant_pair(p1[k], p1[k + 1], r);
        const float2 qh = quant_pair(hf[8 * iy + k], hf[8 * iy + k + 1], r);  // hf = 0: q = 0
        check_pair<CHECK>(q0, qmax);
        check_pair<CHECK>(q1, qmax);
        v[(8 * iy + k) / 2] = sub_pair(q0, qh);
        v[(32 + 8 * iy + k) / 2] = sub_pair(q1, q0);
      }
    }
  } else if constexpr (NDIM == 1) {
#pragma unroll
    for (int row = 0; row < 8; ++row) {
      float f8[8];
      src.row(0, 0, 8 * row, f8);
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        v[(8 * row + k) / 2] = quant_pair(f8[k], f8[k + 1], r);
        check_pair<CHECK>(v[(8 * row + k) / 2], qmax);
      }
    }
  } else {
#pragma unroll
    for (int row = 0; row < 8; ++row) {
      float f8[8];
      src.row(0, row, 0, f8);
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        v[(8 * row + k) / 2] = quant_pair(f8[k], f8[k + 1], r);
        check_pair<CHECK>(v[(8 * row + k) / 2], qmax);
      }
    }
#pragma unroll
    for (int ix = 0; ix < 8; ix += 2) {            // D_y
      float2 up;
      up.x = __shfl_up_sync(full, v[(ix + 56) / 2].x, 8);
      up.y = __shfl_up_sync(full, v[(ix + 56) / 2].y, 8);
      if (q.by == 0) up = quant_pair(hf[ix], hf[ix + 1], r);   // hf = 0 when t == 0: q = 0
#pragma unroll
      for (int iy = 7; iy >= 1; --iy)
        v[(ix + 8 * iy) / 2] = sub_pair(v[(ix + 8 * iy) / 2], v[(ix + 8 * (iy - 1)) / 2]);
      v[ix / 2] = sub_pair(v[ix / 2], up);
    }
  }
}

// Part 2 in fp32: the remaining differences (3-D: D_y, then D_x; 2-D: D_x;
// 1-D: D_x along the lane's 64 elements, whose left neighbour is the
// previous lane's last, or for lane 0 the element before the tile).
template <int NDIM, bool WHOLE = false>
__device__ __forceinline__ void residuals_rest_f(const CompressArgs &a, const TileGeo &q, int g,
                                                 float r, float2 (&v)[32]) {
  const unsigned full = 0xffffffffu;
  if constexpr (NDIM == 1) {
    float hq = kRoundMagic;                          // q = 0 before a chunk's first element
    if (march_halo<NDIM, WHOLE>(q) && g == 0)
      hq = quant_pair((q.x0 - 1 < a.dims[0]) ? __ldcs(a.x + q.x0 - 1) : 0.0f, 0.0f, r).x;
    float left = __shfl_up_sync(full, v[31].y, 1);
    if (g == 0) left = hq;
#pragma unroll
    for (int j = 31; j >= 1; --j) {
      v[j].y = __fsub_rn(v[j].y, v[j].x);
      v[j].x = __fsub_rn(v[j].x, v[j - 1].y);
    }
    v[0].y = __fsub_rn(v[0].y, v[0].x);
    v[0].x = __fsub_rn(v[0].x, left);
    return;
  }
  if constexpr (NDIM == 3) {
#pragma unroll
    for (int iz = 0; iz < 2; ++iz) {               // D_y
#pragma unroll
      for (int ix = 0; ix < 8; ix += 2) {
        float2 up;
        up.x = __shfl_up_sync(full, v[(ix + 24 + 32 * iz) / 2].x, 4);
        up.y = __shfl_up_sync(full, v[(ix + 24 + 32 * iz) / 2].y, 4);
        if (q.by == 0)
          up = WHOLE && q.y0 > 0 ? make_float2(face_up3(a, q, ix, iz, r), face_up3(a, q, ix + 1, iz, r))
                                   : make_float2(0.f, 0.f);
#pragma unroll
        for (int iy = 3; iy >= 1; --iy)
          v[(ix + 8 * iy + 32 * iz) / 2] =
              sub_pair(v[(ix + 8 * iy + 32 * iz) / 2], v[(ix + 8 * (iy - 1) + 32 * iz) / 2]);
        v[(ix + 32 * iz) / 2] = sub_pair(v[(ix + 32 * iz) / 2], up);
      }
    }
  }
#pragma unroll
  for (int row = 0; row < 8; ++row) {              // D_x: element 2j+1 - 2j, 2j - (2j-1)
    float left = __shfl_up_sync(full, v[4 * row + 3].y, 1);
    if (q.bx == 0)
      left = !(WHOLE && q.x0 > 0) ? 0.f
             : NDIM == 3            ? face_left3(a, q, row % 4, row / 4, r)
                                    : face_left2(a, q, row, r);
#pragma unroll
    for (int j = 3; j >= 1; --j) {
      v[4 * row + j].y = __fsub_rn(v[4 * row + j].y, v[4 * row + j].x);
      v[4 * row + j].x = __fsub_rn(v[4 * row + j].x, v[4 * row + j - 1].y);
    }
    v[4 * row].y = __fsub_rn(v[4 * row].y, v[4 * row].x);
    v[4 * row].x = __fsub_rn(v[4 * row].x, left);
  }
}

// Pairs of 16-bit sign-magnitude codes (Sec. 3.2) from exact float
// residuals: the low 16 bits of |d| + 2^23 are |d| for |d| < 2^16, the sign
// is the float's (a difference of equal values is +0, never -0).  Returns
// the OR of the bits of |d| + 2^23: within 0x4B00007F when every |d| < 128,
// within 0x4B007FFF when no residual escapes.
__device__ __forceinline__ uint32_t pack_codes_f(const float2 (&v)[32], uint32_t (&w)[32]) {
  uint32_t o = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const uint32_t m0 = __float_as_uint(__fadd_rn(fabsf(v[i].x), 8388608.0f));
    const uint32_t m1 = __float_as_uint(__fadd_rn(fabsf(v[i].y), 8388608.0f));
    o |= m0 | m1;
    const uint32_t mag = byte_perm(m0, m1, 0x5410);
    const uint32_t sgn = byte_perm(__float_as_uint(v[i].x), __float_as_uint(v[i].y), 0x7030);
    w[i] = mag | (sgn & 0x80008000u);
  }
  return o;
}

// residual 0 (code 0) for the padding positions of a tile that reaches
// past the field
template <int NDIM>
__device__ __forceinline__ void mask_padding(const CompressArgs &a, const TileGeo &q,
                                             float2 (&v)[32]) {
  using G = Geo<NDIM>;
  const uint64_t lx = q.x0 < a.dims[0] ? a.dims[0] - q.x0 : 0;
  const uint64_t ly = q.y0 < a.dims[1] ? a.dims[1] - q.y0 : 0;
  const uint64_t lz = q.z0 < a.dims[2] ? a.dims[2] - q.z0 : 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int ix = (2 * i) % G::BX, iy = (2 * i / G::BX) % G::BY, iz = 2 * i / (G::BX * G::BY);
    const bool row = (uint64_t)iy < ly && (uint64_t)iz < lz;
    if (!(row && (uint64_t)ix < lx)) v[i].x = 0.f;
    if (!(row && (uint64_t)ix + 1 < lx)) v[i].y = 0.f;
  }
}

// Part 2: the remaining differences (no more input reads) and code 0 for
// padding positions.
template <int NDIM, bool WHOLE = false, bool WIDE = false>
__device__ __forceinline__ void residuals_rest(const CompressArgs &a, const TileGeo &q, int g,
                                               float r, int32_t (&v)[64]) {
  constexpr bool wide = WIDE;
  using G = Geo<NDIM>;
  const unsigned full = 0xffffffffu;
  if constexpr (NDIM == 3) {
#pragma unroll
    for (int iz = 0; iz < 2; ++iz) {                 // D_y
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) {
        int32_t up = __shfl_up_sync(full, v[ix + 24 + 32 * iz], 4);
        if (q.by == 0)
          up = WHOLE && q.y0 > 0 ? qi_at(a, q.x0 + ix, q.y0 - 1, q.z0 + iz, r, wide) -
                                         qi_at(a, q.x0 + ix, q.y0 - 1, q.z0 + iz - 1, r, wide)
                                   : 0;
#pragma unroll
        for (int iy = 3; iy >= 1; --iy) v[ix + 8 * iy + 32 * iz] -= v[ix + 8 * (iy - 1) + 32 * iz];
        v[ix + 32 * iz] -= up;
      }
    }
  }
  if constexpr (NDIM >= 2) {
#pragma unroll
    for (int row = 0; row < 8; ++row) {              // D_x
      int32_t left = __shfl_up_sync(full, v[7 + 8 * row], 1);
      if (q.bx == 0) {
        left = 0;
        if (WHOLE && q.x0 > 0) {
          // the column before the brick, differenced like the brick's rows
          const uint64_t x = q.x0 - 1;
          const int iy = NDIM == 3 ? row % 4 : row, iz = NDIM == 3 ? row / 4 : 0;
          const uint64_t y = q.y0 + iy, z = q.z0 + iz;
          left = qi_at(a, x, y, z, r, wide) - qi_at(a, x, y - 1, z, r, wide);
          if (NDIM == 3)
            left -= qi_at(a, x, y, z - 1, r, wide) - qi_at(a, x, y - 1, z - 1, r, wide);
        }
      }
#pragma unroll
      for (int ix = 7; ix >= 1; --ix) v[ix + 8 * row] -= v[ix - 1 + 8 * row];
      v[8 * row] -= left;
    }
  } else {
    int32_t hq = (int32_t)kMagicBits;
    if (march_halo<NDIM, WHOLE>(q) && g == 0)
      hq = quant_bits((q.x0 - 1 < a.dims[0]) ? __ldcs(a.x + q.x0 - 1) : 0.0f, r, wide);
    int32_t left = __shfl_up_sync(full, v[63], 1);
    if (g == 0) left = hq;
#pragma unroll
    for (int e = 63; e >= 1; --e) v[e] -= v[e - 1];
    v[0] -= left;
  }
  if (q.edge) {
    const uint64_t X = a.dims[0];
    const uint64_t lx = q.x0 < X ? X - q.x0 : 0;
    const uint64_t ly = q.y0 < a.dims[1] ? a.dims[1] - q.y0 : 0;
    const uint64_t lz = q.z0 < a.dims[2] ? a.dims[2] - q.z0 : 0;
#pragma unroll
    for (int e = 0; e < 64; ++e) {
      const int ix = e % G::BX, iy = (e / G::BX) % G::BY, iz = e / (G::BX * G::BY);
      if (!((uint64_t)ix < lx && (uint64_t)iy < ly && (uint64_t)iz < lz)) v[e] = 0;
    }
  }
}

// all residuals from global memory (the rare escape repack and the outlier
// pass, when the TMA box no longer holds the tile)
template <int NDIM, int V, bool WHOLE = false, bool WIDE = false>
__device__ __forceinline__ void residuals_global(const CompressArgs &a, uint64_t T, int g,
                                                 float r, int32_t (&v)[64]) {
  const TileGeo q = tile_geo<NDIM>(a, ChunkGrid(a), T, g);
  uint32_t unused = 0;
  float hf[32];
  load_halo<NDIM, V, WHOLE>(a, q, hf);
  residuals_first<NDIM, false, GlobalRows<NDIM, V>, WIDE>(GlobalRows<NDIM, V>{a, q}, q, g, r, hf,
                                                          v, unused);
  residuals_rest<NDIM, WHOLE, WIDE>(a, q, g, r, v);
}

// residuals -> pairs of 16-bit sign-magnitude codes (Sec. 3.2), even code in
// the low half.  Returns the OR of |residual| (bit 15 or above set: escapes).
__device__ __forceinline__ uint32_t pack_codes(const int32_t (&v)[64], uint32_t (&w)[32]) {
  uint32_t orabs = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int32_t d0 = v[2 * i], d1 = v[2 * i + 1];
    const uint32_t a0 = (uint32_t)abs(d0), a1 = (uint32_t)abs(d1);
    orabs |= a0 | a1;
    const uint32_t mag = byte_perm(a0, a1, 0x5410);             // |d0| | |d1|<<16
    const uint32_t sgn = byte_perm((uint32_t)d0, (uint32_t)d1, 0x7030);
    w[i] = mag | (sgn & 0x80008000u);
  }
  return orabs;
}

// escape: a residual whose magnitude needs more than 15 bits gets 0x8000
__device__ __forceinline__ uint32_t pack_codes_escaped(const int32_t (&v)[64], uint32_t (&w)[32]) {
  uint32_t n = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int32_t d0 = v[2 * i], d1 = v[2 * i + 1];
    const uint32_t a0 = (uint32_t)abs(d0), a1 = (uint32_t)abs(d1);
    uint32_t c0 = a0 | ((uint32_t)(d0 >> 16) & 0x8000u);
    uint32_t c1 = a1 | ((uint32_t)(d1 >> 16) & 0x8000u);
    n += (a0 > 32767u) + (a1 > 32767u);
    c0 = a0 > 32767u ? 0x8000u : c0;
    c1 = a1 > 32767u ? 0x8000u : c1;
    w[i] = byte_perm(c0, c1, 0x5410);
  }
  return n;
}

// The rare escape path, kept out of the hot loop: recompute the lane's
// residuals from global memory, pack them with escapes into pb[32g..32g+31]
// and return the lane's escape count.
template <int NDIM, int V, bool WHOLE = false, bool WIDE = false>
__device__ __forceinline__ uint32_t escape_repack(const CompressArgs &a, uint64_t T, int g, float r,
                                               uint32_t *pb) {
  int32_t v[64];
  residuals_global<NDIM, V, WHOLE, WIDE>(a, T, g, r, v);
  uint32_t w[32];
  const uint32_t n = pack_codes_escaped(v, w);
#pragma unroll
  for (int i = 0; i < 32; ++i) pb[32 * g + i] = w[i];
  __syncwarp();
  return n;
}

// TMA box of tile T for this warp: 3-D {32,32,2} (the tile's two planes),
// 2-D two {32,32} x halves of the tile's 32 rows
template <int NDIM>
__device__ __forceinline__ void issue_box(const CompressArgs &a, const ChunkGrid &cg,
                                          const CUtensorMap *tm, uint8_t *box, uint64_t *bar,
                                          uint64_t T) {
  const uint32_t c = (uint32_t)(T >> 2);
  const int t = (int)(T & 3);
  const uint32_t r = cg.x.div(c);
  const uint32_t cx = c - r * cg.x.d, cz = cg.y.div(r), cy = r - cz * cg.y.d;
  mbar_expect_tx(bar, kTileBoxBytes);
  if constexpr (NDIM == 3) {
    tma_load_3d(box, tm, bar, (int)(cx * 32), (int)(cy * 32), (int)(cz * 8 + 2 * t));
  } else {
    const int y = (int)(cy * 128 + 32 * t);
    tma_load_2d(box, tm, bar, (int)(cx * 64), y);
    tma_load_2d(box + kHalf2D, tm, bar, (int)(cx * 64 + 32), y);
  }
}

// The row-class boxes of tile T (fields whose rows are not 16-byte
// aligned; the four class maps cm[0..3] are 2-D, x then row-of-class).
// Every box starts at the tile's x origin (a multiple of 32 floats, so
// 16-byte aligned in the map) and at the class's first row at or after the
// tile's first row R0 on the plane; rows past the field read as zero, and
// rows of the next plane that a tile reaching past y = Y picks up are
// padding the kernel masks.
template <int NDIM>
__device__ __forceinline__ void issue_class_boxes(const CompressArgs &a, const ChunkGrid &cg,
                                                  const CUtensorMap *cm, uint8_t *box,
                                                  uint64_t *bar, uint64_t T) {
  const uint32_t c = (uint32_t)(T >> 2);
  const int t = (int)(T & 3);
  const uint32_t r = cg.x.div(c);
  const uint32_t cx = c - r * cg.x.d, cz = cg.y.div(r), cy = r - cz * cg.y.d;
  if constexpr (NDIM == 3) {
    mbar_expect_tx(bar, 8 * kClassBox3);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const uint64_t R0 = (uint64_t)cy * 32 + a.dims[1] * ((uint64_t)cz * 8 + 2 * t + p);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        tma_load_2d(box + (p * 4 + k) * kClassBox3, cm + k, bar, (int)(cx * 32),
                    (int)((R0 + 3 - k) / 4));
    }
  } else {
    mbar_expect_tx(bar, 4 * kClassBox2);
    const uint64_t R0 = (uint64_t)cy * 128 + 32 * t;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      tma_load_2d(box + k * kClassBox2, cm + k, bar, (int)(cx * 64), (int)((R0 + 3 - k) / 4));
  }
}

// the compacted blocks of a finished tile, stored in a later round
struct Pending {
  uint32_t T;          // tile index in its field (kNoTile: none; < 2^21)
  uint32_t field;      // its field (batches)
  uint64_t agg;        // (blocks << 32) | outliers
  uint32_t round;      // the block round it belongs to (its ring end: round & 1)
};
constexpr uint32_t kNoTile = 0xFFFFFFFFu;

// a ring block's place: the 16-byte column within its 128-byte row XORed
// with the row, so that lanes writing runs of blocks that start 8 apart
// (dense planes) hit distinct banks
__device__ __forceinline__ uint32_t ring_slot(uint32_t k) { return k ^ ((k >> 3) & 7u); }
// the first block of a tile of n blocks at ring end e
template <bool BATCH>
__device__ __forceinline__ uint32_t ring_base(uint32_t e, uint32_t n) {
  return e ? (uint32_t)ring_blocks<BATCH>() - n : 0u;
}

// Take a finished tile's exclusive prefix from the scan warp and store its
// compacted blocks (Listing 2's copy: block (b, i) -> payload[PreSum]); the
// blocks lie in rank order in the ring, so the copy is contiguous.
template <int NDIM, bool BATCH>
__device__ __forceinline__ void finish_tile(const CompressArgs &a, CompShared *sh,
                                            const Pending &d, const uint4 *ring,
                                            const FieldRt &rt, int g, int wid) {
  SetScratch *cur = a.set_cur;
  const uint64_t n_tiles = a.n_chunks * kTilesPerChunk;
  const uint64_t pay = 64 + 32 * n_tiles;
  const EbParams &p = rt.p;
  const float fmin = rt.fmin, fmax = rt.fmax;
  const int s = (int)(d.round % kRing);
  uint64_t excl = 0;
  if (warp_wait(&sh->excl_bar[s], (d.round / kRing) & 1u, a.wait_limit_ns)) {
    excl = sh->slot[s].excl[wid];
  } else if (g == 0) {
    atomicOr(&cur->err, kErrTimeout);
  }
  if (g == 0) {
    a.tile_out_prefix[d.T] = (uint32_t)excl;
    a.tile_out_count[d.T] = (uint32_t)d.agg;
    if (d.T == n_tiles - 1) {
      const uint64_t inc = excl + d.agg;
      StreamHeader *h = reinterpret_cast<StreamHeader *>(a.out);
      h->magic[0] = 'F'; h->magic[1] = 'Z'; h->magic[2] = 'G'; h->magic[3] = '1';
      h->version = a.whole ? 2 : 1;         // 2: whole-field residuals
      h->ndim = (uint8_t)NDIM; h->mode = (uint8_t)a.mode;
      h->reserved0 = rt.wide ? kHdrWide : 0;   // the wide quantiser's streams
      h->dims[0] = (uint32_t)a.dims[0]; h->dims[1] = (uint32_t)a.dims[1];
      h->dims[2] = (uint32_t)a.dims[2];
      h->n_tiles = (uint32_t)n_tiles;
      h->eb_requested = a.eb_req;
      h->eb = p.eb; h->ebx2 = p.ebx2; h->ebx2_r = p.ebx2_r;
      h->nnz_blocks = (uint32_t)(inc >> 32);
      h->n_outliers = (uint32_t)inc;
      h->range_min = fmin; h->range_max = fmax;
      h->reserved1 = 0;
      cur->nnz = inc >> 32;
      cur->nout = inc & 0xffffffffull;
    }
  }
  const uint32_t tile_nnz = (uint32_t)(d.agg >> 32);
  const uint32_t base = ring_base<BATCH>(d.round & 1u, tile_nnz);
  uint8_t *const out = a.out;                        // read once: stores follow
  const uint64_t dst = pay + 16 * (excl >> 32);
  if (dst + 16 * (uint64_t)tile_nnz <= a.out_capacity) {
    for (uint32_t k = (uint32_t)g; k < tile_nnz; k += 32)
      __stcs(reinterpret_cast<uint4 *>(out + dst + 16 * (uint64_t)k), ring[ring_slot(base + k)]);
  } else if (g == 0) {
    atomicOr(&cur->err, kErrCapacity);
  }
  __syncwarp();                                      // ring blocks free again
}

// The scan warp's ticket for block round r: a unit index from the launch's
// counter and the unit's field, posted in the ring (lane 0 only).  A single
// field's launch clears the unit's look-back word in the next call's status
// array here (a batch's status words are cleared before its launch).
template <bool BATCH>
__device__ __forceinline__ void post_ticket(const CompressArgs &a0, const BatchArgs &b,
                                            CompShared *sh, uint32_t r, uint64_t n_units) {
  RoundSlot &slot = sh->slot[r % kRing];
  if constexpr (BATCH) {
    const uint64_t u = atomicAdd(b.ticket, 1u);
    const uint2 m = u < n_units ? b.unit_map[u] : make_uint2(0u, 0u);
    slot.unit = u;
    slot.field = m.x;
    slot.local = m.y;
  } else {
    const uint64_t u = atomicAdd(&a0.set_cur->ticket, 1u);
    if (u < n_units) a0.status_next[u * kStatusStride] = 0;
    slot.unit = u;
    slot.field = 0;
    slot.local = (uint32_t)u;
  }
  mbar_arrive(&sh->ticket_bar[r % kRing]);
}

// The scan warp: tickets two rounds ahead, then per round the unit's
// aggregate, its decoupled look-back (in its field's domain) and the tiles'
// exclusive prefixes.  Round r + 2's ticket reuses round r - 2's ring
// entry, which every compute warp has read once round r's aggregates are
// all posted.
template <bool BATCH>
__device__ __forceinline__ void scan_warp(const CompressArgs &a0, const BatchArgs &b,
                                          CompShared *sh, uint64_t n_units, int g) {
  const unsigned full = 0xffffffffu;
  const uint64_t skip_unit = !BATCH && a0.skip_publish_chunk < a0.n_chunks
                                 ? a0.skip_publish_chunk * kTilesPerChunk / kCompWarps
                                 : ~0ull;
  if (g == 0) {
    post_ticket<BATCH>(a0, b, sh, 0, n_units);
    post_ticket<BATCH>(a0, b, sh, 1, n_units);
  }
  for (uint32_t r = 0;; ++r) {
    const int s = (int)(r % kRing);
    __syncwarp();                                    // lane 0's ticket write
    const uint64_t u = sh->slot[s].unit;
    const uint32_t f = sh->slot[s].field, ul = sh->slot[s].local;
    if (u >= n_units) break;
    const CompressArgs &a = BATCH ? b.fields[f] : a0;
    SetScratch *cur = a.set_cur;
    if (!warp_wait(&sh->agg_bar[s], (r / kRing) & 1u, a.wait_limit_ns)) {
      if (g == 0) atomicOr(&cur->err, kErrTimeout);
      break;
    }
    const uint64_t t_agg = g < kCompWarps ? sh->slot[s].agg[g] : 0;
    uint64_t inc = t_agg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(full, inc, o);
      if (g >= o) inc += y;
    }
    const uint64_t total = __shfl_sync(full, inc, 31);
    const bool publish = ul != skip_unit;
    publish_aggregate(a.status_cur, ul, total, publish);
    // The ticket for round r + 2 is taken once this block has finished
    // round r (and published the round's aggregate, which later units' look-
    // backs wait for): the later units are handed out, the closer their
    // order is to the order in which blocks finish them, and the less a
    // look-back waits for a predecessor's aggregate.  (Taken earlier, or by
    // a compute warp at the start of a round, the compressor ran 1 to 6%
    // slower; taken before the publication, 1% slower.)
    if (g == 0) post_ticket<BATCH>(a0, b, sh, r + 2, n_units);
    // 4 words per lane: a window of 128 units per round trip
    const uint64_t excl =
        resolve_prefix<4>(a.status_cur, ul, total, publish, &cur->err, a.wait_limit_ns);
    if (g < kCompWarps) {
      sh->slot[s].excl[g] = excl + inc - t_agg;
      mbar_arrive(&sh->excl_bar[s]);
    }
  }
}

// One block per SM.  A single field's launch (BATCH = false) reads its field
// from the kernel parameters; a batched launch reads each unit's field from
// the batch's descriptors.
template <int NDIM, int V, bool CHECK, bool TMA, bool BATCH, bool WHOLE = false,
          bool WIDE = false>
__global__ void __launch_bounds__(kCompThreads, 1)
    compress_kernel(const CompressArgs a0, const __grid_constant__ CUtensorMap tmap0,
                    const BatchArgs b) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const unsigned full = 0xffffffffu;
  const int g = threadIdx.x & 31, wid = threadIdx.x >> 5;
  grid_dependency_wait();                // a preceding range pass's result
  grid_launch_dependents();              // the launch after this one may be scheduled
  // [TMA boxes] [rings] [CompShared] [WarpField per compute warp (batches)]
  constexpr int kBox = TMA ? box_bytes<BATCH>() : 0;
  constexpr int kRingOff = kCompWarps * kBox;
  CompShared *sh = reinterpret_cast<CompShared *>(smem + comp_area_bytes<TMA, BATCH>());
  WarpField *wfield = reinterpret_cast<WarpField *>(
      smem + comp_area_bytes<TMA, BATCH>() + kCompShBytes +
      (wid < kCompWarps ? wid : 0) * kWarpFieldBytes);

  uint64_t n_units;
  FieldRt rt0{};
  if constexpr (BATCH) {
    n_units = b.n_units;
  } else {
    n_units = (a0.n_chunks * kTilesPerChunk + kCompWarps - 1) / kCompWarps;
    uint32_t err = 0;
    rt0 = derive_field(a0, err);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (err) atomicOr(&a0.set_cur->err, err);
      SetScratch *nx = a0.set_next;                  // the next call's block
      nx->ticket = 0; nx->err = 0; nx->nnz = 0; nx->nout = 0;
      nx->n_chunks = 0; nx->hdr_nout = 0;
    }
    if (!rt0.ok) return;                             // the same in every thread
  }

  if (threadIdx.x == 0) {
    for (int i = 0; i < kCompWarps; ++i) mbar_init(&sh->box_bar[i], 1);
    for (int i = 0; i < kRing; ++i) {
      mbar_init(&sh->ticket_bar[i], 1);
      mbar_init(&sh->agg_bar[i], kCompWarps);
      mbar_init(&sh->excl_bar[i], kCompWarps);
    }
  }
  __syncthreads();
  if (wid == kCompWarps) {
    scan_warp<BATCH>(a0, b, sh, n_units, g);
    return;
  }

  // ---- compute warp
  uint8_t *box = smem + wid * kBox;
  uint4 *const ring = reinterpret_cast<uint4 *>(smem + kRingOff + wid * ring_bytes<BATCH>());
  uint64_t *bar = &sh->box_bar[wid];
  // a unit's tile for this warp, and whether this warp computes it (the
  // unit exists, the tile lies in the field and the field can be quantised)
  struct Work {
    uint64_t u;
    uint32_t T, field;             // T < 2^21: tiles of one field
    bool run;
  };
  auto work_of = [&](int s) {
    Work w;
    w.u = sh->slot[s].unit;
    w.field = BATCH ? sh->slot[s].field : 0u;
    w.T = sh->slot[s].local * kCompWarps + wid;
    w.run = false;
    if (w.u < n_units) {
      if constexpr (BATCH) {
        w.run = w.T < b.fields[w.field].n_chunks * kTilesPerChunk && b.rt[w.field].ok;
      } else {
        w.run = w.T < a0.n_chunks * kTilesPerChunk;
      }
    }
    return w;
  };
  auto rt_of = [&](uint32_t f) -> FieldRt { return BATCH ? b.rt[f] : rt0; };
  // whether a unit's tile comes by TMA (a batch decides per field: rows
  // 16-byte aligned; the others read global memory directly)
  auto tma_of = [&](const Work &w) -> bool {
    if constexpr (!TMA) return false;
    else if constexpr (BATCH) return w.run && b.fields[w.field].use_tma != 0;
    else return w.run;
  };
  auto issue = [&](const Work &w) {
    if constexpr (TMA) {
      const FieldRt rt = rt_of(w.field);
      fence_proxy_async_smem();          // earlier generic reads of the box first
      bool cls = false;
      if constexpr (BATCH && NDIM >= 2) cls = b.fields[w.field].use_tma == 2;
      if (cls)
        issue_class_boxes<NDIM>(b.fields[w.field], ChunkGrid(rt.dx, rt.dy), &b.cmaps[4 * w.field],
                                box, bar, w.T);
      else
        issue_box<NDIM>(BATCH ? b.fields[w.field] : a0, ChunkGrid(rt.dx, rt.dy),
                        BATCH ? &b.tmaps[w.field] : &tmap0, box, bar, w.T);
    }
  };

  Work cw{n_units, 0u, 0u, false};
  if (warp_wait(&sh->ticket_bar[0], 0, a0.wait_limit_ns)) cw = work_of(0);
  else if (g == 0) atomicOr(&a0.set_cur->err, kErrTimeout);
  uint32_t phase = 0;
  if constexpr (TMA) {
    if (g == 0 && tma_of(cw)) issue(cw);
    __syncwarp();
  }
  Pending prev1{kNoTile, 0, 0, 0};                  // last round's tile (the other end)
  Pending prev2{kNoTile, 0, 0, 0};                  // the round before's (this round's end)
  auto finish = [&](Pending &d) {
    finish_tile<NDIM, BATCH>(BATCH ? b.fields[d.field] : a0, sh, d, ring, rt_of(d.field), g, wid);
    d.T = kNoTile;
  };
  uint32_t cached = ~0u;                             // the field in wfield (batches)
  for (uint32_t r = 0; cw.u < n_units; ++r) {
    const int s = (int)(r % kRing);
    const uint64_t T = cw.T;
    // the next round's unit (the scan warp posts tickets two rounds ahead)
    Work nw{n_units, 0u, 0u, false};
    auto next_unit = [&] {
      const int s1 = (int)((r + 1) % kRing);
      if (warp_wait(&sh->ticket_bar[s1], ((r + 1) / kRing) & 1u, a0.wait_limit_ns))
        nw = work_of(s1);
      else if (g == 0)
        atomicOr(&a0.set_cur->err, kErrTimeout);
    };
    uint64_t agg = 0;
    const uint32_t e = r & 1u;                       // this round's end of the ring
    if (cw.run) {
      if constexpr (BATCH) {
        if (cw.field != cached) {                    // this warp's field changed
          constexpr int kWords = (int)(sizeof(WarpField) / 8);
          const uint64_t *src_a = reinterpret_cast<const uint64_t *>(&b.fields[cw.field]);
          const uint64_t *src_r = reinterpret_cast<const uint64_t *>(&b.rt[cw.field]);
          uint64_t *dst = reinterpret_cast<uint64_t *>(wfield);
          constexpr int kA = (int)(sizeof(CompressArgs) / 8), kR = (int)(sizeof(FieldRt) / 8);
          for (int i = g; i < kA; i += 32) dst[i] = src_a[i];
          for (int i = g; i < kR; i += 32)
            reinterpret_cast<uint64_t *>(&wfield->rt)[i] = src_r[i];
          (void)kWords;
          __syncwarp();
          cached = cw.field;
        }
      }
      const CompressArgs &a = BATCH ? wfield->a : a0;
      const FieldRt rt = BATCH ? wfield->rt : rt0;
      const ChunkGrid cg(rt.dx, rt.dy);
      SetScratch *cur = a.set_cur;
      const TileGeo q = tile_geo<NDIM>(a, cg, T, g);
      uint32_t w[32];
      bool narrow, escape;
      if constexpr (WIDE) {
        // the wide quantiser: every tile takes the integer path below
        (void)q;
        next_unit();
        if (g == 0 && tma_of(nw)) issue(nw);
        narrow = false;
        escape = true;
      } else {
      float hf[32];
      // a batch's one-box TMA fields have 16-byte aligned rows: vector halo
      // loads (the row-class fields' rows are not aligned)
      const int tmode = BATCH ? (tma_of(cw) ? a.use_tma : 0) : (TMA ? 1 : 0);
      if (BATCH && V < 4 && tmode == 1) load_halo<NDIM, 4>(a, q, hf);
      else load_halo<NDIM, V, WHOLE>(a, q, hf);
      float2 vf[32];                                // fp32 residuals, codes 2i, 2i+1 in vf[i]
      uint32_t qmax = 0;
      // a single field's launch compiles one load path; a batch picks per field
      if (tmode != 0) {
        if (!mbar_wait_bounded(bar, phase, a0.wait_limit_ns) && g == 0)
          atomicOr(&cur->err, kErrTimeout);
        phase ^= 1u;
        bool done = false;
        if constexpr (BATCH && NDIM >= 2) {
          if (tmode == 2) {
            // row classes: each class's offset from 16 bytes, and the class
            // of the tile's first row on each plane
            ClassBoxRows<NDIM> cr{box, q.bx, q.by, {0u, 0u}, 0u};
            const uint64_t xw = reinterpret_cast<uintptr_t>(a.x) >> 2;
#pragma unroll
            for (int k = 0; k < 4; ++k)
              cr.shift |= (uint32_t)((xw + k * a.pitch) & 3u) << (2 * k);
            cr.r0[0] = (uint32_t)((q.y0 + (NDIM == 3 ? a.dims[1] * q.z0 : 0)) & 3u);
            cr.r0[1] = (uint32_t)((q.y0 + a.dims[1] * (q.z0 + 1)) & 3u);
            residuals_first_f<NDIM, CHECK>(cr, q, rt.p.ebx2_r, hf, vf, qmax);
            done = true;
          }
        }
        if (!done)
          residuals_first_f<NDIM, CHECK>(BoxRows<NDIM>{box, q.bx, q.by}, q, rt.p.ebx2_r, hf, vf,
                                         qmax);
        __syncwarp();                    // every lane is done with the box
      } else {
        residuals_first_f<NDIM, CHECK>(GlobalRows<NDIM, V>{a, q}, q, rt.p.ebx2_r, hf, vf, qmax);
      }
      // the box is free: fetch the next round's tile into it while this one
      // is finished
      next_unit();
      if (g == 0 && tma_of(nw)) issue(nw);
      residuals_rest_f<NDIM, WHOLE>(a, q, g, rt.p.ebx2_r, vf);
      if (CHECK && __any_sync(full, qmax > kBiasedMax) && g == 0) atomicOr(&cur->err, kErrRange);

      // narrow: every code of the tile fits in 7 bits and the sign, so the
      // planes of magnitude bits 7..14 are zero and half the transpose is
      // skipped; escape: some |residual| needs more than 15 bits
      if (q.edge) mask_padding<NDIM>(a, q, vf);
      const uint32_t o = pack_codes_f(vf, w);        // vf is dead from here on
      narrow = !__any_sync(full, (o & ~0x4B00007Fu) != 0u);
      escape = __any_sync(full, (o & ~0x4B007FFFu) != 0u);
      }
      // this end of the ring: store the tile of two rounds back that waits
      // there, and make the last round's tile at the other end leave the
      // staging area free
      if (prev2.T != kNoTile) finish(prev2);
      if (prev1.T != kNoTile &&
          (uint32_t)(prev1.agg >> 32) > (uint32_t)(ring_blocks<BATCH>() - kStageBlocks))
        finish(prev1);
      uint32_t *const pb =
          reinterpret_cast<uint32_t *>(ring + (e ? ring_blocks<BATCH>() - kStageBlocks : 0));
      uint32_t nout_lane = 0;
      if (!narrow && escape) {
        // rare: some |residual| needs more than 15 bits; recompute and repack
        // with escapes out of line (through the staging area)
        nout_lane = escape_repack<NDIM, V, WHOLE, WIDE>(a, T, g, rt.p.ebx2_r, pb);
#pragma unroll
        for (int i = 0; i < 32; ++i) w[i] = pb[32 * g + i];
        __syncwarp();
      }

      // staging area: lane b collects plane b's 32 words (8 blocks); a
      // narrow tile writes its 16 nonzero planes only
      if (narrow) {
        uint32_t u[16];
        squeeze_narrow(w, u);
        transpose16(u);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int b2 = narrow_row(k);
          pb[32 * b2 + 4 * ((g >> 2) ^ (b2 & 7)) + (g & 3)] = u[k];
        }
      } else {
        transpose32(w);                              // lane g: out[32b + g]
#pragma unroll
        for (int b2 = 0; b2 < 32; ++b2) pb[32 * b2 + 4 * ((g >> 2) ^ (b2 & 7)) + (g & 3)] = w[b2];
      }
      __syncwarp();
      uint4 blk[8];
      uint32_t F = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {                  // lane b: plane b, its flag byte
        blk[i] = *reinterpret_cast<const uint4 *>(pb + 32 * g + 4 * (i ^ (g & 7)));
        F |= ((blk[i].x | blk[i].y | blk[i].z | blk[i].w) != 0u ? 1u : 0u) << i;
      }
      if (narrow && (g & 15) >= 7 && (g & 15) != 15) F = 0;   // rows not written

      const uint32_t pc = __popc(F);
      uint32_t P = pc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, P, o);
        if (g >= o) P += y;
      }
      const uint32_t tile_nnz = __shfl_sync(full, P, 31);
      P -= pc;
      const uint32_t tile_nout = __reduce_add_sync(full, nout_lane);
      a.out[64 + T * 32 + g] = (uint8_t)F;           // Listing 1's flags
      agg = ((uint64_t)tile_nnz << 32) | tile_nout;
      if (g == 0) {
        sh->slot[s].agg[wid] = agg;
        mbar_arrive(&sh->agg_bar[s]);
      }
      // the compacted blocks in rank order over the staging area, once
      // every lane has read its plane
      __syncwarp();
      uint32_t k = ring_base<BATCH>(e, tile_nnz) + P;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if ((F >> i) & 1u) ring[ring_slot(k++)] = blk[i];
      }
      __syncwarp();
    } else {
      next_unit();                                   // no tile here this round
      if (g == 0 && tma_of(nw)) issue(nw);
      if (g == 0) {
        sh->slot[s].agg[wid] = 0;
        mbar_arrive(&sh->agg_bar[s]);
      }
    }
    // a round without a tile stored nothing: store the tile at this end now,
    // so that at most two tiles stay pending
    if (prev2.T != kNoTile) finish(prev2);
    prev2 = prev1;
    prev1 = Pending{cw.run ? (uint32_t)T : kNoTile, BATCH ? cw.field : 0u, agg, r};
    cw = nw;
  }
  if (prev2.T != kNoTile) finish(prev2);
  if (prev1.T != kNoTile) finish(prev1);
}

// ====================================================================
// outlier pass (only tiles that escaped some residual)
// ====================================================================
constexpr int kOutWarps = 4;                    // outlier pass: warps per block, one tile each

template <int NDIM, int V, bool WHOLE = false, bool WIDE = false>
__global__ void __launch_bounds__(kOutWarps * 32)
    outlier_kernel(const CompressArgs a, uint64_t out_section) {
  const int g = threadIdx.x & 31;
  const uint64_t n_tiles = a.n_chunks * kTilesPerChunk;
  const uint64_t T = (uint64_t)blockIdx.x * kOutWarps + (threadIdx.x >> 5);
  if (T >= n_tiles || a.tile_out_count[T] == 0) return;
  uint32_t err = 0;
  const FieldRt rt = derive_field(a, err);         // the compressor's bound and quantiser
  int32_t v[64];
  residuals_global<NDIM, V, WHOLE, WIDE>(a, T, g, rt.p.ebx2_r, v);
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

}  // namespace fz
