// fz_decompress.cu -- GB300 decompression kernel (Sec. 4.4: the compression
// pipeline run backwards).
//
// Persistent warps; each warp takes chunks from a ticket counter in stream
// order and for each chunk:
//   flags -> popcounts -> warp-level decoupled look-back (payload offset);
//   all four tiles' non-zero 16-byte blocks are copied at once with
//   asynchronous zero-filling copies into per-warp plane buffers (Listing 2
//   backwards), then per tile: escape detection on the bit planes, inverse
//   bitshuffle (the register transpose), sign-magnitude decode, outlier
//   patch (rare), chunk-local inverse Lorenzo as prefix sums (in-register and
//   warp scans, a carried plane/row across tiles), q * 2eb, 32-byte stores.
// The header is validated on the device, so the call needs no host read of
// the stream before the launch.
#include <cuda_runtime.h>

#include "fz_device.cuh"
#include "fz_kernels.h"

namespace fz {

constexpr int kDecWarps = 4;                    // decompression: warps per block
constexpr int kOffChunks = 512;                 // offsets pass: chunks (threads) per block
// per warp: four tile buffers (the next chunk's tiles, gathered ahead) and a
// 1 KB staging area for row stores of fields whose rows are not 16-byte aligned
constexpr int kDecWarpSmem = kTilesPerChunk * 4096 + 1024;
constexpr int kDecSmemBytes = kDecWarps * kDecWarpSmem;

struct Hdr {
  int version, ndim, mode;
  bool wide;                     // header byte 7: |q| may pass 2^22 - 1
  uint32_t dims[3];
  uint64_t n_tiles, nnz, nout, n_chunks, ncx, ncy, n_elems;
  float ebx2;
  bool ok;
};

__device__ __forceinline__ uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

__device__ Hdr read_header(const DecompressArgs &a) {
  Hdr h{};
  h.ok = false;
  if (a.in_size < 64) return h;
  const StreamHeader *s = reinterpret_cast<const StreamHeader *>(a.in);
  if (s->magic[0] != 'F' || s->magic[1] != 'Z' || s->magic[2] != 'G' || s->magic[3] != '1')
    return h;
  if (!(s->version == 1 || (s->version == 2 && a.accept_whole)) ||
      (s->reserved0 != 0 && s->reserved0 != kHdrWide) || s->mode > 1)
    return h;
  h.version = s->version;
  h.wide = s->reserved0 == kHdrWide;
  h.ndim = s->ndim;
  h.mode = s->mode;
  if (h.ndim < 1 || h.ndim > 3) return h;
  for (int i = 0; i < 3; ++i) h.dims[i] = s->dims[i];
  for (int i = 0; i < 3; ++i) {
    if (i < h.ndim && h.dims[i] == 0) return h;
    if (i >= h.ndim && h.dims[i] != 1) return h;
  }
  uint64_t cx = h.ndim == 1 ? 8192 : (h.ndim == 2 ? 64 : 32);
  uint64_t cy = h.ndim == 1 ? 1 : (h.ndim == 2 ? 128 : 32);
  uint64_t cz = h.ndim == 3 ? 8 : 1;
  h.ncx = cdiv(h.dims[0], cx);
  h.ncy = cdiv(h.dims[1], cy);
  h.n_chunks = h.ncx * h.ncy * cdiv(h.dims[2], cz);
  h.n_tiles = h.n_chunks * kTilesPerChunk;
  if (h.n_tiles * kTileCodes > 0xFFFFFFFFull) return h;
  if (s->n_tiles != h.n_tiles) return h;
  h.nnz = s->nnz_blocks;
  h.nout = s->n_outliers;
  if (64 + 32 * h.n_tiles + 16 * h.nnz + 8 * h.nout != a.in_size) return h;
  h.n_elems = (uint64_t)h.dims[0] * h.dims[1] * h.dims[2];
  h.ebx2 = s->ebx2;
  h.ok = true;
  return h;
}

// first record index in [0, n) whose stream index is >= key (records sorted)
__device__ __forceinline__ uint64_t lower_bound_rec(const uint2 *rec, uint64_t n,
                                                    uint32_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (__ldg(&rec[mid].x) < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// residual of the escaped code with stream index `key`, searched among the
// chunk's records [lo, hi); false when absent or not a real outlier
__device__ __forceinline__ bool find_outlier(const uint2 *rec, uint64_t lo, uint64_t hi,
                                          uint32_t key, int32_t *val) {
  uint64_t k = lo + lower_bound_rec(rec + lo, hi - lo, key);
  if (k >= hi) return false;
  uint2 r = __ldg(&rec[k]);
  if (r.x != key) return false;
  int32_t v = (int32_t)r.y;
  if (v >= -32767 && v <= 32767) return false;
  *val = v;
  return true;
}

// 16-byte asynchronous copy global -> shared; with `bytes` = 0 nothing is
// read and the destination is zero-filled
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)),
               "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// PRMT with sign-replicating selectors (a selector nibble with its msb set
// copies the sign bit of the chosen byte into all 8 bits); the CUDA
// intrinsic __byte_perm masks that bit off, hence the inline PTX.
__device__ __forceinline__ uint32_t prmt_sign(uint32_t x, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(0u), "r"(sel));
  return r;
}

// decode 32 packed sign-magnitude pairs to residuals (an escape, 0x8000,
// decodes to 0 and is patched later)
__device__ __forceinline__ void decode_codes(const uint32_t (&w)[32], int32_t (&v)[64]) {
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const uint32_t s0 = prmt_sign(w[i], 0x9999);   // sign of the low code, replicated
    const uint32_t s1 = prmt_sign(w[i], 0xBBBB);   // sign of the high code
    v[2 * i] = (int32_t)(((w[i] & 0x7FFFu) ^ s0) - s0);
    v[2 * i + 1] = (int32_t)((((w[i] >> 16) & 0x7FFFu) ^ s1) - s1);
  }
}

// decode a narrow tile's 16 byte-code words (transpose16's output: byte k of
// u[j] is code 2j, 2j+1, 32+2j, 33+2j for k = 0..3; magnitude in bits 0..6,
// sign in bit 7) to residuals; an escape (sign only) decodes to 0
__device__ __forceinline__ void decode_narrow(const uint32_t (&u)[16], int32_t (&v)[64]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t x = u[j];
    const uint32_t s0 = prmt_sign(x, 0x8888), s1 = prmt_sign(x, 0x9999);
    const uint32_t s2 = prmt_sign(x, 0xAAAA), s3 = prmt_sign(x, 0xBBBB);
    v[2 * j] = (int32_t)(((x & 0x7Fu) ^ s0) - s0);
    v[2 * j + 1] = (int32_t)((((x >> 8) & 0x7Fu) ^ s1) - s1);
    v[32 + 2 * j] = (int32_t)((((x >> 16) & 0x7Fu) ^ s2) - s2);
    v[33 + 2 * j] = (int32_t)((((x >> 24) & 0x7Fu) ^ s3) - s3);
  }
}

// inverse Lorenzo inside the tile: v holds residuals in, q out.  `carry`
// holds the previous tile's boundary values of q (3-D: this brick's last
// plane, 2-D: the last row, 1-D: the last element) and is updated.
template <int NDIM>
__device__ __forceinline__ void inverse_lorenzo(int32_t (&v)[64], int32_t (&carry)[32], int g) {
  using G = Geo<NDIM>;
  const unsigned full = 0xffffffffu;
  const int bx = g % G::NBX;
  if constexpr (NDIM == 3) {
    // S_x: rows of 8, then an exclusive scan of row totals over the 4 bx lanes
#pragma unroll
    for (int row = 0; row < 8; ++row) {
#pragma unroll
      for (int ix = 1; ix < 8; ++ix) v[ix + 8 * row] += v[ix - 1 + 8 * row];
      const int32_t tot = v[7 + 8 * row];
      int32_t inc = tot;
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        const int32_t y = __shfl_up_sync(full, inc, o);
        if (bx >= o) inc += y;
      }
      const int32_t ex = inc - tot;
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) v[ix + 8 * row] += ex;
    }
    // S_y: columns of 4, then over the 8 by lanes (lane stride 4)
#pragma unroll
    for (int iz = 0; iz < 2; ++iz) {
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) {
#pragma unroll
        for (int iy = 1; iy < 4; ++iy) v[ix + 8 * iy + 32 * iz] += v[ix + 8 * (iy - 1) + 32 * iz];
        const int32_t tot = v[ix + 24 + 32 * iz];
        int32_t inc = tot;
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
          const int32_t y = __shfl_up_sync(full, inc, o);
          if (g >= o) inc += y;
        }
        const int32_t ex = inc - tot;
#pragma unroll
        for (int iy = 0; iy < 4; ++iy) v[ix + 8 * iy + 32 * iz] += ex;
      }
    }
    // S_z: the two planes of the tile plus the carried plane
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      v[e] += carry[e];
      v[e + 32] += v[e];
      carry[e] = v[e + 32];
    }
  } else if constexpr (NDIM == 2) {
#pragma unroll
    for (int row = 0; row < 8; ++row) {                 // S_x over 8 bx lanes
#pragma unroll
      for (int ix = 1; ix < 8; ++ix) v[ix + 8 * row] += v[ix - 1 + 8 * row];
      const int32_t tot = v[7 + 8 * row];
      int32_t inc = tot;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int32_t y = __shfl_up_sync(full, inc, o);
        if (bx >= o) inc += y;
      }
      const int32_t ex = inc - tot;
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) v[ix + 8 * row] += ex;
    }
#pragma unroll
    for (int ix = 0; ix < 8; ++ix) {                    // S_y over 4 by lanes
#pragma unroll
      for (int iy = 1; iy < 8; ++iy) v[ix + 8 * iy] += v[ix + 8 * (iy - 1)];
      const int32_t tot = v[ix + 56];
      int32_t inc = tot;
#pragma unroll
      for (int o = 8; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(full, inc, o);
        if (g >= o) inc += y;
      }
      const int32_t ex = inc - tot + carry[ix];
#pragma unroll
      for (int iy = 0; iy < 8; ++iy) v[ix + 8 * iy] += ex;
      carry[ix] = __shfl_sync(full, v[ix + 56], bx + 8 * (G::NBY - 1));
    }
  } else {
#pragma unroll
    for (int e = 1; e < 64; ++e) v[e] += v[e - 1];
    const int32_t tot = v[63];
    int32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(full, inc, o);
      if (g >= o) inc += y;
    }
    const int32_t ex = inc - tot + carry[0];
#pragma unroll
    for (int e = 0; e < 64; ++e) v[e] += ex;
    carry[0] = __shfl_sync(full, v[63], 31);
  }
}

// elements of [o, o + n) below the field's extent L
__device__ __forceinline__ uint32_t extent_in(uint64_t o, uint64_t L, uint32_t n) {
  return o >= L ? 0u : (L - o < n ? (uint32_t)(L - o) : n);
}

// lowest n bits set, n in [0, 32]
__device__ __forceinline__ uint32_t low_bits(uint32_t n) {
  return n >= 32 ? 0xFFFFFFFFu : (1u << n) - 1u;
}

// Which of a lane's 64 brick elements lie inside the field, as two masks
// over its 32 code words: bit t of `ev` for element 2t (the low code of word
// t), of `od` for element 2t+1.  l[0..2]: elements of the brick's first row
// / rows / planes that are inside (clamped to the brick).
template <int NDIM>
__device__ __forceinline__ void inside_masks(uint32_t lx, uint32_t ly, uint32_t lz,
                                             uint32_t &ev, uint32_t &od) {
  if constexpr (NDIM == 1) {
    ev = low_bits((lx + 1) / 2);
    od = low_bits(lx / 2);
  } else {
    // rows of 8 elements = 4 words; row r is (iy, iz) = (r % BY, r / BY)
    using G = Geo<NDIM>;
    const uint32_t re = low_bits((lx + 1) / 2), ro = low_bits(lx / 2);
    ev = 0; od = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t iy = r % G::BY, iz = r / G::BY;
      if (iy < ly && iz < lz) { ev |= re << (4 * r); od |= ro << (4 * r); }
    }
  }
}

// the 8 flag bytes of tile t for lane b (plane b), from the chunk's flag
// words held one per lane
__device__ __forceinline__ uint32_t plane_flags(uint32_t fw, int t, int g) {
  return (__shfl_sync(0xffffffffu, fw, 8 * t + (g >> 2)) >> (8 * (g & 3))) & 0xFFu;
}

// Copy tile t's present blocks into its plane buffer (Listing 2 backwards:
// block k comes from payload[PreSum[k]]), as one commit group; lane b
// copies plane b's blocks, `rank` its first block's payload index.  Absent
// blocks are zero-filled; a rank past the payload marks the stream corrupt.
__device__ __forceinline__ bool gather_tile(const uint8_t *payload, uint64_t nnz, uint32_t *dst,
                                            uint32_t F, uint64_t rank, int g) {
  bool oob = false;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool present = (F >> i) & 1u;
    const bool valid = present && rank < nnz;
    oob |= present && !valid;
    cp_async16(dst + 32 * g + 4 * (i ^ (g & 7)), payload + 16 * (valid ? rank : 0),
               valid ? 16u : 0u);
    rank += present;
  }
  cp_async_commit();
  return oob;
}

// A chunk's per-lane gather state: its flag word (lane l: word l of the
// chunk's 32) and, per tile, the payload index of lane b's first block.
struct ChunkPlan {
  uint32_t fw;
  uint32_t narrow;            // bit t: tile t's planes of magnitude bits 7..14 are all absent
  uint64_t base;              // the chunk's first payload block
  uint32_t p01, p23;          // per-lane exclusive ranks, tiles 0/1 and 2/3 (16-bit halves)
  uint32_t c01, c23;          // tile block counts, same packing
};

__device__ __forceinline__ ChunkPlan plan_chunk(uint32_t fw, uint64_t base, int g) {
  const unsigned full = 0xffffffffu;
  ChunkPlan p;
  p.fw = fw;
  p.base = base;
  // lane l holds flag bytes 4(l & 7) .. +3 of tile l >> 3: the bytes of
  // planes 7..14 and 23..30
  const uint32_t wi = (uint32_t)g & 3u;
  const uint32_t hm = wi == 1 ? 0xFF000000u : wi == 2 ? 0xFFFFFFFFu : wi == 3 ? 0x00FFFFFFu : 0u;
  const uint32_t wide = __ballot_sync(full, (fw & hm) != 0u);
  p.narrow = 0;
#pragma unroll
  for (int t = 0; t < kTilesPerChunk; ++t) p.narrow |= (((wide >> (8 * t)) & 0xFFu) == 0u) << t;
  uint32_t a = __popc(plane_flags(fw, 0, g)) | (__popc(plane_flags(fw, 1, g)) << 16);
  uint32_t b = __popc(plane_flags(fw, 2, g)) | (__popc(plane_flags(fw, 3, g)) << 16);
  uint32_t ia = a, ib = b;                    // two tiles per scan: sums <= 256
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t ya = __shfl_up_sync(full, ia, o), yb = __shfl_up_sync(full, ib, o);
    if (g >= o) { ia += ya; ib += yb; }
  }
  p.c01 = __shfl_sync(full, ia, 31);
  p.c23 = __shfl_sync(full, ib, 31);
  p.p01 = ia - a;
  p.p23 = ib - b;
  return p;
}

// payload index of lane g's first block of tile t
__device__ __forceinline__ uint64_t tile_rank(const ChunkPlan &p, int t) {
  const uint32_t lo01 = p.c01 & 0xFFFFu, hi01 = p.c01 >> 16, lo23 = p.c23 & 0xFFFFu;
  switch (t) {
    case 0: return p.base + (p.p01 & 0xFFFFu);
    case 1: return p.base + lo01 + (p.p01 >> 16);
    case 2: return p.base + lo01 + hi01 + (p.p23 & 0xFFFFu);
    default: return p.base + lo01 + hi01 + lo23 + (p.p23 >> 16);
  }
}

// phase 1: L on the chunk's upper faces, from the lanes that hold them
// (layouts at decompress_chunks)
template <int NDIM>
__device__ __forceinline__ void write_faces(const DecompressArgs &a, uint64_t c, int t, int bx,
                                            int by, int g, const int32_t (&v)[64]) {
  if constexpr (NDIM == 3) {
    if (bx == 3) {                                   // x = 31: rows 4by..4by+3, planes 2t, 2t+1
#pragma unroll
      for (int iz = 0; iz < 2; ++iz)
        *reinterpret_cast<int4 *>(a.face[0] + c * 256 + 32 * (2 * t + iz) + 4 * by) =
            make_int4(v[7 + 32 * iz], v[15 + 32 * iz], v[23 + 32 * iz], v[31 + 32 * iz]);
    }
    if (by == 7) {                                   // y = 31
#pragma unroll
      for (int iz = 0; iz < 2; ++iz) {
        int4 *d = reinterpret_cast<int4 *>(a.face[1] + c * 256 + 32 * (2 * t + iz) + 8 * bx);
        d[0] = make_int4(v[24 + 32 * iz], v[25 + 32 * iz], v[26 + 32 * iz], v[27 + 32 * iz]);
        d[1] = make_int4(v[28 + 32 * iz], v[29 + 32 * iz], v[30 + 32 * iz], v[31 + 32 * iz]);
      }
    }
    if (t == kTilesPerChunk - 1) {                   // z = 7: the tile's second plane
#pragma unroll
      for (int iy = 0; iy < 4; ++iy) {
        int4 *d = reinterpret_cast<int4 *>(a.face[2] + c * 1024 + 32 * (4 * by + iy) + 8 * bx);
        d[0] = make_int4(v[32 + 8 * iy], v[33 + 8 * iy], v[34 + 8 * iy], v[35 + 8 * iy]);
        d[1] = make_int4(v[36 + 8 * iy], v[37 + 8 * iy], v[38 + 8 * iy], v[39 + 8 * iy]);
      }
    }
  } else if constexpr (NDIM == 2) {
    if (bx == 7) {                                   // x = 63: rows 32t + 8by .. +7
      int4 *d = reinterpret_cast<int4 *>(a.face[0] + c * 128 + 32 * t + 8 * by);
      d[0] = make_int4(v[7], v[15], v[23], v[31]);
      d[1] = make_int4(v[39], v[47], v[55], v[63]);
    }
    if (t == kTilesPerChunk - 1 && by == 3) {        // y = 127
      int4 *d = reinterpret_cast<int4 *>(a.face[1] + c * 64 + 8 * bx);
      d[0] = make_int4(v[56], v[57], v[58], v[59]);
      d[1] = make_int4(v[60], v[61], v[62], v[63]);
    }
  } else {
    if (t == kTilesPerChunk - 1 && g == 31) a.face[0][c] = v[63];
  }
}

// phase 2: the corrections that change along the chunk's last axis (3-D:
// A'(y, z) + B'(x, z), 2-D: A'(y)); the others came in with the carry
template <int NDIM>
__device__ __forceinline__ void add_corrections(const DecompressArgs &a, uint64_t c, int t,
                                                int bx, int by, int32_t (&v)[64]) {
  if constexpr (NDIM == 3) {
#pragma unroll
    for (int iz = 0; iz < 2; ++iz) {
      const uint64_t o = c * 256 + 32 * (2 * t + iz);
      const int4 ay = __ldg(reinterpret_cast<const int4 *>(a.corr[0] + o + 4 * by));
      const int4 b0 = __ldg(reinterpret_cast<const int4 *>(a.corr[1] + o + 8 * bx));
      const int4 b1 = __ldg(reinterpret_cast<const int4 *>(a.corr[1] + o + 8 * bx) + 1);
      const int32_t A[4] = {ay.x, ay.y, ay.z, ay.w};
      const int32_t B[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int iy = 0; iy < 4; ++iy)
#pragma unroll
        for (int ix = 0; ix < 8; ++ix) v[ix + 8 * iy + 32 * iz] += A[iy] + B[ix];
    }
  } else if constexpr (NDIM == 2) {
    const int4 *p = reinterpret_cast<const int4 *>(a.corr[0] + c * 128 + 32 * t + 8 * by);
    const int4 a0 = __ldg(p), a1 = __ldg(p + 1);
    const int32_t A[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
    for (int row = 0; row < 8; ++row)
#pragma unroll
      for (int ix = 0; ix < 8; ++ix) v[ix + 8 * row] += A[row];
  }
}

// PHASE 0: a version-1 stream written out; 1 and 2: the two passes over a
// version-2 stream (whole-field Lorenzo).  Phase 1 writes each chunk's
// chunk-local prefix sums L on its upper faces and nothing else; phase 2
// adds the cross-chunk corrections to L and writes the field.  Face and
// correction layouts per chunk c (coordinates inside the chunk):
//   3-D: [0] (y, z) at c*256 + 32z + y, [1] (x, z) at c*256 + 32z + x,
//        [2] (x, y) at c*1024 + 32y + x;
//   2-D: [0] y at c*128 + y, [1] x at c*64 + x;   1-D: [0] at c.
// Faces hold L at the chunk's last x ([0]), last y ([1]), last z ([2]).
template <int NDIM, int PHASE, bool WIDE = false>
__device__ void decompress_chunks(const DecompressArgs &a, const Hdr &h, uint32_t *pbuf,
                                  SetScratch *cur) {
  using G = Geo<NDIM>;
  const unsigned full = 0xffffffffu;
  const int g = threadIdx.x & 31;
  const uint8_t *flags = a.in + 64;
  const uint8_t *payload = flags + 32 * h.n_tiles;
  const uint2 *recs = reinterpret_cast<const uint2 *>(payload + 16 * h.nnz);
  const uintptr_t op = reinterpret_cast<uintptr_t>(a.out);
  const int vw = (h.dims[0] % 8 == 0 && op % 32 == 0) ? 8
                 : (h.dims[0] % 4 == 0 && op % 16 == 0) ? 4 : 1;
  const FastDiv dx((uint32_t)h.ncx), dy((uint32_t)h.ncy);
  const uint64_t X = h.dims[0], Y = h.dims[1];
  const float e2 = h.ebx2;
  // the float bias of 1.5 * 2^23 that the prefix sums carry into every q
  // (none for the wide quantiser's streams: q is converted as an integer)
  const int32_t bias = WIDE ? 0 : (int32_t)kMagicBits;
  // chunks are dealt out statically: their payload offsets come from the
  // offsets pass, so no chunk waits for another
  const uint64_t n_warps = (uint64_t)gridDim.x * kDecWarps;
  // the chunks this launch decompresses: [chunk_lo, chunk_hi), chunk_hi 0 for all
  auto live = [&](uint64_t cc) { return cc < h.n_chunks && (a.chunk_hi == 0 || cc < a.chunk_hi); };
  uint64_t c = a.chunk_lo + (uint64_t)blockIdx.x * kDecWarps + (threadIdx.x >> 5);
  bool oob = false;
  uint32_t matched = 0, bad = 0;

  auto load_plan = [&](uint64_t cc) {
    uint32_t fw = 0;
    uint64_t base = 0;
    if (live(cc)) {
      fw = __ldg(reinterpret_cast<const uint32_t *>(flags + 128 * cc) + g);
      base = __ldg(a.chunk_off + cc);
    }
    return plan_chunk(fw, base, g);
  };
  // the first chunk's four tiles are requested up front
  ChunkPlan cp = load_plan(c);
  uint32_t cur_narrow = cp.narrow;   // the current chunk's narrow tiles
#pragma unroll
  for (int t = 0; t < kTilesPerChunk; ++t) {
    if (live(c)) oob |= gather_tile(payload, h.nnz, pbuf + 1024 * t, plane_flags(cp.fw, t, g),
                                           tile_rank(cp, t), g);
    else cp_async_commit();
  }
  while (live(c)) {
    const uint64_t cn = c + n_warps;
    // next chunk's flags and offset: in flight while tile 0 is decoded
    uint32_t fw_n = 0;
    uint64_t base_n = 0;
    if (live(cn)) {
      fw_n = __ldg(reinterpret_cast<const uint32_t *>(flags + 128 * cn) + g);
      base_n = __ldg(a.chunk_off + cn);
    }
    uint64_t o_lo = 0, o_hi = 0;
    if (h.nout) {
      o_lo = __ldg(a.chunk_olo + c);
      o_hi = c + 1 < h.n_chunks ? __ldg(a.chunk_olo + c + 1) : h.nout;
    }
    const uint32_t cr = dx.div((uint32_t)c);
    const uint64_t cx = (uint32_t)c - cr * dx.d, cz = dy.div(cr), cy = cr - (uint32_t)cz * dy.d;
    const bool edge = (cx + 1) * G::CX > h.dims[0] || (cy + 1) * G::CY > h.dims[1] ||
                      (cz + 1) * G::CZ > h.dims[2];
    // origin of lane g's brick in tile 0
    const int bx = g % G::NBX, by = g / G::NBX;
    uint64_t x0, y0, z0;
    if constexpr (NDIM == 3) {
      x0 = cx * 32 + 8 * bx; y0 = cy * 32 + 4 * by; z0 = cz * 8;
    } else if constexpr (NDIM == 2) {
      x0 = cx * 64 + 8 * bx; y0 = cy * 128 + 8 * by; z0 = 0;
    } else {
      x0 = cx * 8192 + 64 * g; y0 = 0; z0 = 0;
    }
    ChunkPlan np{};
    const uint32_t narrow_c = cur_narrow;
    int32_t carry[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) carry[e] = 0;
    if constexpr (PHASE == 2) {
      // the corrections that do not change along the chunk's last axis
      // (3-D: C'(x, y), 2-D: B'(x), 1-D: A') and the float bias enter as the
      // carried plane / row / element, so the prefix sums add them to all
      if constexpr (NDIM == 3) {
        const int4 *cc = reinterpret_cast<const int4 *>(a.corr[2] + c * 1024 + 32 * (4 * by) + 8 * bx);
#pragma unroll
        for (int iy = 0; iy < 4; ++iy) {
          const int4 p = __ldg(cc + 8 * iy), q = __ldg(cc + 8 * iy + 1);
          const int32_t r8[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
#pragma unroll
          for (int ix = 0; ix < 8; ++ix) carry[ix + 8 * iy] = r8[ix] + bias;
        }
      } else if constexpr (NDIM == 2) {
        const int4 *cb = reinterpret_cast<const int4 *>(a.corr[1] + c * 64 + 8 * bx);
        const int4 p = __ldg(cb), q = __ldg(cb + 1);
        const int32_t r8[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
#pragma unroll
        for (int ix = 0; ix < 8; ++ix) carry[ix] = r8[ix] + bias;
      } else {
        carry[0] = __ldg(a.corr[0] + c) + bias;
      }
    }
#pragma unroll 1
    for (int t = 0; t < kTilesPerChunk; ++t) {
      cp_async_wait<3>();                // this tile's group (3 newer ones may pend)
      __syncwarp();
      uint32_t *pb = pbuf + 1024 * t;
      // a narrow tile (every code within 7 bits and the sign) has 16 live
      // planes, read into w[0..15] (plane narrow_row(k) in w[k])
      const bool narrow = (narrow_c >> t) & 1u;
      uint32_t w[32];
      if (narrow) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int b = narrow_row(k);
          w[k] = pb[32 * b + 4 * ((g >> 2) ^ (b & 7)) + (g & 3)];
        }
      } else {
#pragma unroll
        for (int b = 0; b < 32; ++b) w[b] = pb[32 * b + 4 * ((g >> 2) ^ (b & 7)) + (g & 3)];
      }
      __syncwarp();                      // the buffer is free: refill it for the next chunk
      if (t == 0) np = plan_chunk(fw_n, base_n, g);
      if (live(cn))
        oob |= gather_tile(payload, h.nnz, pb, plane_flags(np.fw, t, g), tile_rank(np, t), g);
      else
        cp_async_commit();
      // codes on the bit planes (before the transpose): bit t of a mask is
      // word t of this lane's brick, low code (even element) or high code
      uint32_t lo_or = 0, hi_or = 0, sg_ev, sg_od;
      if (narrow) {
#pragma unroll
        for (int k = 0; k < 7; ++k) { lo_or |= w[k]; hi_or |= w[k + 8]; }
        sg_ev = w[7]; sg_od = w[15];
      } else {
#pragma unroll
        for (int b = 0; b < 15; ++b) { lo_or |= w[b]; hi_or |= w[b + 16]; }
        sg_ev = w[15]; sg_od = w[31];
      }
      uint32_t esc_ev = sg_ev & ~lo_or, esc_od = sg_od & ~hi_or;   // 0x8000: an escape
      // this tile's brick origin
      uint64_t bxo = x0, byo = y0, bzo = z0;
      if constexpr (NDIM == 3) bzo += 2 * t;
      else if constexpr (NDIM == 2) byo += 32 * t;
      else bxo += 2048 * t;
      if (edge) {
        // padding codes must be 0; escapes count only inside the field
        const uint32_t lx = extent_in(bxo, X, G::BX);
        const uint32_t ly = extent_in(byo, Y, G::BY);
        const uint32_t lz = extent_in(bzo, h.dims[2], G::BZ);
        uint32_t in_ev, in_od;
        inside_masks<NDIM>(lx, ly, lz, in_ev, in_od);
        bad |= ((lo_or | sg_ev) & ~in_ev) | ((hi_or | sg_od) & ~in_od);
        esc_ev &= in_ev;
        esc_od &= in_od;
      }
      int32_t v[64];
      if (narrow) {
        uint32_t(&u)[16] = *reinterpret_cast<uint32_t(*)[16]>(&w[0]);
        transpose16(u);                  // lane g: brick g's codes as bytes
        decode_narrow(u, v);
      } else {
        transpose32(w);                  // lane g: the 32 code words of brick g
        decode_codes(w, v);              // an escape decodes to 0
      }
      if (__any_sync(full, (esc_ev | esc_od) != 0)) {
        // rare: patch each escape with its recorded residual
        const uint32_t tile_code0 = (uint32_t)((c * kTilesPerChunk + t) * kTileCodes) + 64 * g;
        while (esc_ev | esc_od) {
          int e;
          if (esc_ev) { e = 2 * (__ffs(esc_ev) - 1); esc_ev &= esc_ev - 1; }
          else { e = 2 * (__ffs(esc_od) - 1) + 1; esc_od &= esc_od - 1; }
          int32_t val;
          if (find_outlier(recs, o_lo, o_hi, tile_code0 + e, &val)) {
            ++matched;
#pragma unroll
            for (int k = 0; k < 64; ++k) v[k] = k == e ? val : v[k];
          } else {
            bad = 1;
          }
        }
      }
      // the chunk origin carries the float bias of 1.5*2^23 into every q
      if (PHASE == 0 && t == 0 && g == 0) v[0] += bias;
      inverse_lorenzo<NDIM>(v, carry, g);
      if constexpr (PHASE == 1) {
        write_faces<NDIM>(a, c, t, bx, by, g, v);
        continue;
      }
      if constexpr (PHASE == 2) add_corrections<NDIM>(a, c, t, bx, by, v);
      // q -> fl(float(q) * 2eb), 8-float rows
      auto row_floats = [&](int row, float (&f)[8]) {
        if constexpr (WIDE) {
          // q beyond 2^22: unbiased integers, converted (the same fl(float(q) * 2eb))
#pragma unroll
          for (int k = 0; k < 8; ++k) f[k] = __fmul_rn(__int2float_rn(v[8 * row + k]), e2);
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k)
            f[k] = __fmul_rn(__fsub_rn(__int_as_float(v[8 * row + k]), kRoundMagic), e2);
        }
      };
      bool staged = false;
      if constexpr (NDIM >= 2) staged = vw == 1;
      if (staged) {
        // rows not 16-byte aligned: per row index, stage the warp's 8 (3-D)
        // or 4 (2-D) row segments in shared memory and store them 32
        // consecutive floats per instruction
        constexpr int SEG = 8 * G::NBX;              // floats per row segment
        float *st = reinterpret_cast<float *>(pbuf + kTilesPerChunk * 1024);
        float4 *s4 = reinterpret_cast<float4 *>(st + (g / G::NBX) * SEG + 8 * (g % G::NBX));
        // segment origin: the chunk's x, this tile's rows
        const uint64_t xc = bxo - 8 * (g % G::NBX);
        const uint64_t yc = byo - (uint64_t)G::BY * (g / G::NBX);
#pragma unroll
        for (int row = 0; row < 8; ++row) {
          float f[8];
          row_floats(row, f);
          const int iy = NDIM == 3 ? row % 4 : row, iz = NDIM == 3 ? row / 4 : 0;
          s4[0] = make_float4(f[0], f[1], f[2], f[3]);
          s4[1] = make_float4(f[4], f[5], f[6], f[7]);
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int e = 32 * j + g, sb = e / SEG, xo = e % SEG;
            const uint64_t x = xc + xo, y = yc + (uint64_t)G::BY * sb + iy, z = bzo + iz;
            if (!edge || (x < X && y < Y && z < h.dims[2]))
              __stcs(a.out + x + X * (y + Y * z), st[e]);
          }
          __syncwarp();                      // the staging area is free again
        }
      } else {
        float *base = a.out + bxo + X * (byo + Y * bzo);
#pragma unroll
        for (int row = 0; row < 8; ++row) {
          float f[8];
          row_floats(row, f);
          int iy, iz, ix;
          if constexpr (NDIM == 3) { ix = 0; iy = row % 4; iz = row / 4; }
          else if constexpr (NDIM == 2) { ix = 0; iy = row; iz = 0; }
          else { ix = 8 * row; iy = 0; iz = 0; }
          float *dst = base + ix + X * (iy + Y * iz);
          const bool row_in = !edge || (byo + iy < Y && bzo + iz < h.dims[2]);
          const bool full_row = !edge || (row_in && bxo + ix + 8 <= X);
          if (full_row && vw == 8) {
            asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(dst),
                         "f"(f[0]), "f"(f[1]), "f"(f[2]), "f"(f[3]), "f"(f[4]), "f"(f[5]),
                         "f"(f[6]), "f"(f[7])
                         : "memory");
          } else if (full_row && vw == 4) {
            __stcs(reinterpret_cast<float4 *>(dst), make_float4(f[0], f[1], f[2], f[3]));
            __stcs(reinterpret_cast<float4 *>(dst) + 1, make_float4(f[4], f[5], f[6], f[7]));
          } else if (row_in) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (bxo + ix + k < X) __stcs(dst + k, f[k]);
          }
        }
      }
    }
    if (h.nout) {
      const uint32_t m = __reduce_add_sync(full, matched);
      if (g == 0 && m != o_hi - o_lo) atomicOr(&cur->err, kErrCorrupt);
      if (g == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&cur->nout), (unsigned long long)m);
      matched = 0;
    }
    cur_narrow = np.narrow;
    c = cn;
  }
  cp_async_wait<0>();
  if (__any_sync(full, oob || bad != 0) && g == 0) atomicOr(&cur->err, kErrCorrupt);
}

// Offsets pass: blocks take units of kOffChunks consecutive chunks from a
// ticket counter (in stream order, as many as the grid holds at once), one
// chunk per thread: a block counts each chunk's non-zero blocks from its 128
// flag bytes, scans the counts over the block and takes the unit's offset by
// decoupled look-back, then writes every chunk's first payload block and,
// with outliers, its first outlier record.  Block 0 also validates the
// header and prepares the next call's scratch.  A unit's predecessors were
// ticketed earlier to blocks that are running, so every look-back ends.
__global__ void __launch_bounds__(kOffChunks) dec_offsets_kernel(const DecompressArgs a) {
  const unsigned full = 0xffffffffu;
  __shared__ uint32_t warp_tot[kOffChunks / 32];
  __shared__ uint64_t s_unit, s_excl;
  grid_launch_dependents();              // the decompressor may be scheduled now
  SetScratch *cur = a.set_cur;
  const int g = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Hdr h = read_header(a);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    SetScratch *nx = a.set_next;
    nx->ticket = 0; nx->err = 0; nx->nnz = 0; nx->nout = 0; nx->n_chunks = 0; nx->hdr_nout = 0;
    nx->version = 0;
    if (!h.ok) atomicOr(&cur->err, kErrCorrupt);
    else if (a.out_cap_elems < h.n_elems) atomicOr(&cur->err, kErrCapacity);
    else if (h.n_chunks > a.status_cap) atomicOr(&cur->err, kErrCorrupt);
    cur->version = h.ok ? (uint32_t)h.version : 0;
    cur->ndim = h.ok ? (uint32_t)h.ndim : 0;
    cur->wide = h.ok && h.wide ? 1u : 0u;
    cur->ncx = h.ok ? (uint32_t)h.ncx : 0;
    cur->ncy = h.ok ? (uint32_t)h.ncy : 0;
    cur->n_chunks = h.ok ? h.n_chunks : 0;
    cur->nnz = h.ok ? h.nnz : 0;
    cur->hdr_nout = h.ok ? (uint32_t)h.nout : 0;
  }
  if (!h.ok || a.out_cap_elems < h.n_elems || h.n_chunks > a.status_cap) return;
  const uint64_t n_units = cdiv(h.n_chunks, kOffChunks);
  const uint2 *recs = reinterpret_cast<const uint2 *>(a.in + 64 + 32 * h.n_tiles + 16 * h.nnz);
  while (true) {
    if (threadIdx.x == 0) s_unit = atomicAdd(&cur->ticket, 1u);
    __syncthreads();
    const uint64_t u = s_unit;
    if (u >= n_units) return;                        // the same in the whole block
    const uint64_t c = u * kOffChunks + threadIdx.x;
    uint32_t cnt = 0;
    if (c < h.n_chunks) {
      const uint4 *f = reinterpret_cast<const uint4 *>(a.in + 64 + 128 * c);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint4 v = __ldg(f + i);
        cnt += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
      }
    }
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(full, inc, o);
      if (g >= o) inc += y;
    }
    if (g == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
      // the unit's total, its look-back, and the warps' exclusive offsets
      const uint32_t t = g < kOffChunks / 32 ? warp_tot[g] : 0u;
      uint32_t ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, ti, o);
        if (g >= o) ti += y;
      }
      const uint32_t total = __shfl_sync(full, ti, 31);
      const bool publish = a.skip_publish_chunk >= h.n_chunks ||
                           u != a.skip_publish_chunk / kOffChunks;
      const uint64_t excl = lookback(a.status_cur, u, total, publish, &cur->err, a.wait_limit_ns);
      if (g < kOffChunks / 32) warp_tot[g] = ti - t;
      if (g == 0) {
        s_excl = excl;
        a.status_next[u * kStatusStride] = 0;          // for the next call
        if (u == n_units - 1 && excl + total != h.nnz) atomicOr(&cur->err, kErrCorrupt);
      }
    }
    __syncthreads();
    if (c < h.n_chunks) {
      const uint64_t off = s_excl + warp_tot[w] + inc - cnt;
      if (off + cnt > h.nnz) atomicOr(&cur->err, kErrCorrupt);
      a.chunk_off[c] = (uint32_t)off;
      if (h.nout) a.chunk_olo[c] = (uint32_t)lower_bound_rec(recs, h.nout, (uint32_t)(c * kChunkCodes));
    }
    __syncthreads();                                 // s_unit, s_excl, warp_tot reused
  }
}

__global__ void __launch_bounds__(kDecWarps * 32, 3) decompress_kernel(const DecompressArgs a) {
  extern __shared__ __align__(16) uint32_t dsmem[];
  grid_launch_dependents();              // the call's result copy may be scheduled now
  SetScratch *cur = a.set_cur;
  const int w = threadIdx.x >> 5;
  const Hdr h = read_header(a);
  if (!h.ok || a.out_cap_elems < h.n_elems || h.n_chunks > a.status_cap) return;
  // version 2 (phases 1 and 2 follow) and the wide quantiser's streams
  // (decompress_wide_kernel follows) are left to their own kernels
  if (h.version != 1 || h.wide) return;
  uint32_t *pbuf = dsmem + w * (kDecWarpSmem / 4);
  grid_dependency_wait();                // the offsets pass's chunk offsets
  if (h.ndim == 3) decompress_chunks<3, 0>(a, h, pbuf, cur);
  else if (h.ndim == 2) decompress_chunks<2, 0>(a, h, pbuf, cur);
  else decompress_chunks<1, 0>(a, h, pbuf, cur);
}

// a version-1 stream of the wide quantiser (header byte 7)
__global__ void __launch_bounds__(kDecWarps * 32, 3) decompress_wide_kernel(const DecompressArgs a) {
  extern __shared__ __align__(16) uint32_t dsmem[];
  SetScratch *cur = a.set_cur;
  const int w = threadIdx.x >> 5;
  const Hdr h = read_header(a);
  if (!h.ok || a.out_cap_elems < h.n_elems || h.n_chunks > a.status_cap) return;
  if (h.version != 1 || !h.wide) return;
  uint32_t *pbuf = dsmem + w * (kDecWarpSmem / 4);
  grid_dependency_wait();
  if (h.ndim == 3) decompress_chunks<3, 0, true>(a, h, pbuf, cur);
  else if (h.ndim == 2) decompress_chunks<2, 0, true>(a, h, pbuf, cur);
  else decompress_chunks<1, 0, true>(a, h, pbuf, cur);
}

// phases 1 and 2 of a version-2 stream (after the offsets pass and phase 0)
template <int PHASE, bool WIDE>
__global__ void __launch_bounds__(kDecWarps * 32, 3) decompress_whole_kernel(const DecompressArgs a) {
  extern __shared__ __align__(16) uint32_t dsmem[];
  SetScratch *cur = a.set_cur;
  const int w = threadIdx.x >> 5;
  const Hdr h = read_header(a);
  if (!h.ok || a.out_cap_elems < h.n_elems || h.n_chunks > a.status_cap) return;
  if (h.version != 2 || h.wide != WIDE) return;
  uint32_t *pbuf = dsmem + w * (kDecWarpSmem / 4);
  if (h.ndim == 3) decompress_chunks<3, PHASE, WIDE>(a, h, pbuf, cur);
  else if (h.ndim == 2) decompress_chunks<2, PHASE, WIDE>(a, h, pbuf, cur);
  else decompress_chunks<1, PHASE, WIDE>(a, h, pbuf, cur);
}

// The grid: enough blocks for max_chunks chunks, at most two per SM (the
// blocks loop over their tickets).
cudaError_t launch_dec_offsets(const DecompressArgs &a, uint64_t max_chunks, int sms,
                               cudaStream_t s) {
  if (sms < 1) sms = 1;
  uint64_t blocks = (max_chunks + kOffChunks - 1) / kOffChunks;
  if (blocks > (uint64_t)sms * 2) blocks = (uint64_t)sms * 2;
  dec_offsets_kernel<<<(unsigned)(blocks ? blocks : 1), kOffChunks, 0, s>>>(a);
  return cudaGetLastError();
}

// The 64-byte result block to (mapped host) memory once the grid before it
// on the stream has finished.
__global__ void __launch_bounds__(32) copy_result_kernel(const SetScratch *src, SetScratch *dst) {
  grid_dependency_wait();
  constexpr int kWords = (int)(sizeof(SetScratch) / 4);
  if (threadIdx.x < kWords)
    reinterpret_cast<uint32_t *>(dst)[threadIdx.x] =
        reinterpret_cast<const uint32_t *>(src)[threadIdx.x];
}

__global__ void __launch_bounds__(32) gather_u32_kernel(const uint32_t *src, GatherIdx idx, int n,
                                                        uint32_t *dst) {
  if ((int)threadIdx.x < n) dst[threadIdx.x] = src[idx.idx[threadIdx.x]];
}

cudaError_t launch_gather_u32(const uint32_t *src, GatherIdx idx, int n, uint32_t *dst,
                              cudaStream_t s) {
  gather_u32_kernel<<<1, 32, 0, s>>>(src, idx, n < 8 ? n : 8, dst);
  return cudaGetLastError();
}

cudaError_t launch_copy_result(const SetScratch *src, SetScratch *dst, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, copy_result_kernel, src, dst);
}

cudaError_t launch_decompress(const DecompressArgs &a, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kDecWarps * 32);
  cfg.dynamicSmemBytes = kDecSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  // phases 1 and 2 wait for everything before them (no dependency wait inside)
  cfg.numAttrs = a.phase == 0 ? 1 : 0;
  if (a.wide) {
    if (a.phase == 1) return cudaLaunchKernelEx(&cfg, decompress_whole_kernel<1, true>, a);
    if (a.phase == 2) return cudaLaunchKernelEx(&cfg, decompress_whole_kernel<2, true>, a);
    return cudaLaunchKernelEx(&cfg, decompress_wide_kernel, a);
  }
  if (a.phase == 1) return cudaLaunchKernelEx(&cfg, decompress_whole_kernel<1, false>, a);
  if (a.phase == 2) return cudaLaunchKernelEx(&cfg, decompress_whole_kernel<2, false>, a);
  return cudaLaunchKernelEx(&cfg, decompress_kernel, a);
}

int decompress_blocks_per_sm() {
  int n = 0;
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaFuncSetAttribute(decompress_whole_kernel<1, false>, at, kDecSmemBytes);
  cudaFuncSetAttribute(decompress_whole_kernel<2, false>, at, kDecSmemBytes);
  cudaFuncSetAttribute(decompress_whole_kernel<1, true>, at, kDecSmemBytes);
  cudaFuncSetAttribute(decompress_whole_kernel<2, true>, at, kDecSmemBytes);
  cudaFuncSetAttribute(decompress_wide_kernel, at, kDecSmemBytes);
  cudaFuncSetAttribute(decompress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kDecSmemBytes);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decompress_kernel, kDecWarps * 32,
                                                    kDecSmemBytes) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

uint64_t decompress_status_words(uint64_t n_chunks) {
  return (n_chunks + kOffChunks - 1) / kOffChunks;
}

}  // namespace fz
