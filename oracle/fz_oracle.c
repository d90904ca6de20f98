/*
 * fz_oracle.c -- plain CPU oracle of the FZ-GPU compression path.
 *
 * TEST INFRASTRUCTURE ONLY (see fz_oracle.h).  Written for clarity, not
 * speed: every step is a direct loop over its definition, in the order the
 * paper gives them.  Floating point is IEEE binary32 with no contraction
 * (compiled with -ffp-contract=off), because the stream format fixes the
 * quantiser's arithmetic to fp32 multiply + round-half-even.
 *
 * Format constants (the paper leaves them open; these are this format's
 * readings):
 *   chunk (Lorenzo independence unit) = 4 tiles of 2048 codes
 *     1-D: 8192          tiles of 2048 along x
 *     2-D: 64 x 128      tiles of 64 x 32 along y
 *     3-D: 32 x 32 x 8   tiles of 32 x 32 x 2 along z
 *   inside a tile the 2048 codes are 32 groups ("bricks") of 64 codes;
 *   group g is the g-th brick, codes x-fastest inside the brick:
 *     1-D: brick 64          g = brick index along x
 *     2-D: brick 8 x 8       g = bx + 8*by   (8 x 4 bricks)
 *     3-D: brick 8 x 4 x 2   g = bx + 4*by   (4 x 8 bricks)
 *   word w of a tile packs codes 2w (low half) and 2w+1 (high half).
 */
#include "fz_oracle.h"

#include <fenv.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* small helpers                                                        */
/* ------------------------------------------------------------------ */

static void put_u32(uint8_t *p, uint32_t v) {
  p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}
static uint32_t get_u32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
         ((uint32_t)p[3] << 24);
}
static void put_f32(uint8_t *p, float f) {
  uint32_t u; memcpy(&u, &f, 4); put_u32(p, u);
}
static float get_f32(const uint8_t *p) {
  uint32_t u = get_u32(p); float f; memcpy(&f, &u, 4); return f;
}
static void put_f64(uint8_t *p, double d) {
  uint64_t u; memcpy(&u, &d, 8);
  put_u32(p, (uint32_t)u); put_u32(p + 4, (uint32_t)(u >> 32));
}

static uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

/* ------------------------------------------------------------------ */
/* Sec. 4.1: error bound.  "relative error bounds (relative to the value  */
/* range of the data field)": eb_abs = rel * (max - min).                 */
/* Reading: computed in double, then rounded DOWN to fp32 so the fp32     */
/* bound never exceeds the request; a constant field (range 0) uses       */
/* |max| (or 1 when the field is all zeros) as its range.                 */
/* ------------------------------------------------------------------ */
int fzo_derive_eb(int mode, double eb_req, float fmin, float fmax,
                  float *eb_f, float *ebx2, float *ebx2_r) {
  double eb_d;
  if (mode == FZO_EB_REL) {
    double range = (double)fmax - (double)fmin;
    if (range == 0.0) {
      range = fabs((double)fmax);
      if (range == 0.0) range = 1.0;
    }
    eb_d = eb_req * range;
  } else {
    eb_d = eb_req;
  }
  if (!(eb_d > 0.0) || !isfinite(eb_d)) return FZO_ERR_EB_RANGE;
  float e = (float)eb_d;                 /* nearest ...            */
  if ((double)e > eb_d) e = nextafterf(e, 0.0f);   /* ... then not above */
  if (!(e >= FLT_MIN)) return FZO_ERR_EB_RANGE;    /* zero or subnormal  */
  float e2 = 2.0f * e;                   /* exact unless it overflows */
  if (isinf(e2)) return FZO_ERR_EB_RANGE;
  *eb_f = e;
  *ebx2 = e2;
  *ebx2_r = (float)(1.0 / (double)e2);
  return FZO_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3: pre-quantisation, the only lossy step:                      */
/*   q = round(d / (2 eb)), error |q*2eb - d| <= eb.                      */
/* Reading: divide = multiply by the stored fp32 reciprocal; round =      */
/* nearest, ties to even; |q| limited to 2^22 - 1.                        */
/* ------------------------------------------------------------------ */
int fzo_prequant1(float x, float ebx2_r, int32_t *q) {
  volatile float v = x * ebx2_r;         /* one binary32 multiply */
  float r = nearbyintf(v);               /* FE_TONEAREST: ties to even */
  if (!(fabs((double)r) <= (double)FZO_QMAX)) return FZO_ERR_EB_RANGE;
  *q = (int32_t)r;
  return FZO_OK;
}

/* ------------------------------------------------------------------ */
/* chunking                                                             */
/* ------------------------------------------------------------------ */
void fzo_chunk_shape(int ndim, uint32_t chunk[3]) {
  if (ndim == 1) { chunk[0] = 8192; chunk[1] = 1; chunk[2] = 1; }
  else if (ndim == 2) { chunk[0] = 64; chunk[1] = 128; chunk[2] = 1; }
  else { chunk[0] = 32; chunk[1] = 32; chunk[2] = 8; }
}

static void norm_dims(int ndim, const uint32_t dims[3], uint64_t d[3]) {
  d[0] = dims[0];
  d[1] = ndim >= 2 ? dims[1] : 1;
  d[2] = ndim >= 3 ? dims[2] : 1;
}

uint64_t fzo_num_tiles(int ndim, const uint32_t dims[3]) {
  uint32_t ch[3]; uint64_t d[3];
  fzo_chunk_shape(ndim, ch); norm_dims(ndim, dims, d);
  return ceil_div(d[0], ch[0]) * ceil_div(d[1], ch[1]) *
         ceil_div(d[2], ch[2]) * FZO_TILES_PER_CHUNK;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2-2.3 / 3.1: Lorenzo prediction on the integer grid inside      */
/* independent chunks.  Reading: first-order ("one layer") Lorenzo;       */
/* neighbours outside the current chunk count as 0.                       */
/* ------------------------------------------------------------------ */

/* q~ : value at (x,y,z) if it lies in the chunk whose origin is o, else 0 */
static int64_t qt(const int32_t *q, const uint64_t d[3], const uint64_t o[3],
                  int64_t x, int64_t y, int64_t z) {
  if (x < (int64_t)o[0] || y < (int64_t)o[1] || z < (int64_t)o[2]) return 0;
  return q[(uint64_t)x + d[0] * ((uint64_t)y + d[1] * (uint64_t)z)];
}

static void chunk_origin(int ndim, uint64_t x, uint64_t y, uint64_t z,
                         uint64_t o[3]) {
  uint32_t ch[3];
  fzo_chunk_shape(ndim, ch);
  o[0] = x / ch[0] * ch[0];
  o[1] = y / ch[1] * ch[1];
  o[2] = z / ch[2] * ch[2];
}

/* the origin neighbours are cut off at: the chunk's, or for the
 * whole-field variant the field's (every neighbour inside the field counts;
 * the paper's chunks trade this for independence, Sec. 2.3) */
static void pred_origin(int ndim, int whole, uint64_t x, uint64_t y, uint64_t z,
                        uint64_t o[3]) {
  if (whole) { o[0] = o[1] = o[2] = 0; return; }
  chunk_origin(ndim, x, y, z, o);
}

/* the 1-, 2- and 3-D Lorenzo predictions (neighbours at lower indices) */
static int64_t lorenzo_pred(const int32_t *q, const uint64_t d[3],
                            const uint64_t o[3], int ndim, int64_t x,
                            int64_t y, int64_t z) {
  if (ndim == 1) return qt(q, d, o, x - 1, y, z);
  if (ndim == 2)
    return qt(q, d, o, x - 1, y, z) + qt(q, d, o, x, y - 1, z) -
           qt(q, d, o, x - 1, y - 1, z);
  return qt(q, d, o, x - 1, y, z) + qt(q, d, o, x, y - 1, z) +
         qt(q, d, o, x, y, z - 1) - qt(q, d, o, x - 1, y - 1, z) -
         qt(q, d, o, x - 1, y, z - 1) - qt(q, d, o, x, y - 1, z - 1) +
         qt(q, d, o, x - 1, y - 1, z - 1);
}

static void lorenzo_mode(const int32_t *q, const uint32_t dims[3], int ndim,
                         int whole, int32_t *delta) {
  uint64_t d[3];
  norm_dims(ndim, dims, d);
  for (uint64_t z = 0; z < d[2]; z++)
    for (uint64_t y = 0; y < d[1]; y++)
      for (uint64_t x = 0; x < d[0]; x++) {
        uint64_t o[3];
        pred_origin(ndim, whole, x, y, z, o);
        uint64_t i = x + d[0] * (y + d[1] * z);
        int64_t pred = lorenzo_pred(q, d, o, ndim, (int64_t)x, (int64_t)y,
                                    (int64_t)z);
        delta[i] = (int32_t)((int64_t)q[i] - pred);
      }
}

void fzo_lorenzo(const int32_t *q, const uint32_t dims[3], int ndim,
                 int32_t *delta) {
  lorenzo_mode(q, dims, ndim, 0, delta);
}

void fzo_lorenzo_whole(const int32_t *q, const uint32_t dims[3], int ndim,
                       int32_t *delta) {
  lorenzo_mode(q, dims, ndim, 1, delta);
}

/* Sec. 4.4 (decompression mirrors compression): rebuild q point by point
 * in increasing index order, q = delta + prediction from the already
 * rebuilt lower neighbours. Works in int64 so corrupt inputs cannot
 * overflow. */
static int64_t qt64(const int64_t *q, const uint64_t d[3], const uint64_t o[3],
                    int64_t x, int64_t y, int64_t z) {
  if (x < (int64_t)o[0] || y < (int64_t)o[1] || z < (int64_t)o[2]) return 0;
  return q[(uint64_t)x + d[0] * ((uint64_t)y + d[1] * (uint64_t)z)];
}

static void lorenzo_inverse_mode(const int32_t *delta, const uint32_t dims[3],
                                 int ndim, int whole, int64_t *q) {
  uint64_t d[3];
  norm_dims(ndim, dims, d);
  for (uint64_t z = 0; z < d[2]; z++)
    for (uint64_t y = 0; y < d[1]; y++)
      for (uint64_t x = 0; x < d[0]; x++) {
        uint64_t o[3];
        pred_origin(ndim, whole, x, y, z, o);
        int64_t X = (int64_t)x, Y = (int64_t)y, Z = (int64_t)z;
        int64_t pred;
        if (ndim == 1)
          pred = qt64(q, d, o, X - 1, Y, Z);
        else if (ndim == 2)
          pred = qt64(q, d, o, X - 1, Y, Z) + qt64(q, d, o, X, Y - 1, Z) -
                 qt64(q, d, o, X - 1, Y - 1, Z);
        else
          pred = qt64(q, d, o, X - 1, Y, Z) + qt64(q, d, o, X, Y - 1, Z) +
                 qt64(q, d, o, X, Y, Z - 1) - qt64(q, d, o, X - 1, Y - 1, Z) -
                 qt64(q, d, o, X - 1, Y, Z - 1) -
                 qt64(q, d, o, X, Y - 1, Z - 1) +
                 qt64(q, d, o, X - 1, Y - 1, Z - 1);
        uint64_t i = x + d[0] * (y + d[1] * z);
        q[i] = (int64_t)delta[i] + pred;
      }
}

void fzo_lorenzo_inverse(const int32_t *delta, const uint32_t dims[3],
                         int ndim, int64_t *q) {
  lorenzo_inverse_mode(delta, dims, ndim, 0, q);
}

void fzo_lorenzo_whole_inverse(const int32_t *delta, const uint32_t dims[3],
                               int ndim, int64_t *q) {
  lorenzo_inverse_mode(delta, dims, ndim, 1, q);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2: 16-bit codes, most significant bit = sign, no shift by a     */
/* radius.  Reading: |delta| > 32767 cannot be represented; such a code   */
/* becomes 0x8000 (negative zero, never produced otherwise) and the exact */
/* residual goes to an outlier list so the error bound still holds.       */
/* ------------------------------------------------------------------ */
uint16_t fzo_encode(int32_t delta) {
  int64_t a = delta < 0 ? -(int64_t)delta : (int64_t)delta;
  if (a > 32767) return 0x8000;
  return (uint16_t)((delta < 0 ? 0x8000u : 0u) | (uint32_t)a);
}

int32_t fzo_decode(uint16_t code) {
  int32_t m = code & 0x7FFF;
  return (code & 0x8000) ? -m : m;
}

/* ------------------------------------------------------------------ */
/* tile geometry                                                        */
/* ------------------------------------------------------------------ */
int fzo_tile_coord(int ndim, const uint32_t dims[3], uint64_t tile,
                   uint32_t p, uint32_t xyz[3]) {
  uint32_t ch[3]; uint64_t d[3];
  fzo_chunk_shape(ndim, ch); norm_dims(ndim, dims, d);
  uint64_t ncx = ceil_div(d[0], ch[0]), ncy = ceil_div(d[1], ch[1]);
  uint64_t c = tile / FZO_TILES_PER_CHUNK;
  uint32_t t = (uint32_t)(tile % FZO_TILES_PER_CHUNK);
  uint64_t cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
  uint32_t g = p / 64, l = p % 64;
  uint64_t x, y, z;
  if (ndim == 1) {
    x = cx * 8192 + (uint64_t)t * 2048 + p; y = 0; z = 0;
  } else if (ndim == 2) {
    uint32_t bx = g % 8, by = g / 8, ix = l % 8, iy = l / 8;
    x = cx * 64 + bx * 8 + ix;
    y = cy * 128 + (uint64_t)t * 32 + by * 8 + iy;
    z = 0;
  } else {
    uint32_t bx = g % 4, by = g / 4;
    uint32_t ix = l % 8, iy = (l / 8) % 4, iz = l / 32;
    x = cx * 32 + bx * 8 + ix;
    y = cy * 32 + by * 4 + iy;
    z = cz * 8 + (uint64_t)t * 2 + iz;
  }
  xyz[0] = (uint32_t)x; xyz[1] = (uint32_t)y; xyz[2] = (uint32_t)z;
  return x < d[0] && y < d[1] && z < d[2];
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3 bitshuffle: per group of 32 words, bit b of word t becomes   */
/* bit t of plane word b; planes are written "column-wise", i.e. plane b  */
/* of group g goes to word 32*b + g of the tile.                          */
/* ------------------------------------------------------------------ */
void fzo_bitshuffle(const uint32_t in[1024], uint32_t out[1024]) {
  for (int g = 0; g < 32; g++)
    for (int b = 0; b < 32; b++) {
      uint32_t w = 0;
      for (int t = 0; t < 32; t++)
        if ((in[32 * g + t] >> b) & 1u) w |= 1u << t;
      out[32 * b + g] = w;
    }
}

void fzo_bitunshuffle(const uint32_t out[1024], uint32_t in[1024]) {
  for (int g = 0; g < 32; g++)
    for (int t = 0; t < 32; t++) {
      uint32_t w = 0;
      for (int b = 0; b < 32; b++)
        if ((out[32 * b + g] >> t) & 1u) w |= 1u << b;
      in[32 * g + t] = w;
    }
}

/* Sec. 3.4 Listing 1: 16-byte data blocks (4 words); a block's flag is 1
 * when any of its words is non-zero; 256 flags per tile packed into 8
 * words, flag of block 32j+t at bit t of word j. */
void fzo_block_flags(const uint32_t out[1024], uint32_t flags[8]) {
  for (int j = 0; j < 8; j++) flags[j] = 0;
  for (int k = 0; k < 256; k++) {
    int nz = 0;
    for (int i = 0; i < 4; i++)
      if (out[4 * k + i] != 0) nz = 1;
    if (nz) flags[k / 32] |= 1u << (k % 32);
  }
}

/* ------------------------------------------------------------------ */
/* stream layout (little-endian)                                        */
/*   0  "FZG1"            4 version     5 ndim   6 eb mode   7 reserved  */
/*      (version 1: chunk-local Lorenzo; 2: whole-field Lorenzo)         */
/*   8  u32 dims[3]      20 u32 n_tiles 24 f64 eb as requested           */
/*  32  f32 eb (abs)     36 f32 2eb     40 f32 1/(2eb)                   */
/*  44  u32 nnz blocks   48 u32 n outliers                               */
/*  52  f32 field min    56 f32 field max (relative mode; else 0)        */
/*  60  u32 reserved                                                     */
/*  64  u32 flags[n_tiles][8]                                            */
/*      payload: non-zero 16-byte blocks in (tile, block) order           */
/*      outliers: (u32 stream code index, i32 residual), increasing index */
/* ------------------------------------------------------------------ */
uint64_t fzo_compress_bound(int ndim, const uint32_t dims[3]) {
  uint64_t nt = fzo_num_tiles(ndim, dims);
  return FZO_HEADER_BYTES + 32 * nt + 16 * 256 * nt + 8 * 2048 * nt;
}

static int check_dims(int ndim, const uint32_t dims[3]) {
  if (ndim < 1 || ndim > 3) return 0;
  for (int i = 0; i < ndim; i++)
    if (dims[i] == 0) return 0;
  if (fzo_num_tiles(ndim, dims) * FZO_TILE_CODES > 0xFFFFFFFFull) return 0;
  return 1;
}

/* Shared by fzo_compress and fzo_compress_ranged: rng == NULL takes the
 * relative bound's value range from x itself. */
static int compress_common(const float *x, const uint32_t dims[3], int ndim,
                           int mode, double eb, const float *rng, int whole,
                           uint8_t *out, uint64_t cap, uint64_t *out_size);

int fzo_compress(const float *x, const uint32_t dims[3], int ndim, int mode,
                 double eb, uint8_t *out, uint64_t cap, uint64_t *out_size) {
  return compress_common(x, dims, ndim, mode, eb, NULL, 0, out, cap, out_size);
}

/* The whole-field Lorenzo variant: the same stream with version 2, whose
 * residuals take every neighbour inside the field (no chunk cut-offs). */
int fzo_compress_whole(const float *x, const uint32_t dims[3], int ndim, int mode,
                       double eb, uint8_t *out, uint64_t cap, uint64_t *out_size) {
  return compress_common(x, dims, ndim, mode, eb, NULL, 1, out, cap, out_size);
}

/* Sec. 4.1's value-range-relative bound with the range supplied by the
 * caller: the range of the whole field when x is one slab of it, so that
 * every slab quantises with the field's bound. */
int fzo_compress_ranged(const float *x, const uint32_t dims[3], int ndim,
                        double eb, float range_min, float range_max,
                        uint8_t *out, uint64_t cap, uint64_t *out_size) {
  float rng[2] = {range_min, range_max};
  if (!isfinite(range_min) || !isfinite(range_max) || range_min > range_max) {
    *out_size = 0;
    return FZO_ERR_ARG;
  }
  return compress_common(x, dims, ndim, FZO_EB_REL, eb, rng, 0, out, cap, out_size);
}

static int compress_common(const float *x, const uint32_t dims[3], int ndim,
                           int mode, double eb, const float *rng, int whole,
                           uint8_t *out, uint64_t cap, uint64_t *out_size) {
  *out_size = 0;
  if (!x || !out || !check_dims(ndim, dims)) return FZO_ERR_ARG;
  if (mode != FZO_EB_ABS && mode != FZO_EB_REL) return FZO_ERR_ARG;
  if (!(eb > 0.0) || !isfinite(eb)) return FZO_ERR_ARG;
  if (fegetround() != FE_TONEAREST) return FZO_ERR_ARG;

  uint64_t d[3];
  norm_dims(ndim, dims, d);
  uint64_t n = d[0] * d[1] * d[2];

  /* non-finite input is rejected before anything else */
  for (uint64_t i = 0; i < n; i++)
    if (!isfinite(x[i])) return FZO_ERR_NONFINITE;

  /* value range (relative mode), +0 for zeros */
  float fmin = 0.0f, fmax = 0.0f;
  if (mode == FZO_EB_REL && rng) {
    fmin = rng[0] + 0.0f;
    fmax = rng[1] + 0.0f;
  } else if (mode == FZO_EB_REL) {
    fmin = x[0]; fmax = x[0];
    for (uint64_t i = 1; i < n; i++) {
      if (x[i] < fmin) fmin = x[i];
      if (x[i] > fmax) fmax = x[i];
    }
    fmin = fmin + 0.0f;
    fmax = fmax + 0.0f;
  }
  float eb_f, ebx2, ebx2_r;
  int st = fzo_derive_eb(mode, eb, fmin, fmax, &eb_f, &ebx2, &ebx2_r);
  if (st) return st;

  /* step 1: pre-quantisation of every point */
  int32_t *q = (int32_t *)malloc(n * sizeof(int32_t));
  int32_t *delta = (int32_t *)malloc(n * sizeof(int32_t));
  if (!q || !delta) { free(q); free(delta); return FZO_ERR_ARG; }
  int wide = 0;                          /* some |q| beyond FZO_QNARROW */
  for (uint64_t i = 0; i < n; i++) {
    if (fzo_prequant1(x[i], ebx2_r, &q[i])) {
      free(q); free(delta);
      return FZO_ERR_EB_RANGE;
    }
    wide |= q[i] > FZO_QNARROW || q[i] < -FZO_QNARROW;
  }

  /* step 2: chunk-local Lorenzo residuals */
  lorenzo_mode(q, dims, ndim, whole, delta);
  free(q);

  /* step 3: codes in stream order, outliers, words, bitshuffle, flags */
  uint64_t nt = fzo_num_tiles(ndim, dims);
  uint32_t *shuf = (uint32_t *)malloc(nt * 1024 * sizeof(uint32_t));
  uint32_t *flags = (uint32_t *)malloc(nt * 8 * sizeof(uint32_t));
  uint64_t n_out = 0, out_capacity = 1024;
  uint32_t *out_idx = (uint32_t *)malloc(out_capacity * sizeof(uint32_t));
  int32_t *out_val = (int32_t *)malloc(out_capacity * sizeof(int32_t));
  for (uint64_t t = 0; t < nt; t++) {
    uint16_t codes[FZO_TILE_CODES];
    uint32_t words[1024];
    for (uint32_t p = 0; p < FZO_TILE_CODES; p++) {
      uint32_t c[3];
      codes[p] = 0;
      if (!fzo_tile_coord(ndim, dims, t, p, c)) continue;   /* padding */
      int32_t dl = delta[c[0] + d[0] * (c[1] + d[1] * (uint64_t)c[2])];
      codes[p] = fzo_encode(dl);
      if (codes[p] == 0x8000) {
        if (n_out == out_capacity) {
          out_capacity *= 2;
          out_idx = (uint32_t *)realloc(out_idx, out_capacity * 4);
          out_val = (int32_t *)realloc(out_val, out_capacity * 4);
        }
        out_idx[n_out] = (uint32_t)(t * FZO_TILE_CODES + p);
        out_val[n_out] = dl;
        n_out++;
      }
    }
    for (int w = 0; w < 1024; w++)
      words[w] = (uint32_t)codes[2 * w] | ((uint32_t)codes[2 * w + 1] << 16);
    fzo_bitshuffle(words, shuf + t * 1024);
    fzo_block_flags(shuf + t * 1024, flags + t * 8);
  }
  free(delta);

  /* step 4 (Listing 2): byte flag per block, exclusive prefix sum over the
   * whole stream, block k goes to PreSum[k] when PreSum[k+1] != PreSum[k] */
  uint64_t nblk = nt * 256;
  uint8_t *byteflag = (uint8_t *)malloc(nblk);
  uint64_t *presum = (uint64_t *)malloc((nblk + 1) * sizeof(uint64_t));
  for (uint64_t k = 0; k < nblk; k++)
    byteflag[k] = (uint8_t)((flags[(k / 256) * 8 + (k % 256) / 32] >>
                             (k % 32)) & 1u);
  presum[0] = 0;
  for (uint64_t k = 0; k < nblk; k++) presum[k + 1] = presum[k] + byteflag[k];
  uint64_t nnz = presum[nblk];

  uint64_t size = FZO_HEADER_BYTES + 32 * nt + 16 * nnz + 8 * n_out;
  if (size > cap) {
    *out_size = size;
    free(shuf); free(flags); free(byteflag); free(presum);
    free(out_idx); free(out_val);
    return FZO_ERR_CAPACITY;
  }
  memset(out, 0, FZO_HEADER_BYTES);
  out[0] = 'F'; out[1] = 'Z'; out[2] = 'G'; out[3] = '1';
  out[4] = whole ? 2 : 1; out[5] = (uint8_t)ndim; out[6] = (uint8_t)mode; out[7] = (uint8_t)wide;
  put_u32(out + 8, (uint32_t)d[0]);
  put_u32(out + 12, (uint32_t)d[1]);
  put_u32(out + 16, (uint32_t)d[2]);
  put_u32(out + 20, (uint32_t)nt);
  put_f64(out + 24, eb);
  put_f32(out + 32, eb_f);
  put_f32(out + 36, ebx2);
  put_f32(out + 40, ebx2_r);
  put_u32(out + 44, (uint32_t)nnz);
  put_u32(out + 48, (uint32_t)n_out);
  put_f32(out + 52, fmin);
  put_f32(out + 56, fmax);
  put_u32(out + 60, 0);
  uint8_t *pf = out + FZO_HEADER_BYTES;
  for (uint64_t i = 0; i < nt * 8; i++) put_u32(pf + 4 * i, flags[i]);
  uint8_t *pp = pf + 32 * nt;
  for (uint64_t k = 0; k < nblk; k++) {
    if (presum[k + 1] != presum[k]) {
      const uint32_t *blk = shuf + 4 * k;   /* tile k/256, words 4(k%256).. */
      for (int i = 0; i < 4; i++) put_u32(pp + 16 * presum[k] + 4 * i, blk[i]);
    }
  }
  uint8_t *po = pp + 16 * nnz;
  for (uint64_t i = 0; i < n_out; i++) {
    put_u32(po + 8 * i, out_idx[i]);
    put_u32(po + 8 * i + 4, (uint32_t)out_val[i]);
  }
  *out_size = size;
  free(shuf); free(flags); free(byteflag); free(presum);
  free(out_idx); free(out_val);
  return FZO_OK;
}

/* ------------------------------------------------------------------ */
/* decompression (Sec. 4.4: the pipeline run backwards)                  */
/* ------------------------------------------------------------------ */
int fzo_decompress(const uint8_t *in, uint64_t in_size, float *x,
                   uint64_t cap_elems) {
  if (!in || !x) return FZO_ERR_ARG;
  if (in_size < FZO_HEADER_BYTES) return FZO_ERR_CORRUPT;
  if (in[0] != 'F' || in[1] != 'Z' || in[2] != 'G' || in[3] != '1' ||
      (in[4] != 1 && in[4] != 2) || in[7] > 1)
    return FZO_ERR_CORRUPT;
  const int whole = in[4] == 2;
  int ndim = in[5], mode = in[6];
  uint32_t dims[3] = {get_u32(in + 8), get_u32(in + 12), get_u32(in + 16)};
  if (ndim < 1 || ndim > 3 || mode > 1) return FZO_ERR_CORRUPT;
  for (int i = ndim; i < 3; i++)
    if (dims[i] != 1) return FZO_ERR_CORRUPT;
  if (!check_dims(ndim, dims)) return FZO_ERR_CORRUPT;
  uint64_t nt = fzo_num_tiles(ndim, dims);
  if (get_u32(in + 20) != nt) return FZO_ERR_CORRUPT;
  float ebx2 = get_f32(in + 36);
  uint64_t nnz = get_u32(in + 44), n_out = get_u32(in + 48);
  if (FZO_HEADER_BYTES + 32 * nt + 16 * nnz + 8 * n_out != in_size)
    return FZO_ERR_CORRUPT;
  uint64_t d[3];
  norm_dims(ndim, dims, d);
  uint64_t n = d[0] * d[1] * d[2];
  if (cap_elems < n) return FZO_ERR_CAPACITY;

  const uint8_t *pf = in + FZO_HEADER_BYTES;
  const uint8_t *pp = pf + 32 * nt;
  const uint8_t *po = pp + 16 * nnz;

  /* flags -> PreSum (Listing 2 run backwards) */
  uint64_t nblk = nt * 256, count = 0;
  for (uint64_t k = 0; k < nblk; k++)
    count += (get_u32(pf + 4 * (k / 32)) >> (k % 32)) & 1u;
  if (count != nnz) return FZO_ERR_CORRUPT;

  /* outliers: strictly increasing, in range, |residual| > 32767 */
  for (uint64_t i = 0; i < n_out; i++) {
    uint32_t idx = get_u32(po + 8 * i);
    int32_t v = (int32_t)get_u32(po + 8 * i + 4);
    if (idx >= nt * FZO_TILE_CODES) return FZO_ERR_CORRUPT;
    if (i > 0 && idx <= get_u32(po + 8 * (i - 1))) return FZO_ERR_CORRUPT;
    if (v >= -32767 && v <= 32767) return FZO_ERR_CORRUPT;
  }

  int32_t *delta = (int32_t *)calloc(n, sizeof(int32_t));
  int64_t *q = (int64_t *)malloc(n * sizeof(int64_t));
  if (!delta || !q) { free(delta); free(q); return FZO_ERR_ARG; }
  uint64_t presum = 0, oi = 0;
  int bad = 0;
  for (uint64_t t = 0; t < nt && !bad; t++) {
    uint32_t shuf[1024], words[1024];
    for (int k = 0; k < 256; k++) {
      uint64_t kk = t * 256 + (uint64_t)k;
      int f = (get_u32(pf + 4 * (kk / 32)) >> (kk % 32)) & 1u;
      for (int i = 0; i < 4; i++)
        shuf[4 * k + i] = f ? get_u32(pp + 16 * presum + 4 * i) : 0;
      presum += (uint64_t)f;
    }
    fzo_bitunshuffle(shuf, words);
    for (uint32_t p = 0; p < FZO_TILE_CODES; p++) {
      uint16_t code = (uint16_t)(words[p / 2] >> (16 * (p % 2)));
      uint32_t c[3];
      int in_field = fzo_tile_coord(ndim, dims, t, p, c);
      uint32_t sidx = (uint32_t)(t * FZO_TILE_CODES + p);
      int32_t dl;
      if (code == 0x8000) {
        if (oi >= n_out || get_u32(po + 8 * oi) != sidx) { bad = 1; break; }
        dl = (int32_t)get_u32(po + 8 * oi + 4);
        oi++;
      } else {
        if (oi < n_out && get_u32(po + 8 * oi) == sidx) { bad = 1; break; }
        dl = fzo_decode(code);
      }
      if (!in_field) {
        if (code != 0) { bad = 1; break; }   /* padding must be zero */
        continue;
      }
      delta[c[0] + d[0] * (c[1] + d[1] * (uint64_t)c[2])] = dl;
    }
  }
  if (!bad && oi != n_out) bad = 1;
  if (bad) { free(delta); free(q); return FZO_ERR_CORRUPT; }

  lorenzo_inverse_mode(delta, dims, ndim, whole, q);
  for (uint64_t i = 0; i < n; i++) {
    volatile float qf = (float)q[i];
    x[i] = qf * ebx2;
  }
  free(delta); free(q);
  return FZO_OK;
}

/* the reconstruction's closed form (all later stages are lossless) */
int fzo_reconstruct_closed_form(const float *x, uint64_t n, float ebx2_r,
                                float ebx2, float *xr) {
  for (uint64_t i = 0; i < n; i++) {
    int32_t q;
    if (fzo_prequant1(x[i], ebx2_r, &q)) return FZO_ERR_EB_RANGE;
    volatile float qf = (float)q;
    xr[i] = qf * ebx2;
  }
  return FZO_OK;
}


/* ====================================================================
 * point-wise relative bounds by log transform (Sec. 4.1)
 * ==================================================================== */
int fzo_pwrel_bound(double eps, double *eb_abs) {
  if (!eb_abs || !(eps >= 1e-4 && eps <= 0.5)) return FZO_ERR_ARG;
  *eb_abs = log2(1.0 + eps) - ldexp(1.0, -14);
  return FZO_OK;
}

static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

float fzo_pw_log2(float a) {
  uint32_t b = f2u(a);
  int e = 0;
  if (b < 0x00800000u) {                 /* subnormal: times 2^23, exact */
    a = a * 8388608.0f;
    b = f2u(a);
    e = -23;
  }
  e += (int)(b >> 23) - 127;
  float m = u2f((b & 0x007FFFFFu) | 0x3F800000u);
  float num = m - 1.0f;
  float den = m + 1.0f;
  float s = num / den;
  float s2 = s * s;
  /* 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + ... + s^12/13), inner sum by Horner */
  float p = 0.07692308f;
  p = p * s2; p = p + 0.09090909f;
  p = p * s2; p = p + 0.11111111f;
  p = p * s2; p = p + 0.14285715f;
  p = p * s2; p = p + 0.2f;
  p = p * s2; p = p + 0.33333334f;
  p = p * s2; p = p + 1.0f;
  float two_s = 2.0f * s;
  float ln_m = two_s * p;
  float l2 = ln_m * 1.442695f;            /* 1 / ln 2 */
  return (float)e + l2;
}

float fzo_pw_exp2(float y) {
  if (!(y < 128.0f)) return FLT_MAX;
  if (y < -150.0f) return 0.0f;
  float k = floorf(y);
  float f = y - k;                        /* exact, in [0, 1) */
  float u = f * 0.6931472f;               /* ln 2 */
  /* exp(u) = 1 + u (1 + u/2 (1 + u/3 (...))), written as the power series
   * sum u^n / n!, n = 0..10, by Horner from the top */
  float p = 2.755732e-07f;
  p = p * u; p = p + 2.7557319e-06f;
  p = p * u; p = p + 2.4801588e-05f;
  p = p * u; p = p + 0.0001984127f;
  p = p * u; p = p + 0.0013888889f;
  p = p * u; p = p + 0.008333334f;
  p = p * u; p = p + 0.041666668f;
  p = p * u; p = p + 0.16666667f;
  p = p * u; p = p + 0.5f;
  p = p * u; p = p + 1.0f;
  p = p * u; p = p + 1.0f;
  int ki = (int)k;
  if (ki >= -126) return p * u2f((uint32_t)(ki + 127) << 23);
  float t = p * u2f((uint32_t)(ki + 126 + 127) << 23);
  return t * 1.17549435e-38f;             /* 2^-126 */
}

int fzo_pwrel_forward(const float *x, uint64_t n, float *y, uint32_t *signs) {
  int bad = 0;
  for (uint64_t w = 0; w < (n + 31) / 32; ++w) signs[w] = 0;
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t b = f2u(x[i]);
    if (b >> 31) signs[i / 32] |= 1u << (i % 32);
    if ((b & 0x7F800000u) == 0x7F800000u) { bad = 1; y[i] = -160.0f; continue; }
    float a = fabsf(x[i]);
    y[i] = a == 0.0f ? -160.0f : fzo_pw_log2(a);
  }
  return bad ? FZO_ERR_NONFINITE : FZO_OK;
}

void fzo_pwrel_inverse(const float *y, uint64_t n, const uint32_t *signs, float *x) {
  for (uint64_t i = 0; i < n; ++i) {
    float a = y[i] < -154.0f ? 0.0f : fzo_pw_exp2(y[i]);
    x[i] = ((signs[i / 32] >> (i % 32)) & 1u) ? -a : a;
  }
}

/* ------------------------------------------------------------------ */
/* All host cores (the paper's multi-threaded CPU version, FZ-OMP, Sec.   */
/* 4.4): the same steps as compress_common and fzo_decompress, with the   */
/* loops whose iterations are independent (points, tiles, chunks) split   */
/* into contiguous ranges over POSIX threads, and the compaction (prefix  */
/* sum and copy) serial.  Every value is computed by the same per-point   */
/* and per-tile functions, so the stream and the reconstruction are       */
/* identical to the one-thread calls.  Chunk-local (version 1) streams.   */
/* ------------------------------------------------------------------ */
#include <pthread.h>
#include <unistd.h>

#define MT_MAX_THREADS 256

int fzo_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  if (n < 1) n = 1;
  if (n > MT_MAX_THREADS) n = MT_MAX_THREADS;
  return (int)n;
}

typedef void (*mt_body)(void *ctx, int64_t lo, int64_t hi, int part);
typedef struct { mt_body fn; void *ctx; int64_t lo, hi; int part; } mt_job;

static void *mt_run(void *p) {
  mt_job *j = (mt_job *)p;
  j->fn(j->ctx, j->lo, j->hi, j->part);
  return NULL;
}

/* fn over [0, n) in `parts` contiguous ranges, one per thread (the calling
 * thread takes the first); parts <= MT_MAX_THREADS */
static void mt_for(int64_t n, int parts, mt_body fn, void *ctx) {
  mt_job jobs[MT_MAX_THREADS];
  pthread_t th[MT_MAX_THREADS];
  int started[MT_MAX_THREADS];
  for (int k = 0; k < parts; k++) {
    jobs[k].fn = fn; jobs[k].ctx = ctx; jobs[k].part = k;
    jobs[k].lo = n * k / parts; jobs[k].hi = n * (k + 1) / parts;
    started[k] = 0;
  }
  for (int k = 1; k < parts; k++)
    started[k] = pthread_create(&th[k], NULL, mt_run, &jobs[k]) == 0;
  mt_run(&jobs[0]);
  for (int k = 1; k < parts; k++) {
    if (started[k]) pthread_join(th[k], NULL);
    else mt_run(&jobs[k]);                /* no thread: run it here */
  }
}

/* codes of tile t (stream order) from the residual field; returns the
 * number of escapes */
static uint32_t tile_codes(const int32_t *delta, const uint32_t dims[3], int ndim,
                           const uint64_t d[3], uint64_t t, uint16_t codes[FZO_TILE_CODES]) {
  uint32_t n_out = 0;
  for (uint32_t p = 0; p < FZO_TILE_CODES; p++) {
    uint32_t c[3];
    codes[p] = 0;
    if (!fzo_tile_coord(ndim, dims, t, p, c)) continue;
    codes[p] = fzo_encode(delta[c[0] + d[0] * (c[1] + d[1] * (uint64_t)c[2])]);
    n_out += codes[p] == 0x8000;
  }
  return n_out;
}

typedef struct {
  const float *x;
  int32_t *q, *delta;
  const uint32_t *dims;
  const uint64_t *d;
  int ndim;
  float ebx2_r;
  uint32_t *shuf, *flags;
  uint64_t *tile_out;
  uint8_t *po;
  int bad[MT_MAX_THREADS];
  int wide[MT_MAX_THREADS];           /* some |q| beyond FZO_QNARROW */
  float lo[MT_MAX_THREADS], hi[MT_MAX_THREADS];
} mt_comp;

static void mt_finite(void *c, int64_t lo, int64_t hi, int k) {
  mt_comp *m = (mt_comp *)c;
  int bad = 0;
  for (int64_t i = lo; i < hi; i++) bad |= !isfinite(m->x[i]);
  m->bad[k] = bad;
}
static void mt_minmax(void *c, int64_t lo, int64_t hi, int k) {
  mt_comp *m = (mt_comp *)c;
  float a = m->x[lo < hi ? lo : 0], b = a;
  for (int64_t i = lo; i < hi; i++) {
    if (m->x[i] < a) a = m->x[i];
    if (m->x[i] > b) b = m->x[i];
  }
  m->lo[k] = a;
  m->hi[k] = b;
}
static void mt_prequant(void *c, int64_t lo, int64_t hi, int k) {
  mt_comp *m = (mt_comp *)c;
  int bad = 0, wide = 0;
  for (int64_t i = lo; i < hi; i++) {
    bad |= fzo_prequant1(m->x[i], m->ebx2_r, &m->q[i]) != FZO_OK;
    wide |= m->q[i] > FZO_QNARROW || m->q[i] < -FZO_QNARROW;
  }
  m->bad[k] = bad;
  m->wide[k] = wide;
}
static void mt_lorenzo(void *c, int64_t lo, int64_t hi, int k) {
  mt_comp *m = (mt_comp *)c;
  const uint64_t *d = m->d;
  (void)k;
  for (int64_t i = lo; i < hi; i++) {
    const uint64_t xx = (uint64_t)i % d[0], yy = ((uint64_t)i / d[0]) % d[1];
    const uint64_t zz = (uint64_t)i / (d[0] * d[1]);
    uint64_t o[3];
    pred_origin(m->ndim, 0, xx, yy, zz, o);
    m->delta[i] = (int32_t)((int64_t)m->q[i] -
                            lorenzo_pred(m->q, d, o, m->ndim, (int64_t)xx, (int64_t)yy, (int64_t)zz));
  }
}
static void mt_tiles(void *c, int64_t lo, int64_t hi, int k) {
  mt_comp *m = (mt_comp *)c;
  (void)k;
  for (int64_t t = lo; t < hi; t++) {
    uint16_t codes[FZO_TILE_CODES];
    uint32_t words[1024];
    m->tile_out[t + 1] = tile_codes(m->delta, m->dims, m->ndim, m->d, (uint64_t)t, codes);
    for (int w = 0; w < 1024; w++)
      words[w] = (uint32_t)codes[2 * w] | ((uint32_t)codes[2 * w + 1] << 16);
    fzo_bitshuffle(words, m->shuf + t * 1024);
    fzo_block_flags(m->shuf + t * 1024, m->flags + t * 8);
  }
}
/* escapes in stream order: each tile writes its own slice of the list */
static void mt_escapes(void *c, int64_t lo, int64_t hi, int k) {
  mt_comp *m = (mt_comp *)c;
  const uint64_t *d = m->d;
  (void)k;
  for (int64_t t = lo; t < hi; t++) {
    if (m->tile_out[t + 1] == m->tile_out[t]) continue;
    uint16_t codes[FZO_TILE_CODES];
    tile_codes(m->delta, m->dims, m->ndim, d, (uint64_t)t, codes);
    uint64_t j = m->tile_out[t];
    for (uint32_t p = 0; p < FZO_TILE_CODES; p++) {
      if (codes[p] != 0x8000) continue;
      uint32_t c3[3];
      fzo_tile_coord(m->ndim, m->dims, (uint64_t)t, p, c3);
      put_u32(m->po + 8 * j, (uint32_t)((uint64_t)t * FZO_TILE_CODES + p));
      put_u32(m->po + 8 * j + 4,
              (uint32_t)m->delta[c3[0] + d[0] * (c3[1] + d[1] * (uint64_t)c3[2])]);
      j++;
    }
  }
}

int fzo_compress_mt(const float *x, const uint32_t dims[3], int ndim, int mode,
                    double eb, uint8_t *out, uint64_t cap, uint64_t *out_size) {
  *out_size = 0;
  if (!x || !out || !check_dims(ndim, dims)) return FZO_ERR_ARG;
  if (mode != FZO_EB_ABS && mode != FZO_EB_REL) return FZO_ERR_ARG;
  if (!(eb > 0.0) || !isfinite(eb)) return FZO_ERR_ARG;
  if (fegetround() != FE_TONEAREST) return FZO_ERR_ARG;
  uint64_t d[3];
  norm_dims(ndim, dims, d);
  const int64_t n = (int64_t)(d[0] * d[1] * d[2]);
  const int T = fzo_threads();
  mt_comp *m = (mt_comp *)calloc(1, sizeof(mt_comp));
  if (!m) return FZO_ERR_ARG;
  m->x = x; m->dims = dims; m->d = d; m->ndim = ndim;

  mt_for(n, T, mt_finite, m);
  int bad = 0;
  for (int k = 0; k < T; k++) bad |= m->bad[k];
  if (bad) { free(m); return FZO_ERR_NONFINITE; }

  /* min and max are exact, so the order of the partial results is free */
  float fmin = 0.0f, fmax = 0.0f;
  if (mode == FZO_EB_REL) {
    mt_for(n, T, mt_minmax, m);
    fmin = m->lo[0]; fmax = m->hi[0];
    for (int k = 1; k < T; k++) {
      if (m->lo[k] < fmin) fmin = m->lo[k];
      if (m->hi[k] > fmax) fmax = m->hi[k];
    }
    fmin = fmin + 0.0f;
    fmax = fmax + 0.0f;
  }
  float eb_f, ebx2, ebx2_r;
  int st = fzo_derive_eb(mode, eb, fmin, fmax, &eb_f, &ebx2, &ebx2_r);
  if (st) { free(m); return st; }

  m->q = (int32_t *)malloc(n * sizeof(int32_t));
  m->delta = (int32_t *)malloc(n * sizeof(int32_t));
  if (!m->q || !m->delta) { free(m->q); free(m->delta); free(m); return FZO_ERR_ARG; }
  m->ebx2_r = ebx2_r;
  mt_for(n, T, mt_prequant, m);
  bad = 0;
  for (int k = 0; k < T; k++) bad |= m->bad[k];
  if (bad) { free(m->q); free(m->delta); free(m); return FZO_ERR_EB_RANGE; }
  int wide = 0;
  for (int k = 0; k < T; k++) wide |= m->wide[k];
  mt_for(n, T, mt_lorenzo, m);
  free(m->q);
  m->q = NULL;

  const int64_t nt = (int64_t)fzo_num_tiles(ndim, dims);
  m->shuf = (uint32_t *)malloc(nt * 1024 * sizeof(uint32_t));
  m->flags = (uint32_t *)malloc(nt * 8 * sizeof(uint32_t));
  m->tile_out = (uint64_t *)malloc((nt + 1) * sizeof(uint64_t));
  mt_for(nt, T, mt_tiles, m);
  m->tile_out[0] = 0;
  for (int64_t t = 0; t < nt; t++) m->tile_out[t + 1] += m->tile_out[t];
  const uint64_t n_out = m->tile_out[nt];
  const uint32_t *flags = m->flags, *shuf = m->shuf;

  /* compaction, serial: block k goes to PreSum[k] (Listing 2) */
  const uint64_t nblk = (uint64_t)nt * 256;
  uint64_t nnz = 0;
  for (uint64_t k = 0; k < nblk; k++) nnz += (flags[k / 32] >> (k % 32)) & 1u;
  const uint64_t size = FZO_HEADER_BYTES + 32 * (uint64_t)nt + 16 * nnz + 8 * n_out;
  if (size > cap) {
    *out_size = size;
    free(m->shuf); free(m->flags); free(m->tile_out); free(m->delta); free(m);
    return FZO_ERR_CAPACITY;
  }
  memset(out, 0, FZO_HEADER_BYTES);
  out[0] = 'F'; out[1] = 'Z'; out[2] = 'G'; out[3] = '1';
  out[4] = 1; out[5] = (uint8_t)ndim; out[6] = (uint8_t)mode; out[7] = (uint8_t)wide;
  put_u32(out + 8, (uint32_t)d[0]);
  put_u32(out + 12, (uint32_t)d[1]);
  put_u32(out + 16, (uint32_t)d[2]);
  put_u32(out + 20, (uint32_t)nt);
  put_f64(out + 24, eb);
  put_f32(out + 32, eb_f);
  put_f32(out + 36, ebx2);
  put_f32(out + 40, ebx2_r);
  put_u32(out + 44, (uint32_t)nnz);
  put_u32(out + 48, (uint32_t)n_out);
  put_f32(out + 52, fmin);
  put_f32(out + 56, fmax);
  uint8_t *pf = out + FZO_HEADER_BYTES;
  for (uint64_t i = 0; i < (uint64_t)nt * 8; i++) put_u32(pf + 4 * i, flags[i]);
  uint8_t *pp = pf + 32 * (uint64_t)nt;
  uint64_t presum = 0;
  for (uint64_t k = 0; k < nblk; k++) {
    if ((flags[k / 32] >> (k % 32)) & 1u) {
      for (int i = 0; i < 4; i++) put_u32(pp + 16 * presum + 4 * i, shuf[4 * k + i]);
      presum++;
    }
  }
  m->po = pp + 16 * nnz;
  mt_for(nt, T, mt_escapes, m);
  *out_size = size;
  free(m->shuf); free(m->flags); free(m->tile_out); free(m->delta); free(m);
  return FZO_OK;
}

typedef struct {
  const uint8_t *pf, *pp, *po;
  const uint32_t *dims;
  const uint64_t *d;
  int ndim;
  uint64_t n_out;
  const uint64_t *tile_pre;
  int32_t *delta;
  int64_t *q;
  float *x;
  float ebx2;
  uint32_t ch[3];
  uint64_t ncx, ncy;
  int bad[MT_MAX_THREADS];
  uint64_t matched[MT_MAX_THREADS];
} mt_dec;

static void mt_unshuffle(void *c, int64_t lo, int64_t hi, int k) {
  mt_dec *m = (mt_dec *)c;
  const uint64_t *d = m->d;
  int bad = 0;
  uint64_t matched = 0;
  for (int64_t t = lo; t < hi && !bad; t++) {
    uint32_t shuf[1024], words[1024];
    uint64_t presum = m->tile_pre[t];
    for (int b = 0; b < 256; b++) {
      int f = (get_u32(m->pf + 32 * t + 4 * (b / 32)) >> (b % 32)) & 1u;
      for (int i = 0; i < 4; i++) shuf[4 * b + i] = f ? get_u32(m->pp + 16 * presum + 4 * i) : 0;
      presum += (uint64_t)f;
    }
    fzo_bitunshuffle(shuf, words);
    /* this tile's first outlier record: the records are sorted by index */
    uint64_t lo2 = 0, hi2 = m->n_out;
    const uint32_t first = (uint32_t)((uint64_t)t * FZO_TILE_CODES);
    while (lo2 < hi2) {
      uint64_t mid = (lo2 + hi2) / 2;
      if (get_u32(m->po + 8 * mid) < first) lo2 = mid + 1; else hi2 = mid;
    }
    uint64_t oi = lo2;
    for (uint32_t p = 0; p < FZO_TILE_CODES; p++) {
      uint16_t code = (uint16_t)(words[p / 2] >> (16 * (p % 2)));
      uint32_t c3[3];
      int in_field = fzo_tile_coord(m->ndim, m->dims, (uint64_t)t, p, c3);
      uint32_t sidx = first + p;
      int32_t dl;
      if (code == 0x8000) {
        if (oi >= m->n_out || get_u32(m->po + 8 * oi) != sidx) { bad = 1; break; }
        dl = (int32_t)get_u32(m->po + 8 * oi + 4);
        oi++;
        matched++;
      } else {
        if (oi < m->n_out && get_u32(m->po + 8 * oi) == sidx) { bad = 1; break; }
        dl = fzo_decode(code);
      }
      if (!in_field) {
        if (code != 0) { bad = 1; break; }
        continue;
      }
      m->delta[c3[0] + d[0] * (c3[1] + d[1] * (uint64_t)c3[2])] = dl;
    }
  }
  m->bad[k] = bad;
  m->matched[k] = matched;
}
/* the predictor recurrence chunk by chunk (chunks are independent) */
static void mt_inverse(void *c, int64_t lo, int64_t hi, int k) {
  mt_dec *m = (mt_dec *)c;
  const uint64_t *d = m->d;
  const int64_t *q = m->q;
  (void)k;
  for (int64_t ci = lo; ci < hi; ci++) {
    const uint64_t o[3] = {((uint64_t)ci % m->ncx) * m->ch[0],
                           (((uint64_t)ci / m->ncx) % m->ncy) * m->ch[1],
                           ((uint64_t)ci / (m->ncx * m->ncy)) * m->ch[2]};
    for (uint64_t z = o[2]; z < o[2] + m->ch[2] && z < d[2]; z++)
      for (uint64_t y = o[1]; y < o[1] + m->ch[1] && y < d[1]; y++)
        for (uint64_t xx = o[0]; xx < o[0] + m->ch[0] && xx < d[0]; xx++) {
          int64_t X = (int64_t)xx, Y = (int64_t)y, Z = (int64_t)z;
          int64_t pred;
          if (m->ndim == 1)
            pred = qt64(q, d, o, X - 1, Y, Z);
          else if (m->ndim == 2)
            pred = qt64(q, d, o, X - 1, Y, Z) + qt64(q, d, o, X, Y - 1, Z) -
                   qt64(q, d, o, X - 1, Y - 1, Z);
          else
            pred = qt64(q, d, o, X - 1, Y, Z) + qt64(q, d, o, X, Y - 1, Z) +
                   qt64(q, d, o, X, Y, Z - 1) - qt64(q, d, o, X - 1, Y - 1, Z) -
                   qt64(q, d, o, X - 1, Y, Z - 1) - qt64(q, d, o, X, Y - 1, Z - 1) +
                   qt64(q, d, o, X - 1, Y - 1, Z - 1);
          const uint64_t i = xx + d[0] * (y + d[1] * z);
          m->q[i] = (int64_t)m->delta[i] + pred;
        }
  }
}
static void mt_dequant(void *c, int64_t lo, int64_t hi, int k) {
  mt_dec *m = (mt_dec *)c;
  (void)k;
  for (int64_t i = lo; i < hi; i++) {
    volatile float qf = (float)m->q[i];
    m->x[i] = qf * m->ebx2;
  }
}

int fzo_decompress_mt(const uint8_t *in, uint64_t in_size, float *x, uint64_t cap_elems) {
  if (!in || !x) return FZO_ERR_ARG;
  if (in_size < FZO_HEADER_BYTES) return FZO_ERR_CORRUPT;
  if (in[4] == 2) return fzo_decompress(in, in_size, x, cap_elems);   /* whole-field */
  if (in[0] != 'F' || in[1] != 'Z' || in[2] != 'G' || in[3] != '1' || in[4] != 1 ||
      in[7] > 1)
    return FZO_ERR_CORRUPT;
  int ndim = in[5], mode = in[6];
  uint32_t dims[3] = {get_u32(in + 8), get_u32(in + 12), get_u32(in + 16)};
  if (ndim < 1 || ndim > 3 || mode > 1) return FZO_ERR_CORRUPT;
  for (int i = ndim; i < 3; i++)
    if (dims[i] != 1) return FZO_ERR_CORRUPT;
  if (!check_dims(ndim, dims)) return FZO_ERR_CORRUPT;
  const int64_t nt = (int64_t)fzo_num_tiles(ndim, dims);
  if (get_u32(in + 20) != (uint64_t)nt) return FZO_ERR_CORRUPT;
  float ebx2 = get_f32(in + 36);
  uint64_t nnz = get_u32(in + 44), n_out = get_u32(in + 48);
  if (FZO_HEADER_BYTES + 32 * (uint64_t)nt + 16 * nnz + 8 * n_out != in_size)
    return FZO_ERR_CORRUPT;
  uint64_t d[3];
  norm_dims(ndim, dims, d);
  const int64_t n = (int64_t)(d[0] * d[1] * d[2]);
  if (cap_elems < (uint64_t)n) return FZO_ERR_CAPACITY;
  const int T = fzo_threads();
  mt_dec *m = (mt_dec *)calloc(1, sizeof(mt_dec));
  uint64_t *tile_pre = (uint64_t *)malloc((nt + 1) * sizeof(uint64_t));
  if (!m || !tile_pre) { free(m); free(tile_pre); return FZO_ERR_ARG; }
  m->pf = in + FZO_HEADER_BYTES;
  m->pp = m->pf + 32 * (uint64_t)nt;
  m->po = m->pp + 16 * nnz;
  m->dims = dims; m->d = d; m->ndim = ndim; m->n_out = n_out; m->ebx2 = ebx2;

  /* each tile's first payload block (serial prefix of the flag counts) */
  tile_pre[0] = 0;
  for (int64_t t = 0; t < nt; t++) {
    uint64_t c = 0;
    for (int j = 0; j < 8; j++) c += (uint64_t)__builtin_popcount(get_u32(m->pf + 32 * t + 4 * j));
    tile_pre[t + 1] = tile_pre[t] + c;
  }
  int bad = tile_pre[nt] != nnz;
  for (uint64_t i = 0; i < n_out && !bad; i++) {
    uint32_t idx = get_u32(m->po + 8 * i);
    int32_t v = (int32_t)get_u32(m->po + 8 * i + 4);
    if (idx >= (uint64_t)nt * FZO_TILE_CODES) bad = 1;
    if (i > 0 && idx <= get_u32(m->po + 8 * (i - 1))) bad = 1;
    if (v >= -32767 && v <= 32767) bad = 1;
  }
  if (bad) { free(tile_pre); free(m); return FZO_ERR_CORRUPT; }
  m->tile_pre = tile_pre;
  m->delta = (int32_t *)calloc(n, sizeof(int32_t));
  m->q = (int64_t *)malloc(n * sizeof(int64_t));
  if (!m->delta || !m->q) {
    free(m->delta); free(m->q); free(tile_pre); free(m);
    return FZO_ERR_ARG;
  }
  mt_for(nt, T, mt_unshuffle, m);
  uint64_t matched = 0;
  for (int k = 0; k < T; k++) { bad |= m->bad[k]; matched += m->matched[k]; }
  free(tile_pre);
  if (!bad && matched != n_out) bad = 1;
  if (bad) { free(m->delta); free(m->q); free(m); return FZO_ERR_CORRUPT; }

  fzo_chunk_shape(ndim, m->ch);
  m->ncx = ceil_div(d[0], m->ch[0]);
  m->ncy = ceil_div(d[1], m->ch[1]);
  const int64_t nc = (int64_t)(m->ncx * m->ncy * ceil_div(d[2], m->ch[2]));
  mt_for(nc, T, mt_inverse, m);
  m->x = x;
  mt_for(n, T, mt_dequant, m);
  free(m->delta); free(m->q); free(m);
  return FZO_OK;
}
