/*
 * fz_oracle.h -- plain, slow, single-threaded CPU oracle for the FZ-GPU
 * compression path (Zhang, Tian et al., HPDC'23, arXiv 2304.12557).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the package
 * entry module and the CPU-baseline leg of the benchmark may load this code.
 * The product path (the CUDA library) neither includes this header nor links
 * this library, and this oracle includes nothing from the product path.
 *
 * What it computes, step by step (paper sections):
 *   eb derivation ........... Sec. 4.1 (value-range-relative error bound)
 *   pre-quantization ........ Sec. 2.3 (error-control equation)
 *   chunked Lorenzo residual  Sec. 2.2-2.3 (independent chunks), Sec. 3.1
 *   sign-magnitude u16 code . Sec. 3.2
 *   bitshuffle .............. Sec. 3.3 (32x32 u32 tile, planes written column-wise)
 *   zero-block flags ........ Sec. 3.4 (Listing 1: 16-byte blocks, bit flags)
 *   prefix-sum compaction ... Sec. 3.4 (Listing 2: copy block k to PreSum[k]
 *                             when PreSum[k+1] != PreSum[k])
 *   decompression ........... Sec. 4.4 (pipeline run backwards)
 * Readings where the paper is silent are listed in the repository's design
 * notes and restated at each function below.
 */
#ifndef FZ_ORACLE_H
#define FZ_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (same numeric values as the product library's, by design of
 * the format; the oracle defines its own copies) */
#define FZO_OK            0
#define FZO_ERR_ARG      -1
#define FZO_ERR_CAPACITY -2
#define FZO_ERR_NONFINITE -3
#define FZO_ERR_EB_RANGE -4
#define FZO_ERR_CORRUPT  -6

#define FZO_EB_ABS 0
#define FZO_EB_REL 1

#define FZO_HEADER_BYTES 64
#define FZO_TILE_CODES 2048
#define FZO_TILES_PER_CHUNK 4
#define FZO_QMAX 268435455    /* 2^28 - 1: largest |q| accepted (every 3-D
                                 residual, a signed sum of 8 q, fits an i32
                                 outlier record) */
#define FZO_QNARROW 4194303   /* 2^22 - 1: a stream whose every |q| is at most
                                 this has header byte 7 = 0, else 1 */

/* --- individual steps (exported so the tests can pin each one) --- */

/* Sec. 4.1: absolute bound from the request.  Writes eb_f, ebx2, ebx2_r.
 * Returns FZO_OK or FZO_ERR_EB_RANGE (bound not a positive normal float). */
int fzo_derive_eb(int mode, double eb_req, float fmin, float fmax,
                  float *eb_f, float *ebx2, float *ebx2_r);

/* Sec. 2.3: q = round-half-even(fl32(x * ebx2_r)).  Returns 0 and writes *q
 * when |q| <= FZO_QMAX, else returns FZO_ERR_EB_RANGE. */
int fzo_prequant1(float x, float ebx2_r, int32_t *q);

/* chunk shape for ndim (x, y, z extents) */
void fzo_chunk_shape(int ndim, uint32_t chunk[3]);

/* Chunk-local first-order Lorenzo residual of an integer field q laid out
 * x-fastest with extents dims[0..2] (unused dims = 1). */
void fzo_lorenzo(const int32_t *q, const uint32_t dims[3], int ndim,
                 int32_t *delta);

/* Inverse of fzo_lorenzo by the predictor recurrence q = delta + pred(q). */
void fzo_lorenzo_inverse(const int32_t *delta, const uint32_t dims[3],
                         int ndim, int64_t *q);

/* Sec. 3.2 sign-magnitude code; 0x8000 (negative zero) marks an escape. */
uint16_t fzo_encode(int32_t delta);
int32_t fzo_decode(uint16_t code);     /* escape decodes to 0 */

/* field coordinates of code position p (0..2047) of tile `tile`; returns 1
 * when the position lies inside the field, 0 when it is padding */
int fzo_tile_coord(int ndim, const uint32_t dims[3], uint64_t tile,
                   uint32_t p, uint32_t xyz[3]);
uint64_t fzo_num_tiles(int ndim, const uint32_t dims[3]);

/* Sec. 3.3: out[32*b + g] bit t = bit b of in[32*g + t] (1024 words) */
void fzo_bitshuffle(const uint32_t in[1024], uint32_t out[1024]);
void fzo_bitunshuffle(const uint32_t out[1024], uint32_t in[1024]);

/* Sec. 3.4 Listing 1: flag of 16-byte block k (words 4k..4k+3) is 1 when any
 * word is non-zero; flags[j] bit t = flag of block 32*j + t. */
void fzo_block_flags(const uint32_t out[1024], uint32_t flags[8]);

/* --- whole pipeline --- */

/* Worst-case stream size (every block non-zero, every code an escape). */
uint64_t fzo_compress_bound(int ndim, const uint32_t dims[3]);

/* Compress x (dims x-fastest).  Returns FZO_OK and writes *out_size, or an
 * error (with *out_size = required size on FZO_ERR_CAPACITY, else 0). */
int fzo_compress(const float *x, const uint32_t dims[3], int ndim, int mode,
                 double eb, uint8_t *out, uint64_t cap, uint64_t *out_size);

/* The relative bound (Sec. 4.1) against a caller-supplied value range
 * [range_min, range_max] instead of x's own (x a slab of a larger field whose
 * range this is).  Header mode REL, header range = the supplied one.
 * FZO_ERR_ARG for a non-finite or inverted range. */
int fzo_compress_ranged(const float *x, const uint32_t dims[3], int ndim,
                        double eb, float range_min, float range_max,
                        uint8_t *out, uint64_t cap, uint64_t *out_size);

/* Decompress a stream into x (capacity in elements). */
int fzo_decompress(const uint8_t *in, uint64_t in_size, float *x,
                   uint64_t cap_elems);

/* The reconstruction's plain definition: xr[i] = fl32(float(q_i) * ebx2). */
int fzo_reconstruct_closed_form(const float *x, uint64_t n, float ebx2_r,
                                float ebx2, float *xr);

/* --- the whole-field Lorenzo variant ----------------------------------
 * The paper's chunks make every chunk independent (Sec. 2.3) at the price
 * of a residual spike at each chunk's lower faces.  The variant takes every
 * neighbour inside the field instead (zero only outside the field).  Its
 * stream is the same apart from the version byte (2), which the
 * decompressor reads to choose the inverse.  Only the oracle has it; the
 * GPU library rejects version-2 streams. */
void fzo_lorenzo_whole(const int32_t *q, const uint32_t dims[3], int ndim,
                       int32_t *delta);
void fzo_lorenzo_whole_inverse(const int32_t *delta, const uint32_t dims[3],
                               int ndim, int64_t *q);
int fzo_compress_whole(const float *x, const uint32_t dims[3], int ndim, int mode,
                       double eb, uint8_t *out, uint64_t cap, uint64_t *out_size);

/* --- point-wise relative bounds by log transform ---------------------
 * Sec. 4.1 compresses the particle dataset log-transformed, with the
 * absolute bound a point-wise relative bound implies.  The transform is
 * y = log2|x| with the sign kept as a bit; a zero becomes -160 (every
 * nonzero float has log2 >= -149) and comes back as 0 below -154.
 * log2 and exp2 are evaluated in fp32 by fixed formulas, one IEEE
 * round-to-nearest operation at a time:
 *   log2 a = e + ln(m) / ln 2 for a = m 2^e, m in [1, 2), with
 *     ln m = 2 (s + s^3/3 + ... + s^13/13), s = (m - 1) / (m + 1);
 *   2^y = 2^k exp(u), k = floor(y), u = (y - k) ln 2, with
 *     exp(u) = sum of u^n / n! for n <= 10 (Horner).
 * These are approximations, pinned by the tests against the closed forms
 * (math.log2, 2**y), exact at powers of two, and by the end-to-end bound
 * |x' - x| <= eps |x| through the compressor. */

/* eb_abs = log2(1 + eps) - 2^-14; FZO_ERR_ARG unless 1e-4 <= eps <= 0.5 */
int fzo_pwrel_bound(double eps, double *eb_abs);
float fzo_pw_log2(float a);     /* a > 0, finite */
float fzo_pw_exp2(float y);     /* finite y */
/* y[i] = log2|x[i]| (-160 for zeros); signs: (n + 31) / 32 words, bit i % 32
 * of word i / 32 set for a negative (or -0) x[i].  FZO_OK or
 * FZO_ERR_NONFINITE (y then unspecified). */
int fzo_pwrel_forward(const float *x, uint64_t n, float *y, uint32_t *signs);
/* x[i] = +-2^y[i] (0 below -154, +-FLT_MAX from 128 up) */
void fzo_pwrel_inverse(const float *y, uint64_t n, const uint32_t *signs, float *x);

/* --- all host cores (the paper's multi-threaded FZ-OMP, Sec. 4.4) -------
 * The same steps with the loops over points, tiles and chunks split over
 * POSIX threads, one per online core; the compaction stays serial.  Streams
 * and reconstructions are identical to fzo_compress / fzo_decompress.
 * fzo_threads: the threads these calls use. */
int fzo_threads(void);
int fzo_compress_mt(const float *x, const uint32_t dims[3], int ndim, int mode,
                    double eb, uint8_t *out, uint64_t cap, uint64_t *out_size);
int fzo_decompress_mt(const uint8_t *in, uint64_t in_size, float *x, uint64_t cap_elems);

#ifdef __cplusplus
}
#endif
#endif
