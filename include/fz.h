/*
 * fz.h -- C ABI of the GB300 (sm_103a) FZ-GPU compression library.
 *
 * Method: FZ-GPU (Zhang, Tian et al., HPDC'23, arXiv 2304.12557).  A float32
 * field already resident in GPU memory is compressed on the GPU (Sec. 2.4:
 * data produced on the GPU is compressed from GPU memory, the compressed
 * bytes are kept in GPU memory or copied out through the CPU, and
 * decompressed on the GPU when needed):
 *   1. dual-quantisation (Sec. 2.3, 3.2): q = round(x / 2eb), then the
 *      chunk-local Lorenzo residual of q, as 16-bit sign-magnitude codes;
 *   2. bitshuffle of the codes in tiles of 32x32 u32 words (Sec. 3.3);
 *   3. zero-block encoding: 16-byte blocks, bit flags and prefix-sum
 *      compaction of the non-zero blocks (Sec. 3.4, Listings 1-2);
 *   4. the matching decompressor (Sec. 4.4: symmetric pipeline).
 *
 * Conventions for every entry point:
 *  - Plain pointers and sizes only.  "d_" pointers are device pointers on the
 *    context's device, "h_" pointers are host pointers.  `stream` is a
 *    cudaStream_t passed as void* (NULL = legacy default stream).
 *  - The caller owns every input and output buffer.  The library owns only
 *    the context's scratch (look-back status words, counters, a small
 *    result block), allocated by fz_create and grown when a larger field
 *    arrives; no other call allocates device memory.
 *  - Calls are stream-ordered and return after a synchronisation of
 *    `stream` (they report sizes and status to the host).  A context serves
 *    one call at a time: use one context per concurrently used stream.
 *  - Status: FZ_OK (0) or a negative FZ_ERR_* code.  On error no output size
 *    is reported (0), except FZ_ERR_CAPACITY, which reports the size needed.
 *  - Dims are given fastest-varying first: dims[0] = x (contiguous),
 *    dims[1] = y, dims[2] = z; entries beyond ndim are ignored.  The element
 *    (x,y,z) lives at index x + dims[0]*(y + dims[1]*z).
 */
#ifndef FZ_GB300_H
#define FZ_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status */
#define FZ_OK               0
#define FZ_ERR_ARG         -1  /* bad pointer, ndim, dims, eb, alignment   */
#define FZ_ERR_CAPACITY    -2  /* output buffer too small                  */
#define FZ_ERR_NONFINITE   -3  /* NaN or Inf in the input field            */
#define FZ_ERR_EB_RANGE    -4  /* some |x|/(2eb) rounds beyond 2^28-1
                                  (2^22-1 for a batch, a server request,
                                  the no-alloc and the unfused entries), or
                                  the derived bound is not a normal float   */
#define FZ_ERR_CORRUPT     -6  /* stream fails a structural check          */
#define FZ_ERR_TIMEOUT     -7  /* a bounded device wait gave up            */
#define FZ_ERR_CUDA        -8  /* a CUDA runtime call failed               */
#define FZ_ERR_VERSION     -9  /* a version-2 stream (whole-field Lorenzo)
                                  where the call reads version 1 only      */

/* error-bound modes (Sec. 4.1) */
#define FZ_EB_ABS 0   /* eb is the absolute bound                          */
#define FZ_EB_REL 1   /* eb is relative to the field's value range         */

#define FZ_HEADER_BYTES 64

typedef struct fz_ctx fz_ctx;

/* Stream facts decoded from a 64-byte header (fz_inspect). */
typedef struct fz_info {
  int32_t ndim;           /* 1..3                                          */
  int32_t mode;           /* FZ_EB_ABS or FZ_EB_REL                        */
  uint64_t dims[3];       /* fastest first; unused dims = 1                */
  double eb_requested;    /* the eb argument of fz_compress                */
  float eb;               /* absolute bound in effect (fp32, <= request)   */
  float ebx2;             /* 2*eb                                          */
  float ebx2_r;           /* fl(1/(2eb)), the quantiser's multiplier       */
  float range_min;        /* field min/max in relative mode, else 0        */
  float range_max;
  uint64_t n_tiles;       /* 2048-code tiles                               */
  uint64_t nnz_blocks;    /* non-zero 16-byte blocks in the payload        */
  uint64_t n_outliers;    /* escaped residuals                             */
  uint64_t stream_bytes;  /* 64 + 32*n_tiles + 16*nnz_blocks + 8*n_outliers*/
  uint32_t version;       /* 1: chunk-local Lorenzo (fz_compress), 2:
                             whole-field Lorenzo (fz_compress_whole)       */
  uint32_t wide;          /* 1: some |q| passes 2^22 - 1 (header byte 7)   */
} fz_info;

/* Create a context on CUDA device `device`: allocates the scratch used by
 * the prefix-sum look-back and the result block.  Returns FZ_OK,
 * FZ_ERR_ARG (ctx == NULL) or FZ_ERR_CUDA. */
int fz_create(fz_ctx **ctx, int device);

/* Release a context and its scratch.  NULL is allowed. */
void fz_destroy(fz_ctx *ctx);

/* Worst-case stream size in bytes for a field of these dims (every 16-byte
 * block non-zero and every code escaped).  0 for invalid dims. */
uint64_t fz_compress_bound(const uint64_t dims[3], int ndim);

/* Size of the stream's fixed part (header + flags): any stream of these dims
 * is at least this large.  0 for invalid dims. */
uint64_t fz_stream_min_bytes(const uint64_t dims[3], int ndim);

/* Compress a float32 field (Sec. 3.1 pipeline).
 *   d_in      device pointer to prod(dims[0..ndim)) floats, x fastest
 *   dims/ndim field extents, fastest first, 1 <= ndim <= 3; the field must
 *             have fewer than 2^32 codes after padding to whole tiles
 *   mode/eb   FZ_EB_ABS: eb is the absolute bound; FZ_EB_REL: eb times the
 *             field's value range (Sec. 4.1); eb finite and > 0
 *   d_out     device pointer, 16-byte aligned, out_capacity bytes
 *   out_size  host pointer; receives the stream size on success
 * The stream is a pure function of (input bytes, dims, mode, eb).  A field
 * whose |q| passes 2^22 - 1 (up to 2^28 - 1) takes a second launch with
 * integer quantisation; its stream sets header byte 7 (fz_info.wide).
 * Errors: FZ_ERR_ARG, FZ_ERR_NONFINITE, FZ_ERR_EB_RANGE, FZ_ERR_CAPACITY
 * (*out_size = bytes needed), FZ_ERR_TIMEOUT, FZ_ERR_CUDA. */
int fz_compress(fz_ctx *ctx, const float *d_in, const uint64_t dims[3],
                int ndim, int mode, double eb, void *d_out,
                uint64_t out_capacity, uint64_t *out_size, void *stream);

/* The whole-field Lorenzo variant of fz_compress: the same quantisation,
 * encoding and stream layout, but the residual of every element takes its
 * Lorenzo neighbours anywhere in the field (Eq. 1 with q = 0 only outside
 * the field) instead of inside its chunk (Sec. 2.3), so chunk faces see
 * full-order predictors.  The stream's version byte is 2; fz_decompress
 * reads it (three passes instead of one: the chunks are no longer
 * independent).  The reconstruction equals fz_compress's, element for
 * element.  Same arguments and errors as fz_compress. */
int fz_compress_whole(fz_ctx *ctx, const float *d_in, const uint64_t dims[3],
                      int ndim, int mode, double eb, void *d_out,
                      uint64_t out_capacity, uint64_t *out_size, void *stream);

/* Decompress a stream made by fz_compress or fz_compress_whole (Sec. 4.4).
 *   d_in       device pointer to the stream, 16-byte aligned, in_size bytes
 *   d_out      device pointer to out_capacity_elems floats
 * Writes every element of the field; the reconstruction x' satisfies
 * x' = fl(q * 2eb) with q the pre-quantised value of the original x.  A
 * version-2 stream takes context scratch of 3/2 (3-D), 3/16 (2-D) or
 * 1/1024 (1-D) bytes per element, allocated on first use and kept.
 * Errors: FZ_ERR_ARG, FZ_ERR_CORRUPT (header, sizes, flags or outlier list
 * inconsistent), FZ_ERR_CAPACITY, FZ_ERR_TIMEOUT, FZ_ERR_CUDA. */
int fz_decompress(fz_ctx *ctx, const void *d_in, uint64_t in_size,
                  float *d_out, uint64_t out_capacity_elems, void *stream);

/* Host-buffer forms of the two calls: copy h_in to the device, run the
 * device call on context-owned staging buffers (grown as needed), copy the
 * result back to h_out.  Same arguments and errors as the device forms.
 * fz_decompress_host of a version-1 stream whose field is 64 MiB or more
 * works in up to four slabs of whole chunk planes (3-D), chunk rows (2-D)
 * or chunks (1-D): the stream is copied in on a second stream of the
 * context (header, flags and outlier records first, then the payload in
 * pieces), each slab is decoded once its payload is in, and its part of the
 * field is copied out on a third stream while later slabs are decoded and
 * the rest of the stream comes in.  The call orders itself after earlier
 * work on `stream` and returns when h_out is complete.  h_in and h_out in
 * pinned memory let the copies overlap; pageable buffers work too. */
int fz_compress_host(fz_ctx *ctx, const float *h_in, const uint64_t dims[3],
                     int ndim, int mode, double eb, void *h_out,
                     uint64_t out_capacity, uint64_t *out_size, void *stream);
int fz_decompress_host(fz_ctx *ctx, const void *h_in, uint64_t in_size,
                       float *h_out, uint64_t out_capacity_elems,
                       void *stream);

/* Decode a host copy of a stream's first n >= 64 bytes.  FZ_OK or
 * FZ_ERR_CORRUPT / FZ_ERR_ARG. */
int fz_inspect(const void *h_header, uint64_t n, fz_info *out);

/* Static English message for a status code. */
const char *fz_strerror(int status);

/* Bound, in nanoseconds, on every device-side wait of this context (the
 * prefix-sum look-back and the tile-load barrier).  Default 2e9. */
int fz_set_wait_limit_ns(fz_ctx *ctx, uint64_t ns);

/* Fault injection for tests of the bounded waits: the look-back unit that
 * holds this chunk (the compressor's unit of 14 consecutive tiles, the
 * decompressor's unit of 512 consecutive chunks) skips publishing its
 * aggregate, so later units' waits run out and the call returns
 * FZ_ERR_TIMEOUT.  UINT64_MAX disables. */
int fz_debug_skip_publish(fz_ctx *ctx, uint64_t chunk);

/* Kernel timing for profiling (off by default).  When on, each call
 * records CUDA events around every kernel it launches, on the call's
 * stream, and fz_get_kernel_times fills ms[0..4] with the last call's
 * durations in milliseconds: [0] range pass, [1] compression kernel,
 * [2] outlier pass, [3] decompression kernel, [4] the decompressor's
 * offsets pass (0 for kernels not run).
 * Returns FZ_OK, FZ_ERR_ARG or FZ_ERR_CUDA. */
int fz_set_profiling(fz_ctx *ctx, int on);
int fz_get_kernel_times(fz_ctx *ctx, double ms[5]);

/* Whole-call timing (off by default).  When on, fz_compress and
 * fz_decompress record one CUDA event on their stream when they are
 * entered and one after their last operation on it (the result read-back
 * they wait for), and fz_get_call_times fills ms[0] / ms[1] with the last
 * fz_compress / fz_decompress call's time between the two, in milliseconds
 * (0 before the first such call): the launches, kernels, gaps and read-back
 * of the call, without the caller's own overhead.  Independent of
 * fz_set_profiling.  Returns FZ_OK, FZ_ERR_ARG or FZ_ERR_CUDA. */
int fz_set_call_timing(fz_ctx *ctx, int on);
int fz_get_call_times(fz_ctx *ctx, double ms[2]);

/* ---------------------------------------------------------------------
 * One field split across ranks.  Chunks are independent (Sec. 2.3: the
 * Lorenzo residual never reaches across a chunk), so a field can be cut
 * into slabs of whole chunk rows along its slowest axis, each slab
 * compressed on its own rank, and the slabs' streams concatenated into the
 * stream of the whole field, byte for byte the stream fz_compress makes of
 * it.  The relative bound needs one exchange first: the field's value range
 * (Sec. 4.1), the min and max over every slab.
 *
 * fz_range: value range of a device field of n floats (the relative mode's
 * range pass).  Writes *h_min, *h_max (+0 for zeros of either sign) and
 * *h_nonfinite (1 if some element is NaN or Inf; min/max then unspecified).
 * Synchronises `stream`.  FZ_OK, FZ_ERR_ARG (n == 0, NULL pointer, d_in
 * not 4-byte aligned) or FZ_ERR_CUDA. */
int fz_range(fz_ctx *ctx, const float *d_in, uint64_t n, float *h_min,
             float *h_max, int *h_nonfinite, void *stream);

/* fz_compress in relative mode (Sec. 4.1) against a value range supplied by
 * the caller, [range_min, range_max], instead of d_in's own: the bound is
 * eb * (range_max - range_min), as fz_compress would derive it from a field
 * with that range, and the header records that range.  No range pass runs;
 * every element is still checked (FZ_ERR_NONFINITE, FZ_ERR_EB_RANGE).  A
 * non-finite or inverted range is FZ_ERR_ARG.  Other arguments and errors
 * as fz_compress. */
int fz_compress_ranged(fz_ctx *ctx, const float *d_in, const uint64_t dims[3],
                       int ndim, double eb, float range_min, float range_max,
                       void *d_out, uint64_t out_capacity, uint64_t *out_size,
                       void *stream);

/* Slab `shard` of `n_shards` of a field: the range [*begin, *end) of its
 * slowest axis (z for 3-D, y for 2-D, x for 1-D), whole chunk rows, the rows
 * dealt out as evenly as possible in order.  A shard may be empty
 * (*begin == *end) when there are fewer rows than shards.  Host only.
 * FZ_OK or FZ_ERR_ARG. */
int fz_shard_extent(const uint64_t dims[3], int ndim, int n_shards, int shard,
                    uint64_t *begin, uint64_t *end);

/* Concatenate the streams of consecutive slabs of one field, in slab order,
 * into the stream of the whole field (header totals summed, flags, payloads
 * and outlier lists appended, outlier code indices moved by the codes before
 * each slab).  Every part must come from fz_compress (ABS) or
 * fz_compress_ranged (REL, same range) with the same ndim, mode, eb and
 * non-slowest dims; every part but the last must span whole chunk rows.
 *   d_parts[i]   device pointer to part i, 8-byte aligned, part_sizes[i] bytes
 *   d_out        device pointer, 16-byte aligned, out_capacity bytes
 *   out_size     host pointer; receives the stream size (also on
 *                FZ_ERR_CAPACITY: the size needed)
 * Synchronises `stream`.  FZ_OK, FZ_ERR_ARG, FZ_ERR_CORRUPT (a part's
 * header or size is inconsistent, or the parts do not fit together),
 * FZ_ERR_VERSION (a version-2 part), FZ_ERR_CAPACITY or FZ_ERR_CUDA. */
int fz_concat_streams(fz_ctx *ctx, const void *const *d_parts,
                      const uint64_t *part_sizes, int n_parts, void *d_out,
                      uint64_t out_capacity, uint64_t *out_size, void *stream);

/* The same concatenation of host copies of the parts into host memory (no
 * GPU involved; usable on a rank without one).  h_out may be NULL with
 * out_capacity 0: a size query (FZ_ERR_CAPACITY, *out_size = the size). */
int fz_concat_streams_host(const void *const *h_parts,
                           const uint64_t *part_sizes, int n_parts, void *h_out,
                           uint64_t out_capacity, uint64_t *out_size);

/* The same compression as fz_compress (byte for byte the same stream), run
 * as the paper's sequence of separate kernels with the intermediate data in
 * HBM (Sec. 3; the per-kernel evaluation of Sec. 4.5): pre-quantisation + Lorenzo
 * writing the 16-bit codes, bitshuffle + mark writing the shuffled words and
 * flags, the prefix sum, and the encoding copy.  For measuring what fusing
 * them into one kernel saves.  ms (host, 5 entries, may be NULL) receives
 * the times of the range pass (0 for absolute bounds) and of the four
 * kernels, in ms.  Allocates its intermediate buffers (4 KiB per tile
 * each) in the context on first use.  Same arguments and errors as
 * fz_compress otherwise. */
int fz_compress_staged(fz_ctx *ctx, const float *d_in, const uint64_t dims[3],
                       int ndim, int mode, double eb, void *d_out,
                       uint64_t out_capacity, uint64_t *out_size, double ms[5],
                       void *stream);

/* The bitshuffle of fz_compress_staged (Sec. 3.3, Listing 1):
 * FZ_SHUFFLE_REGISTER (default) transposes each lane's 32 code words in
 * registers; FZ_SHUFFLE_BALLOT is Listing 1's form, 32 warp ballots per
 * 32-word group, one word per lane (plane b of group g to word 32b + g).
 * The stream is the same byte for byte; the choice only changes the time.
 * The fused fz_compress always uses the register transpose.  FZ_OK or
 * FZ_ERR_ARG. */
#define FZ_SHUFFLE_REGISTER 0
#define FZ_SHUFFLE_BALLOT 1
int fz_set_staged_shuffle(fz_ctx *ctx, int kind);

/* ---------------------------------------------------------------------
 * Many fields in one persistent launch.  A batch is planned once for a fixed
 * list of fields (their device buffers, dims and bounds); every run
 * compresses the fields' current contents.  A run is one range pass over the
 * relative-bound fields, one small per-field preparation, one persistent
 * compression launch per dimensionality present (every field with its own
 * look-back domain, so each field's stream is byte for byte what
 * fz_compress makes of it alone), one escape pass per dimensionality and one
 * copy of the per-field results to the host: a fixed sequence, captured in a
 * CUDA graph and replayed on later runs (fz_batch_set_graph).  The paper
 * has no counterpart; its future-work section asks for fusing the kernels. */

typedef struct fz_field {
  const float *d_in;      /* device, 4-byte aligned; dims as fz_compress     */
  uint64_t dims[3];
  int32_t ndim;
  int32_t mode;           /* FZ_EB_ABS or FZ_EB_REL                          */
  double eb;
  void *d_out;            /* device, 16-byte aligned                         */
  uint64_t out_capacity;  /* bytes                                           */
} fz_field;

typedef struct fz_batch fz_batch;

#define FZ_BATCH_MAX_FIELDS 65536

/* Plan a batch of n fields on ctx's device: validates every field (FZ_ERR_ARG;
 * FZ_ERR_CAPACITY when an output cannot hold the header and flags) and
 * allocates the batch's descriptors and scratch (FZ_ERR_CUDA).  Fields
 * whose rows are 16-byte aligned take TMA tile loads, the other 2-D/3-D
 * fields of four rows or more row-class TMA boxes, the rest direct loads
 * (load path [3] of fz_batch_autotune).  The batch keeps ctx for later
 * calls; destroy the batch before the context. */
int fz_batch_create(fz_ctx *ctx, const fz_field *fields, int n, fz_batch **batch);

/* Release a batch.  NULL is allowed. */
void fz_batch_destroy(fz_batch *batch);

/* Run the batch on `stream` and wait for it.  out_sizes[i] and statuses[i]
 * (host arrays of n) receive each field's stream size and status, as
 * fz_compress would report them.  Returns FZ_OK when every field succeeded,
 * else the first failing field's status (FZ_ERR_CUDA for the run itself). */
int fz_batch_compress(fz_batch *batch, uint64_t *out_sizes, int *statuses, void *stream);

/* Capture runs in a CUDA graph (default on) or launch them directly. */
int fz_batch_set_graph(fz_batch *batch, int on);

/* Autotune the batch's load path over four choices, `reps` timed runs
 * each: [0] direct loads for every field; [1] TMA tile loads for the
 * fields whose rows allow them (2-D/3-D, rows 16-byte aligned), direct
 * loads for the others; [2] TMA tile loads for every 2-D/3-D
 * field, the others through staging copies with the row pitch padded to 4
 * elements, written by each run's first pass (about 4 bytes of device
 * memory per element of those fields); [3] TMA for every 2-D/3-D field of
 * four rows or more, the unaligned ones by four row-class boxes per tile
 * (rows grouped by index mod 4 share a 16-byte offset and form a tensor of
 * their own), read in place (the default).  Keeps the fastest.
 * The outputs are overwritten by the trial runs.  fz_batch_tuning reports
 * the choice (tma 0/1/2, staged) and the median run times in ms of the four
 * paths (0 before tuning). */
int fz_batch_autotune(fz_batch *batch, int reps, void *stream);
/* Set the load path by hand: tma 0 (direct loads), 1 (TMA for aligned
 * rows), 2 (TMA for aligned rows, row-class boxes for the others); staged 1
 * with tma 1 (TMA for every 2-D/3-D field through staging copies).
 * Allocates the staging copies when first needed.  FZ_OK, FZ_ERR_ARG or
 * FZ_ERR_CUDA. */
int fz_batch_set_load_path(fz_batch *batch, int tma, int staged);
int fz_batch_tuning(const fz_batch *batch, int *tma, int *staged, double ms[4]);

/* ---------------------------------------------------------------------
 * A request server with continuous batching.  Clients submit compress and
 * decompress requests at any time, from any thread; a worker thread admits
 * them in arrival order while a device-resident pool of pool_bytes has room
 * for the request's input, output and scratch (a later request may pass
 * one that does not fit yet), copies their inputs in, and runs them:
 * every admitted compress request joins the next batched launch (as in
 * fz_batch_*; two batches alternate on two streams, so the next batch is
 * formed, queued and started on the device while one runs), and
 * decompressions run on a third stream beside the batches.  Results stay
 * in the pool until fetched.  Each result equals what fz_compress /
 * fz_decompress return for that input alone.  The paper has no counterpart. */

#define FZ_PENDING 1            /* poll/fetch: the request is not done yet */
#define FZ_OP_COMPRESS 0
#define FZ_OP_DECOMPRESS 1

typedef struct fz_request {
  int32_t op;             /* FZ_OP_COMPRESS or FZ_OP_DECOMPRESS               */
  int32_t ndim;           /* compress: the field (as fz_compress)              */
  uint64_t dims[3];
  int32_t mode;
  int32_t reserved;
  double eb;
  const void *h_in;       /* host: the field (compress) or the stream; must
                             stay valid until the request is done; pinned
                             memory copies without blocking the worker         */
  uint64_t in_bytes;      /* 4 * elements, or the stream's size               */
} fz_request;

typedef struct fz_server_stats {
  uint64_t completed;     /* requests done (since the last reset)             */
  uint64_t failed;        /* of which with an error status                     */
  uint64_t queued;        /* waiting for pool room                             */
  uint64_t in_flight;     /* admitted, not yet done                            */
  uint64_t pool_used, pool_bytes;
  double p50_ms, p99_ms;  /* submit-to-done latency of the completed requests  */
  double seconds;         /* since the last reset                              */
} fz_server_stats;

typedef struct fz_server fz_server;

/* Start a server on `device` with a pool of pool_bytes (>= 1 MiB) and at most
 * max_batch fields per batched launch.  FZ_OK, FZ_ERR_ARG or FZ_ERR_CUDA. */
int fz_server_create(int device, uint64_t pool_bytes, int max_batch, fz_server **server);

/* Stop the worker (requests not done are dropped) and free everything. */
void fz_server_destroy(fz_server *server);

/* Queue a request; *id names it.  FZ_ERR_ARG (bad request), FZ_ERR_CORRUPT
 * (a decompress input whose header or size is inconsistent), FZ_ERR_VERSION
 * (a version-2 stream: fz_decompress reads those) or
 * FZ_ERR_CAPACITY (the request needs more than the whole pool). */
int fz_server_submit(fz_server *server, const fz_request *request, uint64_t *id);

/* FZ_PENDING while the request runs; FZ_OK when done, with *status its
 * result (as the single call would return it) and *size its output bytes
 * (the stream, or 4 * elements). */
int fz_server_poll(fz_server *server, uint64_t id, int *status, uint64_t *size);

/* Copy a done request's output to h_out (capacity bytes; NULL discards it)
 * and release the request.  FZ_PENDING while it runs, FZ_ERR_CAPACITY when
 * h_out is too small (the request stays), FZ_ERR_ARG for an unknown id or a
 * request that failed (which is released). */
int fz_server_fetch(fz_server *server, uint64_t id, void *h_out, uint64_t capacity);

/* Counters and latency percentiles; reset != 0 starts a new window. */
int fz_server_get_stats(fz_server *server, fz_server_stats *stats, int reset);

/* Where a request's time went, for a request not yet fetched.  Host times
 * are ms since the server's creation (steady clock); GPU times are ms since
 * an event the server recorded at its creation, from CUDA events around the
 * request's kernels (the whole batch's, for a compress request).  Fields not
 * reached yet are negative. */
typedef struct fz_request_info {
  uint64_t batch;         /* compress: the batch it ran in, numbered from 1
                             in launch order; decompress: 0                     */
  uint64_t launch_seq;    /* the order in which its GPU work was launched,
                             batches and decompressions counted together
                             from 1                                             */
  double submit_ms;       /* fz_server_submit                                   */
  double admit_ms;        /* pool room found, input copy queued                 */
  double launch_ms;       /* its kernels queued                                 */
  double done_ms;         /* the worker saw them complete                       */
  double gpu_start_ms;    /* its kernels (its batch) began on the device        */
  double gpu_end_ms;      /* ... and ended                                      */
} fz_request_info;
int fz_server_request_info(fz_server *server, uint64_t id, fz_request_info *info);

/* ---------------------------------------------------------------------
 * Compression without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * GPU memory while they run, e.g. an application whose memory pool has
 * already reserved the free HBM (a cudaMalloc would fail or fragment it),
 * a latency-critical loop that cannot pay for cudaMalloc/cudaFree and
 * their device-wide synchronisation, or a deployment with a memory plan
 * fixed in advance.
 *
 * Same arguments, stream format and statuses as fz_compress, but with no
 * context: the look-back and result scratch lives in one statically sized
 * device array inside the library, FZ_NOALLOC_SCRATCH_BYTES (at most
 * 1.75 MiB) per device, kept until the process exits.  That array is not
 * allocated by this call, but the CUDA driver reserves it in device memory
 * when it loads the library's device code on a device, which under lazy
 * module loading (the default) happens at the first call on that device.
 * So make one call on each device at start-up, before a memory pool takes
 * the free HBM, and before any stream capture (the first call also looks up
 * the array's device address).  Fields are limited to FZ_NOALLOC_MAX_CODES
 * codes after padding to whole chunks (a 512^3 field fits); larger fields
 * return FZ_ERR_ARG.  The call uses the calling thread's current device.
 * Every call on a device shares the one array and clears the parts that
 * must start at zero; calls whose GPU work overlaps (different streams or
 * threads at the same time) race on it and must be serialised by the
 * caller.  No cudaMalloc, cudaFree or other allocating routine is called. */
#define FZ_NOALLOC_MAX_CODES 134217728ull
#define FZ_NOALLOC_SCRATCH_BYTES 1835008ull
int fz_compress_noalloc(const float *d_in, const uint64_t dims[3], int ndim,
                        int mode, double eb, void *d_out,
                        uint64_t out_capacity, uint64_t *out_size,
                        void *stream);

/* ---------------------------------------------------------------------
 * Point-wise relative error bounds by log transform (Sec. 4.1: the
 * particle dataset is compressed log-transformed, with the absolute bound
 * that the point-wise relative bound implies).  The caller runs
 *
 *   fz_pwrel_forward(x) -> y, signs;   fz_compress(y, FZ_EB_ABS, eb_abs)
 *   fz_decompress -> y';               fz_pwrel_inverse(y', signs) -> x'
 *
 * with eb_abs from fz_pwrel_bound(eps); then |x' - x| <= eps |x| for every
 * element whose magnitude is 0 or at least FLT_MIN (2^-126), and
 * |x' - x| <= max(eps |x|, 2^-149) for the subnormal ones (the spacing of
 * the subnormal grid).  The sign bits travel beside the stream: one 32-bit
 * word per 32 elements, bit i % 32 of word i / 32 set for a negative x[i]
 * (or -0).
 *
 * fz_pwrel_bound: eb_abs = log2(1 + eps) - 2^-14 (the margin covers the
 * fp32 rounding of the log values, of the quantiser and of the
 * reconstruction at log magnitudes up to 160, and of the transforms
 * themselves).  FZ_OK, or FZ_ERR_ARG unless 1e-4 <= eps <= 0.5.
 *
 * fz_pwrel_forward: y[i] = log2|x[i]| (fp32; -160 for a zero, which
 * fz_pwrel_inverse maps back to 0 exactly: every nonzero float has
 * log2 >= -149), signs as above.  d_x, d_y: n floats each, 4-byte aligned;
 * d_signs: (n + 31) / 32 words.  Synchronises `stream`.  FZ_OK,
 * FZ_ERR_NONFINITE (NaN or Inf in x; y and signs are then unspecified),
 * FZ_ERR_ARG or FZ_ERR_CUDA.
 *
 * fz_pwrel_inverse: x[i] = +-2^y[i] with the sign from d_signs, 0 where
 * y[i] < -154, +-FLT_MAX where y[i] >= 128.  Asynchronous on `stream`.
 * FZ_OK, FZ_ERR_ARG or FZ_ERR_CUDA. */
int fz_pwrel_bound(double eps, double *eb_abs);
int fz_pwrel_forward(fz_ctx *ctx, const float *d_x, uint64_t n, float *d_y,
                     uint32_t *d_signs, void *stream);
int fz_pwrel_inverse(fz_ctx *ctx, const float *d_y, uint64_t n, const uint32_t *d_signs,
                     float *d_x, void *stream);

#ifdef __cplusplus
}
#endif
#endif
