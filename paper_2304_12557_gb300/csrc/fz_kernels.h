// fz_kernels.h -- launch interface between the C ABI (fz_api.cu) and the
// kernels (fz_compress.cu, fz_decompress.cu).  Internal to the library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

struct fz_ctx;

namespace fz {

// the CUDA device a context was created on (-1 for NULL)
int context_device(const fz_ctx *c);

// kernels timed by fz_get_kernel_times: range, compress, outliers,
// decompress, decompression offsets
constexpr int kProfSlots = 5;

struct SetScratch;
struct RangeResult;
struct FastDiv;

struct CompressArgs {
  const float *x;
  uint64_t dims[3];            // unused dims = 1
  uint64_t pitch;              // elements from one x row to the next: dims[0], or
                               // a batch's row-aligned staging copy's padded pitch
  uint32_t ncx, ncy;           // chunk grid (x, y)
  uint64_t n_chunks;
  int mode;                    // 0 abs, 1 rel
  double eb_req;
  const RangeResult *range;    // relative mode: min/max/non-finite of a range pass
  int range_given;             // relative mode: use [range_lo, range_hi] instead
  float range_lo, range_hi;
  int use_tma;                 // batches: 0 direct loads, 1 one TMA box per tile (rows
                               // 16-byte aligned), 2 row-class boxes (rows not aligned)
  int ndim;                    // batches: the field's dimensionality
  int whole;                   // whole-field Lorenzo (stream version 2): residuals
                               // across chunk faces
  int allow_wide;              // a field past |q| = 2^22 - 1 stops with kErrWide for
                               // a second launch (else kErrRange)
  int wide;                    // this launch uses the wide quantiser (|q| up to
                               // 2^28 - 1), checked against the range pass's
                               // result in *range
  SetScratch *set_cur, *set_next;
  uint64_t *status_cur, *status_next;
  uint32_t *tile_out_prefix;   // per tile: exclusive outlier prefix
  uint32_t *tile_out_count;    // per tile: outliers
  uint8_t *out;
  uint64_t out_capacity;
  uint64_t wait_limit_ns;
  uint64_t skip_publish_chunk; // fault injection for timeout tests
};

struct DecompressArgs {
  const uint8_t *in;
  uint64_t in_size;
  float *out;
  uint64_t out_cap_elems;
  SetScratch *set_cur, *set_next;
  uint64_t *status_cur, *status_next;
  uint64_t status_cap;         // entries available in the status and chunk arrays
  uint32_t *chunk_off;         // per chunk: first payload block (offsets pass)
  uint32_t *chunk_olo;         // per chunk: first outlier record (offsets pass)
  uint64_t wait_limit_ns;
  uint64_t skip_publish_chunk;
  // Stream version 2 (whole-field Lorenzo).  accept_whole: the offsets pass
  // takes version-2 headers (else they fail the header check).  phase 0:
  // version 1 written out, a version-2 stream left alone (the caller runs
  // phases 1 and 2); phase 1: each chunk's chunk-local prefix sums L on its
  // three upper faces to face[0..2]; phase 2: L plus the cross-chunk
  // corrections corr[0..2], written out.  Face layouts in fz_whole.cu.
  int accept_whole;
  int phase;
  int wide;                    // streams of the wide quantiser (header byte 7): the
                               // kernels that convert q as integers
  int32_t *face[3];
  const int32_t *corr[3];
  // decompress only the chunks [chunk_lo, chunk_hi) (chunk_hi 0: to the
  // last chunk); the offsets pass always covers the whole stream
  uint64_t chunk_lo, chunk_hi;
};

// Version-2 decompression, between phases 1 and 2: the cross-chunk sums of
// the faces (fz_whole.cu).  face[k] and work[k] hold face_elems(ndim, k)
// words per chunk; the corrections end up in corr[k], which points into
// face or work.  n_chunk[3]: the chunk grid.
int whole_face_elems(int ndim, int k);
cudaError_t launch_whole_scans(int ndim, const uint32_t n_chunk[3], int32_t *const face[3],
                               int32_t *const work[3], const int32_t *corr[3], cudaStream_t s);

void launch_range(const float *x, uint64_t n, float2 *partial, int nblocks,
                  RangeResult *res, cudaStream_t s);
// True when the compression kernel for this field reads its tiles through
// TMA (2-D/3-D fields whose rows are 16-byte aligned); the caller then
// passes a tensor map from encode_field_tmap.
bool compress_uses_tma(int ndim, const CompressArgs &a);
bool encode_field_tmap(int ndim, const uint64_t dims[3], const float *x, CUtensorMap *tm);
// the same for rows `pitch` elements apart (pitch * 4 a multiple of 16)
// The four row-class maps of a 2-D/3-D field whose rows need not be 16-byte
// aligned (rows R = y + Y z by R mod 4; see issue_class_boxes): false when
// the field has fewer than four rows or a map does not encode.
bool encode_class_tmaps(int ndim, const uint64_t dims[3], uint64_t pitch, const float *x,
                        CUtensorMap tm[4]);
bool encode_field_tmap_pitch(int ndim, const uint64_t dims[3], uint64_t pitch, const float *x,
                             CUtensorMap *tm);
// Tiles per look-back unit of a single-field compression (the compression
// kernel's compute warps per block; fz_compress_impl.cuh checks the two agree).
constexpr uint64_t kCompressUnitTiles = 15;
// look-back status words (one per unit of consecutive tiles) a compression
// of n_tiles tiles uses and clears in the other set
constexpr uint64_t compress_status_words(uint64_t n_tiles) {
  return (n_tiles + kCompressUnitTiles - 1) / kCompressUnitTiles;
}
// after_range: the launch directly follows launch_range on stream s; the
// compressor is then scheduled while the range pass finishes and waits for
// its result on the device (programmatic dependent launch)
cudaError_t launch_compress(int ndim, const CompressArgs &a, const CUtensorMap *tm, int sms,
                            cudaStream_t s, bool after_range = false);
cudaError_t launch_outliers(int ndim, const CompressArgs &a, uint64_t out_section,
                            cudaStream_t s);
// offsets pass (header check, per-chunk payload and outlier offsets) over
// at most max_chunks chunks on a grid of at most 2 * sms blocks, then the
// decompression proper, which may be scheduled while the offsets pass
// finishes (it waits for the pass's results on the device).  The kernel's
// shared-memory attribute is set by decompress_blocks_per_sm(), which a
// context or server calls on its device before its first launch.
cudaError_t launch_dec_offsets(const DecompressArgs &a, uint64_t max_chunks, int sms,
                               cudaStream_t s);
cudaError_t launch_decompress(const DecompressArgs &a, int grid, cudaStream_t s);
// look-back status words the offsets pass uses and clears in the other set
// one warp copies a 64-byte result block to (mapped host) memory, after the
// kernel before it on the stream (programmatic dependent launch)
cudaError_t launch_copy_result(const SetScratch *src, SetScratch *dst, cudaStream_t s);
// dst[i] = src[idx[i]] for i < n <= 8 (one warp; dst may be mapped host memory)
struct GatherIdx {
  uint64_t idx[8];
};
cudaError_t launch_gather_u32(const uint32_t *src, GatherIdx idx, int n, uint32_t *dst,
                              cudaStream_t s);
uint64_t decompress_status_words(uint64_t n_chunks);

// the unfused compression path (fz_staged.cu): intermediate data in HBM
struct StagedScratch {
  uint32_t *codes;             // per tile: 1024 code words
  uint32_t *shuf;              // per tile: 1024 shuffled words
  uint32_t *tile_nnz;          // per tile: non-zero blocks
  uint64_t *tile_excl;         // per tile: exclusive (blocks << 32 | escapes)
  uint64_t *status;            // look-back words of the scan (zero at launch)
};
// ballot: the bitshuffle step by warp ballots (Listing 1) instead of the
// register transpose; ev (may be NULL): 5 events recorded before, between
// and after the 4 kernels
cudaError_t launch_staged(int ndim, const CompressArgs &a, const StagedScratch &w, int sms,
                          bool ballot, cudaEvent_t *ev, cudaStream_t s);
uint64_t staged_status_words(uint64_t n_tiles);

// concatenation of slab streams (fz_shard.cu)
struct ConcatPart {
  uint64_t tiles, nnz, nout;              // the part's own counts
  uint64_t tile_off, nnz_off, out_off;    // counts of the parts before it
};
struct ConcatPlan {
  uint8_t hdr[64];                        // the whole field's header
  uint64_t n_tiles, nnz, nout, total;
};
// Validate the parts' headers (host copies) and sizes; FZ_OK or an FZ_ERR_*.
int concat_plan(const uint8_t (*hdrs)[64], const uint64_t *sizes, int n, ConcatPart *parts,
                ConcatPlan *plan);
// dst[i] = src[i] with the code index moved by `add` (n 8-byte records)
cudaError_t launch_rebase_outliers(const void *src, void *dst, uint64_t n, uint32_t add,
                                   cudaStream_t s);
int decompress_blocks_per_sm();

}  // namespace fz
