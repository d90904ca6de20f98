// fz_batch_ws.h -- the host side of batched compression: a reusable
// workspace that lays out a list of fields, uploads their descriptors and
// puts one batched run on a stream.  Used by the planned batch (fz_batch_*)
// and by the request server (fz_server_*).  Internal to the library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "fz.h"
#include "fz_device.cuh"

namespace fz {

struct CompressArgs;
struct FieldRt;
struct RangeResult;
struct SetScratch;
struct RangeSlots;

// A segment of one field for the batch's first pass: its value range (a
// relative bound's field) and, for a field whose rows are not 16-byte
// aligned, its elements copied into a staging copy with a padded row pitch
// that the compressor then reads with TMA boxes.
struct RangeSeg {
  const float *x;
  uint64_t n;          // elements in this segment
  uint32_t field;
  uint32_t range;      // 1: the field's relative bound needs its range
  float *dst;          // the field's staging copy (NULL: none this run)
  uint64_t row0;       // x row of the segment's first element
  uint32_t col0;       // and its column
  uint32_t pitch;      // the staging copy's row pitch (elements)
  FastDiv X;           // the field's row length dims[0]
  uint32_t pad;
};


struct WsClass {                   // the fields of one dimensionality
  int ndim = 0;
  bool check = false;              // some field needs the per-element check
  std::vector<uint32_t> fields;
  uint64_t n_units = 0;
  uint64_t unit_off = 0;           // into the unit map
};

class BatchWs {
 public:
  BatchWs() = default;
  BatchWs(const BatchWs &) = delete;
  BatchWs &operator=(const BatchWs &) = delete;
  ~BatchWs() { release(); }

  // Lay out `fields`, growing the device and staging memory when needed,
  // and upload the descriptors on `s` (asynchronously, from pinned
  // staging).  The workspace must be idle: no earlier run still on a stream.
  // FZ_OK, FZ_ERR_ARG, FZ_ERR_CAPACITY (an output smaller than header and
  // flags) or FZ_ERR_CUDA.
  int set(int device, const fz_field *fields, int n, cudaStream_t s);
  // One run of the current fields on `s`: clear, range pass, preparation,
  // compression per dimensionality, escapes, results to pinned memory.
  int enqueue(cudaStream_t s);
  // Per-field sizes and statuses of the last run (after it has completed);
  // ctx (may be NULL) classifies absolute-bound failures as NaN/Inf or range.
  int collect(fz_ctx *ctx, uint64_t *sizes, int *statuses, cudaStream_t s) const;
  // Re-encode the tensor maps for a new load-path choice (idle workspace):
  // tma 1, TMA boxes for fields whose rows are 16-byte aligned; tma 2, also
  // the row-class boxes for the other 2-D/3-D fields (four maps each, see
  // issue_class_boxes); staged (with tma 1), TMA boxes for the others
  // through a staging copy with a padded row pitch that the first pass
  // writes (device memory grown as needed).
  int set_load_path(int tma, bool staged, cudaStream_t s);
  void release();

  uint32_t size() const { return n_; }
  int tma_mode() const { return tma_mode_; }
  bool staged_on() const { return tma_mode_ == 1 && stage_on_; }
  uint64_t wait_limit_ns = 2000000000ull;

 private:
  int upload(cudaStream_t s);

  int device_ = 0;
  int num_sms_ = 1;
  int tma_mode_ = 2;
  bool stage_on_ = false;
  // per field: its offset (floats) in the staging memory, or ~0 when its
  // rows are read in place; the first pass's segments (host copy)
  std::vector<uint64_t> stage_off_;
  std::vector<RangeSeg> segs_;
  size_t o_segs_ = 0;
  uint64_t stage_floats_ = 0;
  float *d_stage_ = nullptr;
  size_t stage_mem_ = 0;
  uint32_t n_ = 0;
  std::vector<fz_field> host_;
  std::vector<CompressArgs> args_;
  std::vector<WsClass> cls_;
  uint64_t total_tiles_ = 0, total_units_ = 0, n_segs_ = 0;
  // device memory: [descriptors | ranges, FieldRt | zeroed: results, slots,
  // counters, status words, outlier prefixes and counts]
  void *d_mem_ = nullptr;
  size_t d_cap_ = 0;
  size_t desc_bytes_ = 0;          // the uploaded prefix
  size_t zero_off_ = 0, zero_bytes_ = 0;
  CompressArgs *d_args_ = nullptr;
  CUtensorMap *d_tmaps_ = nullptr;
  CUtensorMap *d_cmaps_ = nullptr;   // 4 per field: the row-class maps
  uint2 *d_unit_map_ = nullptr;
  RangeSeg *d_segs_ = nullptr;
  uint64_t *d_tile_off_ = nullptr;
  FieldRt *d_rt_ = nullptr;
  RangeResult *d_ranges_ = nullptr;
  SetScratch *d_sets_ = nullptr;   // n fields + one launch-level block
  RangeSlots *d_slots_ = nullptr;
  uint32_t *d_tickets_ = nullptr;
  uint32_t *d_tile_out_ = nullptr;
  // pinned host memory: the descriptor image and the result blocks
  void *h_stage_ = nullptr;
  size_t stage_cap_ = 0;
  SetScratch *h_res_ = nullptr;     // pinned, mapped
  SetScratch *h_res_dev_ = nullptr; // h_res_ as the device addresses it
  uint32_t res_cap_ = 0;
};

// the batch kernels' shared-memory limits (set once, before any capture)
cudaError_t batch_kernel_attrs();

}  // namespace fz
