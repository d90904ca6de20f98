// fz_server.cu -- a request server with continuous batching on one GPU.
//
// Clients submit compress and decompress requests at any time (host
// buffers in, results kept in a device-resident pool until fetched).  A
// worker thread runs the loop:
//   completions  batches and decompressions whose events have fired;
//   admission    queued requests in arrival order (a later, smaller request
//                may pass one that does not fit yet) while the pool has room
//                for the request's input, output and scratch;
//   uploads      host -> pool copies of the admitted inputs (upload stream);
//   compression  every admitted compress request joins the next batched
//                launch (fz_batch_ws.h); two workspaces alternate, each on
//                its own stream, so the next batch is formed, queued and
//                started on the device while the previous one runs;
//   decompression admitted streams, each with its own scratch, on a third
//                stream: its kernels fill the device beside the batches.
// CUDA events around every batch and decompression, against one recorded
// at start-up, give each request's device interval (fz_server_request_info).
// Every request's result is computed exactly as the single calls compute it
// (the batch keeps one look-back domain per field; a decompression has its
// own scratch), so it does not depend on what else is in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fz.h"
#include "fz_batch_ws.h"
#include "fz_device.cuh"
#include "fz_kernels.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr uint64_t kAlign = 256;
constexpr uint64_t kNone = ~0ull;

uint64_t align_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// first fit over one device allocation; offsets 256-byte aligned
class Pool {
 public:
  bool init(uint64_t bytes) {
    bytes = bytes / kAlign * kAlign;
    if (bytes == 0 || cudaMalloc(&base_, bytes) != cudaSuccess) return false;
    cap_ = bytes;
    free_[0] = bytes;
    return true;
  }
  void destroy() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  uint64_t alloc(uint64_t bytes) {
    bytes = align_up(bytes ? bytes : 1, kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const uint64_t off = it->first, size = it->second;
      free_.erase(it);
      if (size > bytes) free_[off + bytes] = size - bytes;
      used_ += bytes;
      return off;
    }
    return kNone;
  }
  void release(uint64_t off, uint64_t bytes) {
    if (off == kNone) return;
    bytes = align_up(bytes ? bytes : 1, kAlign);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint8_t *ptr(uint64_t off) const { return static_cast<uint8_t *>(base_) + off; }
  uint64_t used() const { return used_; }
  uint64_t capacity() const { return cap_; }

 private:
  void *base_ = nullptr;
  uint64_t cap_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

enum State { kQueued, kAdmitted, kRunning, kDone, kFetched };

struct Req {
  uint64_t id = 0;
  int op = FZ_OP_COMPRESS;
  State state = kQueued;
  // compress: the field; decompress: the stream
  const void *h_in = nullptr;
  uint64_t in_bytes = 0;
  uint64_t dims[3] = {1, 1, 1};
  int ndim = 0, mode = FZ_EB_REL;
  double eb = 0.0;
  bool wide = false;             // decompress: a stream of the wide quantiser
  // pool memory
  uint64_t in_off = kNone, out_off = kNone, scratch_off = kNone;
  uint64_t out_cap = 0, scratch_bytes = 0;
  bool full_bound = false;         // compress: output sized for every escape
  // decompress
  uint64_t n_elems = 0, n_chunks = 0, max_chunks = 0;
  int slot = -1;                   // pinned result slot
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  // result
  int status = FZ_OK;
  uint64_t size = 0;
  Clock::time_point t_submit, t_done;
  // where the time went (fz_server_request_info)
  uint64_t batch = 0, launch_seq = 0;
  double admit_ms = -1.0, launch_ms = -1.0, gpu_start_ms = -1.0, gpu_end_ms = -1.0;
};

}  // namespace

struct fz_server {
  int device = 0;
  fz_ctx *ctx = nullptr;
  int max_batch = 256, max_dec = 8;
  int dec_grid = 1, num_sms = 1;
  Pool pool;
  cudaStream_t s_up = nullptr, s_comp[2] = {nullptr, nullptr}, s_dec = nullptr, s_down = nullptr;
  fz::BatchWs ws[2];
  bool ws_busy[2] = {false, false};
  cudaEvent_t ws_ev[2] = {nullptr, nullptr};       // batch done (also its end time)
  cudaEvent_t ws_start[2] = {nullptr, nullptr};    // batch start time
  uint64_t ws_batch[2] = {0, 0};
  cudaEvent_t ev_epoch = nullptr;                  // device time zero
  Clock::time_point t_epoch = Clock::now();        // host time zero
  uint64_t n_batches = 0, n_launches = 0;
  std::vector<uint64_t> ws_ids[2];
  int ws_next = 0;
  cudaEvent_t ev_uploads = nullptr;
  fz::SetScratch *h_slots = nullptr;   // pinned, max_dec
  std::vector<int> free_slots;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> queued;
  std::vector<uint64_t> adm_comp, adm_dec, run_dec;
  uint64_t next_id = 1;
  std::vector<double> lat_ms;
  uint64_t completed = 0, failed = 0;
  Clock::time_point t_stats = Clock::now();
};

namespace {

uint64_t compress_out_cap(const Req &r, uint64_t tiles) {
  // header, flags and every block of every tile; escapes (8 bytes each) are
  // rare: 64 KiB for them first, every code when that was not enough
  if (r.full_bound) return 64 + 32 * tiles + 4096 * tiles + 8ull * fz::kTileCodes * tiles;
  return 64 + 32 * tiles + 4096 * tiles + 65536;
}

double host_ms(const fz_server *S, Clock::time_point t) {
  return std::chrono::duration<double, std::milli>(t - S->t_epoch).count();
}
double gpu_ms(const fz_server *S, cudaEvent_t e) {
  float ms = -1.f;
  if (!e || cudaEventElapsedTime(&ms, S->ev_epoch, e) != cudaSuccess) return -1.0;
  return ms;
}

// pool memory a request needs; false when it can never fit
bool sizes_of(fz_server *S, Req &r) {
  if (r.op == FZ_OP_COMPRESS) {
    const uint64_t tiles = (fz_stream_min_bytes(r.dims, r.ndim) - 64) / 32;
    r.out_cap = compress_out_cap(r, tiles);
    r.scratch_bytes = 0;
  } else {
    const uint64_t units = fz::decompress_status_words(r.max_chunks);
    r.out_cap = 4 * r.n_elems;
    r.scratch_bytes = 2 * sizeof(fz::SetScratch) + 2 * units * fz::kStatusStride * 8 +
                      2 * align_up(4 * r.max_chunks, kAlign);
  }
  const uint64_t need = align_up(r.in_bytes, kAlign) + align_up(r.out_cap, kAlign) +
                        align_up(r.scratch_bytes, kAlign);
  return need <= S->pool.capacity();
}

// under S->mu: admit in arrival order, letting a later request pass one that
// does not fit yet (a window of 64)
void admit(fz_server *S, std::vector<uint64_t> &uploads) {
  int seen = 0;
  for (auto it = S->queued.begin(); it != S->queued.end() && seen < 64; ++seen) {
    Req &r = S->reqs[*it];
    const uint64_t in = S->pool.alloc(r.in_bytes);
    if (in == kNone) {
      ++it;
      continue;
    }
    const uint64_t out = S->pool.alloc(r.out_cap);
    const uint64_t scr = r.scratch_bytes ? S->pool.alloc(r.scratch_bytes) : 0;
    if (out == kNone || (r.scratch_bytes && scr == kNone)) {
      S->pool.release(in, r.in_bytes);
      if (out != kNone) S->pool.release(out, r.out_cap);
      ++it;
      continue;
    }
    r.in_off = in;
    r.out_off = out;
    r.scratch_off = r.scratch_bytes ? scr : kNone;
    r.state = kAdmitted;
    r.admit_ms = host_ms(S, Clock::now());
    (r.op == FZ_OP_COMPRESS ? S->adm_comp : S->adm_dec).push_back(r.id);
    uploads.push_back(r.id);
    it = S->queued.erase(it);
  }
}

void finish(fz_server *S, Req &r, int status, uint64_t size) {
  r.status = status;
  r.size = size;
  r.state = kDone;
  r.t_done = Clock::now();
  S->pool.release(r.in_off, r.in_bytes);
  r.in_off = kNone;
  if (r.scratch_off != kNone) S->pool.release(r.scratch_off, r.scratch_bytes);
  r.scratch_off = kNone;
  if (status != FZ_OK) {
    S->pool.release(r.out_off, r.out_cap);
    r.out_off = kNone;
    ++S->failed;
  }
  ++S->completed;
  S->lat_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
}

// one pass of the loop; returns whether anything happened
bool step(fz_server *S) {
  bool did = false;
  // ---- completions: batches
  for (int w = 0; w < 2; ++w) {
    if (!S->ws_busy[w] || cudaEventQuery(S->ws_ev[w]) != cudaSuccess) continue;
    const uint32_t n = (uint32_t)S->ws_ids[w].size();
    std::vector<uint64_t> sizes(n);
    std::vector<int> sts(n);
    S->ws[w].collect(S->ctx, sizes.data(), sts.data(), S->s_comp[w]);
    const double g0 = gpu_ms(S, S->ws_start[w]), g1 = gpu_ms(S, S->ws_ev[w]);
    std::lock_guard<std::mutex> lk(S->mu);
    for (uint32_t i = 0; i < n; ++i) {
      Req &r = S->reqs[S->ws_ids[w][i]];
      r.gpu_start_ms = g0;
      r.gpu_end_ms = g1;
      if (sts[i] == FZ_ERR_CAPACITY && !r.full_bound) {
        // escapes overflowed the first output: again with room for all of them
        S->pool.release(r.out_off, r.out_cap);
        r.full_bound = true;
        sizes_of(S, r);
        r.out_off = kNone;
        S->pool.release(r.in_off, r.in_bytes);
        r.in_off = kNone;
        r.state = kQueued;
        S->queued.push_front(r.id);
        continue;
      }
      finish(S, r, sts[i], sizes[i]);
    }
    S->ws_ids[w].clear();
    S->ws_busy[w] = false;
    did = true;
  }
  // ---- completions: decompressions
  for (auto it = S->run_dec.begin(); it != S->run_dec.end();) {
    Req *rp;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      rp = &S->reqs[*it];
    }
    Req &r = *rp;
    if (cudaEventQuery(r.ev_done) != cudaSuccess) {
      ++it;
      continue;
    }
    const fz::SetScratch res = S->h_slots[r.slot];
    r.gpu_start_ms = gpu_ms(S, r.ev_start);
    r.gpu_end_ms = gpu_ms(S, r.ev_done);
    int st = FZ_OK;
    if (res.err & fz::kErrTimeout) st = FZ_ERR_TIMEOUT;
    else if (res.err & fz::kErrCorrupt) st = FZ_ERR_CORRUPT;
    else if (res.err & fz::kErrCapacity) st = FZ_ERR_CAPACITY;
    else if (res.nout != res.hdr_nout) st = FZ_ERR_CORRUPT;
    std::lock_guard<std::mutex> lk(S->mu);
    S->free_slots.push_back(r.slot);
    r.slot = -1;
    finish(S, r, st, st == FZ_OK ? 4 * r.n_elems : 0);
    it = S->run_dec.erase(it);
    did = true;
  }
  // ---- admission and uploads
  std::vector<uint64_t> uploads;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    admit(S, uploads);
  }
  for (uint64_t id : uploads) {
    Req *rp;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      rp = &S->reqs[id];
    }
    cudaMemcpyAsync(S->pool.ptr(rp->in_off), rp->h_in, rp->in_bytes, cudaMemcpyHostToDevice,
                    S->s_up);
    did = true;
  }
  if (!uploads.empty()) cudaEventRecord(S->ev_uploads, S->s_up);
  // ---- compression: the admitted requests join the next batch
  for (int k = 0; k < 2; ++k) {
    const int w = S->ws_next;
    std::vector<uint64_t> ids;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->ws_busy[w] || S->adm_comp.empty()) break;
      const size_t take = std::min<size_t>(S->adm_comp.size(), (size_t)S->max_batch);
      ids.assign(S->adm_comp.begin(), S->adm_comp.begin() + take);
      S->adm_comp.erase(S->adm_comp.begin(), S->adm_comp.begin() + take);
    }
    std::vector<fz_field> fields(ids.size());
    const uint64_t batch = ++S->n_batches, seq = ++S->n_launches;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const double now = host_ms(S, Clock::now());
      for (size_t i = 0; i < ids.size(); ++i) {
        Req &r = S->reqs[ids[i]];
        fz_field &f = fields[i];
        f.d_in = reinterpret_cast<const float *>(S->pool.ptr(r.in_off));
        for (int d = 0; d < 3; ++d) f.dims[d] = r.dims[d];
        f.ndim = r.ndim;
        f.mode = r.mode;
        f.eb = r.eb;
        f.d_out = S->pool.ptr(r.out_off);
        f.out_capacity = r.out_cap;
        r.state = kRunning;
        r.batch = batch;
        r.launch_seq = seq;
        r.launch_ms = now;
      }
    }
    cudaStream_t sc = S->s_comp[w];
    cudaStreamWaitEvent(sc, S->ev_uploads, 0);
    int st = S->ws[w].set(S->device, fields.data(), (int)fields.size(), sc);
    if (st == FZ_OK) st = cudaEventRecord(S->ws_start[w], sc) == cudaSuccess ? FZ_OK : FZ_ERR_CUDA;
    if (st == FZ_OK) st = S->ws[w].enqueue(sc);
    if (st == FZ_OK) cudaEventRecord(S->ws_ev[w], sc);
    if (st != FZ_OK) {
      std::lock_guard<std::mutex> lk(S->mu);
      for (uint64_t id : ids) finish(S, S->reqs[id], st, 0);
      continue;
    }
    S->ws_ids[w] = ids;
    S->ws_batch[w] = batch;
    S->ws_busy[w] = true;
    S->ws_next = 1 - w;
    did = true;
  }
  // ---- decompression: each admitted stream on the second stream
  while (true) {
    Req *rp = nullptr;
    int slot = -1;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->adm_dec.empty() || S->free_slots.empty()) break;
      rp = &S->reqs[S->adm_dec.front()];
      S->adm_dec.erase(S->adm_dec.begin());
      slot = S->free_slots.back();
      S->free_slots.pop_back();
      rp->state = kRunning;
      rp->slot = slot;
      rp->launch_seq = ++S->n_launches;
      rp->launch_ms = host_ms(S, Clock::now());
    }
    Req &r = *rp;
    uint8_t *scr = S->pool.ptr(r.scratch_off);
    const uint64_t units = fz::decompress_status_words(r.max_chunks);
    fz::DecompressArgs a{};
    a.in = S->pool.ptr(r.in_off);
    a.in_size = r.in_bytes;
    a.out = reinterpret_cast<float *>(S->pool.ptr(r.out_off));
    a.out_cap_elems = r.n_elems;
    a.set_cur = reinterpret_cast<fz::SetScratch *>(scr);
    a.set_next = a.set_cur + 1;
    a.status_cur = reinterpret_cast<uint64_t *>(scr + 2 * sizeof(fz::SetScratch));
    a.status_next = a.status_cur + units * fz::kStatusStride;
    a.status_cap = r.max_chunks;
    uint8_t *arrays = scr + 2 * sizeof(fz::SetScratch) + 2 * units * fz::kStatusStride * 8;
    a.chunk_off = reinterpret_cast<uint32_t *>(arrays);
    a.chunk_olo = reinterpret_cast<uint32_t *>(arrays + align_up(4 * r.max_chunks, kAlign));
    a.wait_limit_ns = 2000000000ull;
    a.skip_publish_chunk = ~0ull;
    a.wide = r.wide ? 1 : 0;
    a.chunk_lo = 0;
    a.chunk_hi = 0;                                // every chunk
    cudaStreamWaitEvent(S->s_dec, S->ev_uploads, 0);
    cudaEventRecord(r.ev_start, S->s_dec);
    cudaMemsetAsync(scr, 0, 2 * sizeof(fz::SetScratch) + units * fz::kStatusStride * 8, S->s_dec);
    fz::launch_dec_offsets(a, r.max_chunks, S->num_sms, S->s_dec);
    fz::launch_decompress(a, S->dec_grid, S->s_dec);
    cudaMemcpyAsync(&S->h_slots[slot], a.set_cur, sizeof(fz::SetScratch), cudaMemcpyDeviceToHost,
                    S->s_dec);
    cudaEventRecord(r.ev_done, S->s_dec);
    S->run_dec.push_back(r.id);
    did = true;
  }
  return did;
}

void loop(fz_server *S) {
  cudaSetDevice(S->device);
  while (true) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) break;
    }
    if (!step(S)) {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) break;
      S->cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int fz_server_create(int device, uint64_t pool_bytes, int max_batch, fz_server **out) {
  if (!out) return FZ_ERR_ARG;
  *out = nullptr;
  if (pool_bytes < (1ull << 20) || max_batch < 1 || max_batch > FZ_BATCH_MAX_FIELDS)
    return FZ_ERR_ARG;
  fz_server *S = new (std::nothrow) fz_server();
  if (!S) return FZ_ERR_CUDA;
  S->device = device;
  S->max_batch = max_batch;
  int prev = -1;
  cudaGetDevice(&prev);
  bool ok = fz_create(&S->ctx, device) == FZ_OK && cudaSetDevice(device) == cudaSuccess &&
            S->pool.init(pool_bytes) &&
            cudaStreamCreateWithFlags(&S->s_up, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->s_comp[0], cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->s_comp[1], cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->s_dec, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->s_down, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&S->ev_uploads, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreate(&S->ws_ev[0]) == cudaSuccess &&
            cudaEventCreate(&S->ws_ev[1]) == cudaSuccess &&
            cudaEventCreate(&S->ws_start[0]) == cudaSuccess &&
            cudaEventCreate(&S->ws_start[1]) == cudaSuccess &&
            cudaEventCreate(&S->ev_epoch) == cudaSuccess &&
            cudaMallocHost(&S->h_slots, S->max_dec * sizeof(fz::SetScratch)) == cudaSuccess;
  if (ok) {
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    S->num_sms = sms;
    S->dec_grid = sms * fz::decompress_blocks_per_sm();
    for (int i = 0; i < S->max_dec; ++i) S->free_slots.push_back(i);
    cudaEventRecord(S->ev_uploads, S->s_up);
    cudaEventRecord(S->ev_epoch, S->s_up);
    cudaEventSynchronize(S->ev_epoch);
    S->t_epoch = Clock::now();
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (!ok) {
    fz_server_destroy(S);
    return FZ_ERR_CUDA;
  }
  S->worker = std::thread(loop, S);
  *out = S;
  return FZ_OK;
}

void fz_server_destroy(fz_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  for (cudaStream_t s : {S->s_up, S->s_comp[0], S->s_comp[1], S->s_dec, S->s_down})
    if (s) cudaStreamSynchronize(s);
  for (auto &kv : S->reqs) {
    if (kv.second.ev_done) cudaEventDestroy(kv.second.ev_done);
    if (kv.second.ev_start) cudaEventDestroy(kv.second.ev_start);
  }
  S->ws[0].release();
  S->ws[1].release();
  for (cudaStream_t s : {S->s_up, S->s_comp[0], S->s_comp[1], S->s_dec, S->s_down})
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : {S->ev_uploads, S->ws_ev[0], S->ws_ev[1], S->ws_start[0], S->ws_start[1],
                        S->ev_epoch})
    if (e) cudaEventDestroy(e);
  if (S->h_slots) cudaFreeHost(S->h_slots);
  S->pool.destroy();
  if (S->ctx) fz_destroy(S->ctx);
  if (prev >= 0) cudaSetDevice(prev);
  delete S;
}

int fz_server_submit(fz_server *S, const fz_request *q, uint64_t *id) {
  if (!S || !q || !id || !q->h_in) return FZ_ERR_ARG;
  *id = 0;
  Req r;
  r.op = q->op;
  r.h_in = q->h_in;
  if (q->op == FZ_OP_COMPRESS) {
    if (q->ndim < 1 || q->ndim > 3 || (q->mode != FZ_EB_ABS && q->mode != FZ_EB_REL) ||
        !(q->eb > 0.0) || fz_stream_min_bytes(q->dims, q->ndim) == 0)
      return FZ_ERR_ARG;
    r.ndim = q->ndim;
    r.mode = q->mode;
    r.eb = q->eb;
    uint64_t n = 1;
    for (int d = 0; d < 3; ++d) {
      r.dims[d] = d < q->ndim ? q->dims[d] : 1;
      n *= r.dims[d];
    }
    r.in_bytes = 4 * n;
    if (q->in_bytes != r.in_bytes) return FZ_ERR_ARG;
  } else if (q->op == FZ_OP_DECOMPRESS) {
    fz_info info;
    if (fz_inspect(q->h_in, q->in_bytes, &info) != FZ_OK) return FZ_ERR_CORRUPT;
    if (info.stream_bytes != q->in_bytes) return FZ_ERR_CORRUPT;
    if (info.version != 1) return FZ_ERR_VERSION;
    r.wide = info.wide != 0;
    r.in_bytes = q->in_bytes;
    r.n_elems = info.dims[0] * info.dims[1] * info.dims[2];
    r.n_chunks = info.n_tiles / fz::kTilesPerChunk;
    r.max_chunks = r.n_chunks;
  } else {
    return FZ_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (!sizes_of(S, r)) return FZ_ERR_CAPACITY;     // larger than the whole pool
  if (r.op == FZ_OP_DECOMPRESS &&
      (cudaEventCreate(&r.ev_done) != cudaSuccess || cudaEventCreate(&r.ev_start) != cudaSuccess)) {
    if (r.ev_done) cudaEventDestroy(r.ev_done);
    return FZ_ERR_CUDA;
  }
  r.id = S->next_id++;
  r.t_submit = Clock::now();
  S->reqs.emplace(r.id, r);
  S->queued.push_back(r.id);
  S->cv.notify_all();
  *id = r.id;
  return FZ_OK;
}

int fz_server_poll(fz_server *S, uint64_t id, int *status, uint64_t *size) {
  if (!S || !status || !size) return FZ_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end() || it->second.state == kFetched) return FZ_ERR_ARG;
  if (it->second.state != kDone) return FZ_PENDING;
  *status = it->second.status;
  *size = it->second.size;
  return FZ_OK;
}

int fz_server_fetch(fz_server *S, uint64_t id, void *h_out, uint64_t capacity) {
  if (!S) return FZ_ERR_ARG;
  uint64_t off, size;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || it->second.state == kFetched) return FZ_ERR_ARG;
    Req &r = it->second;
    if (r.state != kDone) return FZ_PENDING;
    if (r.status != FZ_OK) {
      if (r.ev_done) cudaEventDestroy(r.ev_done);
      if (r.ev_start) cudaEventDestroy(r.ev_start);
      S->reqs.erase(it);
      return FZ_ERR_ARG;
    }
    if (h_out && capacity < r.size) return FZ_ERR_CAPACITY;
    off = r.out_off;
    size = r.size;
  }
  int st = FZ_OK;
  if (h_out) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    if (cudaMemcpyAsync(h_out, S->pool.ptr(off), size, cudaMemcpyDeviceToHost, S->s_down) !=
            cudaSuccess ||
        cudaStreamSynchronize(S->s_down) != cudaSuccess)
      st = FZ_ERR_CUDA;
    if (prev >= 0) cudaSetDevice(prev);
  }
  std::lock_guard<std::mutex> lk(S->mu);
  Req &r = S->reqs[id];
  S->pool.release(r.out_off, r.out_cap);
  if (r.ev_done) cudaEventDestroy(r.ev_done);
  if (r.ev_start) cudaEventDestroy(r.ev_start);
  S->reqs.erase(id);
  S->cv.notify_all();
  return st;
}

int fz_server_request_info(fz_server *S, uint64_t id, fz_request_info *info) {
  if (!S || !info) return FZ_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end() || it->second.state == kFetched) return FZ_ERR_ARG;
  const Req &r = it->second;
  info->batch = r.batch;
  info->launch_seq = r.launch_seq;
  info->submit_ms = host_ms(S, r.t_submit);
  info->admit_ms = r.admit_ms;
  info->launch_ms = r.launch_ms;
  info->done_ms = r.state == kDone ? host_ms(S, r.t_done) : -1.0;
  info->gpu_start_ms = r.gpu_start_ms;
  info->gpu_end_ms = r.gpu_end_ms;
  return FZ_OK;
}

int fz_server_get_stats(fz_server *S, fz_server_stats *out, int reset) {
  if (!S || !out) return FZ_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = S->queued.size();
  out->in_flight = S->adm_comp.size() + S->adm_dec.size() + S->run_dec.size() +
                   S->ws_ids[0].size() + S->ws_ids[1].size();
  out->pool_used = S->pool.used();
  out->pool_bytes = S->pool.capacity();
  out->p50_ms = percentile(S->lat_ms, 0.5);
  out->p99_ms = percentile(S->lat_ms, 0.99);
  out->seconds = std::chrono::duration<double>(Clock::now() - S->t_stats).count();
  if (reset) {
    S->lat_ms.clear();
    S->completed = 0;
    S->failed = 0;
    S->t_stats = Clock::now();
  }
  return FZ_OK;
}

}  // extern "C"
