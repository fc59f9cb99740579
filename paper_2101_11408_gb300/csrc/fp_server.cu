// fp_server.cu -- the request server of include/fpparse.h (fp_server_*):
// continuous batching of host-memory parse requests on one GPU.
//
// One scheduler thread per server runs a polling loop of four steps:
//   retire  a slot whose launch has ended completes its requests (after
//           copying back the results of any request whose host arrays the
//           device cannot reach) and releases their arena units;
//   take    new submissions move to the pending queue (FIFO);
//   admit   pending requests get arena units in arrival order while they
//           fit;
//   launch  each free slot takes the admitted requests not yet launched, in
//           order, up to launch_bytes of text (at least one request, at most
//           max_batch) and queues on its own stream: the texts in
//           (one gather kernel for the small requests, a copy call for each
//           request of 1 MB or more), the persistent batched parse and its
//           fallback, one scatter kernel for the small requests' results
//           (first min(count, cap), arena -> the caller's pinned arrays) and
//           the copy of the counts; large requests' results follow by copy
//           calls of exactly their counts once those are back.
// The slots' streams overlap on the device: one batch's texts come in
// while another is parsed and a third one's results go out.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fpparse.h"
#include "fp_arena.h"
#include "fp_copy.h"
#include "fp_internal.h"

namespace {

constexpr uint64_t UNIT_ROUND = 256;       // units of a request are rounded up to this
// Requests of at least this many bytes move by copy engines (one copy call
// each way costs little next to their bytes, and copy engines leave the SMs
// to the parse); smaller ones by the gather / scatter kernels.
constexpr uint64_t ENGINE_BYTES = 1u << 20;
// By default a launch takes admitted requests up to this many text bytes (at
// least one request), so that under load consecutive launches on different
// slots overlap their copies in, parses and copies out.
constexpr uint64_t LAUNCH_BYTES = 32u << 20;
constexpr uint64_t MIN_BUDGET = 4096;
constexpr uint32_t MAX_SLOTS = 8;
constexpr uint32_t MAX_BATCH = 65536;
constexpr unsigned long long MAX_LEN = 1ull << 40;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t id = 0;
  const char* h_text = nullptr;
  size_t len = 0;
  double* h_f64 = nullptr;
  uint8_t* h_status = nullptr;
  size_t out_cap = 0;           // entries of h_f64 / h_status
  // device views of the host arrays (null: the device cannot reach them,
  // so the copy calls move them)
  const uint8_t* dv_text = nullptr;
  unsigned long long* dv_f64 = nullptr;
  uint8_t* dv_status = nullptr;
  uint64_t off = 0, units = 0;  // arena range while admitted
  uint64_t text_off = 0;        // where the text starts: off + (h_text mod 16)
  fp_request_info_t info{};
  bool done = false;
  std::atomic<bool> done_flag{false};  // set with `done`, read by waiters without the lock
};

// The address the device uses for host memory p, or null when p is not
// pinned (page-locked) memory.
template <class T>
T* device_view(T* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of an unknown pointer
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return static_cast<T*>(a.devicePointer);
}

enum class Phase { FREE, PARSING, PIPELINED, COPYING };

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_counts = nullptr, ev_done = nullptr;
  uint64_t* d_counts = nullptr;  // max_batch field counts
  uint64_t* h_counts = nullptr;  // pinned copy
  unsigned int* d_err = nullptr; // the parse scratch's error word of this stream
  unsigned int* h_err = nullptr; // pinned copy, written by the fallback kernel at the end of each launch
  unsigned int* h_err_dv = nullptr;  // device view of h_err
  // piece tables in pinned host memory, read by the copy kernels
  fp::CopyPiece* gpieces = nullptr;   // written here ...
  fp::ScatterItem* sitems = nullptr;
  fp::ScatterPiece* spieces = nullptr;
  const fp::CopyPiece* gpieces_dv = nullptr;  // ... read there (device views)
  const fp::ScatterItem* sitems_dv = nullptr;
  const fp::ScatterPiece* spieces_dv = nullptr;
  uint32_t cap_gpieces = 0, cap_spieces = 0;
  bool unmapped_out = false;     // some request's results go back by copy calls
  bool direct = false;           // one request, results and count written to host memory by the parse
  uint64_t* h_counts_dv = nullptr;  // device view of h_counts
  // one large request in segments (Phase::PIPELINED): copies in on s_in,
  // parses on `stream`, copies out on s_out, segment i's count in h_counts[i]
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[fp::PIPE_MAX_SEGS] = {}, ev_parsed[fp::PIPE_MAX_SEGS] = {};
  size_t cuts[fp::PIPE_MAX_SEGS + 1] = {};
  int nseg = 0, next_seg = 0;  // segments, and the first whose results are not yet queued
  uint64_t seg_total = 0;      // fields of the segments before next_seg
  Phase phase = Phase::FREE;
  std::vector<Request*> reqs;
  std::vector<const char*> texts;
  std::vector<size_t> lens;
  std::vector<uint64_t> base, cap;
};

}  // namespace

struct fp_server {
  fp_server_config_t cfg{};
  int device = 0;
  uint64_t units = 0;
  void* dmem = nullptr;
  char* d_text = nullptr;
  double* d_f64 = nullptr;
  uint8_t* d_status = nullptr;
  fp::Arena arena{0};
  int sms = 1;
  std::vector<Slot> slots;
  std::thread thread;

  std::mutex mu;  // guards everything below up to `st`
  std::condition_variable cv_submit, cv_done;
  std::deque<Request*> incoming;
  std::unordered_map<uint64_t, Request*> live;  // submitted, not yet waited for
  uint64_t next_id = 1;
  uint64_t outstanding = 0;                     // submitted, not yet completed
  bool stop = false;
  fp_server_stats_t st{};

  // scheduler thread only
  std::deque<Request*> pending, admitted;
  uint64_t held_requests = 0;
};

namespace {

void finish(fp_server* S, Request* r, fp_err_t err) {
  r->info.error = (int32_t)err;
  r->info.done_ns = now_ns();
  if (r->units) S->arena.release(r->off, r->units);
  r->units = 0;
  S->held_requests--;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->done = true;
    r->done_flag.store(true, std::memory_order_release);
    S->outstanding--;
    S->st.completed++;
    if (err == FP_OK) S->st.fields += r->info.count;
  }
  S->cv_done.notify_all();
}

void fail_slot(fp_server* S, Slot& sl, fp_err_t err) {
  // Whatever the slot had queued before the failure (copies from or to the
  // callers' host arrays, kernels writing arena units) ends before the
  // requests complete and their units return to the arena.
  cudaStreamSynchronize(sl.stream);
  cudaStreamSynchronize(sl.s_in);
  cudaStreamSynchronize(sl.s_out);
  cudaGetLastError();  // the failure is reported through the requests
  for (Request* r : sl.reqs) finish(S, r, err);
  sl.reqs.clear();
  sl.phase = Phase::FREE;
}

// Retire step for one slot; returns true if it changed state.
bool retire(fp_server* S, Slot& sl) {
  if (sl.phase == Phase::PARSING) {
    const cudaError_t q = cudaEventQuery(sl.ev_counts);
    if (q == cudaErrorNotReady) return false;
    if (q != cudaSuccess) {
      fail_slot(S, sl, FP_ERR_CUDA);
      return true;
    }
    const unsigned int derr = *(volatile unsigned int*)sl.h_err;
    if (derr) {  // a bounded device wait ran out: the batch's results are void
      const fp_err_t e = (fp_err_t)derr;
      *sl.h_err = 0;
      cudaMemsetAsync(sl.d_err, 0, sizeof(unsigned int), sl.stream);
      fail_slot(S, sl, e);
      return true;
    }
    for (size_t i = 0; i < sl.reqs.size(); i++) {
      Request* r = sl.reqs[i];
      const uint64_t count = *(volatile uint64_t*)&sl.h_counts[i];
      r->info.count = count;
      if (count > r->len) {  // cannot happen: a text of len bytes has at most len fields
        r->info.error = FP_ERR_INTERNAL;
        continue;
      }
      if (r->dv_f64) continue;  // already written by the scatter kernel
      const uint64_t n = std::min<uint64_t>(count, r->out_cap);
      if (n) {
        if (cudaMemcpyAsync(r->h_f64, S->d_f64 + r->off, n * sizeof(double),
                            cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
            cudaMemcpyAsync(r->h_status, S->d_status + r->off, n, cudaMemcpyDeviceToHost,
                            sl.stream) != cudaSuccess)
          r->info.error = FP_ERR_CUDA;
      }
    }
    if (!sl.unmapped_out) {
      for (Request* r : sl.reqs) finish(S, r, (fp_err_t)r->info.error);
      sl.reqs.clear();
      sl.phase = Phase::FREE;
      return true;
    }
    if (cudaEventRecord(sl.ev_done, sl.stream) != cudaSuccess) {
      fail_slot(S, sl, FP_ERR_CUDA);
      return true;
    }
    sl.phase = Phase::COPYING;
    return true;
  }
  if (sl.phase == Phase::PIPELINED) {
    // segments in order: once one is parsed, its results go to the caller's
    // arrays at the running field total
    Request* r = sl.reqs[0];
    bool moved = false;
    while (sl.next_seg < sl.nseg) {
      const int i = sl.next_seg;
      const cudaError_t q = cudaEventQuery(sl.ev_parsed[i]);
      if (q == cudaErrorNotReady) return moved;
      if (q != cudaSuccess) {
        fail_slot(S, sl, FP_ERR_CUDA);
        return true;
      }
      const unsigned int derr = *(volatile unsigned int*)sl.h_err;
      if (derr) {  // a bounded device wait ran out: the request's results are void
        *sl.h_err = 0;
        cudaMemsetAsync(sl.d_err, 0, sizeof(unsigned int), sl.stream);
        fail_slot(S, sl, (fp_err_t)derr);
        return true;
      }
      const uint64_t count = *(volatile uint64_t*)&sl.h_counts[i];
      if (count > sl.cuts[i + 1] - sl.cuts[i]) {  // at most one field per byte
        fail_slot(S, sl, FP_ERR_INTERNAL);
        return true;
      }
      const uint64_t room = r->out_cap > sl.seg_total ? r->out_cap - sl.seg_total : 0;
      const uint64_t n = std::min<uint64_t>(count, room);
      const uint64_t src = r->off + sl.cuts[i];
      if (n && (cudaMemcpyAsync(r->h_f64 + sl.seg_total, S->d_f64 + src, n * sizeof(double),
                                cudaMemcpyDeviceToHost, sl.s_out) != cudaSuccess ||
                cudaMemcpyAsync(r->h_status + sl.seg_total, S->d_status + src, n,
                                cudaMemcpyDeviceToHost, sl.s_out) != cudaSuccess)) {
        fail_slot(S, sl, FP_ERR_CUDA);
        return true;
      }
      sl.seg_total += count;
      sl.next_seg++;
      moved = true;
    }
    r->info.count = sl.seg_total;
    if (cudaEventRecord(sl.ev_done, sl.s_out) != cudaSuccess) {
      fail_slot(S, sl, FP_ERR_CUDA);
      return true;
    }
    sl.phase = Phase::COPYING;
    return true;
  }
  if (sl.phase == Phase::COPYING) {
    const cudaError_t q = cudaEventQuery(sl.ev_done);
    if (q == cudaErrorNotReady) return false;
    for (Request* r : sl.reqs) {
      fp_err_t e = (fp_err_t)r->info.error;
      if (q != cudaSuccess) e = FP_ERR_CUDA;
      finish(S, r, e);
    }
    sl.reqs.clear();
    sl.phase = Phase::FREE;
    return true;
  }
  return false;
}

// A launch of one request whose host arrays the device can reach and whose
// text is below DIRECT_BYTES: one copy in, then the parse writes the results
// and the count straight into the caller's pinned arrays (no gather, scatter
// or count copy), as fp_parse_f64_host does for such texts alone.
constexpr uint64_t DIRECT_BYTES = 8u << 20;

bool launch_direct(fp_server* S, Slot& sl, Request* r) {
  uint8_t* dst = reinterpret_cast<uint8_t*>(S->d_text) + r->text_off;
  if (r->len && cudaMemcpyAsync(dst, r->h_text, r->len, cudaMemcpyHostToDevice, sl.stream) !=
                    cudaSuccess)
    return false;
  const char* text = reinterpret_cast<const char*>(dst);
  const size_t len = r->len;
  const uint64_t base = 0, cap = std::min<uint64_t>(r->out_cap, r->len);
  *(volatile uint64_t*)&sl.h_counts[0] = ~0ull;
  if (fp::parse_batch_ranges(&text, &len, 1, S->cfg.delim,
                             reinterpret_cast<double*>(r->dv_f64), r->dv_status, &base, &cap,
                             sl.h_counts_dv, sl.stream, sl.h_err_dv) != FP_OK)
    return false;
  return cudaEventRecord(sl.ev_counts, sl.stream) == cudaSuccess;
}

// One large request alone, with pinned host arrays: its text is cut at
// separators into segments (as fp_parse_f64_host cuts a large pinned text),
// copied into its arena range on s_in back to back; segment i is parsed on
// the slot's stream once it has landed, into the request's arena slots from
// its own byte offset on, its count going to pinned memory; the retire step
// then queues each segment's results on s_out at the running total.  Copies
// in, parses and copies out of different segments overlap.
bool launch_pipelined(fp_server* S, Slot& sl, Request* r) {
  sl.nseg = fp::plan_host_segments(r->h_text, r->len, S->cfg.delim, sl.cuts);
  sl.next_seg = 0;
  sl.seg_total = 0;
  uint8_t* dst = reinterpret_cast<uint8_t*>(S->d_text) + r->text_off;
  for (int i = 0; i < sl.nseg; i++) {
    if (cudaMemcpyAsync(dst + sl.cuts[i], r->h_text + sl.cuts[i], sl.cuts[i + 1] - sl.cuts[i],
                        cudaMemcpyHostToDevice, sl.s_in) != cudaSuccess ||
        cudaEventRecord(sl.ev_in[i], sl.s_in) != cudaSuccess)
      return false;
  }
  for (int i = 0; i < sl.nseg; i++) {
    const char* text = reinterpret_cast<const char*>(dst + sl.cuts[i]);
    const size_t len = sl.cuts[i + 1] - sl.cuts[i];
    const uint64_t base = r->off + sl.cuts[i], cap = len;  // at most one field per byte
    *(volatile uint64_t*)&sl.h_counts[i] = ~0ull;
    if (cudaStreamWaitEvent(sl.stream, sl.ev_in[i], 0) != cudaSuccess ||
        fp::parse_batch_ranges(&text, &len, 1, S->cfg.delim, S->d_f64, S->d_status, &base, &cap,
                               sl.h_counts_dv + i, sl.stream, sl.h_err_dv) != FP_OK ||
        cudaEventRecord(sl.ev_parsed[i], sl.stream) != cudaSuccess)
      return false;
  }
  return true;
}

// Launch step for one free slot.
void launch(fp_server* S, Slot& sl) {
  const size_t kmax = std::min<size_t>(S->admitted.size(), S->cfg.max_batch);
  size_t k = 1;
  uint64_t bytes = S->admitted[0]->len;
  const uint64_t cap = S->cfg.launch_bytes ? S->cfg.launch_bytes : LAUNCH_BYTES;
  while (k < kmax && bytes + S->admitted[k]->len <= cap) bytes += S->admitted[k++]->len;
  sl.reqs.assign(S->admitted.begin(), S->admitted.begin() + k);
  S->admitted.erase(S->admitted.begin(), S->admitted.begin() + k);
  sl.unmapped_out = false;
  sl.direct = false;
  if (k == 1) {
    Request* r = sl.reqs[0];
    if (r->len < DIRECT_BYTES && r->dv_f64 && r->dv_status && sl.h_counts_dv) {
      sl.direct = true;
      if (!launch_direct(S, sl, r)) {
        fail_slot(S, sl, FP_ERR_CUDA);
        return;
      }
      r->info.launch_ns = now_ns();
      r->info.batch_size = 1;
      sl.phase = Phase::PARSING;
      std::lock_guard<std::mutex> lk(S->mu);
      S->st.launches++;
      S->st.max_batch_seen = std::max<uint64_t>(S->st.max_batch_seen, 1);
      return;
    }
    if (r->len >= fp::PIPE_MIN_BYTES && r->dv_text && r->dv_f64 && r->dv_status) {
      if (!launch_pipelined(S, sl, r)) {
        fail_slot(S, sl, FP_ERR_CUDA);
        return;
      }
      r->info.launch_ns = now_ns();
      r->info.batch_size = 1;
      sl.phase = Phase::PIPELINED;
      std::lock_guard<std::mutex> lk(S->mu);
      S->st.launches += (uint64_t)sl.nseg;
      S->st.max_batch_seen = std::max<uint64_t>(S->st.max_batch_seen, 1);
      return;
    }
  }
  sl.texts.resize(k);
  sl.lens.resize(k);
  sl.base.resize(k);
  sl.cap.resize(k);
  sl.unmapped_out = false;
  fp_err_t e = FP_OK;
  uint32_t ng = 0, ns = 0;
  for (size_t i = 0; i < k && e == FP_OK; i++) {
    Request* r = sl.reqs[i];
    uint8_t* dst = reinterpret_cast<uint8_t*>(S->d_text) + r->text_off;
    sl.texts[i] = reinterpret_cast<const char*>(dst);
    sl.lens[i] = r->len;
    sl.base[i] = r->off;
    sl.cap[i] = r->len;  // fp_max_fields(len)
    // text in: by the gather kernel, else by a copy call
    const bool engine = r->len >= ENGINE_BYTES;
    if (r->len && r->dv_text && !engine) {
      for (uint64_t p = 0; p < r->len; p += fp::GATHER_PIECE) {
        if (ng >= sl.cap_gpieces) {
          e = FP_ERR_INTERNAL;
          break;
        }
        const uint64_t nb = std::min<uint64_t>(fp::GATHER_PIECE, r->len - p);
        sl.gpieces[ng++] = fp::CopyPiece{r->dv_text + p, dst + p, (uint32_t)nb, 0};
      }
    } else if (r->len && cudaMemcpyAsync(dst, r->h_text, r->len, cudaMemcpyHostToDevice,
                                         sl.stream) != cudaSuccess) {
      e = FP_ERR_CUDA;
    }
    // results out: by the scatter kernel, else by copy calls after the counts
    const uint64_t cap = std::min<uint64_t>(r->out_cap, r->len);
    if (r->dv_f64 && r->dv_status && !engine) {
      sl.sitems[i] = fp::ScatterItem{reinterpret_cast<const unsigned long long*>(S->d_f64) + r->off,
                                     S->d_status + r->off, r->dv_f64, r->dv_status,
                                     reinterpret_cast<const unsigned long long*>(sl.d_counts) + i,
                                     cap};
      for (uint64_t f = 0; f < cap; f += fp::SCATTER_PIECE) {
        if (ns >= sl.cap_spieces) {
          e = FP_ERR_INTERNAL;
          break;
        }
        sl.spieces[ns++] = fp::ScatterPiece{(uint32_t)i, 0, f};
      }
    } else {
      r->dv_f64 = nullptr;
      sl.unmapped_out = true;
    }
  }
  const int grid = S->sms * 4;
  if (e == FP_OK &&
      fp::launch_gather(sl.gpieces_dv, ng, (int)std::min<uint32_t>(ng ? ng : 1, grid), sl.stream) !=
          cudaSuccess)
    e = FP_ERR_CUDA;
  if (e == FP_OK)
    e = fp::parse_batch_ranges(sl.texts.data(), sl.lens.data(), (uint32_t)k, S->cfg.delim,
                               S->d_f64, S->d_status, sl.base.data(), sl.cap.data(), sl.d_counts,
                               sl.stream, sl.h_err_dv);
  if (e == FP_OK &&
      fp::launch_scatter(sl.sitems_dv, sl.spieces_dv, ns, (int)std::min<uint32_t>(ns ? ns : 1, grid),
                         sl.stream) != cudaSuccess)
    e = FP_ERR_CUDA;
  if (e == FP_OK &&
      (cudaMemcpyAsync(sl.h_counts, sl.d_counts, k * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                       sl.stream) != cudaSuccess ||
       cudaEventRecord(sl.ev_counts, sl.stream) != cudaSuccess))
    e = FP_ERR_CUDA;
  if (e != FP_OK) {
    fail_slot(S, sl, e);
    return;
  }
  const int64_t t = now_ns();
  for (Request* r : sl.reqs) {
    r->info.launch_ns = t;
    r->info.batch_size = (uint32_t)k;
  }
  sl.phase = Phase::PARSING;
  std::lock_guard<std::mutex> lk(S->mu);
  S->st.launches++;
  S->st.max_batch_seen = std::max<uint64_t>(S->st.max_batch_seen, k);
}

// After its last piece of work the scheduler keeps polling for this long
// before it sleeps on the submission condition (a sleeping thread takes tens
// of microseconds to wake, which a request arriving soon after would wait).
constexpr int64_t SPIN_NS = 2000000;

void scheduler(fp_server* S) {
  cudaSetDevice(S->device);
  int64_t last_work = now_ns();
  for (;;) {
    bool progressed = false, busy = false;
    for (Slot& sl : S->slots) {
      progressed |= retire(S, sl);
      busy |= sl.phase != Phase::FREE;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      while (!S->incoming.empty()) {
        S->pending.push_back(S->incoming.front());
        S->incoming.pop_front();
      }
      if (S->stop && S->outstanding == 0) break;
    }
    bool admitted_any = false;
    while (!S->pending.empty()) {
      Request* r = S->pending.front();
      uint64_t off = 0;
      if (!S->arena.alloc(r->units, &off)) break;  // first come, first served
      S->pending.pop_front();
      r->off = off;
      r->text_off = off + (reinterpret_cast<uintptr_t>(r->h_text) & 15);
      S->held_requests++;
      r->info.admit_ns = now_ns();
      S->admitted.push_back(r);
      admitted_any = true;
    }
    if (admitted_any) {
      progressed = true;
      std::lock_guard<std::mutex> lk(S->mu);
      S->st.peak_units = std::max<uint64_t>(S->st.peak_units, S->arena.used_units());
      S->st.peak_requests = std::max<uint64_t>(S->st.peak_requests, S->held_requests);
    }
    for (Slot& sl : S->slots) {
      if (S->admitted.empty()) break;
      if (sl.phase != Phase::FREE) continue;
      launch(S, sl);
      progressed = true;
      busy = true;
    }
    if (progressed) {
      last_work = now_ns();
      continue;
    }
    if (busy || !S->admitted.empty() || now_ns() - last_work < SPIN_NS) {
      std::this_thread::yield();
    } else {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_submit.wait_for(lk, std::chrono::milliseconds(1),
                            [&] { return !S->incoming.empty() || S->stop; });
    }
  }
}

void free_server(fp_server* S) {
  cudaSetDevice(S->device);
  for (Slot& sl : S->slots) {
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      fp::release_stream_scratch(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
    for (cudaStream_t x : {sl.s_in, sl.s_out}) {
      if (x) {
        cudaStreamSynchronize(x);
        cudaStreamDestroy(x);
      }
    }
    for (int i = 0; i < fp::PIPE_MAX_SEGS; i++) {
      if (sl.ev_in[i]) cudaEventDestroy(sl.ev_in[i]);
      if (sl.ev_parsed[i]) cudaEventDestroy(sl.ev_parsed[i]);
    }
    if (sl.ev_counts) cudaEventDestroy(sl.ev_counts);
    if (sl.ev_done) cudaEventDestroy(sl.ev_done);
    cudaFree(sl.d_counts);
    cudaFreeHost(sl.h_counts);
    cudaFreeHost(sl.h_err);
    cudaFreeHost(sl.gpieces);
    cudaFreeHost(sl.sitems);
    cudaFreeHost(sl.spieces);
  }
  cudaFree(S->dmem);
  for (auto& kv : S->live) delete kv.second;
  delete S;
}

}  // namespace

#define SRV_CUDA(x)                 \
  do {                              \
    if ((x) != cudaSuccess) {       \
      free_server(S);               \
      return FP_ERR_CUDA;           \
    }                               \
  } while (0)

extern "C" fp_err_t fp_server_create(const fp_server_config_t* cfg, fp_server** server) {
  if (!cfg || !server) return FP_ERR_ARG;
  *server = nullptr;
  if (cfg->device_budget < MIN_BUDGET || cfg->max_batch < 1 || cfg->max_batch > MAX_BATCH ||
      cfg->max_inflight < 1 || cfg->max_inflight > MAX_SLOTS)
    return FP_ERR_ARG;
  fp_server* S = new fp_server();
  S->cfg = *cfg;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return FP_ERR_CUDA;
  }
  // units: 1 text byte + 8 value bytes + 1 status byte each
  S->units = cfg->device_budget / 10 / UNIT_ROUND * UNIT_ROUND;
  if (S->units == 0) {
    delete S;
    return FP_ERR_ARG;
  }
  SRV_CUDA(cudaMalloc(&S->dmem, S->units * 10));
  S->d_text = static_cast<char*>(S->dmem);
  S->d_f64 = reinterpret_cast<double*>(S->d_text + S->units);
  S->d_status = reinterpret_cast<uint8_t*>(S->d_text + 9 * S->units);
  S->arena = fp::Arena(S->units);
  SRV_CUDA(cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device));
  S->slots.resize(cfg->max_inflight);
  // the most chunks one launch can hold: every unit of text at the smallest
  // chunk size, plus one partial chunk per request at each end
  const unsigned long long chunks = S->units / 4096 + 2ull * cfg->max_batch + 16;
  for (Slot& sl : S->slots) {
    SRV_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
    SRV_CUDA(cudaEventCreateWithFlags(&sl.ev_counts, cudaEventDisableTiming));
    SRV_CUDA(cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming));
    SRV_CUDA(cudaMalloc(&sl.d_counts, cfg->max_batch * sizeof(uint64_t)));
    SRV_CUDA(cudaMallocHost(&sl.h_counts, std::max<uint32_t>(cfg->max_batch, fp::PIPE_MAX_SEGS) *
                                              sizeof(uint64_t)));
    SRV_CUDA(cudaStreamCreateWithFlags(&sl.s_in, cudaStreamNonBlocking));
    SRV_CUDA(cudaStreamCreateWithFlags(&sl.s_out, cudaStreamNonBlocking));
    for (int i = 0; i < fp::PIPE_MAX_SEGS; i++) {
      SRV_CUDA(cudaEventCreateWithFlags(&sl.ev_in[i], cudaEventDisableTiming));
      SRV_CUDA(cudaEventCreateWithFlags(&sl.ev_parsed[i], cudaEventDisableTiming));
    }
    sl.h_counts_dv = device_view(sl.h_counts);
    SRV_CUDA(cudaMallocHost(&sl.h_err, sizeof(unsigned int)));
    *sl.h_err = 0;
    sl.h_err_dv = device_view(sl.h_err);
    // piece tables: every unit of a batch once, plus one partial piece per request
    sl.cap_gpieces = (uint32_t)(S->units / fp::GATHER_PIECE + cfg->max_batch + 1);
    sl.cap_spieces = (uint32_t)(S->units / fp::SCATTER_PIECE + cfg->max_batch + 1);
    SRV_CUDA(cudaHostAlloc(&sl.gpieces, sl.cap_gpieces * sizeof(fp::CopyPiece), cudaHostAllocMapped));
    SRV_CUDA(cudaHostAlloc(&sl.sitems, cfg->max_batch * sizeof(fp::ScatterItem), cudaHostAllocMapped));
    SRV_CUDA(cudaHostAlloc(&sl.spieces, sl.cap_spieces * sizeof(fp::ScatterPiece), cudaHostAllocMapped));
    sl.gpieces_dv = device_view(sl.gpieces);
    sl.sitems_dv = device_view(sl.sitems);
    sl.spieces_dv = device_view(sl.spieces);
    if (!sl.gpieces_dv || !sl.sitems_dv || !sl.spieces_dv || !sl.h_err_dv) {
      free_server(S);
      return FP_ERR_CUDA;
    }
    if (fp::reserve_stream_scratch(sl.stream, chunks, cfg->max_batch) != FP_OK ||
        fp::stream_error_word(sl.stream, &sl.d_err) != FP_OK) {
      free_server(S);
      return FP_ERR_CUDA;
    }
    sl.reqs.reserve(cfg->max_batch);
  }
  SRV_CUDA(cudaDeviceSynchronize());
  S->thread = std::thread(scheduler, S);
  *server = S;
  return FP_OK;
}

extern "C" fp_err_t fp_server_submit(fp_server* S, const char* host_text, size_t len,
                                     double* host_f64, uint8_t* host_status, size_t out_cap,
                                     uint64_t* request_id) {
  if (!S || !request_id) return FP_ERR_ARG;
  if (len >= MAX_LEN) return FP_ERR_ARG;
  if (len > 0 && !host_text) return FP_ERR_ARG;
  if (out_cap > 0 && (!host_f64 || !host_status)) return FP_ERR_ARG;
  // len text bytes placed at the source's address mod 16 (+15), and len
  // value / status slots (fp_max_fields)
  const uint64_t units = (len + 16 + UNIT_ROUND - 1) / UNIT_ROUND * UNIT_ROUND;
  if (units > S->units) return FP_ERR_BUDGET;
  Request* r = new Request();
  r->h_text = host_text;
  r->len = len;
  r->h_f64 = host_f64;
  r->h_status = host_status;
  r->out_cap = out_cap;
  r->units = units;
  r->dv_text = device_view(reinterpret_cast<const uint8_t*>(host_text));
  if (out_cap) {
    r->dv_f64 = device_view(reinterpret_cast<unsigned long long*>(host_f64));
    r->dv_status = device_view(host_status);
  }
  r->info.submit_ns = now_ns();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete r;
      return FP_ERR_ARG;
    }
    r->id = S->next_id++;
    S->live[r->id] = r;
    S->incoming.push_back(r);
    S->outstanding++;
    S->st.submitted++;
    S->st.bytes += len;
  }
  S->cv_submit.notify_one();
  *request_id = r->id;
  return FP_OK;
}

extern "C" fp_err_t fp_server_wait(fp_server* S, uint64_t id, int64_t timeout_ns,
                                   fp_request_info_t* info) {
  if (!S) return FP_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->live.find(id);
  if (it == S->live.end()) return FP_ERR_ARG;
  Request* r = it->second;
  if (!r->done && timeout_ns != 0) {
    // most requests end within a few hundred microseconds: poll for that
    // long (lock released) before sleeping on the completion condition
    lk.unlock();
    const int64_t t_end = now_ns() + SPIN_NS / 4;
    while (!r->done_flag.load(std::memory_order_acquire) && now_ns() < t_end)
      std::this_thread::yield();
    lk.lock();
    it = S->live.find(id);  // other submissions may have rehashed the map meanwhile
  }
  if (!r->done) {
    if (timeout_ns == 0) return FP_ERR_TIMEOUT;
    auto pred = [&] { return r->done; };
    if (timeout_ns < 0) {
      S->cv_done.wait(lk, pred);
    } else if (!S->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), pred)) {
      return FP_ERR_TIMEOUT;
    }
  }
  if (info) *info = r->info;
  const fp_err_t e = (fp_err_t)r->info.error;
  S->live.erase(it);
  delete r;
  return e;
}

extern "C" fp_err_t fp_server_get_stats(fp_server* S, fp_server_stats_t* out) {
  if (!S || !out) return FP_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  return FP_OK;
}

extern "C" fp_err_t fp_server_destroy(fp_server* S) {
  if (!S) return FP_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_submit.notify_all();
  if (S->thread.joinable()) S->thread.join();
  free_server(S);
  return FP_OK;
}
