// fp_api.cu -- the C ABI (include/fpparse.h): argument checks, per-stream
// scratch, launch configuration, counters and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fpparse.h"
#include "../../include/fpparse_test.h"
#include "fp_device.cuh"
#include "fp_internal.h"
#include "fp_copy.h"
#include "fp_launch.h"
#include "fp_types.cuh"

namespace {

using fp::BufDesc;
using fp::Ctl;
using fp::LaunchParams;

constexpr unsigned long long MAX_LEN = 1ull << 40;
constexpr uint32_t MAX_BUFS = 1u << 24;

struct Config {
  uint32_t chunk_bytes = 16384;
  uint32_t ctas_per_sm = 0;  // 0: as many as fit
  uint32_t fallback_queue = 1u << 20;
};

// Launch parameters; FP_CHUNK_BYTES, FP_CTAS_PER_SM and FP_FALLBACK_QUEUE in
// the environment override the defaults when the library is loaded.
Config initial_config() {
  Config c;
  if (const char* v = getenv("FP_CHUNK_BYTES")) {
    unsigned long x = strtoul(v, nullptr, 10);
    if (x == 4096 || x == 8192 || x == 12288 || x == 16384) c.chunk_bytes = (uint32_t)x;
  }
  if (const char* v = getenv("FP_CTAS_PER_SM")) {
    unsigned long x = strtoul(v, nullptr, 10);
    if (x <= 8) c.ctas_per_sm = (uint32_t)x;
  }
  if (const char* v = getenv("FP_FALLBACK_QUEUE")) {
    unsigned long x = strtoul(v, nullptr, 10);
    if (x >= 1024 && x <= (1u << 28)) c.fallback_queue = (uint32_t)x;
  }
  return c;
}

std::mutex g_mu;
Config g_cfg = initial_config();

struct DeviceInfo {
  int sms = 0;
  std::map<int, int> parse_occ;    // chunk bytes -> resident blocks per SM (binary64)
  std::map<int, int> parse_occ32;  // the same for the binary32 kernels
  std::map<int, int> parse_occ_ext;  // JSON / column-major kernels (8 and 16 KiB chunks)
  int fb_occ = 0, fb_occ32 = 0;          // the fallback kernel's idle build
  int fb_busy = 0, fb_busy32 = 0;        // and its busy build (fp_launch.h)
  char name[256] = {0};
};
std::map<int, DeviceInfo> g_dev;

struct Scratch {
  int device = -1;
  cudaStream_t stream = nullptr;
  Ctl* ctl = nullptr;
  unsigned long long* chunk_status = nullptr;
  unsigned long long cap_chunks = 0;
  unsigned long long* queue = nullptr;
  unsigned long long qcap = 0;
  unsigned long long* ovf = nullptr;
  unsigned long long ovf_cap = 0;
  BufDesc* d_descs = nullptr;
  BufDesc* h_descs = nullptr;  // pinned staging for the descriptor upload
  uint32_t cap_descs = 0;
  cudaEvent_t desc_copied = nullptr;
  bool desc_pending = false;
  unsigned int epoch = 1;
  unsigned long long calls = 0, bytes = 0;
  // kernel timing (optional): a ring of event triples harvested as they complete
  static constexpr int RING = 256;
  cudaEvent_t ev[RING][3] = {};
  bool ev_used[RING] = {};
  int ev_head = 0;
  double acc_parse_ms = 0, acc_fb_ms = 0;
  unsigned long long acc_calls = 0;
  // staging for fp_parse_f64_host
  uint8_t* stage_text = nullptr;
  double* stage_out = nullptr;
  uint8_t* stage_status = nullptr;
  unsigned long long* stage_count = nullptr;
  size_t stage_cap = 0;      // bytes of stage_text
  size_t stage_out_cap = 0;  // entries of stage_out and stage_status
  // binary32 calls: pending fields' locations, indexed like the outputs
  unsigned long long* loc = nullptr;
  unsigned long long cap_loc = 0;
  // the pipelined host parse: copy-in and copy-out streams, per-segment
  // events, segment counts
  static constexpr int PIPE_SEGS = fp::PIPE_MAX_SEGS;
  cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
  cudaEvent_t pipe_ev_in[PIPE_SEGS] = {}, pipe_ev_parsed[PIPE_SEGS] = {};
  cudaEvent_t pipe_ev_start = nullptr, pipe_ev_done = nullptr;
  unsigned long long* pipe_counts = nullptr;     // segment counts (pinned) ...
  unsigned long long* pipe_counts_dv = nullptr;  // ... and the address the parse kernel writes them at
  // how many fields the stream's last finished call queued for the fallback
  // kernel (pinned; written by that kernel), and its device address
  unsigned long long* pend_host = nullptr;
  unsigned long long* pend_dv = nullptr;
  unsigned long long* pipe_host = nullptr;       // one count (pinned) ...
  unsigned long long* pipe_host_dv = nullptr;    // ... and the address the parse kernel writes it at
  // fp_test_arm_stalled_lookback: the next call skips chunk 0 and waits at
  // most test_wait_ns on the device
  bool test_stall = false;
  unsigned long long test_wait_ns = 0;
};
// fp_timing_enable: 0 off, else every g_timing-th call on a stream is timed
int g_timing = 0;

std::map<std::pair<int, cudaStream_t>, Scratch*> g_scratch;

#define FP_CUDA(x)                                  \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) {                        \
      fprintf(stderr, "fpparse: %s failed: %s\n", #x, cudaGetErrorString(e_)); \
      return FP_ERR_CUDA;                           \
    }                                               \
  } while (0)

fp_err_t harvest(Scratch* s, int slot, bool wait) {
  if (!s->ev_used[slot]) return FP_OK;
  if (wait) {
    FP_CUDA(cudaEventSynchronize(s->ev[slot][2]));
  } else if (cudaEventQuery(s->ev[slot][2]) != cudaSuccess) {
    return FP_OK;
  }
  float a = 0, b = 0;
  FP_CUDA(cudaEventElapsedTime(&a, s->ev[slot][0], s->ev[slot][1]));
  FP_CUDA(cudaEventElapsedTime(&b, s->ev[slot][1], s->ev[slot][2]));
  s->acc_parse_ms += a;
  s->acc_fb_ms += b;
  s->acc_calls++;
  s->ev_used[slot] = false;
  return FP_OK;
}

fp_err_t device_info(int dev, DeviceInfo** out) {
  auto it = g_dev.find(dev);
  if (it == g_dev.end()) {
    DeviceInfo di;
    cudaDeviceProp prop;
    FP_CUDA(cudaGetDeviceProperties(&prop, dev));
    di.sms = prop.multiProcessorCount;
    snprintf(di.name, sizeof(di.name), "%s", prop.name);
    for (int c : {4096, 8192, 12288, 16384}) {
      int occ = 0;
      FP_CUDA(fp::parse_occupancy(c, &occ, false));
      di.parse_occ[c] = std::max(occ, 1);
      FP_CUDA(fp::parse_occupancy(c, &occ, true));
      di.parse_occ32[c] = std::max(occ, 1);
    }
    for (int c : {8192, 16384}) {
      int occ = 0;
      FP_CUDA(fp::parse_occupancy_ext(c, &occ));
      di.parse_occ_ext[c] = std::max(occ, 1);
    }
    FP_CUDA(fp::fallback_occupancy(&di.fb_occ, false));
    di.fb_occ = std::max(di.fb_occ, 1);
    FP_CUDA(fp::fallback_occupancy(&di.fb_occ32, true));
    di.fb_occ32 = std::max(di.fb_occ32, 1);
    FP_CUDA(fp::fallback_occupancy(&di.fb_busy, false, true));
    di.fb_busy = std::max(di.fb_busy, 1);
    FP_CUDA(fp::fallback_occupancy(&di.fb_busy32, true, true));
    di.fb_busy32 = std::max(di.fb_busy32, 1);
    it = g_dev.emplace(dev, di).first;
  }
  *out = &it->second;
  return FP_OK;
}

void free_scratch(Scratch* s) {
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  cudaFree(s->ctl);
  cudaFree(s->chunk_status);
  cudaFree(s->queue);
  cudaFree(s->ovf);
  cudaFree(s->d_descs);
  cudaFreeHost(s->h_descs);
  if (s->desc_copied) cudaEventDestroy(s->desc_copied);
  for (auto& tri : s->ev)
    for (cudaEvent_t e : tri)
      if (e) cudaEventDestroy(e);
  cudaFree(s->stage_text);
  cudaFree(s->stage_out);
  cudaFree(s->stage_status);
  cudaFree(s->stage_count);
  cudaFree(s->loc);
  if (s->pipe_in) {
    cudaStreamSynchronize(s->pipe_in);
    cudaStreamDestroy(s->pipe_in);
  }
  if (s->pipe_out) {
    cudaStreamSynchronize(s->pipe_out);
    cudaStreamDestroy(s->pipe_out);
  }
  for (int i = 0; i < Scratch::PIPE_SEGS; i++) {
    if (s->pipe_ev_in[i]) cudaEventDestroy(s->pipe_ev_in[i]);
    if (s->pipe_ev_parsed[i]) cudaEventDestroy(s->pipe_ev_parsed[i]);
  }
  if (s->pipe_ev_start) cudaEventDestroy(s->pipe_ev_start);
  if (s->pipe_ev_done) cudaEventDestroy(s->pipe_ev_done);
  cudaFreeHost(s->pipe_counts);
  cudaFreeHost(s->pipe_host);
  cudaFreeHost(s->pend_host);
  if (prev >= 0) cudaSetDevice(prev);
  delete s;
}

// Scratch of (current device, stream) with room for `chunks` chunks and
// `nbuf` descriptors.
fp_err_t get_scratch(cudaStream_t stream, unsigned long long chunks, uint32_t nbuf,
                     uint32_t qcap, Scratch** out) {
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  auto key = std::make_pair(dev, stream);
  Scratch*& s = g_scratch[key];
  if (!s) {
    s = new Scratch();
    s->device = dev;
    s->stream = stream;
    if (cudaMalloc(&s->ctl, sizeof(Ctl)) != cudaSuccess) {
      delete s;
      s = nullptr;
      return FP_ERR_CUDA;
    }
    FP_CUDA(cudaMemsetAsync(s->ctl, 0, sizeof(Ctl), stream));
    FP_CUDA(cudaEventCreateWithFlags(&s->desc_copied, cudaEventDisableTiming));
  }
  if (chunks > s->cap_chunks) {
    unsigned long long cap = std::max<unsigned long long>(chunks, 1ull << 15);
    FP_CUDA(cudaStreamSynchronize(stream));
    cudaFree(s->chunk_status);
    cudaFree(s->ovf);
    s->chunk_status = nullptr;
    s->ovf = nullptr;
    s->cap_chunks = 0;
    FP_CUDA(cudaMalloc(&s->chunk_status, cap * sizeof(unsigned long long)));
    FP_CUDA(cudaMalloc(&s->ovf, 2 * cap * sizeof(unsigned long long)));
    FP_CUDA(cudaMemsetAsync(s->chunk_status, 0, cap * sizeof(unsigned long long), stream));
    s->cap_chunks = cap;
    s->ovf_cap = cap;
    s->epoch = 1;
  }
  if (qcap != s->qcap) {
    FP_CUDA(cudaStreamSynchronize(stream));
    cudaFree(s->queue);
    s->queue = nullptr;
    s->qcap = 0;
    FP_CUDA(cudaMalloc(&s->queue, (size_t)qcap * sizeof(unsigned long long)));
    s->qcap = qcap;
  }
  if (nbuf > 1 && nbuf > s->cap_descs) {
    uint32_t cap = std::max<uint32_t>(nbuf, 256);
    FP_CUDA(cudaStreamSynchronize(stream));
    cudaFree(s->d_descs);
    cudaFreeHost(s->h_descs);
    s->d_descs = nullptr;
    s->h_descs = nullptr;
    s->cap_descs = 0;
    FP_CUDA(cudaMalloc(&s->d_descs, (size_t)cap * sizeof(BufDesc)));
    FP_CUDA(cudaMallocHost(&s->h_descs, (size_t)cap * sizeof(BufDesc)));
    s->cap_descs = cap;
    s->desc_pending = false;
  }
  *out = s;
  return FP_OK;
}

unsigned long long chunks_of(unsigned long long o, unsigned long long len, uint32_t C) {
  unsigned long long n = (o + len + C - 1) / C;
  return n ? n : 1;
}

void fill_desc(BufDesc& d, const char* text, size_t len, unsigned long long chunk0,
               unsigned long long nchunks, unsigned long long out_base, unsigned long long out_cap,
               uint64_t* out_count) {
  const uintptr_t t = reinterpret_cast<uintptr_t>(text);
  d.base = reinterpret_cast<const uint8_t*>(t & ~(uintptr_t)15);
  d.o = t & 15;
  d.len = len;
  d.chunk0 = chunk0;
  d.nchunks = nchunks;
  d.out_base = out_base;
  d.out_cap = out_cap;
  d.out_count = reinterpret_cast<unsigned long long*>(out_count);
}

// Texts below this many bytes are parsed in 4 KiB chunks when the configured
// chunk size is the default 16 KiB (more blocks share a small text), and
// their fallback launch is one block per SM (its blocks only look at the
// queue when nothing is pending).
constexpr size_t SMALL_TEXT_BYTES = 4u << 20;
constexpr uint32_t DEFAULT_CHUNK = 16384;
Config text_config(Config cfg, size_t len) {
  if (len < SMALL_TEXT_BYTES && cfg.chunk_bytes == DEFAULT_CHUNK) cfg.chunk_bytes = 4096;
  return cfg;
}

// Queue the two kernels of one call (binary32 results when f32).
fp_err_t run(Scratch* s, const Config& cfg, const DeviceInfo& di, LaunchParams& p,
             unsigned long long total_chunks, unsigned long long total_bytes, cudaStream_t stream,
             bool f32 = false, int mode = 0) {
  if (s->epoch >= fp::LB_EPOCH_MAX) {
    FP_CUDA(cudaMemsetAsync(s->chunk_status, 0, s->cap_chunks * sizeof(unsigned long long), stream));
    s->epoch = 1;
  }
  p.ctl = s->ctl;
  p.chunk_status = s->chunk_status;
  if (!s->pend_host) {
    FP_CUDA(cudaMallocHost(&s->pend_host, sizeof(unsigned long long)));
    *s->pend_host = 0;
    FP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->pend_dv), s->pend_host, 0));
  }
  p.pending_out = s->pend_dv;
  // When the stream's last finished call had fallback work, a one-block
  // launch separates this call's parse and fallback kernels, so that the
  // fallback kernel's blocks start in their own division of the SMs' on-chip
  // memory (large L1) instead of the parse kernel's (fp_fallback_kernel.cu).
  const bool separate = *reinterpret_cast<volatile unsigned long long*>(s->pend_host) != 0;
  p.epoch = s->epoch++;
  p.queue = s->queue;
  p.qcap = s->qcap;
  p.ovf = s->ovf;
  p.ovf_cap = s->ovf_cap;
  p.total_chunks = total_chunks;
  if (!p.loc) p.loc = p.out_bits;  // binary64: the location sits in the output slot
  if (s->test_stall) {
    // the test hook: tickets start at 1, so no block ever takes chunk 0 and
    // the look-back of the chunks after it waits for a word nothing writes
    static const unsigned long long first_ticket = 1;
    FP_CUDA(cudaMemcpyAsync(&s->ctl->ticket, &first_ticket, sizeof(first_ticket),
                            cudaMemcpyHostToDevice, stream));
    p.wait_ns = s->test_wait_ns;
    s->test_stall = false;
  }
  const int occ = (mode ? di.parse_occ_ext : (f32 ? di.parse_occ32 : di.parse_occ))
                      .at((int)cfg.chunk_bytes);
  const int per_sm = cfg.ctas_per_sm ? std::min<int>((int)cfg.ctas_per_sm, occ) : occ;
  unsigned long long grid = (unsigned long long)di.sms * per_sm;
  if (grid > total_chunks) grid = total_chunks;
  const bool timing = g_timing > 0 && s->calls % (unsigned long long)g_timing == 0;
  int slot = -1;
  if (timing) {
    slot = s->ev_head;
    s->ev_head = (s->ev_head + 1) % Scratch::RING;
    fp_err_t e = harvest(s, slot, true);  // only blocks with RING calls in flight
    if (e != FP_OK) return e;
    if (!s->ev[slot][0])
      for (cudaEvent_t& ev : s->ev[slot]) FP_CUDA(cudaEventCreate(&ev));
    FP_CUDA(cudaEventRecord(s->ev[slot][0], stream));
  }
  if (mode) FP_CUDA(fp::launch_parse_ext(p, (int)cfg.chunk_bytes, (int)grid, stream, f32, mode));
  else FP_CUDA(fp::launch_parse(p, (int)cfg.chunk_bytes, (int)grid, stream, f32));
  if (timing) FP_CUDA(cudaEventRecord(s->ev[slot][1], stream));
  if (separate) FP_CUDA(fp::launch_fallback_separator(stream));
  // the fallback kernel's busy build on a stream with fallback work, else its
  // idle build (fp_launch.h); either decides whatever is queued
  const int fb_occ = separate ? (f32 ? di.fb_busy32 : di.fb_busy) : (f32 ? di.fb_occ32 : di.fb_occ);
  const int fb_grid = total_bytes < SMALL_TEXT_BYTES ? di.sms : di.sms * fb_occ;
  FP_CUDA(fp::launch_fallback(p, fb_grid, stream, f32, separate));
  if (timing) {
    FP_CUDA(cudaEventRecord(s->ev[slot][2], stream));
    s->ev_used[slot] = true;
    for (int k = 1; k <= 2; k++) {  // harvest a couple of older slots, non-blocking
      int old = (slot - k + Scratch::RING) % Scratch::RING;
      fp_err_t e = harvest(s, old, false);
      if (e != FP_OK) return e;
    }
  }
  s->calls++;
  s->bytes += total_bytes;
  return FP_OK;
}

// One persistent launch over nbuf device buffers; range(b) gives buffer b's
// output range (first entry, capacity) in out_f64 / out_status.
template <class Range>
fp_err_t batch_impl(const char* const* texts, const size_t* lens, uint32_t nbuf, char delim,
                    double* out_f64, uint8_t* out_status, uint64_t* out_counts,
                    cudaStream_t stream, Range range, unsigned int* err_out = nullptr) {
  if (!texts || !lens || !out_counts) return FP_ERR_ARG;
  if (nbuf == 0 || nbuf > MAX_BUFS) return FP_ERR_ARG;
  bool any = false;
  for (uint32_t b = 0; b < nbuf; b++) {
    if (lens[b] >= MAX_LEN) return FP_ERR_ARG;
    if (lens[b] > 0 && !texts[b]) return FP_ERR_ARG;
    any |= range(b).second > 0;
  }
  if (any && (!out_f64 || !out_status)) return FP_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  const Config cfg = g_cfg;
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  DeviceInfo* di = nullptr;
  fp_err_t e = device_info(dev, &di);
  if (e != FP_OK) return e;
  unsigned long long total = 0, bytes = 0;
  for (uint32_t b = 0; b < nbuf; b++) {
    total += chunks_of(reinterpret_cast<uintptr_t>(texts[b]) & 15, lens[b], cfg.chunk_bytes);
    bytes += lens[b];
  }
  Scratch* s = nullptr;
  e = get_scratch(stream, total, nbuf, cfg.fallback_queue, &s);
  if (e != FP_OK) return e;
  LaunchParams p;
  memset(&p, 0, sizeof(p));
  p.nbuf = nbuf;
  p.delim = (unsigned char)delim;
  p.out_bits = reinterpret_cast<unsigned long long*>(out_f64);
  p.out_status = out_status;
  p.err_out = err_out;
  if (nbuf == 1) {
    const auto r = range(0);
    fill_desc(p.one, texts[0], lens[0], 0, total, r.first, r.second, out_counts);
  } else {
    // the staging buffer may still feed the previous call's upload
    if (s->desc_pending) FP_CUDA(cudaEventSynchronize(s->desc_copied));
    unsigned long long c = 0;
    for (uint32_t b = 0; b < nbuf; b++) {
      const unsigned long long nch =
          chunks_of(reinterpret_cast<uintptr_t>(texts[b]) & 15, lens[b], cfg.chunk_bytes);
      const auto r = range(b);
      fill_desc(s->h_descs[b], texts[b], lens[b], c, nch, r.first, r.second, out_counts + b);
      c += nch;
    }
    FP_CUDA(cudaMemcpyAsync(s->d_descs, s->h_descs, (size_t)nbuf * sizeof(BufDesc),
                            cudaMemcpyHostToDevice, stream));
    FP_CUDA(cudaEventRecord(s->desc_copied, stream));
    s->desc_pending = true;
    p.descs = s->d_descs;
  }
  return run(s, cfg, *di, p, total, bytes, stream);
}

}  // namespace

// Entry points for the library's own host runtime (fp_internal.h).
namespace fp {

// Segments of the pipelined path: at most this many bytes (each copy in and
// each parse call has a fixed cost; 32 MB measured fastest on a 188 MB text,
// 3% above 16 MB), and at least PIPE_MIN_SEGS of them so that copies in,
// parses and copies out still overlap on texts near PIPE_MIN_BYTES.
constexpr size_t PIPE_SEG_BYTES = 32u << 20;
constexpr size_t PIPE_MIN_SEGS = 4;

// Segment starts of the pipelined host parse, cuts[0] = 0 < cuts[1] < ... <
// cuts[K] = len (returns K): each cut follows a separator near a target
// position, so a segment's fields are exactly the text's fields in that
// range.  Segments hold at most about PIPE_SEG_BYTES, there are at least
// PIPE_MIN_SEGS of them, and on long texts the last three shrink to 1/2, 1/4
// and 1/8 of a full one, so that little parse and copy work is left once the
// last bytes have arrived.
int plan_host_segments(const char* host_text, size_t len, char delim, size_t* cuts) {
  const size_t S = PIPE_SEG_BYTES;
  const size_t tail[3] = {S / 2, S / 4, S / 8};
  size_t front = len;
  int ntail = 0;
  for (int j = 0; j < 3 && front >= 2 * S; j++) {
    front -= tail[j];
    ntail++;
  }
  size_t nf = (front + S - 1) / S;
  if (nf + ntail < PIPE_MIN_SEGS) nf = PIPE_MIN_SEGS - ntail;
  if (nf + ntail > (size_t)PIPE_MAX_SEGS) nf = PIPE_MAX_SEGS - ntail;
  size_t targets[PIPE_MAX_SEGS];
  size_t nt = 0;
  for (size_t i = 1; i < nf; i++) targets[nt++] = i * (front / nf);
  size_t at = front;
  for (int j = 0; j < ntail; j++) {
    targets[nt++] = at;
    at += tail[j];
  }
  const unsigned char d = (unsigned char)delim;
  int K = 0;
  cuts[K++] = 0;
  for (size_t t = 0; t < nt; t++) {
    size_t c = targets[t];
    if (c <= cuts[K - 1]) continue;
    const size_t stop = c + (1u << 20) < len ? c + (1u << 20) : len;
    while (c < stop && host_text[c - 1] != '\n' && (unsigned char)host_text[c - 1] != d) c++;
    if (c < stop && c < len) cuts[K++] = c;  // else: no separator near, no cut here
  }
  cuts[K] = len;
  return K;
}


fp_err_t parse_batch_ranges(const char* const* texts, const size_t* lens, uint32_t nbuf,
                            char delim, double* out_f64, uint8_t* out_status,
                            const uint64_t* out_base, const uint64_t* out_cap,
                            uint64_t* out_counts, cudaStream_t stream, unsigned int* err_out) {
  if (!out_base || !out_cap) return FP_ERR_ARG;
  return batch_impl(texts, lens, nbuf, delim, out_f64, out_status, out_counts, stream,
                    [&](uint32_t b) { return std::make_pair(out_base[b], out_cap[b]); },
                    err_out);
}

fp_err_t reserve_stream_scratch(cudaStream_t stream, unsigned long long chunks, uint32_t nbuf) {
  std::lock_guard<std::mutex> lk(g_mu);
  Scratch* s = nullptr;
  return get_scratch(stream, chunks, nbuf, g_cfg.fallback_queue, &s);
}

fp_err_t release_stream_scratch(cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  auto it = g_scratch.find(std::make_pair(dev, stream));
  if (it == g_scratch.end()) return FP_OK;
  if (it->second) {
    cudaStreamSynchronize(stream);
    free_scratch(it->second);
  }
  g_scratch.erase(it);
  return FP_OK;
}

fp_err_t stream_error_word(cudaStream_t stream, unsigned int** word) {
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  auto it = g_scratch.find(std::make_pair(dev, stream));
  if (it == g_scratch.end()) return FP_ERR_ARG;
  *word = &it->second->ctl->error;
  return FP_OK;
}

}  // namespace fp

namespace {
// ---------------------------------------------------------------------------
// host-buffer parse
// ---------------------------------------------------------------------------
// Below this many bytes the simple path lets the parse kernel write the
// results into pinned host arrays directly (no count round trip, no copy
// calls); larger result sets move faster by copy engine.
constexpr size_t DIRECT_MAX_BYTES = 8u << 20;

// The address the device uses for host memory p, or null when p is not
// pinned (page-locked) memory.
const void* device_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return a.devicePointer;
}
void* device_view(void* p) { return const_cast<void*>(device_view(static_cast<const void*>(p))); }

// Staging of (stream) for texts of len bytes, and for their results when
// `results` (room for len of them).  Call with g_mu held.
fp_err_t stage_for(cudaStream_t stream, size_t len, bool results, Scratch** out) {
  Scratch* s = nullptr;
  fp_err_t e = get_scratch(stream, 1, 1, g_cfg.fallback_queue, &s);
  if (e != FP_OK) return e;
  if (!s->stage_count) FP_CUDA(cudaMalloc(&s->stage_count, sizeof(unsigned long long)));
  if (len > s->stage_cap) {
    FP_CUDA(cudaStreamSynchronize(stream));
    cudaFree(s->stage_text);
    s->stage_text = nullptr;
    s->stage_cap = 0;
    FP_CUDA(cudaMalloc(&s->stage_text, len));
    s->stage_cap = len;
  }
  if (results && len > s->stage_out_cap) {
    FP_CUDA(cudaStreamSynchronize(stream));
    cudaFree(s->stage_out);
    cudaFree(s->stage_status);
    s->stage_out = nullptr;
    s->stage_status = nullptr;
    s->stage_out_cap = 0;
    FP_CUDA(cudaMalloc(&s->stage_out, len * sizeof(double)));
    FP_CUDA(cudaMalloc(&s->stage_status, len));
    s->stage_out_cap = len;
  }
  *out = s;
  return FP_OK;
}

// One-buffer binary64 parse of device text into out_f64 / out_status (room
// for out_cap results; device memory, or pinned host memory through its
// device address).  out_count may be null.
fp_err_t parse_one(const char* text, size_t len, char delim, double* out_f64, uint8_t* out_status,
                   size_t out_cap, uint64_t* out_count, cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  const Config cfg = text_config(g_cfg, len);
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  DeviceInfo* di = nullptr;
  fp_err_t e = device_info(dev, &di);
  if (e != FP_OK) return e;
  const uintptr_t t = reinterpret_cast<uintptr_t>(text);
  const unsigned long long nch = chunks_of(t & 15, len, cfg.chunk_bytes);
  Scratch* s = nullptr;
  e = get_scratch(stream, nch, 1, cfg.fallback_queue, &s);
  if (e != FP_OK) return e;
  LaunchParams p;
  memset(&p, 0, sizeof(p));
  fill_desc(p.one, text, len, 0, nch, 0, out_cap, out_count);
  p.descs = nullptr;
  p.nbuf = 1;
  p.delim = (unsigned char)delim;
  p.out_bits = reinterpret_cast<unsigned long long*>(out_f64);
  p.out_status = out_status;
  return run(s, cfg, *di, p, nch, len, stream);
}

// The mapped count word of (stream)'s scratch (pinned; `dv` is its device
// address).  Call with g_mu held.
fp_err_t count_word(Scratch* s, volatile unsigned long long** host,
                    unsigned long long** dv) {
  if (!s->pipe_host) {
    FP_CUDA(cudaMallocHost(&s->pipe_host, sizeof(unsigned long long)));
    FP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->pipe_host_dv), s->pipe_host, 0));
  }
  *host = s->pipe_host;
  *dv = s->pipe_host_dv;
  return FP_OK;
}

// One copy in, one parse, the count, then exactly that many results back.
// When both result arrays are pinned and the text is below DIRECT_MAX_BYTES
// the parse kernel writes them (and the count) in host memory directly, so
// nothing is copied back.
fp_err_t host_simple(const char* host_text, size_t len, char delim, double* host_f64,
                     uint8_t* host_status, uint64_t* host_count, cudaStream_t stream) {
  double* dv_f64 = static_cast<double*>(device_view(host_f64));
  uint8_t* dv_st = static_cast<uint8_t*>(device_view(host_status));
  const bool direct = dv_f64 && dv_st && len < DIRECT_MAX_BYTES;
  Scratch* s = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    fp_err_t e = stage_for(stream, len, !direct, &s);
    if (e != FP_OK) return e;
  }
  if (len) FP_CUDA(cudaMemcpyAsync(s->stage_text, host_text, len, cudaMemcpyHostToDevice, stream));
  const char* text = len ? (const char*)s->stage_text : nullptr;
  if (direct) {  // results straight into the caller's pinned arrays
    volatile unsigned long long* hc = nullptr;
    unsigned long long* dc = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      fp_err_t e = count_word(s, &hc, &dc);
      if (e != FP_OK) return e;
    }
    fp_err_t e = parse_one(text, len, delim, dv_f64, dv_st, len, (uint64_t*)dc, stream);
    if (e != FP_OK) return e;
    FP_CUDA(cudaStreamSynchronize(stream));
    const unsigned long long n = *hc;
    if (n > len) return FP_ERR_INTERNAL;
    *host_count = n;
    return FP_OK;
  }
  fp_err_t e = parse_one(text, len, delim, s->stage_out, s->stage_status, len,
                         (uint64_t*)s->stage_count, stream);
  if (e != FP_OK) return e;
  unsigned long long n = 0;
  FP_CUDA(cudaMemcpyAsync(&n, s->stage_count, sizeof(n), cudaMemcpyDeviceToHost, stream));
  FP_CUDA(cudaStreamSynchronize(stream));
  if (n > len) return FP_ERR_INTERNAL;
  if (n) {
    FP_CUDA(cudaMemcpyAsync(host_f64, s->stage_out, n * sizeof(double), cudaMemcpyDeviceToHost,
                            stream));
    FP_CUDA(cudaMemcpyAsync(host_status, s->stage_status, n, cudaMemcpyDeviceToHost, stream));
  }
  FP_CUDA(cudaStreamSynchronize(stream));
  *host_count = n;
  return FP_OK;
}

// Pinned host memory: the text is cut at separators into segments
// (fp::plan_host_segments).  All segments are copied in on
// pipe_in, back to back; segment i is parsed on the caller's stream once it
// has landed, and the parse kernel writes its field count straight into
// pinned host memory (no copy call queues behind the result copies); this
// thread waits for each parse in turn and queues the copies of exactly that
// many results (copy engine, pipe_out) at the running total.  (Results
// written by the parse kernels into the caller's pinned arrays directly
// were slower here: the kernels' writes share the link less well than the
// copy engine's, 127 against 146 GB/s end to end on the 188 MB bulk text.)
// Copies in, parses and copies out of different segments overlap, and the
// SMs only parse; with both directions busy the link moved about 260 GB/s
// in all (161 in, 99 out), which bounds this path.
fp_err_t host_pipelined(const char* host_text, size_t len, char delim, double* host_f64,
                        uint8_t* host_status, uint64_t* host_count, cudaStream_t stream) {
  size_t cuts[Scratch::PIPE_SEGS + 1];
  const int K = fp::plan_host_segments(host_text, len, delim, cuts);
  Scratch* s = nullptr;
  Config cfg;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    cfg = g_cfg;
    fp_err_t e = stage_for(stream, len, true, &s);
    if (e != FP_OK) return e;
    size_t maxseg = 0;
    for (int i = 0; i < K; i++) maxseg = std::max(maxseg, cuts[i + 1] - cuts[i]);
    e = get_scratch(stream, chunks_of(15, maxseg, cfg.chunk_bytes), 1, cfg.fallback_queue, &s);
    if (e != FP_OK) return e;
    if (!s->pipe_in) {
      FP_CUDA(cudaStreamCreateWithFlags(&s->pipe_in, cudaStreamNonBlocking));
      FP_CUDA(cudaStreamCreateWithFlags(&s->pipe_out, cudaStreamNonBlocking));
      for (int i = 0; i < Scratch::PIPE_SEGS; i++) {
        FP_CUDA(cudaEventCreateWithFlags(&s->pipe_ev_in[i], cudaEventDisableTiming));
        FP_CUDA(cudaEventCreateWithFlags(&s->pipe_ev_parsed[i], cudaEventDisableTiming));
      }
      FP_CUDA(cudaEventCreateWithFlags(&s->pipe_ev_start, cudaEventDisableTiming));
      FP_CUDA(cudaEventCreateWithFlags(&s->pipe_ev_done, cudaEventDisableTiming));
      FP_CUDA(cudaMallocHost(&s->pipe_counts, Scratch::PIPE_SEGS * sizeof(unsigned long long)));
      FP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->pipe_counts_dv), s->pipe_counts,
                                       0));
    }
  }
  unsigned long long* counts = s->pipe_counts_dv;  // written by the parse kernels
  volatile unsigned long long* hcounts = s->pipe_counts;
  // everything queued before on the caller's stream comes first
  FP_CUDA(cudaEventRecord(s->pipe_ev_start, stream));
  FP_CUDA(cudaStreamWaitEvent(s->pipe_in, s->pipe_ev_start, 0));
  FP_CUDA(cudaStreamWaitEvent(s->pipe_out, s->pipe_ev_start, 0));
  for (int i = 0; i < K; i++) {  // all copies in, back to back
    FP_CUDA(cudaMemcpyAsync(s->stage_text + cuts[i], host_text + cuts[i], cuts[i + 1] - cuts[i],
                            cudaMemcpyHostToDevice, s->pipe_in));
    FP_CUDA(cudaEventRecord(s->pipe_ev_in[i], s->pipe_in));
  }
  for (int i = 0; i < K; i++) {  // the parses, each once its bytes have landed
    const size_t c = cuts[i];
    FP_CUDA(cudaStreamWaitEvent(stream, s->pipe_ev_in[i], 0));
    fp_err_t e = fp_parse_f64((const char*)s->stage_text + c, cuts[i + 1] - c, delim,
                              s->stage_out + c, s->stage_status + c, (uint64_t*)(counts + i),
                              reinterpret_cast<struct CUstream_st*>(stream));
    if (e != FP_OK) return e;
    FP_CUDA(cudaEventRecord(s->pipe_ev_parsed[i], stream));
  }
  unsigned long long total = 0;
  for (int i = 0; i < K; i++) {  // results out, segment by segment
    FP_CUDA(cudaEventSynchronize(s->pipe_ev_parsed[i]));
    const unsigned long long n = hcounts[i];
    if (n > cuts[i + 1] - cuts[i]) return FP_ERR_INTERNAL;
    if (n) {
      FP_CUDA(cudaMemcpyAsync(host_f64 + total, s->stage_out + cuts[i], n * sizeof(double),
                              cudaMemcpyDeviceToHost, s->pipe_out));
      FP_CUDA(cudaMemcpyAsync(host_status + total, s->stage_status + cuts[i], n,
                              cudaMemcpyDeviceToHost, s->pipe_out));
    }
    total += n;
  }
  FP_CUDA(cudaStreamSynchronize(s->pipe_out));
  *host_count = total;
  return FP_OK;
}

// A host call that failed part-way may still have copies queued that read or
// write the caller's host arrays: wait for them, so that the arrays are the
// caller's again when the call returns (its documented synchronous contract
// holds on errors too).  The error itself was already returned.
void drain_host_call(cudaStream_t stream) {
  cudaStreamSynchronize(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_scratch.find({dev, stream});
    if (it != g_scratch.end() && it->second) {
      if (it->second->pipe_in) cudaStreamSynchronize(it->second->pipe_in);
      if (it->second->pipe_out) cudaStreamSynchronize(it->second->pipe_out);
    }
  }
  cudaGetLastError();  // the failure is reported by the call's return value
}

}  // namespace

extern "C" {

size_t fp_max_fields(size_t len) { return len; }

fp_err_t fp_parse_f64(const char* text, size_t len, char delim, double* out_f64,
                      uint8_t* out_status, uint64_t* out_count, struct CUstream_st* stream_) {
  if (len >= MAX_LEN) return FP_ERR_ARG;
  if (!out_count) return FP_ERR_ARG;
  if (len > 0 && (!text || !out_f64 || !out_status)) return FP_ERR_ARG;
  return parse_one(text, len, delim, out_f64, out_status, len, out_count,
                   reinterpret_cast<cudaStream_t>(stream_));
}

fp_err_t fp_parse_f32(const char* text, size_t len, char delim, float* out_f32,
                      uint8_t* out_status, uint64_t* out_count, struct CUstream_st* stream_) {
  if (len >= MAX_LEN) return FP_ERR_ARG;
  if (!out_count) return FP_ERR_ARG;
  if (len > 0 && (!text || !out_f32 || !out_status)) return FP_ERR_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(g_mu);
  const Config cfg = text_config(g_cfg, len);
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  DeviceInfo* di = nullptr;
  fp_err_t e = device_info(dev, &di);
  if (e != FP_OK) return e;
  const uintptr_t t = reinterpret_cast<uintptr_t>(text);
  const unsigned long long nch = chunks_of(t & 15, len, cfg.chunk_bytes);
  Scratch* s = nullptr;
  e = get_scratch(stream, nch, 1, cfg.fallback_queue, &s);
  if (e != FP_OK) return e;
  if (len > s->cap_loc) {  // one location slot per possible field
    FP_CUDA(cudaStreamSynchronize(stream));
    cudaFree(s->loc);
    s->loc = nullptr;
    s->cap_loc = 0;
    FP_CUDA(cudaMalloc(&s->loc, len * sizeof(unsigned long long)));
    s->cap_loc = len;
  }
  LaunchParams p;
  memset(&p, 0, sizeof(p));
  fill_desc(p.one, text, len, 0, nch, 0, len, out_count);
  p.descs = nullptr;
  p.nbuf = 1;
  p.delim = (unsigned char)delim;
  p.out_bits = reinterpret_cast<unsigned long long*>(out_f32);
  p.out_status = out_status;
  p.loc = s->loc;
  return run(s, cfg, *di, p, nch, len, stream, true);
}

fp_err_t fp_parse_ex(const char* text, size_t len, const fp_options_t* opt, void* out_values,
                     uint8_t* out_status, uint64_t* out_count, struct CUstream_st* stream_) {
  if (!opt || !out_count || len >= MAX_LEN) return FP_ERR_ARG;
  if (opt->format > FP_FORMAT_F32 || opt->grammar > FP_GRAMMAR_JSON || opt->reserved)
    return FP_ERR_ARG;
  const uint64_t K = opt->columns;
  if (K == 1 || K >= (1u << 24)) return FP_ERR_ARG;
  unsigned long long out_cap = len;
  if (K) {
    if (opt->rows_cap == 0 || opt->rows_cap > (~0ull) / K) return FP_ERR_ARG;
    out_cap = K * opt->rows_cap;
  }
  if (len > 0 && (!text || !out_values || !out_status)) return FP_ERR_ARG;
  const bool f32 = opt->format == FP_FORMAT_F32;
  // MODE_* bits of the parse kernel: JSON 1, column-major 2, hexadecimal 4
  const int mode = (opt->grammar == FP_GRAMMAR_JSON ? 1 : 0) | (K ? 2 : 0) |
                   (opt->grammar == FP_GRAMMAR_HEX ? 4 : 0);
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(g_mu);
  Config cfg = g_cfg;
  if (mode) cfg.chunk_bytes = cfg.chunk_bytes <= 8192 ? 8192 : 16384;
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  DeviceInfo* di = nullptr;
  fp_err_t e = device_info(dev, &di);
  if (e != FP_OK) return e;
  const uintptr_t t = reinterpret_cast<uintptr_t>(text);
  const unsigned long long nch = chunks_of(t & 15, len, cfg.chunk_bytes);
  Scratch* s = nullptr;
  e = get_scratch(stream, nch, 1, cfg.fallback_queue, &s);
  if (e != FP_OK) return e;
  const bool side_loc = f32 || K;  // pending locations outside the output slots
  if (side_loc && len > s->cap_loc) {
    FP_CUDA(cudaStreamSynchronize(stream));
    cudaFree(s->loc);
    s->loc = nullptr;
    s->cap_loc = 0;
    FP_CUDA(cudaMalloc(&s->loc, len * sizeof(unsigned long long)));
    s->cap_loc = len;
  }
  LaunchParams p;
  memset(&p, 0, sizeof(p));
  fill_desc(p.one, text, len, 0, nch, 0, out_cap, out_count);
  p.descs = nullptr;
  p.nbuf = 1;
  p.delim = (unsigned char)opt->delim;
  p.out_bits = reinterpret_cast<unsigned long long*>(out_values);
  p.out_status = out_status;
  p.loc = side_loc ? s->loc : nullptr;
  p.grammar = opt->grammar;
  if (K) {
    p.columns = (unsigned int)K;
    p.rows_cap = opt->rows_cap;
    p.col_magic = (unsigned long long)((((unsigned __int128)1 << 64) + K - 1) / K);
  }
  return run(s, cfg, *di, p, nch, len, stream, f32, mode);
}

fp_err_t fp_parse_f64_batch(const char* const* texts, const size_t* lens, uint32_t nbuf,
                            char delim, double* out_f64, uint8_t* out_status,
                            const uint64_t* out_offsets, uint64_t* out_counts,
                            struct CUstream_st* stream_) {
  if (!texts || !lens || !out_offsets || !out_counts) return FP_ERR_ARG;
  if (nbuf == 0 || nbuf > MAX_BUFS) return FP_ERR_ARG;
  for (uint32_t b = 0; b < nbuf; b++)
    if (out_offsets[b + 1] < out_offsets[b]) return FP_ERR_ARG;
  return batch_impl(texts, lens, nbuf, delim, out_f64, out_status, out_counts,
                    reinterpret_cast<cudaStream_t>(stream_), [&](uint32_t b) {
                      return std::make_pair(out_offsets[b], out_offsets[b + 1] - out_offsets[b]);
                    });
}

fp_err_t fp_get_stats(fp_stats_t* host_out, int reset, struct CUstream_st* stream_) {
  if (!host_out) return FP_ERR_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  memset(host_out, 0, sizeof(*host_out));
  auto it = g_scratch.find(std::make_pair(dev, stream));
  if (it == g_scratch.end()) return FP_OK;
  Scratch* s = it->second;
  unsigned long long st[16];
  FP_CUDA(cudaMemcpyAsync(st, s->ctl->stats, sizeof(st), cudaMemcpyDeviceToHost, stream));
  FP_CUDA(cudaStreamSynchronize(stream));
  host_out->calls = s->calls;
  host_out->bytes = s->bytes;
  host_out->fields = st[fp::CNT_FIELDS];
  host_out->one_multiply = st[fp::CNT_EL] - std::min(st[fp::CNT_EL], st[fp::CNT_TWO_MUL]);
  host_out->two_multiplies = st[fp::CNT_TWO_MUL];
  host_out->long_fields = st[fp::CNT_LONG];
  host_out->long_settled = st[fp::CNT_LONG_SETTLED];
  host_out->fallback = st[fp::CNT_FALLBACK];
  host_out->fallback_bignum = st[fp::CNT_FALLBACK_BIGNUM];
  host_out->queue_overflow = st[fp::CNT_QUEUE_OVERFLOW];
  host_out->general_tokenizer = st[fp::CNT_SLOW];
  if (reset) {
    FP_CUDA(cudaMemsetAsync(s->ctl->stats, 0, sizeof(st), stream));
    FP_CUDA(cudaStreamSynchronize(stream));
    s->calls = s->bytes = 0;
  }
  return FP_OK;
}

fp_err_t fp_get_error(struct CUstream_st* stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  auto it = g_scratch.find(std::make_pair(dev, stream));
  if (it == g_scratch.end()) return FP_OK;
  Scratch* s = it->second;
  unsigned int err = 0;
  FP_CUDA(cudaMemcpyAsync(&err, &s->ctl->error, sizeof(err), cudaMemcpyDeviceToHost, stream));
  FP_CUDA(cudaStreamSynchronize(stream));
  if (err) {
    FP_CUDA(cudaMemsetAsync(&s->ctl->error, 0, sizeof(err), stream));
    FP_CUDA(cudaStreamSynchronize(stream));
  }
  return (fp_err_t)err;
}

fp_err_t fp_test_arm_stalled_lookback(struct CUstream_st* stream_, uint64_t wait_limit_ns) {
  if (wait_limit_ns == 0 || wait_limit_ns > fp::WAIT_NS_DEFAULT) return FP_ERR_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(g_mu);
  Scratch* s = nullptr;
  fp_err_t e = get_scratch(stream, 1, 1, g_cfg.fallback_queue, &s);
  if (e != FP_OK) return e;
  s->test_stall = true;
  s->test_wait_ns = wait_limit_ns;
  return FP_OK;
}

fp_err_t fp_set_config(const fp_config_t* cfg) {
  if (!cfg) return FP_ERR_ARG;
  if (cfg->chunk_bytes != 4096 && cfg->chunk_bytes != 8192 && cfg->chunk_bytes != 12288 &&
      cfg->chunk_bytes != 16384)
    return FP_ERR_ARG;
  if (cfg->ctas_per_sm > 8) return FP_ERR_ARG;
  if (cfg->fallback_queue < 1024 || cfg->fallback_queue > (1u << 28)) return FP_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  g_cfg.chunk_bytes = cfg->chunk_bytes;
  g_cfg.ctas_per_sm = cfg->ctas_per_sm;
  g_cfg.fallback_queue = cfg->fallback_queue;
  return FP_OK;
}

fp_err_t fp_get_config(fp_config_t* cfg) {
  if (!cfg) return FP_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  cfg->chunk_bytes = g_cfg.chunk_bytes;
  cfg->ctas_per_sm = g_cfg.ctas_per_sm;
  cfg->fallback_queue = g_cfg.fallback_queue;
  return FP_OK;
}

fp_err_t fp_timing_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_timing = on > 0 ? on : 0;
  return FP_OK;
}

fp_err_t fp_timing_read(struct CUstream_st* stream_, double* parse_ms, double* fallback_ms,
                        uint64_t* calls) {
  if (!parse_ms || !fallback_ms || !calls) return FP_ERR_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  *parse_ms = *fallback_ms = 0;
  *calls = 0;
  auto it = g_scratch.find(std::make_pair(dev, stream));
  if (it == g_scratch.end()) return FP_OK;
  Scratch* s = it->second;
  for (int k = 0; k < Scratch::RING; k++) {
    fp_err_t e = harvest(s, k, true);
    if (e != FP_OK) return e;
  }
  *parse_ms = s->acc_parse_ms;
  *fallback_ms = s->acc_fb_ms;
  *calls = s->acc_calls;
  s->acc_parse_ms = s->acc_fb_ms = 0;
  s->acc_calls = 0;
  return FP_OK;
}

fp_err_t fp_parse_f64_host(const char* host_text, size_t len, char delim, double* host_f64,
                           uint8_t* host_status, uint64_t* host_count,
                           struct CUstream_st* stream_) {
  if (len >= MAX_LEN || !host_count) return FP_ERR_ARG;
  if (len > 0 && (!host_text || !host_f64 || !host_status)) return FP_ERR_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (len >= fp::PIPE_MIN_BYTES) {
    const void* dv_text = device_view(host_text);
    void* dv_f64 = device_view(host_f64);
    void* dv_st = device_view(host_status);
    if (dv_text && dv_f64 && dv_st) {
      const fp_err_t e =
          host_pipelined(host_text, len, delim, host_f64, host_status, host_count, stream);
      if (e != FP_OK) drain_host_call(stream);
      return e;
    }
  }
  const fp_err_t e = host_simple(host_text, len, delim, host_f64, host_status, host_count, stream);
  if (e != FP_OK) drain_host_call(stream);
  return e;
}

fp_err_t fp_shutdown(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : g_scratch) {
    if (kv.second) {
      cudaSetDevice(kv.second->device);
      cudaStreamSynchronize(kv.second->stream);
      free_scratch(kv.second);
    }
  }
  g_scratch.clear();
  return FP_OK;
}

const char* fp_strerror(fp_err_t err) {
  switch (err) {
    case FP_OK: return "ok";
    case FP_ERR_ARG: return "invalid argument";
    case FP_ERR_CAPACITY: return "capacity exceeded";
    case FP_ERR_CUDA: return "CUDA call failed";
    case FP_ERR_BUDGET: return "device memory budget exceeded";
    case FP_ERR_TIMEOUT: return "bounded device wait ran out";
    case FP_ERR_INTERNAL: return "internal device error";
  }
  return "unknown error";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
namespace {

// The class of a workload, part of the cache key beside the GPU's name: the
// text's size (small texts take 4 KiB chunks by default and do not fill the
// GPU with 16 KiB ones) and how many of its fields reach the fallback kernel
// (long digit strings and near-midpoints, Section 11: the queue depth only
// matters when there are many).
std::string workload_class(size_t len, unsigned long long fields, unsigned long long pending) {
  const char* size = len < SMALL_TEXT_BYTES ? "small" : (len < (64u << 20) ? "medium" : "large");
  const double rate = fields ? (double)pending / (double)fields : 0.0;
  const char* fb = rate < 0.001 ? "rare" : (rate < 0.1 ? "some" : "many");
  return std::string("size=") + size + ",fallback=" + fb;
}

// The cache: one JSON object per line, one line per (GPU, class).
bool read_cache(const char* path, const std::string& gpu, const std::string& cls,
                fp_config_t* cfg) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  const std::string kg = "\"gpu\": \"" + gpu + "\"", kc = "\"class\": \"" + cls + "\"";
  while (!found && fgets(line, sizeof(line), f)) {
    std::string s(line);
    if (s.find(kg) == std::string::npos || s.find(kc) == std::string::npos) continue;
    auto num = [&](const char* k, uint32_t* v) -> bool {
      std::string kk = std::string("\"") + k + "\": ";
      size_t p = s.find(kk);
      if (p == std::string::npos) return false;
      *v = (uint32_t)strtoul(s.c_str() + p + kk.size(), nullptr, 10);
      return true;
    };
    found = num("chunk_bytes", &cfg->chunk_bytes) && num("ctas_per_sm", &cfg->ctas_per_sm) &&
            num("fallback_queue", &cfg->fallback_queue);
  }
  fclose(f);
  return found;
}

// Replace (GPU, class)'s line of the cache, keeping the others.
void write_cache(const char* path, const std::string& gpu, const std::string& cls,
                 const fp_config_t& c, float ms, size_t len) {
  std::vector<std::string> keep;
  const std::string kg = "\"gpu\": \"" + gpu + "\"", kc = "\"class\": \"" + cls + "\"";
  if (FILE* f = fopen(path, "r")) {
    char line[1024];
    while (fgets(line, sizeof(line), f)) {
      std::string s(line);
      if (s.find(kg) != std::string::npos && s.find(kc) != std::string::npos) continue;
      if (s.find('{') != std::string::npos) keep.push_back(s);
    }
    fclose(f);
  }
  FILE* f = fopen(path, "w");
  if (!f) return;
  for (const std::string& s : keep) fputs(s.c_str(), f);
  fprintf(f,
          "{\"gpu\": \"%s\", \"class\": \"%s\", \"chunk_bytes\": %u, \"ctas_per_sm\": %u, "
          "\"fallback_queue\": %u, \"ms\": %.6f, \"bytes\": %zu}\n",
          gpu.c_str(), cls.c_str(), c.chunk_bytes, c.ctas_per_sm, c.fallback_queue, ms, len);
  fclose(f);
}

}  // namespace

extern "C" fp_err_t fp_autotune(const char* text, size_t len, char delim, const char* cache_path,
                                fp_config_t* chosen) {
  if (!text || len == 0 || len >= MAX_LEN) return FP_ERR_ARG;
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  std::string gpu;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo* di = nullptr;
    fp_err_t e = device_info(dev, &di);
    if (e != FP_OK) return e;
    gpu = di->name;
  }
  fp_config_t cur;
  fp_get_config(&cur);
  double* out = nullptr;
  uint8_t* st = nullptr;
  uint64_t* cnt = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fp_config_t best = cur;
  float best_ms = 1e30f;
  fp_err_t err = FP_OK;
  bool from_cache = false;
  std::string cls;
  // every resource is released below, also when one of these fails
  if (cudaMalloc(&out, len * sizeof(double)) != cudaSuccess || cudaMalloc(&st, len) != cudaSuccess ||
      cudaMalloc(&cnt, sizeof(uint64_t)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    err = FP_ERR_CUDA;
  // Time one configuration: the best of three calls after one warm-up.
  auto time_config = [&](const fp_config_t& c, float* ms_out) -> fp_err_t {
    if (fp_set_config(&c) != FP_OK) return FP_ERR_ARG;
    float ms_min = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
      if (cudaEventRecord(e0, stream) != cudaSuccess) return FP_ERR_CUDA;
      fp_err_t e = fp_parse_f64(text, len, delim, out, st, cnt, stream);
      if (e != FP_OK) return e;
      if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        return FP_ERR_CUDA;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) ms_min = std::min(ms_min, ms);
    }
    *ms_out = ms_min;
    return FP_OK;
  };
  // The workload's class: one call with the current configuration, and the
  // share of its fields that reached the fallback kernel.
  if (err == FP_OK) {
    fp_stats_t before, after;
    float ms = 0;
    err = fp_get_stats(&before, 0, stream);
    if (err == FP_OK) err = time_config(cur, &ms);
    if (err == FP_OK) err = fp_get_stats(&after, 0, stream);
    if (err == FP_OK) {
      const unsigned long long calls = std::max<unsigned long long>(after.calls - before.calls, 1);
      cls = workload_class(len, (after.fields - before.fields) / calls,
                           (after.fallback - before.fallback) / calls);
    }
  }
  if (err == FP_OK && cache_path) {
    fp_config_t c = cur;
    if (read_cache(cache_path, gpu, cls, &c) && fp_set_config(&c) == FP_OK) {
      best = c;
      from_cache = true;
    }
  }
  // chunk size x blocks per SM, at the current queue depth
  for (uint32_t chunk : {4096u, 8192u, 12288u, 16384u}) {
    if (err != FP_OK || from_cache) break;
    for (uint32_t per_sm : {1u, 2u, 3u, 4u, 0u}) {
      fp_config_t c = cur;
      c.chunk_bytes = chunk;
      c.ctas_per_sm = per_sm;
      float ms = 0;
      err = time_config(c, &ms);
      if (err != FP_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  }
  // the fallback queue's depth, for the best launch shape: fields beyond the
  // queue are found by scanning their chunks instead, which costs time when
  // many fields are pending and nothing when none are; the smallest depth
  // within 2% of the fastest is kept (it is per-stream device memory)
  if (err == FP_OK && !from_cache) {
    fp_config_t base = best;
    float t_cur = best_ms;
    std::vector<std::pair<uint32_t, float>> qt;
    for (uint32_t q : {1u << 16, 1u << 18, 1u << 20, 1u << 22}) {
      fp_config_t c = base;
      c.fallback_queue = q;
      float ms = 0;
      if (q == base.fallback_queue) {
        ms = t_cur;
      } else {
        err = time_config(c, &ms);
        if (err != FP_OK) break;
      }
      qt.emplace_back(q, ms);
    }
    if (err == FP_OK) {
      float fastest = 1e30f;
      for (auto& x : qt) fastest = std::min(fastest, x.second);
      for (auto& x : qt) {  // ascending depths: the first within 2% wins
        if (x.second <= fastest * 1.02f) {
          best.fallback_queue = x.first;
          best_ms = x.second;
          break;
        }
      }
    }
  }
  if (stream) {
    // release this temporary stream's scratch
    cudaStreamSynchronize(stream);
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_scratch.find(std::make_pair(dev, stream));
    if (it != g_scratch.end()) {
      free_scratch(it->second);
      g_scratch.erase(it);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (stream) cudaStreamDestroy(stream);
  cudaFree(out);
  cudaFree(st);
  cudaFree(cnt);
  if (err == FP_ERR_CUDA) cudaGetLastError();  // reported by the return value
  if (err != FP_OK) {
    fp_set_config(&cur);
    return err;
  }
  fp_set_config(&best);
  if (chosen) *chosen = best;
  if (cache_path && !from_cache) write_cache(cache_path, gpu, cls, best, best_ms, len);
  return FP_OK;
}

// ---------------------------------------------------------------------------
// batch plans
// ---------------------------------------------------------------------------
struct fp_batch_plan {
  int device;
  LaunchParams p;                  // descriptors, outputs and scratch pointers
  unsigned long long total_chunks;
  unsigned long long total_bytes;
  uint32_t chunk_bytes, ctas_per_sm;
  void* dmem;                      // one allocation: ctl, look-back words, overflow list, queue, descriptors
  size_t scratch_bytes;            // bytes cleared before each launch (ctl + look-back words)
  int grid_parse, grid_fallback;
  cudaGraphExec_t graph;           // the captured launch sequence, or null
  // packing of the results (fp_batch_plan_gather)
  const unsigned long long* counts;  // the caller's out_counts (device)
  void* pack;                      // one allocation: bases[nbuf + 1], starts[nbuf + 1], pieces
  const unsigned long long* bases;
  unsigned long long* starts;
  const unsigned long long* pieces;
  unsigned long long npieces;
  int grid_pack;
};

namespace {
fp_err_t plan_enqueue(fp_batch_plan* pl, cudaStream_t stream) {
  FP_CUDA(cudaMemsetAsync(pl->dmem, 0, pl->scratch_bytes, stream));
  FP_CUDA(fp::launch_parse(pl->p, (int)pl->chunk_bytes, pl->grid_parse, stream));
  FP_CUDA(fp::launch_fallback(pl->p, pl->grid_fallback, stream));
  return FP_OK;
}

// Capture the plan's launch sequence on a private stream and instantiate it.
fp_err_t plan_capture(fp_batch_plan* pl) {
  cudaStream_t cs = nullptr;
  FP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  fp_err_t e = FP_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    e = FP_ERR_CUDA;
  } else {
    e = plan_enqueue(pl, cs);
    cudaError_t ce = cudaStreamEndCapture(cs, &g);  // always end the capture
    if (e == FP_OK && ce != cudaSuccess) e = FP_ERR_CUDA;
  }
  if (e == FP_OK && cudaGraphInstantiate(&pl->graph, g, 0) != cudaSuccess) {
    pl->graph = nullptr;
    e = FP_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  return e;
}
}  // namespace

extern "C" fp_err_t fp_batch_plan_create(const char* const* texts, const size_t* lens,
                                         uint32_t nbuf, char delim, double* out_f64,
                                         uint8_t* out_status, const uint64_t* out_offsets,
                                         uint64_t* out_counts, uint32_t flags,
                                         fp_batch_plan** plan) {
  if (!plan || !texts || !lens || !out_offsets || !out_counts) return FP_ERR_ARG;
  *plan = nullptr;
  if (nbuf == 0 || nbuf > MAX_BUFS || (flags & ~FP_PLAN_GRAPH)) return FP_ERR_ARG;
  bool any = false;
  for (uint32_t b = 0; b < nbuf; b++) {
    if (lens[b] >= MAX_LEN) return FP_ERR_ARG;
    if (lens[b] > 0 && !texts[b]) return FP_ERR_ARG;
    if (out_offsets[b + 1] < out_offsets[b]) return FP_ERR_ARG;
    any |= out_offsets[b + 1] > out_offsets[b];
  }
  if (any && (!out_f64 || !out_status)) return FP_ERR_ARG;
  fp_config_t cfg;
  fp_get_config(&cfg);
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  DeviceInfo* di = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    fp_err_t e = device_info(dev, &di);
    if (e != FP_OK) return e;
  }
  std::vector<BufDesc> h(nbuf);
  unsigned long long c = 0, bytes = 0;
  for (uint32_t b = 0; b < nbuf; b++) {
    const unsigned long long nch =
        chunks_of(reinterpret_cast<uintptr_t>(texts[b]) & 15, lens[b], cfg.chunk_bytes);
    fill_desc(h[b], texts[b], lens[b], c, nch, out_offsets[b], out_offsets[b + 1] - out_offsets[b],
              out_counts + b);
    c += nch;
    bytes += lens[b];
  }
  const unsigned long long qcap = cfg.fallback_queue;
  const size_t off_status = 256;
  const size_t off_ovf = off_status + c * 8;
  const size_t off_queue = off_ovf + 2 * c * 8;
  const size_t off_desc = (off_queue + qcap * 8 + 255) & ~(size_t)255;
  const size_t total = off_desc + (size_t)nbuf * sizeof(BufDesc);
  fp_batch_plan* pl = new fp_batch_plan();
  memset(&pl->p, 0, sizeof(pl->p));
  pl->device = dev;
  if (cudaMalloc(&pl->dmem, total) != cudaSuccess) {
    delete pl;
    return FP_ERR_CUDA;
  }
  unsigned char* base = static_cast<unsigned char*>(pl->dmem);
  if (cudaMemcpy(base + off_desc, h.data(), (size_t)nbuf * sizeof(BufDesc),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(base, 0, off_ovf) != cudaSuccess) {
    cudaFree(pl->dmem);
    delete pl;
    return FP_ERR_CUDA;
  }
  LaunchParams& p = pl->p;
  p.nbuf = nbuf;
  if (nbuf == 1) p.one = h[0];
  p.descs = reinterpret_cast<const BufDesc*>(base + off_desc);
  p.delim = (unsigned char)delim;
  p.total_chunks = c;
  p.out_bits = reinterpret_cast<unsigned long long*>(out_f64);
  p.out_status = out_status;
  p.ctl = reinterpret_cast<Ctl*>(base);
  p.chunk_status = reinterpret_cast<unsigned long long*>(base + off_status);
  p.epoch = 1;  // the look-back words are cleared before every launch
  p.queue = reinterpret_cast<unsigned long long*>(base + off_queue);
  p.qcap = qcap;
  p.ovf = reinterpret_cast<unsigned long long*>(base + off_ovf);
  p.ovf_cap = c;
  p.loc = p.out_bits;
  pl->total_chunks = c;
  pl->total_bytes = bytes;
  pl->scratch_bytes = off_ovf;
  pl->chunk_bytes = cfg.chunk_bytes;
  const int occ = di->parse_occ.at((int)cfg.chunk_bytes);
  const int per_sm = cfg.ctas_per_sm ? std::min<int>((int)cfg.ctas_per_sm, occ) : occ;
  unsigned long long grid = (unsigned long long)di->sms * per_sm;
  pl->grid_parse = (int)(grid > c ? c : grid);
  pl->grid_fallback = di->sms * di->fb_occ;
  pl->graph = nullptr;
  // the packing pieces: each buffer's output range cut into PACK_PIECE fields
  {
    std::vector<unsigned long long> pk;
    for (uint32_t b = 0; b < nbuf; b++)
      for (unsigned long long f0 = 0; f0 < out_offsets[b + 1] - out_offsets[b]; f0 += fp::PACK_PIECE)
        pk.push_back(((unsigned long long)b << 40) | f0);
    pl->npieces = pk.size();
    const size_t n_words = (size_t)(nbuf + 1) + (nbuf + 1) + pk.size();
    if (cudaMalloc(&pl->pack, n_words * sizeof(unsigned long long)) != cudaSuccess) {
      cudaFree(pl->dmem);
      delete pl;
      return FP_ERR_CUDA;
    }
    unsigned long long* w = static_cast<unsigned long long*>(pl->pack);
    pl->bases = w;  // the nbuf + 1 output offsets (capacities are their differences)
    pl->starts = w + nbuf + 1;
    pl->pieces = w + 2 * (nbuf + 1);
    std::vector<unsigned long long> bs(out_offsets, out_offsets + nbuf + 1);
    if (cudaMemcpy(w, bs.data(), (nbuf + 1) * sizeof(unsigned long long), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        (!pk.empty() && cudaMemcpy(w + 2 * (nbuf + 1), pk.data(),
                                   pk.size() * sizeof(unsigned long long),
                                   cudaMemcpyHostToDevice) != cudaSuccess)) {
      cudaFree(pl->pack);
      cudaFree(pl->dmem);
      delete pl;
      return FP_ERR_CUDA;
    }
    pl->counts = reinterpret_cast<const unsigned long long*>(out_counts);
    pl->grid_pack = di->sms * 8;
  }
  if (flags & FP_PLAN_GRAPH) {
    fp_err_t e = plan_capture(pl);
    if (e != FP_OK) {
      cudaFree(pl->pack);
      cudaFree(pl->dmem);
      delete pl;
      return e;
    }
  }
  *plan = pl;
  return FP_OK;
}

extern "C" fp_err_t fp_batch_plan_launch(fp_batch_plan* pl, struct CUstream_st* stream_) {
  if (!pl) return FP_ERR_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (pl->graph) {
    FP_CUDA(cudaGraphLaunch(pl->graph, stream));
    return FP_OK;
  }
  return plan_enqueue(pl, stream);
}

extern "C" fp_err_t fp_batch_plan_gather(fp_batch_plan* pl, double* dst_f64, uint8_t* dst_status,
                                         uint64_t* dst_total, struct CUstream_st* stream_) {
  if (!pl) return FP_ERR_ARG;
  if (pl->npieces && (!dst_f64 || !dst_status)) return FP_ERR_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  FP_CUDA(fp::launch_pack_scan(pl->counts, pl->bases, pl->p.nbuf, pl->starts,
                               reinterpret_cast<unsigned long long*>(dst_total), stream));
  FP_CUDA(fp::launch_pack_copy(pl->pieces, pl->npieces, pl->counts, pl->bases, pl->starts,
                               pl->p.out_bits, pl->p.out_status,
                               reinterpret_cast<unsigned long long*>(dst_f64), dst_status,
                               pl->grid_pack, stream));
  return FP_OK;
}

extern "C" fp_err_t fp_batch_plan_destroy(fp_batch_plan* pl) {
  if (!pl) return FP_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(pl->device);
  cudaDeviceSynchronize();
  if (pl->graph) cudaGraphExecDestroy(pl->graph);
  cudaFree(pl->pack);
  cudaFree(pl->dmem);
  if (prev >= 0) cudaSetDevice(prev);
  delete pl;
  return FP_OK;
}
