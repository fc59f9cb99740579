// fp_noalloc.cu -- fp_parse_f64_noalloc: the parse without any allocation.
//
// Some callers may not allocate memory once they are running: a process
// whose memory is fixed at start-up (real-time or certified code, a plugin
// whose host owns every allocation, a service that must not fail on an
// allocation mid-request), or code that already holds a device-wide
// allocator lock.  fp_parse_f64 allocates its per-stream scratch on first
// use; this entry point instead keeps the scratch of the same two kernels
// in one fixed device array below, which every GPU that loads the library
// holds until the process exits.
#include <algorithm>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/fpparse.h"
#include "fp_launch.h"
#include "fp_types.cuh"

namespace {

using fp::BufDesc;
using fp::Ctl;
using fp::LaunchParams;

// Capacity of the fixed scratch: look-back words and overflow entries for
// up to NOALLOC_MAX_CHUNKS chunks, and a fallback queue of NOALLOC_QUEUE
// entries (fields beyond it are found by scanning their chunks).
constexpr unsigned long long NOALLOC_MAX_CHUNKS = 65536;
constexpr unsigned long long NOALLOC_QUEUE = 65536;
constexpr size_t OFF_CTL = 0;
constexpr size_t OFF_STATUS = 256;
constexpr size_t OFF_OVF = OFF_STATUS + NOALLOC_MAX_CHUNKS * 8;
constexpr size_t OFF_QUEUE = OFF_OVF + 2 * NOALLOC_MAX_CHUNKS * 8;
constexpr size_t NOALLOC_BYTES = OFF_QUEUE + NOALLOC_QUEUE * 8;  // 2 MiB + 256 B
static_assert(sizeof(Ctl) <= OFF_STATUS, "control block fits");

// The scratch.  In host code this name is only a stand-in for the device
// array: its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char fp_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
struct DeviceSlot {
  bool ready;
  unsigned char* scratch;  // device address of fp_noalloc_scratch on this device
  int sms, parse_occ, fallback_occ;
};
DeviceSlot g_slots[MAX_DEVICES];
std::mutex g_noalloc_mu;

// Once per device, with that device current: the array's device address and
// the launch shape.  Returns FP_OK or FP_ERR_CUDA.
fp_err_t setup_device(int dev, int chunk_bytes, DeviceSlot** out) {
  DeviceSlot& s = g_slots[dev];
  if (!s.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, fp_noalloc_scratch) != cudaSuccess) return FP_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return FP_ERR_CUDA;
    int fb = 0;
    if (fp::fallback_occupancy(&fb) != cudaSuccess) return FP_ERR_CUDA;
    s.scratch = static_cast<unsigned char*>(ptr);
    s.sms = sms;
    s.fallback_occ = fb > 0 ? fb : 1;
    s.parse_occ = 0;
    s.ready = true;
  }
  int occ = 0;  // may change with the chunk size; cheap to ask
  if (fp::parse_occupancy(chunk_bytes, &occ) != cudaSuccess) return FP_ERR_CUDA;
  s.parse_occ = occ > 0 ? occ : 1;
  *out = &s;
  return FP_OK;
}

// Same bound on a buffer's length as the other entry points (pending
// fields keep a 40-bit offset).
constexpr unsigned long long NOALLOC_MAX_LEN = 1ull << 40;
// Texts below this many bytes take 4 KiB chunks when the configured chunk is
// the default 16 KiB, as fp_parse_f64 does (more blocks share a small text).
constexpr size_t NOALLOC_SMALL_TEXT = 4u << 20;

// Argument and capacity checks of fp_parse_f64_noalloc, before anything is
// queued: the chunk size to use and the number of chunks, or an error.  The
// length is compared with the fixed capacity before any sum that could wrap.
fp_err_t noalloc_plan(const void* text, size_t len, const void* out_f64, const void* out_status,
                         const void* out_count, uint32_t cfg_chunk, uint32_t* chunk_bytes,
                         unsigned long long* nchunks) {
  if (!out_count) return FP_ERR_ARG;
  if (len >= NOALLOC_MAX_LEN) return FP_ERR_ARG;
  if (len > 0 && (!text || !out_f64 || !out_status)) return FP_ERR_ARG;
  uint32_t c = cfg_chunk;
  if (len < NOALLOC_SMALL_TEXT && c == 16384) c = 4096;
  const unsigned long long o = reinterpret_cast<uintptr_t>(text) & 15;
  // o + len <= NOALLOC_MAX_CHUNKS * c, with len < 2^40 so the sum cannot wrap
  if (o + len > NOALLOC_MAX_CHUNKS * (unsigned long long)c) return FP_ERR_CAPACITY;
  unsigned long long n = (o + len + c - 1) / c;
  *chunk_bytes = c;
  *nchunks = n ? n : 1;
  return FP_OK;
}

}  // namespace

extern "C" fp_err_t fp_parse_f64_noalloc(const char* text, size_t len, char delim, double* out_f64,
                                         uint8_t* out_status, uint64_t* out_count,
                                         struct CUstream_st* stream_) {
  fp_config_t cfg;
  fp_get_config(&cfg);
  uint32_t chunk_bytes = 0;
  unsigned long long nchunks = 0;
  const fp_err_t ce = noalloc_plan(text, len, out_f64, out_status, out_count, cfg.chunk_bytes,
                                      &chunk_bytes, &nchunks);
  if (ce != FP_OK) return ce;
  const unsigned long long o = reinterpret_cast<uintptr_t>(text) & 15;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return FP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  DeviceSlot* slot = nullptr;
  fp_err_t e = setup_device(dev, (int)chunk_bytes, &slot);
  if (e != FP_OK) return e;
  unsigned char* base = slot->scratch;
  // The array keeps the previous call's contents: the control block and the
  // look-back words must start at zero.
  if (cudaMemsetAsync(base + OFF_CTL, 0, OFF_STATUS, stream) != cudaSuccess) return FP_ERR_CUDA;
  if (cudaMemsetAsync(base + OFF_STATUS, 0, nchunks * 8, stream) != cudaSuccess) return FP_ERR_CUDA;

  LaunchParams p;
  memset(&p, 0, sizeof(p));
  const uintptr_t t = reinterpret_cast<uintptr_t>(text);
  p.one.base = reinterpret_cast<const uint8_t*>(t & ~(uintptr_t)15);
  p.one.o = o;
  p.one.len = len;
  p.one.chunk0 = 0;
  p.one.nchunks = nchunks;
  p.one.out_base = 0;
  p.one.out_cap = len;
  p.one.out_count = reinterpret_cast<unsigned long long*>(out_count);
  p.descs = nullptr;
  p.nbuf = 1;
  p.delim = (unsigned char)delim;
  p.total_chunks = nchunks;
  p.out_bits = reinterpret_cast<unsigned long long*>(out_f64);
  p.out_status = out_status;
  p.ctl = reinterpret_cast<Ctl*>(base + OFF_CTL);
  p.chunk_status = reinterpret_cast<unsigned long long*>(base + OFF_STATUS);
  p.epoch = 1;
  p.queue = reinterpret_cast<unsigned long long*>(base + OFF_QUEUE);
  p.qcap = NOALLOC_QUEUE;
  p.ovf = reinterpret_cast<unsigned long long*>(base + OFF_OVF);
  p.ovf_cap = NOALLOC_MAX_CHUNKS;
  p.loc = p.out_bits;
  const int per_sm = cfg.ctas_per_sm ? ((int)cfg.ctas_per_sm < slot->parse_occ ? (int)cfg.ctas_per_sm
                                                                              : slot->parse_occ)
                                     : slot->parse_occ;
  unsigned long long grid = (unsigned long long)slot->sms * per_sm;
  if (grid > nchunks) grid = nchunks;
  if (fp::launch_parse(p, (int)chunk_bytes, (int)grid, stream) != cudaSuccess) return FP_ERR_CUDA;
  if (fp::launch_fallback(p, slot->sms * slot->fallback_occ, stream) != cudaSuccess)
    return FP_ERR_CUDA;
  return FP_OK;
}
