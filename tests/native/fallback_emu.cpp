// fallback_emu.cpp -- the fallback kernel's per-field code (warp_field and
// its big-number helpers, taken from fp_fallback_kernel.cu at build time as
// fallback_body.inc) run on the host: the 32 lanes of a warp are 32
// coroutines (POSIX ucontext) scheduled in lockstep, and each warp
// intrinsic (__ballot_sync, __shfl_*_sync, __syncwarp) is a rendezvous of
// all 32: every lane posts its value and yields, and once all have posted,
// each reads the posted values (double-buffered by phase).  A lane that
// reaches an intrinsic the others do not is reported as divergence.
//
// usage: fallback_emu <64|32> <grammar 0|1|2> < text    ('\n'-separated)
// One line per field: "<bits hex> <status>", as the kernel stores them.
#include <ucontext.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#define __device__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))

#include "fp_device.cuh"
#include "fp_types.cuh"
#include "dec_tables.inc"

namespace fp {
const unsigned long long fp_pow5_table_dev[2 * FP_POW5_ENTRIES] = {FP_POW5_TABLE_VALUES};
}

// ---------------------------------------------------------------------------
// warp emulation
// ---------------------------------------------------------------------------
struct uint4 {
  unsigned int x, y, z, w;
};

namespace emu {
constexpr int W = 32;
ucontext_t sched, lanes[W];
int cur = 0;
bool done[W];
int kind[2][W];
uint64_t slot[2][W];
unsigned phase[W];
bool diverged = false;

// post v for this lane's current phase, yield, and return the phase's slots
const uint64_t* post(uint64_t v, int k) {
  const int me = cur;
  const unsigned p = phase[me] & 1;
  slot[p][me] = v;
  kind[p][me] = k;
  phase[me]++;
  swapcontext(&lanes[me], &sched);
  return slot[p];
}
int lane() { return cur; }
}  // namespace emu

enum { K_BALLOT = 1, K_SHFL, K_UP, K_XOR, K_SYNC };

unsigned int __ballot_sync(unsigned int, int pred) {
  const uint64_t* s = emu::post(pred ? 1 : 0, K_BALLOT);
  unsigned int m = 0;
  for (int i = 0; i < emu::W; i++) m |= (unsigned int)(s[i] & 1) << i;
  return m;
}
template <class T>
T __shfl_sync(unsigned int, T v, int src) {
  uint64_t u = 0;
  std::memcpy(&u, &v, sizeof(T));
  const uint64_t* s = emu::post(u, K_SHFL);
  T r;
  std::memcpy(&r, &s[src & 31], sizeof(T));
  return r;
}
template <class T>
T __shfl_up_sync(unsigned int, T v, unsigned int d) {
  uint64_t u = 0;
  std::memcpy(&u, &v, sizeof(T));
  const uint64_t* s = emu::post(u, K_UP);
  const int me = emu::lane();
  T r;
  std::memcpy(&r, &s[me >= (int)d ? me - (int)d : me], sizeof(T));
  return r;
}
template <class T>
T __shfl_xor_sync(unsigned int, T v, int m) {
  uint64_t u = 0;
  std::memcpy(&u, &v, sizeof(T));
  const uint64_t* s = emu::post(u, K_XOR);
  T r;
  std::memcpy(&r, &s[(emu::lane() ^ m) & 31], sizeof(T));
  return r;
}
void __syncwarp() { emu::post(0, K_SYNC); }
int __popc(unsigned int x) { return __builtin_popcount(x); }
int __popcll(unsigned long long x) { return __builtin_popcountll(x); }
int __ffs(int x) { return __builtin_ffs(x); }
int __ffsll(long long x) { return __builtin_ffsll(x); }
int __clz(int x) { return x ? __builtin_clz((unsigned)x) : 32; }
int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }

namespace fp {
namespace {
#include "fallback_body.inc"
}  // namespace
}  // namespace fp

// ---------------------------------------------------------------------------
// one warp per field
// ---------------------------------------------------------------------------
namespace {
struct Job {
  const uint8_t* f;
  unsigned long long lim;
  uint32_t grammar;
  bool f32;
  fp::WarpSmem* sm;
  fp::LongResult r[emu::W];
};
Job g_job;

void lane_main(int l) {
  bool nl = true;
  g_job.r[l] = g_job.f32
                   ? fp::warp_field<fp::F32>(g_job.f, g_job.lim, '\n', g_job.grammar, *g_job.sm, &nl, l)
                   : fp::warp_field<fp::F64>(g_job.f, g_job.lim, '\n', g_job.grammar, *g_job.sm, &nl, l);
  emu::done[l] = true;
  swapcontext(&emu::lanes[l], &emu::sched);
}

void lane_entry(int l) { lane_main(l); }

constexpr size_t STACK = 256 << 10;
std::vector<char> g_stacks(emu::W * STACK);

bool run_field() {
  for (int l = 0; l < emu::W; l++) {
    emu::done[l] = false;
    emu::phase[l] = 0;
    getcontext(&emu::lanes[l]);
    emu::lanes[l].uc_stack.ss_sp = &g_stacks[l * STACK];
    emu::lanes[l].uc_stack.ss_size = STACK;
    emu::lanes[l].uc_link = nullptr;
    makecontext(&emu::lanes[l], (void (*)())lane_entry, 1, l);
  }
  for (;;) {
    for (int l = 0; l < emu::W; l++) {
      emu::cur = l;
      swapcontext(&emu::sched, &emu::lanes[l]);
    }
    int nd = 0;
    for (int l = 0; l < emu::W; l++) nd += emu::done[l];
    if (nd == emu::W) return true;
    if (nd) return false;  // some lanes returned while others wait at an intrinsic
    const unsigned p = (emu::phase[0] - 1) & 1;
    for (int l = 1; l < emu::W; l++)
      if (emu::phase[l] != emu::phase[0] || emu::kind[p][l] != emu::kind[p][0]) return false;
  }
}
}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) {
    std::fprintf(stderr, "usage: %s <64|32> <grammar>\n", argv[0]);
    return 2;
  }
  const bool f32 = std::atoi(argv[1]) == 32;
  const uint32_t grammar = (uint32_t)std::atoi(argv[2]);
  std::string text;
  char buf[1 << 16];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), stdin)) > 0) text.append(buf, got);
  // the buffer 16-byte aligned with padding, as device memory would be read
  // (whole aligned 16-byte granules)
  std::vector<uint8_t> mem(text.size() + 64);
  uint8_t* base = mem.data() + ((16 - (reinterpret_cast<uintptr_t>(mem.data()) & 15)) & 15) + 16;
  std::memcpy(base, text.data(), text.size());
  static fp::WarpSmem sm;
  size_t p = 0;
  while (p < text.size()) {
    g_job.f = base + p;
    g_job.lim = text.size() - p;
    g_job.grammar = grammar;
    g_job.f32 = f32;
    g_job.sm = &sm;
    if (!run_field()) {
      std::printf("DIVERGED at byte %zu\n", p);
      return 1;
    }
    const fp::LongResult& r = g_job.r[0];
    if (r.error) {
      std::printf("ERROR at byte %zu\n", p);
      return 1;
    }
    std::printf("%016llx %u\n", (unsigned long long)r.bits, (unsigned)r.status);
    size_t q = text.find('\n', p);
    p = q == std::string::npos ? text.size() : q + 1;
  }
  return 0;
}
