// parse_block_emu.cpp -- the parse kernel (fp_parse_kernel.cuh, as it is)
// run on the host as 1 to 4 blocks of 256 emulated threads: each thread is a
// coroutine (POSIX ucontext), and the scheduler releases a warp once its 32
// lanes wait at the same warp intrinsic (values posted, double-buffered by
// phase), and a block once all its threads wait at __syncthreads.  The
// kernel's PTX helpers are replaced by host_sync_stub.h (bulk copies
// complete when issued) and its dynamic shared memory by one buffer per
// block.  Blocks take chunk tickets in turn, so a chunk's look-back reads
// other blocks' words.  The text is placed at a chosen offset modulo 16.
//
// usage: parse_block_emu <64|32> <grammar 0|1|2> <chunk bytes> <offset 0..15> [blocks
//        [columns rows_cap]] < text   (grammar 1 runs the hexadecimal mode, 2 the
//        JSON mode; columns K >= 2 the column-major mode, '\n' rows of K
//        ','-separated fields)
// One line per field: "<bits hex> <status>" as stored (pending fields keep
// their location word and a pending status), then "count <n>".
#include <ucontext.h>

#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#define __device__
#define __global__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))
#define __launch_bounds__(...)
#define __align__(n)
#define __shared__

struct emu_dim {
  unsigned int x, y, z;
};
struct uint4 {
  unsigned int x, y, z, w;
};

namespace emu {
constexpr int BT = 256, MAXB = 4, NT = BT * MAXB, NW = NT / 32;
int nthreads = BT, nblocks = 1;
// SPIN: a lane in a bounded wait (it slept); it runs again once no other
// thread can, so that the other blocks publish what it waits for
enum State { RUN, WAIT_WARP, WAIT_BLOCK, DONE, SPIN };
ucontext_t sched, th[NT];
int cur = 0;
State st[NT];
int wkind[NT];
unsigned wphase[NT];
uint64_t slot[NW][2][32];
bool failed = false;
const char* why = "";

void yield() { swapcontext(&th[cur], &sched); }
const uint64_t* post(uint64_t v, int kind) {
  const int me = cur, w = me / 32, l = me % 32;
  const unsigned p = wphase[me] & 1;
  slot[w][p][l] = v;
  wkind[me] = kind;
  wphase[me]++;
  st[me] = WAIT_WARP;
  yield();
  return slot[w][p];
}
}  // namespace emu

inline emu_dim emu_tid() { return emu_dim{(unsigned)(emu::cur % emu::BT), 0, 0}; }
inline emu_dim emu_bid() { return emu_dim{(unsigned)(emu::cur / emu::BT), 0, 0}; }
#define threadIdx (emu_tid())
#define blockIdx (emu_bid())
#define gridDim (emu_dim{(unsigned)emu::nblocks, 1, 1})

enum { K_BALLOT = 1, K_ANY, K_ALL, K_SHFL, K_UP, K_XOR, K_RADD, K_RMIN, K_SYNC };
template <class T>
uint64_t to_u(T v) {
  uint64_t u = 0;
  std::memcpy(&u, &v, sizeof(T));
  return u;
}
template <class T>
T from_u(uint64_t u) {
  T r;
  std::memcpy(&r, &u, sizeof(T));
  return r;
}
unsigned int __ballot_sync(unsigned int, int pred) {
  const uint64_t* s = emu::post(pred ? 1 : 0, K_BALLOT);
  unsigned int m = 0;
  for (int i = 0; i < 32; i++) m |= (unsigned int)(s[i] & 1) << i;
  return m;
}
int __all_sync(unsigned int, int pred) {
  const uint64_t* s = emu::post(pred ? 1 : 0, K_ALL);
  for (int i = 0; i < 32; i++)
    if (!s[i]) return 0;
  return 1;
}
int __any_sync(unsigned int, int pred) {
  const uint64_t* s = emu::post(pred ? 1 : 0, K_ANY);
  for (int i = 0; i < 32; i++)
    if (s[i]) return 1;
  return 0;
}
template <class T>
T __shfl_sync(unsigned int, T v, int src) {
  return from_u<T>(emu::post(to_u(v), K_SHFL)[src & 31]);
}
template <class T>
T __shfl_up_sync(unsigned int, T v, unsigned int d) {
  const uint64_t* s = emu::post(to_u(v), K_UP);
  const int l = emu::cur % 32;
  return from_u<T>(s[l >= (int)d ? l - (int)d : l]);
}
template <class T>
T __shfl_xor_sync(unsigned int, T v, int m) {
  return from_u<T>(emu::post(to_u(v), K_XOR)[((emu::cur % 32) ^ m) & 31]);
}
unsigned int __reduce_add_sync(unsigned int, unsigned int v) {
  const uint64_t* s = emu::post(v, K_RADD);
  unsigned int t = 0;
  for (int i = 0; i < 32; i++) t += (unsigned int)s[i];
  return t;
}
unsigned int __reduce_min_sync(unsigned int, unsigned int v) {
  const uint64_t* s = emu::post(v, K_RMIN);
  unsigned int t = 0xFFFFFFFFu;
  for (int i = 0; i < 32; i++) t = (unsigned int)s[i] < t ? (unsigned int)s[i] : t;
  return t;
}
void __syncwarp(unsigned int = 0xFFFFFFFFu) { emu::post(0, K_SYNC); }
void __syncthreads() {
  emu::st[emu::cur] = emu::WAIT_BLOCK;
  emu::yield();
}
void __nanosleep(unsigned int) {  // let the others run first
  emu::st[emu::cur] = emu::SPIN;
  emu::yield();
}
void __threadfence() {}
int __popc(unsigned int x) { return __builtin_popcount(x); }
int __popcll(unsigned long long x) { return __builtin_popcountll(x); }
int __ffs(int x) { return __builtin_ffs(x); }
int __ffsll(long long x) { return __builtin_ffsll(x); }
int __clz(int x) { return x ? __builtin_clz((unsigned)x) : 32; }
int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
unsigned long long __umul64hi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
template <class T, class U>
T atomicAdd(T* p, U v) {  // the emulated threads run one at a time
  const T old = *p;
  *p = (T)(old + (T)v);
  return old;
}
template <class T, class U>
T atomicCAS(T* p, U cmp, U val) {
  const T old = *p;
  if (old == (T)cmp) *p = (T)val;
  return old;
}

// CUDA's global min / max (by value, in the operands' common type)
template <class A, class B>
typename std::common_type<A, B>::type min(A a, B b) {
  return a < b ? a : b;
}
template <class A, class B>
typename std::common_type<A, B>::type max(A a, B b) {
  return a < b ? b : a;
}

#include "fp_device.cuh"
namespace fp {
const unsigned long long fp_pow5_table_dev[2 * FP_POW5_ENTRIES] = {FP_POW5_TABLE_VALUES};
}  // namespace fp
// each block's dynamic shared memory (the kernel header's copy takes it from here)
alignas(128) uint8_t emu_smem_all[emu::MAXB][96 * 1024];
inline uint8_t* emu_block_smem() { return emu_smem_all[emu::cur / emu::BT]; }
#include "fp_parse_kernel_host.cuh"  // the kernel header: CUDA runtime include removed, smem per block

namespace {
fp::LaunchParams g_p;
int g_f32 = 0, g_chunk = 16384, g_mode = 0;

template <int C, class F>
void body() {
  switch (g_mode) {
    case fp::MODE_JSON: fp::parse_kernel<C, F, fp::MODE_JSON>(g_p); break;
    case fp::MODE_COLUMNS: fp::parse_kernel<C, F, fp::MODE_COLUMNS>(g_p); break;
    case fp::MODE_HEX: fp::parse_kernel<C, F, fp::MODE_HEX>(g_p); break;
    case fp::MODE_HEX | fp::MODE_COLUMNS: fp::parse_kernel<C, F, fp::MODE_HEX | fp::MODE_COLUMNS>(g_p); break;
    default: fp::parse_kernel<C, F, 0>(g_p); break;
  }
}
void thread_entry(int t) {
  (void)t;
  switch (g_chunk * 2 + g_f32) {
    case 4096 * 2: body<4096, fp::F64>(); break;
    case 4096 * 2 + 1: body<4096, fp::F32>(); break;
    case 16384 * 2: body<16384, fp::F64>(); break;
    case 16384 * 2 + 1: body<16384, fp::F32>(); break;
    default: break;
  }
  emu::st[emu::cur] = emu::DONE;
  emu::yield();
}

#ifndef EMU_LIMIT_S
#define EMU_LIMIT_S 120
#endif
constexpr size_t STACK = 64 << 10;

bool run_block() {
  static std::vector<char> stacks(emu::NT * STACK);
  const int NTH = emu::nthreads;
  for (int t = 0; t < NTH; t++) {
    emu::st[t] = emu::RUN;
    emu::wphase[t] = 0;
    getcontext(&emu::th[t]);
    emu::th[t].uc_stack.ss_sp = &stacks[t * STACK];
    emu::th[t].uc_stack.ss_size = STACK;
    emu::th[t].uc_link = nullptr;
    makecontext(&emu::th[t], (void (*)())thread_entry, 1, t);
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    bool ran = false;
    for (int t = 0; t < NTH; t++) {
      if (emu::st[t] != emu::RUN) continue;
      emu::cur = t;
      swapcontext(&emu::sched, &emu::th[t]);
      ran = true;
    }
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(EMU_LIMIT_S)) {
      int n[5] = {0, 0, 0, 0, 0};
      for (int t = 0; t < NTH; t++) n[emu::st[t]]++;
      std::fprintf(stderr, "states: run %d warp %d block %d done %d spin %d; running warps:", n[0],
                   n[1], n[2], n[3], n[4]);
      for (int t = 0; t < NTH; t += 32)
        if (emu::st[t] == emu::RUN) std::fprintf(stderr, " %d", t / 32);
      std::fprintf(stderr, "\n");
      for (int w = 0; w < NTH / 32; w++)
        std::fprintf(stderr, "warp %d: phase %u kind %d\n", w, emu::wphase[32 * w],
                     emu::wkind[32 * w]);
      emu::why = "no progress within the time limit";
      return false;
    }
    if (ran) continue;
    bool released = false;
    for (int w = 0; w < NTH / 32; w++) {
      int waiting = 0;
      for (int l = 0; l < 32; l++) waiting += emu::st[32 * w + l] == emu::WAIT_WARP;
      if (waiting == 0) continue;
      if (waiting != 32) continue;  // the rest of the warp is elsewhere: not yet
      for (int l = 1; l < 32; l++)
        if (emu::wphase[32 * w + l] != emu::wphase[32 * w] ||
            emu::wkind[32 * w + l] != emu::wkind[32 * w]) {
          emu::why = "warp lanes at different intrinsics";
          return false;
        }
      for (int l = 0; l < 32; l++) emu::st[32 * w + l] = emu::RUN;
      released = true;
    }
    if (released) continue;
    int nd_all = 0;
    for (int b = 0; b < emu::nblocks; b++) {
      int nb = 0, nd = 0;
      for (int t = b * emu::BT; t < (b + 1) * emu::BT; t++) {
        nb += emu::st[t] == emu::WAIT_BLOCK;
        nd += emu::st[t] == emu::DONE;
      }
      nd_all += nd;
      if (nb == emu::BT) {  // the whole block at __syncthreads
        for (int t = b * emu::BT; t < (b + 1) * emu::BT; t++) emu::st[t] = emu::RUN;
        released = true;
      } else if (nb && nd) {
        emu::why = "a barrier after some of the block's threads returned";
        return false;
      }
    }
    if (released) continue;
    if (nd_all == NTH) return true;
    bool spinning = false;
    for (int t = 0; t < NTH; t++)
      if (emu::st[t] == emu::SPIN) {
        emu::st[t] = emu::RUN;
        spinning = true;
      }
    if (spinning) continue;  // (a wait that nothing ends runs out on the timer)
    emu::why = "deadlock";
    return false;
  }
}
}  // namespace

int main(int argc, char** argv) {
  if (argc != 5 && argc != 6 && argc != 8) {
    std::fprintf(stderr, "usage: %s <64|32> <grammar> <chunk> <offset> [blocks]\n", argv[0]);
    return 2;
  }
  emu::nblocks = argc >= 6 ? std::atoi(argv[5]) : 1;
  const unsigned long long columns = argc == 8 ? std::strtoull(argv[6], nullptr, 10) : 0;
  const unsigned long long rows_cap = argc == 8 ? std::strtoull(argv[7], nullptr, 10) : 0;
  if (emu::nblocks < 1 || emu::nblocks > emu::MAXB) return 2;
  emu::nthreads = emu::nblocks * emu::BT;
  g_f32 = std::atoi(argv[1]) == 32;
  const uint32_t grammar = (uint32_t)std::atoi(argv[2]);
  g_chunk = std::atoi(argv[3]);
  const int offset = std::atoi(argv[4]) & 15;
  std::string text;
  char buf[1 << 16];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), stdin)) > 0) text.append(buf, got);
  const size_t len = text.size();
  g_mode = columns ? fp::MODE_COLUMNS : (grammar == fp::GRAMMAR_JSON ? fp::MODE_JSON : 0);
  if (grammar == fp::GRAMMAR_HEX) g_mode |= fp::MODE_HEX;
  const size_t cap = columns ? columns * rows_cap : len;
  // the text at `offset` modulo 16, with digits around it (never used)
  std::vector<uint8_t> mem(len + 256, '7');
  uint8_t* a16 = mem.data() + ((16 - (reinterpret_cast<uintptr_t>(mem.data()) & 15)) & 15) + 64;
  uint8_t* tp = a16 + offset;
  std::memcpy(tp, text.data(), len);
  const unsigned long long o = reinterpret_cast<uintptr_t>(tp) & 15;
  unsigned long long nch = (o + len + g_chunk - 1) / g_chunk;
  if (nch == 0) nch = 1;
  std::vector<unsigned long long> out(cap + 1, 0x5A5A5A5A5A5A5A5Aull), loc(len + 1, 0),
      chunk_status(nch, 0), queue(1 << 20), ovf(2 * nch);
  std::vector<uint8_t> status(cap + 1, 0xEE);
  static fp::Ctl ctl;
  std::memset(&ctl, 0, sizeof(ctl));
  unsigned long long count = ~0ull;
  fp::LaunchParams& p = g_p;
  std::memset(&p, 0, sizeof(p));
  p.one.base = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(tp) & ~(uintptr_t)15);
  p.one.o = o;
  p.one.len = len;
  p.one.chunk0 = 0;
  p.one.nchunks = nch;
  p.one.out_base = 0;
  p.one.out_cap = columns ? columns * rows_cap : len;  // as fp_parse_ex sets it
  p.one.out_count = &count;
  p.nbuf = 1;
  p.delim = columns ? ',' : '\n';
  p.total_chunks = nch;
  p.out_bits = out.data();
  p.out_status = status.data();
  p.ctl = &ctl;
  p.chunk_status = chunk_status.data();
  p.epoch = 1;
  p.queue = queue.data();
  p.qcap = queue.size();
  p.ovf = ovf.data();
  p.ovf_cap = nch;
  p.loc = g_f32 ? loc.data() : p.out_bits;
  p.grammar = grammar;
  if (columns) {
    p.columns = (unsigned int)columns;
    p.rows_cap = rows_cap;
    p.col_magic = (unsigned long long)((((unsigned __int128)1 << 64) + columns - 1) / columns);
    p.loc = loc.data();  // pending locations beside the column-major results
  }
  if (!run_block()) {
    std::printf("EMULATION %s\n", emu::why);
    return 1;
  }
  if (ctl.error) {
    std::printf("DEVICE ERROR %u\n", ctl.error);
    return 1;
  }
  for (unsigned long long i = 0; i < count && i < len; i++) {
    // field i's slot: i, or column i mod K, row i div K
    const unsigned long long k = columns ? (i % columns) * rows_cap + i / columns : i;
    const unsigned long long b =
        g_f32 ? (unsigned long long)reinterpret_cast<const uint32_t*>(out.data())[k] : out[k];
    std::printf("%016llx %u\n", b, (unsigned)status[k]);
  }
  std::printf("count %llu\n", count);
  return 0;
}
