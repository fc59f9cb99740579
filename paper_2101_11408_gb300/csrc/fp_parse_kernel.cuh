// fp_parse_kernel.cuh -- fused field index + parse + Algorithm 1 (persistent).
//
// One launch covers every chunk of every buffer of a call.  Each block is
// persistent: it takes chunk tickets in increasing order from a device
// counter, so a chunk only ever waits on chunks that are already owned by
// running blocks (deadlock-free look-back).  Per chunk:
//
//   1. stage  : the chunk's text plus a 16-byte pad before it and a 64-byte
//               margin after it is copied into shared memory by the bulk-copy
//               (TMA) engine, two chunks ahead of the one being parsed (three
//               buffers);
//   2. index  : one iteration ahead of its parse, separators are found four
//               bytes per 32-bit word with exact SWAR zero-byte tests; a
//               block scan ranks the field starts, whose positions are
//               scattered in order into one of two lists (a chunk of more
//               than 1024 fields is listed window by window at its parse);
//               the chunk's field count is published at once for the
//               decoupled look-back;
//   3. parse  : one thread per field, warps taking groups of 32 fields from a
//               shared counter: the window tokenizer for the common
//               shape, else the general tokenizer of Section 4; quick exits
//               and Algorithm 1 against the table held in shared memory; the
//               w / w+1 check of Section 11; results are staged in shared
//               memory;
//   4. prefix : one warp looks back over the preceding chunks for this
//               chunk's first field index (the 32 nearest first, then wider
//               rounds) while the others parse, then joins them;
//   5. store  : coalesced stores of the doubles and status bytes; fields that
//               cannot be settled here are queued for the fallback kernel.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "fp_device.cuh"
#include "fp_sync.cuh"
#include "fp_types.cuh"

namespace fp {

// Kernel modes beside the format (compile-time, so that the default mode
// carries none of their instructions): MODE_JSON checks the JSON number
// grammar on the fast path's fields; MODE_COLUMNS stores field i at column
// i mod K, row i div K, and flags fields whose terminator disagrees with
// their column; MODE_HEX (the decimal-or-hexadecimal grammar) sends fields
// with an "0x" to the hexadecimal window tokenizer.
constexpr int MODE_JSON = 1;
constexpr int MODE_COLUMNS = 2;
constexpr int MODE_HEX = 4;

constexpr int NT = 256;       // threads per block
constexpr int PAD = 16;       // bytes staged before the chunk (holds the byte at c0-1)
constexpr int MARGIN = LMAX;  // bytes staged after the chunk
constexpr int NSTAGE = 3;     // tile buffers: one being parsed, two being fetched
constexpr int STAGE = 1024;   // results held in shared memory until the prefix is known

template <int C>
struct Layout {
  static constexpr int TILE = PAD + C + MARGIN;  // staged bytes
  static constexpr int TILE_ALLOC = (TILE + 16 + 127) / 128 * 128;  // + over-read slack
  static constexpr int SEG_PER_THREAD = C / 16 / NT;  // 16-byte granules per thread
  static constexpr int S_CAP = STAGE;  // field starts listed at a time (denser chunks: windows)
  static constexpr int TABLE_BYTES = FP_POW5_ENTRIES * 8;  // high words only
  static constexpr int OFF_TABLE = 0;
  static constexpr int OFF_WTAB = (TABLE_BYTES + 127) / 128 * 128;  // the window tokenizer's tables
  static constexpr int OFF_TILE = (OFF_WTAB + (int)sizeof(WindowTables) + 127) / 128 * 128;
  static constexpr int OFF_S = OFF_TILE + NSTAGE * TILE_ALLOC;
  static constexpr int S_BYTES = ((S_CAP + 2) * 2 + 15) / 16 * 16;  // one list of field starts
  static constexpr int S_STRIDE = S_BYTES / 2;                       // in uint16 entries
  static constexpr int OFF_STAGE_BITS = OFF_S + 2 * S_BYTES;         // two lists
  static constexpr int OFF_STAGE_ST = OFF_STAGE_BITS + STAGE * 8;
  static constexpr int OFF_MISC = OFF_STAGE_ST + STAGE;
  static constexpr int MISC_BYTES = 1024;
  static constexpr int TOTAL = OFF_MISC + MISC_BYTES;
  static_assert(C % (16 * NT) == 0, "whole granules per thread");
  static_assert(TILE < 65536, "u16 positions");
  static_assert(S_CAP == STAGE, "one window of fields is staged at a time");
  static_assert(S_CAP <= 32 * 32, "a window's groups of 32 fields fit a 32-bit mask");
};

// Miscellaneous shared state of a block.
struct Misc {
  uint64_t bar[NSTAGE];
  BufDesc desc[NSTAGE];              // descriptor of the chunk staged in each buffer
  unsigned long long chunk[NSTAGE];  // global chunk staged in each buffer (or >= total)
  unsigned int desc_index[NSTAGE];
  unsigned int warp_sum[NT / 32];
  unsigned int overflowed;  // a pending field of this chunk did not fit the queue
  unsigned long long lb_part[NT / 32];
  int last_start[NSTAGE];  // tile offset of the last field start of each staged chunk
  unsigned long long cnt[CNT_NUM];
  unsigned int group[2];  // next group of 32 fields to parse, per list of field starts
};
static_assert(sizeof(Misc) <= 1024, "misc");

__device__ __forceinline__ unsigned long long lb_word(unsigned int epoch, unsigned long long flag,
                                                      unsigned long long value) {
  return ((unsigned long long)epoch << 40) | (flag << LB_VALUE_BITS) | (value & LB_VALUE_MASK);
}

__device__ __forceinline__ void set_error(Ctl* ctl, unsigned int code) {
  atomicCAS(&ctl->error, 0u, code);
}

// Find the descriptor of global chunk g (descriptors sorted by chunk0).
__device__ __forceinline__ unsigned int find_desc(const LaunchParams& p, unsigned long long g) {
  if (p.nbuf == 1) return 0;
  unsigned int lo = 0, hi = p.nbuf - 1;
  while (lo < hi) {
    unsigned int mid = (lo + hi + 1) >> 1;
    if (p.descs[mid].chunk0 <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Thread 0: stage chunk g (descriptor d) into a tile buffer.
template <int C>
__device__ __forceinline__ void issue_stage(uint8_t* tile, uint64_t* bar, const BufDesc& d,
                                            unsigned long long g) {
  const long long lc = (long long)(g - d.chunk0);
  const long long c0 = lc * C;
  const long long t0 = c0 - PAD;  // aligned coordinate of tile byte 0
  const long long a_end = (long long)((d.o + d.len + 15) & ~15ull);
  long long s = t0 < 0 ? 0 : t0;
  long long e = c0 + C + MARGIN;
  if (e > a_end) e = a_end;
  if (e > s) {
    const uint32_t bytes = (uint32_t)(e - s);
    fence_proxy_async_smem();  // the buffer was last read by generic loads
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(tile + (s - t0), d.base + s, bytes, bar);
  } else {
    mbar_arrive(bar);
  }
}

// Decoupled look-back for chunk g, by one warp: its first field index is the
// sum of the field counts of the chunks [first, g) of its buffer, where
// either `first` is the buffer's first chunk and `known` is 0, or first-1 is
// a chunk whose inclusive prefix `known` this block already has (its own
// previous chunk).  Chunks publish their counts (aggregates) as soon as they
// are counted, one iteration before they are parsed, and their inclusive
// prefixes once known; the warp reads PER entries per lane per round, newest
// first, and stops at the nearest inclusive prefix.  Each wait is bounded.
// One round of PER*32 entries: returns the sum of the entries up to and
// including the nearest inclusive one (or of all of them when there is none)
// to every lane, and whether one was found.
template <int PER>
__device__ __forceinline__ unsigned long long lookback_round(const LaunchParams& p, long long top,
                                                             long long first, int lane,
                                                             bool& found) {
  // Entry at distance 32u + lane from top is this lane's u-th: the newest 32
  // (the ones most likely not yet published) are on 32 lanes, waited for in
  // parallel.
  unsigned long long wv[PER];
#pragma unroll
  for (int u = 0; u < PER; u++) {
    const long long idx = top - (lane + 32 * u);
    wv[u] = idx >= first ? ld_relaxed_u64(&p.chunk_status[idx]) : lb_word(p.epoch, LB_FLAG_AGG, 0);
  }
  unsigned int nearest = 0xFFFFFFFFu;  // distance of this lane's nearest inclusive entry
#pragma unroll
  for (int u = 0; u < PER; u++) {
    const long long idx = top - (lane + 32 * u);
    if ((unsigned int)(wv[u] >> 40) != p.epoch || ((wv[u] >> LB_VALUE_BITS) & 3) == 0) {
      const uint64_t ts = globaltimer_ns();
      const uint64_t limit = p.wait_ns ? p.wait_ns : WAIT_NS_DEFAULT;
      do {
        __nanosleep(64);
        wv[u] = ld_relaxed_u64(&p.chunk_status[idx]);
        if (globaltimer_ns() - ts > limit) {
          set_error(p.ctl, DERR_TIMEOUT);
          wv[u] = lb_word(p.epoch, LB_FLAG_INC, 0);
          break;
        }
      } while ((unsigned int)(wv[u] >> 40) != p.epoch || ((wv[u] >> LB_VALUE_BITS) & 3) == 0);
    }
    if (nearest == 0xFFFFFFFFu && ((wv[u] >> LB_VALUE_BITS) & 3) == LB_FLAG_INC)
      nearest = (unsigned int)(lane + 32 * u);
  }
  // the sum of the entries up to and including the nearest inclusive one
  const unsigned int stop = __reduce_min_sync(0xFFFFFFFFu, nearest);
  unsigned long long part = 0;
#pragma unroll
  for (int u = 0; u < PER; u++)
    if ((unsigned int)(lane + 32 * u) <= stop) part += wv[u] & LB_VALUE_MASK;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, off);
  found = stop != 0xFFFFFFFFu;
  return part;
}

// Rounds of 32*LB_PER_LANE entries, newest first, all of a round's loads
// issued at once.  One block takes one ticket per iteration, so this block's
// own previous chunk, whose inclusive prefix it knows, is about one grid of
// chunks back: the first round reaches it whether or not the chunks in
// between have published inclusive prefixes yet (a chain of those would make
// the look-back as slow as its slowest link).  Every lane returns the prefix.
constexpr int LB_PER_LANE = 16;
__device__ __forceinline__ unsigned long long warp_lookback(const LaunchParams& p, long long g,
                                                            long long first,
                                                            unsigned long long known, int lane) {
  long long top = g - 1;
  unsigned long long prefix = 0;
  while (top >= first) {
    bool found = false;
    prefix += lookback_round<LB_PER_LANE>(p, top, first, lane, found);
    if (found) return prefix;
    top -= 32 * LB_PER_LANE;
  }
  return prefix + known;
}

__device__ __forceinline__ bool is_sep_byte(uint32_t c, uint32_t delim) {
  return c == '\n' || c == delim;
}

template <int C, class F, int MODE>
__global__ void __launch_bounds__(NT, (C >= 16384 ? 3 : 4)) parse_kernel(const LaunchParams p) {
  using L = Layout<C>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* table = reinterpret_cast<uint64_t*>(smem + L::OFF_TABLE);
  WindowTables* wtab = reinterpret_cast<WindowTables*>(smem + L::OFF_WTAB);
  uint8_t* tiles = smem + L::OFF_TILE;
  uint16_t* S = reinterpret_cast<uint16_t*>(smem + L::OFF_S);
  Misc* ms = reinterpret_cast<Misc*>(smem + L::OFF_MISC);
  unsigned long long* stage_bits = reinterpret_cast<unsigned long long*>(smem + L::OFF_STAGE_BITS);
  uint8_t* stage_st = smem + L::OFF_STAGE_ST;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  Ctl* ctl = p.ctl;
  const uint32_t delim = p.delim & 0xFFu;

  // the fallback kernel launched after this one may be set up now (it waits
  // on the device for this grid to finish); every block of this persistent
  // grid is resident by the time all of them have executed this
  grid_launch_dependents();
  // This launch is itself a programmatic dependent of the kernel before it
  // on the stream (usually the previous call's fallback kernel, which
  // releases it as it starts): its blocks are set up while that kernel
  // runs and wait here until it has completed and its writes are visible.
  // Nothing is read or written before this point.
  grid_dependency_wait();
  if (tid == 0) {
    for (int b = 0; b < NSTAGE; b++) mbar_init(&ms->bar[b], 1);
    fence_mbar_init();
    for (int i = 0; i < CNT_NUM; i++) ms->cnt[i] = 0;
    ms->overflowed = 0;
    // tickets for all but one buffer; the loop keeps them that far ahead
    for (int b = 0; b < NSTAGE - 1; b++) {
      const unsigned long long g = atomicAdd(&ctl->ticket, 1ull);
      ms->chunk[b] = g;
      if (g < p.total_chunks) {
        const unsigned int di = find_desc(p, g);
        ms->desc_index[b] = di;
        ms->desc[b] = p.nbuf == 1 ? p.one : p.descs[di];
        issue_stage<C>(tiles + b * L::TILE_ALLOC, &ms->bar[b], ms->desc[b], g);
      }
    }
  }
  // The high words of the power-of-five table, once per block (Appendix
  // table; 5,208 bytes); the low words, needed only for a second product,
  // are read from global memory.
  for (int i = tid; i < FP_POW5_ENTRIES; i += NT) table[i] = fp_pow5_table_dev[2 * i];
  for (int i = tid; i < WINDOW_TABLE_WORDS; i += NT)
    reinterpret_cast<uint32_t*>(wtab)[i] = window_table_word(i);
  const Pow5 pow5{table, 1, reinterpret_cast<const uint64_t*>(fp_pow5_table_dev) + 1};
  __syncthreads();

  // Path counters: the second products of this thread's fields in a
  // register (added up once, at the end); the rare paths count in shared
  // memory; fields settled by the window tokenizer and Algorithm 1 at once
  // are the block's fields less those that needed anything else.
  uint32_t c_two = 0;
  auto flush_counters = [&]() {
    const uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, c_two);
    if (lane == 0 && tot) atomicAdd(&ms->cnt[CNT_TWO_MUL], (unsigned long long)tot);
    c_two = 0;
  };
  uint32_t phases = 0;  // bit b: parity of buffer b's next phase
  const uint32_t NLW = 0x0A0A0A0Au;
  const uint32_t DLW = delim * 0x01010101u;
  const bool one_sep = (delim == '\n');
  const bool dl_ascii = delim < 0x80u;  // the two-separator test's shortcut needs bit 7 clear

  // Wait until buffer b's bytes have landed (bounded).
  auto wait_buf = [&](int b) {
    const uint32_t par = (phases >> b) & 1u;
    if (!mbar_try_wait(&ms->bar[b], par)) {
      const uint64_t t_start = globaltimer_ns();
      const uint64_t limit = p.wait_ns ? p.wait_ns : WAIT_NS_DEFAULT;
      while (!mbar_try_wait(&ms->bar[b], par)) {
        if (globaltimer_ns() - t_start > limit) {
          set_error(ctl, DERR_TIMEOUT);
          break;
        }
      }
    }
    phases ^= 1u << b;
  };

  // ---- 2. index ----------------------------------------------------------
  // Count the fields that start in the chunk staged in buffer b and publish
  // the count for the look-back.  A field starts at x in [o, endx) if x == o
  // or byte x-1 is a separator; the chunk owns the starts in [c0, c1), i.e.
  // the boundaries b = x-1 in [c0-1, c1-1).  Thread t scans the granules of
  // bytes [c0 + 16*K*t, c0 + 16*K*(t+1)); thread 0 also decides b = c0-1.
  // The per-word boundary flags and the thread's rank stay in registers for
  // the iteration that parses the chunk.
  using MaskT = typename std::conditional<(L::SEG_PER_THREAD > 2), unsigned long long, uint32_t>::type;
  struct Counted {
    MaskT mask;  // bit i: a field starts at byte i+1 of this thread's granules
    uint32_t pad_bit, rank0, n;
  };
  // When the chunk fits one window, the field starts are listed into Sx
  // right away (and Sx[n] = one past the last field's terminator), and
  // group counter gs is reset: the chunk's parse, an iteration later, then
  // needs no barrier of its own.
  auto count_chunk = [&](int b, Counted& cn, uint16_t* Sx, int gs) {
    const uint8_t* tile = tiles + b * L::TILE_ALLOC;
    const BufDesc& d = ms->desc[b];
    const unsigned long long g = ms->chunk[b];
    const long long lc = (long long)(g - d.chunk0);
    const long long c0 = lc * C;
    const long long o = (long long)d.o;
    const long long endx = o + (long long)d.len;
    uint32_t cnt = 0;
    cn.pad_bit = 0;
    if (tid == 0) {
      const long long bb = c0 - 1;
      bool isb;
      if (bb == o - 1) isb = true;
      else if (bb < o || bb >= endx - 1) isb = false;
      else isb = is_sep_byte(tile[PAD - 1], delim);
      cn.pad_bit = isb && (bb + 1 < endx);
      cnt = cn.pad_bit;
    }
    MaskT mask = 0;
    // one loop per separator test (the choice is block-uniform), so that no
    // word pays for the tests it does not use
    auto scan_granules = [&](auto flags) {
#pragma unroll
      for (int k = 0; k < L::SEG_PER_THREAD; k++) {
        const int j = tid * L::SEG_PER_THREAD + k;  // granule within the chunk
        const uint4 v = *reinterpret_cast<const uint4*>(tile + PAD + 16 * j);
        // one bit per byte position
        const uint32_t m16 = flag_pair(flags(v.x), flags(v.y), flag_pair(flags(v.z), flags(v.w)) << 8) >> 7;
        mask |= (MaskT)m16 << (16 * k);
      }
    };
    if (one_sep)
      scan_granules([&](uint32_t w) { return sep_flags_one(w, NLW); });
    else if (dl_ascii)
      scan_granules([&](uint32_t w) { return sep_flags_two(w, NLW, DLW); });
    else
      scan_granules([&](uint32_t w) { return sep_flags_one(w, NLW) | zero_bytes(w ^ DLW); });
    {
      // A boundary at byte b is a field start iff o <= b < endx - 1, plus
      // the virtual boundary o - 1 (the buffer's first field, when it has
      // one); the chunk's last byte is the next chunk's.  Interior threads
      // (all but the chunk's last and those at a buffer's edges) keep every
      // separator.
      constexpr int NB = 16 * L::SEG_PER_THREAD;  // bytes (mask bits) per thread
      const long long x0t = c0 + NB * tid;
      if (x0t < o || x0t + NB > endx - 1 || tid == NT - 1) {
        const long long lo = o - x0t, hi = endx - 1 - x0t;  // valid bit range [lo, hi)
        const int lo_c = lo < 0 ? 0 : (lo > NB ? NB : (int)lo);
        const int hi_c = hi < 0 ? 0 : (hi > NB ? NB : (int)hi);
        MaskT valid = 0;
        if (hi_c > lo_c) {
          const MaskT ones = ~(MaskT)0;
          valid = (ones << lo_c) & (hi_c >= (int)(8 * sizeof(MaskT)) ? ones : ~(ones << hi_c));
        }
        mask &= valid;
        const long long vb = o - 1 - x0t;
        if (vb >= 0 && vb < NB && o < endx) mask |= (MaskT)1 << vb;
        if (tid == NT - 1) mask &= ~((MaskT)1 << (NB - 1));
      }
    }
    cn.mask = mask;
    cnt += (sizeof(MaskT) == 8) ? __popcll((unsigned long long)mask) : __popc((uint32_t)mask);
    // block exclusive scan of the per-thread counts
    uint32_t incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
      if (lane >= off) incl += t;
    }
    if (lane == 31) ms->warp_sum[warp] = incl;
    __syncthreads();
    // the warps' totals: lane l holds warp l's (l < 8); the block's total and
    // this warp's exclusive prefix are two warp reductions
    const uint32_t wsum = lane < NT / 32 ? ms->warp_sum[lane] : 0u;
    const uint32_t n = __reduce_add_sync(0xFFFFFFFFu, wsum);
    const uint32_t wpre = __reduce_add_sync(0xFFFFFFFFu, lane < warp ? wsum : 0u);
    cn.n = n;
    cn.rank0 = wpre + incl - cnt;
    // publish at once so that later chunks can look past this one; the
    // first chunk of a buffer already knows its prefix
    if (tid == 0)
      st_relaxed_u64(&p.chunk_status[g], lb_word(p.epoch, lc == 0 ? LB_FLAG_INC : LB_FLAG_AGG, n));
    // the thread holding the chunk's last field start records it, for the
    // scan that finds where that field ends
    int last = -1;
    if (cnt && wpre + incl == n) {
      const int hb = mask ? (int)(8 * sizeof(MaskT)) - 1 -
                                ((sizeof(MaskT) == 8) ? __clzll((long long)mask) : __clz((uint32_t)mask))
                          : -1;
      last = hb >= 0 ? PAD + 16 * tid * L::SEG_PER_THREAD + hb + 1 : PAD;
      ms->last_start[b] = last;
    }
    if (n <= (uint32_t)L::S_CAP) {
      uint32_t rank = cn.rank0;
      if (cn.pad_bit) Sx[rank++] = PAD;
      const int base_off = PAD + 16 * tid * L::SEG_PER_THREAD + 1;
      // the set bits in order, 32 at a time (32-bit bit scans)
#pragma unroll
      for (int h = 0; h < (int)sizeof(MaskT) / 4; h++) {
        uint32_t m = (uint32_t)(mask >> (32 * h));
        while (m) {
          Sx[rank++] = (uint16_t)(base_off + 32 * h + __ffs(m) - 1);
          m &= m - 1;
        }
      }
      if (last >= 0) {
        // the last field ends at the first separator after its start, at the
        // end of the text, or (if neither is staged) it is long
        const long long vend = endx - (c0 - PAD);
        const int lim = vend < L::TILE ? (int)vend : L::TILE;
        int term = last + 128;
        const int w0 = last & ~3;
        for (int wb = w0; wb < w0 + 128; wb += 4) {
          const uint32_t wv = *reinterpret_cast<const uint32_t*>(tile + wb);
          uint32_t f = one_sep ? zero_bytes(wv ^ NLW) : (zero_bytes(wv ^ NLW) | zero_bytes(wv ^ DLW));
          if (wb == w0) f &= 0xFFFFFFFFu << (8 * (last & 3));
          if (f) {
            term = wb + (ctz32(f) >> 3);
            break;
          }
        }
        if (term > lim) term = lim;
        Sx[n] = (uint16_t)(term + 1);
      }
      if (tid == 0) ms->group[gs] = 0;
    }
    // (warp_sum is next written after at least one more barrier)
  };

  Counted cur, nxt;
  int buf = 0;
  int sset = 0;  // list of field starts of the current chunk
  // this block's previous chunk and the inclusive prefix after it
  long long prev_g = -1;
  unsigned long long prev_inc = 0;
  if (ms->chunk[0] < p.total_chunks) {
    wait_buf(0);
    count_chunk(0, cur, S, 0);
  }
  __syncthreads();

  while (true) {
    const unsigned long long g = ms->chunk[buf];
    if (g >= p.total_chunks) break;
    uint8_t* tile = tiles + buf * L::TILE_ALLOC;
    const int b1 = (buf + 1) % NSTAGE, b2 = (buf + 2) % NSTAGE;
    // Thread 0 takes the ticket of a further chunk now; the atomic's round
    // trip overlaps with the count below, and its bytes are requested after.
    unsigned long long gn = 0;
    if (tid == 0) gn = atomicAdd(&ctl->ticket, 1ull);
    // Count the next chunk now, one iteration before parsing it, so that its
    // field count is public long before any later chunk looks back at it.
    if (ms->chunk[b1] < p.total_chunks) {
      wait_buf(b1);
      count_chunk(b1, nxt, S + (sset ^ 1) * L::S_STRIDE, sset ^ 1);
    }
    if (tid == 0) {
      // stage the ticketed chunk into the buffer that the previous iteration
      // parsed (freed by the barrier that ended it)
      ms->chunk[b2] = gn;
      if (gn < p.total_chunks) {
        const unsigned int di = find_desc(p, gn);
        ms->desc_index[b2] = di;
        ms->desc[b2] = p.nbuf == 1 ? p.one : p.descs[di];
        issue_stage<C>(tiles + b2 * L::TILE_ALLOC, &ms->bar[b2], ms->desc[b2], gn);
      }
    }

    const BufDesc d = ms->desc[buf];
    const unsigned int dix = ms->desc_index[buf];
    const long long lc = (long long)(g - d.chunk0);
    const long long c0 = lc * C;
    const long long t0 = c0 - PAD;
    const long long o = (long long)d.o;
    const long long endx = o + (long long)d.len;  // one past the last text byte
    // tile offsets: bytes at or beyond `limit` are not text (or not staged)
    const long long vend = endx - t0;
    const int limit = vend < L::TILE ? (int)vend : L::TILE;
    const uint32_t n = cur.n;

    // The hot path for one field [s, e): the window tokenizer and
    // Algorithm 1.  Fields it cannot settle are marked for the general
    // tokenizer, which runs in a separate pass so that this loop stays free
    // of rare branches.
    auto parse_hot = [&](int s, int e, unsigned long long& bits, uint8_t& status) {
      if constexpr ((MODE & MODE_HEX) != 0) {
        // a hexadecimal float (Appendix C): its own window tokenizer, whose
        // value needs no Algorithm 1 (the digits give the bits)
        const uint32_t c0 = tile[s];
        const int s1 = s + ((c0 == '-') | (c0 == '+'));
        if ((tile[s1 + 1] | 0x20u) == 'x') {
          uint64_t hbits = 0;
          uint8_t hst = ST_GENERAL;
          if (!parse_hex_window<F>(tile, *wtab, s, e, hbits, hst)) hst = ST_GENERAL;
          bits = hbits;
          status = hst;
          return;
        }
      }
      FastToken ft;
      ft.w = 0;
      ft.q = 0;
      ft.sign = 0;
      bool ok = parse_window(tile, *wtab, s, e, ft);
      if constexpr ((MODE & MODE_JSON) != 0) ok = ok && json_ok_fast(tile, s, ft);
      const ElResult r = convert_wq<F>(ft.w ? ft.w : 1ull, ok ? ft.q : 0, pow5, true);
      c_two += ok & (uint32_t)r.two_mul;
      uint64_t sgn = ft.sign;  // the binary64 sign bit
      if constexpr (F::MBITS != F64::MBITS) sgn = ft.sign ? F::SIGN : 0;
      bits = ft.w ? (r.bits | sgn) : sgn;
      status = !ok ? (uint8_t)ST_GENERAL : (ft.w ? r.status : (uint8_t)ST_OK);
    };
    // The rest: the general tokenizer on the field's exact extent, else the
    // fallback kernel (pending, with the field's location as the value).
    auto parse_general = [&](int s, int e, unsigned long long& bits, uint8_t& status) {
      atomicAdd(&ms->cnt[CNT_NOT_FAST], 1ull);
      if (e - s <= LMAX) {
        atomicAdd(&ms->cnt[CNT_SLOW], 1ull);
        const FieldResult r = parse_short_field<F>(tile + s, e - s, pow5, p.grammar);
        c_two += r.two_mul;
        if (r.is_long) atomicAdd(&ms->cnt[CNT_LONG], 1ull);
        if (r.long_settled) atomicAdd(&ms->cnt[CNT_LONG_SETTLED], 1ull);
        if (r.status != ST_PENDING) {
          bits = r.bits;
          status = r.status;
          return;
        }
      }
      bits = ((unsigned long long)dix << LOC_OFF_BITS) | (unsigned long long)(t0 + s - o);
      status = ST_PENDING;
    };

    // Where the look-back starts: after this block's previous chunk when
    // that chunk belongs to the same buffer, else at the buffer's start.
    const bool same_buf = prev_g >= (long long)d.chunk0;
    const long long lb_first = same_buf ? prev_g + 1 : (long long)d.chunk0;
    const unsigned long long lb_known = same_buf ? prev_inc : 0ull;

    unsigned long long base = 0, cap = 0;
    typename F::word* ob = nullptr;
    uint8_t* os = nullptr;
    // Field k of the chunk (its terminator at tile offset tpos) to the
    // outputs, for the lanes with `act`; every lane of the warp calls it
    // together (the queue append is one atomic per warp).  In field order the
    // field's slot is k; in column-major order it is column i mod K, row
    // i div K of the field's index i.
    auto store_one = [&](bool act, uint32_t k, unsigned long long bits, uint8_t status, int tpos) {
      const bool live = act && k < cap;
      typename F::word* vo = ob + k;
      uint8_t* so = os + k;
      if constexpr ((MODE & MODE_COLUMNS) != 0) {
        if (live) {
          const unsigned long long i = d.out_base + base + k;
          const unsigned long long row = __umul64hi(i, p.col_magic);
          const unsigned long long col = i - row * p.columns;
          // the last column ends at '\n' (or the end of the text), the others
          // at the delimiter
          const bool nl = tpos >= limit || tile[tpos] == '\n';
          if (status != ST_PENDING && nl != (col == p.columns - 1)) status = ST_BAD_SHAPE;
          const unsigned long long dest = col * p.rows_cap + row;
          vo = reinterpret_cast<typename F::word*>(p.out_bits) + dest;
          so = p.out_status + dest;
        }
      }
      const bool pend = live && status == ST_PENDING;
      constexpr bool in_slot = sizeof(typename F::word) == 8 && (MODE & MODE_COLUMNS) == 0;
      if (live) {
        if constexpr (in_slot) {
          *vo = bits;  // a pending field's location stays in its own slot
        } else {
          if (pend) p.loc[d.out_base + base + k] = bits;
          else *vo = (typename F::word)bits;
        }
        if (!pend) *so = status;
      }
      // pending fields: one queue append per warp (Section 11's rare slow path)
      const unsigned int pm = __ballot_sync(0xFFFFFFFFu, pend);
      if (pm) {
        const int leader = __ffs(pm) - 1;
        unsigned long long slot0 = 0;
        if (lane == leader) slot0 = atomicAdd(&ctl->qcount, (unsigned long long)__popc(pm));
        slot0 = __shfl_sync(0xFFFFFFFFu, slot0, leader);
        if (pend) {
          const unsigned long long slot = slot0 + __popc(pm & ((1u << lane) - 1u));
          if (slot < p.qcap) {
            p.queue[slot] = d.out_base + base + k;
            *so = ST_PENDING_QUEUED;
          } else {
            *so = ST_PENDING_SCAN;
            ms->overflowed = 1;
          }
        }
      }
    };

    // The chunk's list of field starts: listed when the chunk was counted if
    // it fits one window (visible since the barrier that ended the previous
    // iteration), else window by window below.
    uint16_t* Sw = S + sset * L::S_STRIDE;
    const bool one_window = n <= (uint32_t)L::S_CAP;
    for (uint32_t lo = 0;; lo += L::S_CAP) {
      const uint32_t hi = min(lo + (uint32_t)L::S_CAP, n);
      if (!one_window) {
        // list the starts of fields lo..hi (hi included: it ends field hi-1)
        uint32_t rank = cur.rank0;
        const int base_off = PAD + 16 * tid * L::SEG_PER_THREAD + 1;
        MaskT m = cur.mask;
        if (cur.pad_bit) {
          if (rank >= lo && rank <= hi) Sw[rank - lo] = PAD;
          rank++;
        }
        while (m) {
          const int bpos = (sizeof(MaskT) == 8) ? __ffsll((long long)m) - 1 : __ffs((uint32_t)m) - 1;
          if (rank >= lo && rank <= hi) Sw[rank - lo] = (uint16_t)(base_off + bpos);
          rank++;
          m &= m - 1;
        }
        if (tid == 0) ms->group[sset] = 0;
        if (hi == n && n > lo && warp == 0) {
          // the last field ends at the first separator after its start, at the
          // end of the text, or (if neither is staged) it is long
          const int st = ms->last_start[buf];
          const int wb = (st & ~3) + 4 * lane;
          const uint32_t wv = *reinterpret_cast<const uint32_t*>(tile + wb);
          uint32_t f = one_sep ? zero_bytes(wv ^ NLW) : (zero_bytes(wv ^ NLW) | zero_bytes(wv ^ DLW));
          if (lane == 0) f &= 0xFFFFFFFFu << (8 * (st & 3));
          const unsigned int hit = __ballot_sync(0xFFFFFFFFu, f != 0);
          int term = st + 128;
          if (hit) {
            const int l = __ffs(hit) - 1;
            const uint32_t fl = __shfl_sync(0xFFFFFFFFu, f, l);
            term = (st & ~3) + 4 * l + (ctz32(fl) >> 3);
          }
          if (term > limit) term = limit;
          if (lane == 0) Sw[n - lo] = (uint16_t)(term + 1);
        }
        __syncthreads();  // S ready
      }
      if (lo == 0 && warp == 0) {
        // the prefix, while the other warps parse; published at once
        const unsigned long long b =
            lc == 0 ? 0ull : warp_lookback(p, (long long)g, lb_first, lb_known, lane);
        if (lane == 0) {
          ms->lb_part[0] = b;
          if (lc != 0) st_relaxed_u64(&p.chunk_status[g], lb_word(p.epoch, LB_FLAG_INC, b + n));
          if (lc + 1 == (long long)d.nchunks && d.out_count) *d.out_count = b + n;
        }
      }
      // Warps take groups of 32 fields until none is left, so that the warp
      // that ran the look-back, or one that met general fields, does less.
      // The general tokenizer then runs on the fields of the warp's own
      // groups that need it, in a second pass (the hot loop stays free of
      // its rare branches).
      const uint32_t cntw = hi - lo;
      const uint32_t ngroups = (cntw + 31) / 32;  // at most S_CAP / 32 = 32
      uint32_t general = 0;  // this warp's groups with a field for the general tokenizer
      // each group's ticket is taken before the group ahead of it is parsed,
      // so the atomic's round trip overlaps that parse
      uint32_t gnext = 0;
      if (lane == 0) gnext = atomicAdd(&ms->group[sset], 1u);
      for (;;) {
        const uint32_t gi = __shfl_sync(0xFFFFFFFFu, gnext, 0);
        if (gi >= ngroups) break;
        if (lane == 0) gnext = atomicAdd(&ms->group[sset], 1u);
        const uint32_t k = 32 * gi + lane;
        uint8_t status = ST_OK;
        if (k < cntw) {
          unsigned long long bits;
          parse_hot(Sw[k], Sw[k + 1] - 1, bits, status);
          stage_bits[k] = bits;
          stage_st[k] = status;
        }
        if (__any_sync(0xFFFFFFFFu, status == ST_GENERAL)) general |= 1u << gi;
      }
      while (general) {
        const uint32_t k = 32 * (__ffs(general) - 1) + lane;
        general &= general - 1;
        if (k < cntw && stage_st[k] == ST_GENERAL)
          parse_general(Sw[k], Sw[k + 1] - 1, stage_bits[k], stage_st[k]);
      }
      // stores: each warp a contiguous, equal share of the window
      const uint32_t share = (cntw + NT / 32 - 1) / (NT / 32);
      const uint32_t k_end = min(warp * share + share, cntw);
      __syncthreads();  // the prefix and the results are in shared memory
      if (lo == 0) {
        base = ms->lb_part[0];
        cap = d.out_cap > base ? d.out_cap - base : 0;
        ob = reinterpret_cast<typename F::word*>(p.out_bits) + d.out_base + base;
        os = p.out_status + d.out_base + base;
      }
      for (uint32_t k0 = warp * share; k0 < k_end; k0 += 32) {  // warp-uniform trip count
        const uint32_t k = k0 + lane;
        const bool act = k < k_end;
        store_one(act, lo + k, act ? stage_bits[k] : 0ull, act ? stage_st[k] : (uint8_t)ST_OK,
                  act ? (int)Sw[k + 1] - 1 : 0);
      }
      if (hi >= n) break;
      __syncthreads();  // S and the staged results are rewritten for the next window
    }
    if (tid == 0) ms->cnt[CNT_FIELDS] += n;
    __syncthreads();
    if (tid == 0 && ms->overflowed) {
      // The fallback kernel will scan this chunk's outputs for pending fields.
      const unsigned long long slot = atomicAdd(&ctl->ovf_count, 1ull);
      if (slot < p.ovf_cap) {
        // (descriptor << 40 | fields of the chunk that were stored, first output index)
        const unsigned long long stored = n < cap ? n : cap;
        p.ovf[2 * slot] = ((unsigned long long)dix << LOC_OFF_BITS) | stored;
        p.ovf[2 * slot + 1] = d.out_base + base;
      } else {
        set_error(ctl, DERR_INTERNAL);
      }
      ms->overflowed = 0;
    }
    prev_g = (long long)g;
    prev_inc = base + n;
    cur = nxt;
    buf = b1;
    sset ^= 1;
  }

  // ---- counters and end-of-launch reset ---------------------------------
  {
    flush_counters();
  }
  __syncthreads();
  if (tid == 0) {
    ms->cnt[CNT_EL] = ms->cnt[CNT_FIELDS] - ms->cnt[CNT_NOT_FAST];
    for (int i = 0; i < CNT_NUM; i++)
      if (ms->cnt[i]) atomicAdd(&ctl->stats[i], ms->cnt[i]);
    __threadfence();
    const unsigned int prev = atomicAdd(&ctl->done_parse, 1u);
    if (prev == gridDim.x - 1) {
      // every block has taken its last ticket: reset for the next call
      ctl->ticket = 0;
      ctl->done_parse = 0;
      __threadfence();
    }
  }
}

}  // namespace fp
