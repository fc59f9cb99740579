// fp_parse_kernel.cu -- fused field index + parse + Algorithm 1 (persistent).
//
// One launch covers every chunk of every buffer of a call.  Each block is
// persistent: it takes chunk tickets in increasing order from a device
// counter, so a chunk only ever waits on chunks that are already owned by
// running blocks (deadlock-free look-back).  Per chunk:
//
//   1. stage  : the chunk's text plus a 16-byte pad before it and a 64-byte
//               margin after it is copied into shared memory by the bulk-copy
//               (TMA) engine, double buffered with the previous chunk's work;
//   2. index  : separators are found 16 bytes per thread with 32-bit SWAR
//               tests; a block scan ranks them and scatters their positions;
//               the number of fields that start in the chunk is published for
//               the decoupled look-back, which yields the chunk's first field
//               index;
//   3. parse  : one thread per field: tokenizer (Section 4), quick exits,
//               Algorithm 1 against the table held in shared memory, the
//               w / w+1 check for long significands (Section 10);
//   4. store  : coalesced stores of the double and the status byte; fields
//               that cannot be settled here are queued for the fallback kernel.
#include <cuda_runtime.h>

#include "fp_device.cuh"
#include "fp_sync.cuh"
#include "fp_types.cuh"

namespace fp {

constexpr int NT = 256;  // threads per block
constexpr int PAD = 16;  // bytes staged before the chunk (holds the byte at c0-1)
constexpr int MARGIN = LMAX;  // bytes staged after the chunk

template <int C>
struct Layout {
  static constexpr int TILE = PAD + C + MARGIN;            // staged bytes
  static constexpr int TILE_ALLOC = (TILE + 127) / 128 * 128;
  static constexpr int NSEG = TILE / 16;
  static constexpr int SEG_PER_THREAD = (NSEG + NT - 1) / NT;
  static constexpr int TABLE_BYTES = 2 * FP_POW5_ENTRIES * 8;
  static constexpr int OFF_TABLE = 0;
  static constexpr int OFF_TILE = (TABLE_BYTES + 127) / 128 * 128;
  static constexpr int OFF_S = OFF_TILE + 2 * TILE_ALLOC;
  static constexpr int S_BYTES = ((TILE + 2) * 2 + 15) / 16 * 16;
  static constexpr int OFF_MISC = OFF_S + S_BYTES;
  static constexpr int MISC_BYTES = 1024;
  static constexpr int TOTAL = OFF_MISC + MISC_BYTES;
  static_assert(TILE % 16 == 0, "tile must be whole granules");
  static_assert(TILE < 65536, "u16 positions");
};

// Miscellaneous shared state of a block.
struct Misc {
  uint64_t bar[2];
  BufDesc desc[2];            // descriptor of the chunk staged in each buffer
  unsigned long long chunk[2];  // global chunk staged in each buffer (or >= total)
  unsigned long long base;    // first field index of the current chunk
  unsigned int desc_index[2];
  unsigned int warp_sum[NT / 32];
  unsigned int nb, n;         // boundaries staged, fields owned
  unsigned int overflowed;    // a pending field of this chunk did not fit the queue
  unsigned int pad;
  unsigned long long cnt[CNT_NUM];
};
static_assert(sizeof(Misc) <= 1024, "misc");

// 0x80 in every byte of t that is zero, exactly (no false positives).
__device__ __forceinline__ uint32_t zero_bytes(uint32_t t) {
  return ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u;
}
// Gather the high bit of each byte into 4 bits (byte k -> bit k).
__device__ __forceinline__ uint32_t gather4(uint32_t hb) {
  return (((hb >> 7) * 0x00204081u) >> 21) & 0xFu;
}

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

// Thread 0: stage chunk g (descriptor d) into tile buffer `buf`.
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

template <int C>
__global__ void __launch_bounds__(NT) parse_kernel(const LaunchParams p) {
  using L = Layout<C>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* table = reinterpret_cast<uint64_t*>(smem + L::OFF_TABLE);
  uint8_t* tiles = smem + L::OFF_TILE;
  uint16_t* S = reinterpret_cast<uint16_t*>(smem + L::OFF_S);
  Misc* ms = reinterpret_cast<Misc*>(smem + L::OFF_MISC);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  Ctl* ctl = p.ctl;

  if (tid == 0) {
    mbar_init(&ms->bar[0], 1);
    mbar_init(&ms->bar[1], 1);
    fence_mbar_init();
    for (int i = 0; i < CNT_NUM; i++) ms->cnt[i] = 0;
    ms->overflowed = 0;
    unsigned long long g = atomicAdd(&ctl->ticket, 1ull);
    ms->chunk[0] = g;
    if (g < p.total_chunks) {
      unsigned int di = find_desc(p, g);
      ms->desc_index[0] = di;
      ms->desc[0] = p.nbuf == 1 ? p.one : p.descs[di];
      issue_stage<C>(tiles, &ms->bar[0], ms->desc[0], g);
    }
  }
  // The power-of-five table, once per block (Appendix table; 10,416 bytes).
  {
    const uint4* src = reinterpret_cast<const uint4*>(fp_pow5_table_dev);
    uint4* dst = reinterpret_cast<uint4*>(table);
    for (int i = tid; i < FP_POW5_ENTRIES; i += NT) dst[i] = src[i];
  }
  __syncthreads();

  unsigned long long c_fields = 0, c_one = 0, c_two = 0, c_long = 0, c_long_ok = 0;
  uint32_t phase0 = 0, phase1 = 0;
  int buf = 0;
  const uint32_t NLW = 0x0A0A0A0Au;
  const uint32_t DLW = (p.delim & 0xFFu) * 0x01010101u;

  while (true) {
    const unsigned long long g = ms->chunk[buf];
    if (g >= p.total_chunks) break;
    uint8_t* tile = tiles + buf * L::TILE_ALLOC;
    // Hand out the next chunk and start staging it into the other buffer
    // (freed by the barrier that ended the previous iteration).
    if (tid == 0) {
      unsigned long long gn = atomicAdd(&ctl->ticket, 1ull);
      ms->chunk[buf ^ 1] = gn;
      if (gn < p.total_chunks) {
        unsigned int di = find_desc(p, gn);
        ms->desc_index[buf ^ 1] = di;
        ms->desc[buf ^ 1] = p.nbuf == 1 ? p.one : p.descs[di];
        issue_stage<C>(tiles + (buf ^ 1) * L::TILE_ALLOC, &ms->bar[buf ^ 1], ms->desc[buf ^ 1], gn);
      }
    }
    // Wait for this chunk's bytes (bounded).
    {
      const uint32_t par = buf ? phase1 : phase0;
      if (!mbar_try_wait(&ms->bar[buf], par)) {
        const uint64_t t_start = globaltimer_ns();
        while (!mbar_try_wait(&ms->bar[buf], par)) {
          if (globaltimer_ns() - t_start > 2000000000ull) {
            set_error(ctl, DERR_TIMEOUT);
            break;
          }
        }
      }
      if (buf) phase1 ^= 1; else phase0 ^= 1;
    }
    const BufDesc d = ms->desc[buf];
    const unsigned int dix = ms->desc_index[buf];
    const long long lc = (long long)(g - d.chunk0);
    const long long c0 = lc * C;
    const long long t0 = c0 - PAD;
    const long long o = (long long)d.o;
    const long long endx = o + (long long)d.len;  // one past the last text byte
    // owned boundaries: positions b with c0-1 <= b < lim
    const long long lim = (c0 + C - 1 < endx - 1) ? c0 + C - 1 : endx - 1;

    // ---- 2. index -------------------------------------------------------
    uint32_t bm[L::SEG_PER_THREAD];
    uint32_t cnt_b = 0, cnt_o = 0;
#pragma unroll
    for (int k = 0; k < L::SEG_PER_THREAD; k++) {
      const int j = tid * L::SEG_PER_THREAD + k;
      uint32_t m = 0, om = 0;
      if (j < L::NSEG) {
        const uint4 v = *reinterpret_cast<const uint4*>(tile + 16 * j);
        m = gather4(zero_bytes(v.x ^ NLW) | zero_bytes(v.x ^ DLW)) |
            (gather4(zero_bytes(v.y ^ NLW) | zero_bytes(v.y ^ DLW)) << 4) |
            (gather4(zero_bytes(v.z ^ NLW) | zero_bytes(v.z ^ DLW)) << 8) |
            (gather4(zero_bytes(v.w ^ NLW) | zero_bytes(v.w ^ DLW)) << 12);
        const long long x0 = t0 + 16 * j;
        const long long lo_in = o - x0, hi_in = endx - x0;
        if (lo_in > 0 || hi_in < 16) {
          // edge of the buffer: keep real separators inside [o, endx) and
          // add the virtual boundaries at o-1 and endx
          uint32_t in = 0;
          for (int b = 0; b < 16; b++) in |= (uint32_t)(b >= lo_in && b < hi_in) << b;
          m &= in;
          if (lo_in - 1 >= 0 && lo_in - 1 < 16) m |= 1u << (lo_in - 1);
          if (hi_in >= 0 && hi_in < 16) m |= 1u << hi_in;
        }
        // the pad granule only contributes the boundary at c0-1: earlier ones
        // close fields of the previous chunk and must not enter the list
        if (j == 0) m &= 0x8000u;
        const long long ol = (c0 - 1) - x0, oh = lim - x0;
        uint32_t own;
        if (ol <= 0 && oh >= 16) {
          own = 0xFFFFu;
        } else {
          own = 0;
          for (int b = 0; b < 16; b++) own |= (uint32_t)(b >= ol && b < oh) << b;
        }
        om = m & own;
      }
      bm[k] = m;
      cnt_b += __popc(m);
      cnt_o += __popc(om);
    }
    // Block exclusive scan of (cnt_b, cnt_o) packed in one word.
    uint32_t packed = cnt_b | (cnt_o << 16);
    uint32_t incl = packed;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
      if (lane >= off) incl += t;
    }
    if (lane == 31) ms->warp_sum[warp] = incl;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
#pragma unroll
    for (int w2 = 0; w2 < NT / 32; w2++) {
      uint32_t v = ms->warp_sum[w2];
      wpre += (w2 < warp) ? v : 0;
      tot += v;
    }
    uint32_t rank = (wpre + incl - packed) & 0xFFFFu;
#pragma unroll
    for (int k = 0; k < L::SEG_PER_THREAD; k++) {
      uint32_t m = bm[k];
      const int j = tid * L::SEG_PER_THREAD + k;
      while (m) {
        const int b = __ffs(m) - 1;
        S[rank++] = (uint16_t)(16 * j + b);
        m &= m - 1;
      }
    }
    const uint32_t nb = tot & 0xFFFFu;
    const uint32_t n = tot >> 16;

    // ---- decoupled look-back: first field index of this chunk -----------
    if (warp == 0) {
      unsigned long long prefix = 0;
      if (lc == 0) {
        if (lane == 0) st_release_u64(&p.chunk_status[g], lb_word(p.epoch, LB_FLAG_INC, n));
      } else {
        if (lane == 0) st_release_u64(&p.chunk_status[g], lb_word(p.epoch, LB_FLAG_AGG, n));
        long long pos = (long long)g - 1;
        const long long first = (long long)d.chunk0;
        bool done = false;
        while (!done) {
          const long long idx = pos - lane;
          unsigned long long wv = 0;
          unsigned long long flag = 0, val = 0;
          if (idx >= first) {
            wv = ld_acquire_u64(&p.chunk_status[idx]);
            if ((unsigned int)(wv >> 40) != p.epoch || ((wv >> LB_VALUE_BITS) & 3) == 0) {
              const uint64_t ts = globaltimer_ns();
              do {
                __nanosleep(64);
                wv = ld_acquire_u64(&p.chunk_status[idx]);
                if (globaltimer_ns() - ts > 2000000000ull) {
                  set_error(ctl, DERR_TIMEOUT);
                  wv = lb_word(p.epoch, LB_FLAG_INC, 0);
                  break;
                }
              } while ((unsigned int)(wv >> 40) != p.epoch || ((wv >> LB_VALUE_BITS) & 3) == 0);
            }
            flag = (wv >> LB_VALUE_BITS) & 3;
            val = wv & LB_VALUE_MASK;
          }
          const unsigned int inc = __ballot_sync(0xFFFFFFFFu, idx >= first && flag == LB_FLAG_INC);
          unsigned long long take;
          if (inc) {
            const int stop = __ffs(inc) - 1;  // nearest inclusive prefix
            take = lane <= stop ? val : 0;
            done = true;
          } else {
            take = val;  // all aggregates (lanes beyond the buffer give 0)
            pos -= 32;
            if (pos < first) done = true;  // cannot happen: chunk `first` is inclusive
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) take += __shfl_xor_sync(0xFFFFFFFFu, take, off);
          prefix += take;
        }
        if (lane == 0) st_release_u64(&p.chunk_status[g], lb_word(p.epoch, LB_FLAG_INC, prefix + n));
      }
      if (lane == 0) {
        ms->base = prefix;
        ms->nb = nb;
        ms->n = n;
        if (lc + 1 == (long long)d.nchunks && d.out_count) *d.out_count = prefix + n;
      }
    }
    __syncthreads();
    const unsigned long long base = ms->base;

    // ---- 3./4. parse and store -----------------------------------------
    for (uint32_t k = tid; k < n; k += NT) {
      const int s = S[k] + 1;  // tile offset of the field's first byte
      const unsigned long long fi = base + k;
      const unsigned long long oi = d.out_base + fi;
      FieldResult r;
      bool pending = true;
      c_fields++;
      if (k + 1 < nb) {
        const int e = S[k + 1];
        if (e - s <= LMAX) {
          r = parse_short_field(tile + s, e - s, table);
          pending = (r.status == ST_PENDING);
          c_one += !r.two_mul;
          c_two += r.two_mul;
          c_long += r.is_long;
          c_long_ok += r.long_settled;
        }
      }
      if (fi < d.out_cap) {
        if (pending) {
          const unsigned long long off = (unsigned long long)(t0 + s - o);
          p.out_bits[oi] = ((unsigned long long)dix << LOC_OFF_BITS) | off;
          const unsigned long long slot = atomicAdd(&ctl->qcount, 1ull);
          if (slot < p.qcap) {
            p.queue[slot] = oi;
            p.out_status[oi] = ST_PENDING_QUEUED;
          } else {
            p.out_status[oi] = ST_PENDING_SCAN;
            ms->overflowed = 1;
          }
        } else {
          p.out_bits[oi] = r.bits;
          p.out_status[oi] = r.status;
        }
      }
    }
    __syncthreads();
    if (tid == 0 && ms->overflowed) {
      // The fallback kernel will scan this chunk's outputs for pending fields.
      const unsigned long long slot = atomicAdd(&ctl->ovf_count, 1ull);
      if (slot < p.ovf_cap) {
        // (descriptor << 40 | fields of the chunk that were stored, first output index)
        const unsigned long long stored =
            base + n <= d.out_cap ? n : (d.out_cap > base ? d.out_cap - base : 0);
        p.ovf[2 * slot] = ((unsigned long long)dix << LOC_OFF_BITS) | stored;
        p.ovf[2 * slot + 1] = d.out_base + base;
      } else {
        set_error(ctl, DERR_INTERNAL);
      }
      ms->overflowed = 0;
    }
    buf ^= 1;
  }

  // ---- counters and end-of-launch reset ---------------------------------
  {
    unsigned long long v[5] = {c_fields, c_one, c_two, c_long, c_long_ok};
#pragma unroll
    for (int i = 0; i < 5; i++) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xFFFFFFFFu, v[i], off);
    }
    if (lane == 0) {
      atomicAdd(&ms->cnt[CNT_FIELDS], v[0]);
      atomicAdd(&ms->cnt[CNT_ONE_MUL], v[1]);
      atomicAdd(&ms->cnt[CNT_TWO_MUL], v[2]);
      atomicAdd(&ms->cnt[CNT_LONG], v[3]);
      atomicAdd(&ms->cnt[CNT_LONG_SETTLED], v[4]);
    }
  }
  __syncthreads();
  if (tid == 0) {
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

template __global__ void parse_kernel<4096>(const LaunchParams);
template __global__ void parse_kernel<8192>(const LaunchParams);
template __global__ void parse_kernel<16384>(const LaunchParams);

// Host-side launch helper (same translation unit as the kernels).
cudaError_t launch_parse(const LaunchParams& p, int chunk_bytes, int grid, cudaStream_t stream) {
  switch (chunk_bytes) {
    case 4096: {
      auto k = parse_kernel<4096>;
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Layout<4096>::TOTAL);
      k<<<grid, NT, Layout<4096>::TOTAL, stream>>>(p);
      break;
    }
    case 8192: {
      auto k = parse_kernel<8192>;
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Layout<8192>::TOTAL);
      k<<<grid, NT, Layout<8192>::TOTAL, stream>>>(p);
      break;
    }
    case 16384: {
      auto k = parse_kernel<16384>;
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Layout<16384>::TOTAL);
      k<<<grid, NT, Layout<16384>::TOTAL, stream>>>(p);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int parse_smem_bytes(int chunk_bytes) {
  switch (chunk_bytes) {
    case 4096: return Layout<4096>::TOTAL;
    case 8192: return Layout<8192>::TOTAL;
    case 16384: return Layout<16384>::TOTAL;
    default: return -1;
  }
}

cudaError_t parse_occupancy(int chunk_bytes, int* blocks_per_sm) {
  switch (chunk_bytes) {
    case 4096:
      cudaFuncSetAttribute(parse_kernel<4096>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           Layout<4096>::TOTAL);
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, parse_kernel<4096>, NT,
                                                           Layout<4096>::TOTAL);
    case 8192:
      cudaFuncSetAttribute(parse_kernel<8192>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           Layout<8192>::TOTAL);
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, parse_kernel<8192>, NT,
                                                           Layout<8192>::TOTAL);
    case 16384:
      cudaFuncSetAttribute(parse_kernel<16384>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           Layout<16384>::TOTAL);
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, parse_kernel<16384>, NT,
                                                           Layout<16384>::TOTAL);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace fp
