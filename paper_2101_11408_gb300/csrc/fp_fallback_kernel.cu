// fp_fallback_kernel.cu -- exact resolution of the fields the parse kernel
// could not settle (Section 11 "higher-precision approach"; the design here
// is this library's own: a big-number comparison against midpoints).
//
// A field arrives here when it is longer than the parse kernel's limit, when
// Algorithm 1 gave up (second product word all ones outside [-27, 55]), or
// when its 19-digit truncation w and w+1 round differently (Section 11).
//
// Method, per field (one thread per field, limbs in shared memory):
//   1. tokenize the whole field from global memory (Section 4 grammar);
//   2. D = its first 800 significant digits, with one extra digit 1 appended
//      when any later digit is nonzero.  Every midpoint between adjacent
//      doubles has at most 768 significant digits (Section 11), so D 10^E and
//      the exact value lie on the same side of every midpoint;
//   3. candidate x = the rounded truncated product of the 19-digit prefix
//      (within one unit of the answer);
//   4. compare D 10^E exactly with the midpoint between x and its neighbour
//      above, and below, as integers scaled by powers of two and five; step
//      x up or down until it is the nearest double; a tie picks the even one.
#include <cuda_runtime.h>

#include "fp_device.cuh"
#include "fp_sync.cuh"
#include "fp_types.cuh"

namespace fp {

constexpr int FB_NT = 64;     // threads per block
constexpr int LIMBS = 88;     // 32-bit limbs per big number (2816 bits)
constexpr int KMAX = 800;     // significant digits kept before the sticky digit
constexpr long long EXP_SAT = 1000000000000000ll;  // explicit exponent saturation


// A big natural: limb i at p[i * FB_NT] (threads interleaved, no bank conflicts).
struct Big {
  uint32_t* p;
  int n;
  __device__ uint32_t& at(int i) const { return p[i * FB_NT]; }
};

__device__ __forceinline__ bool big_mul_add(Big& a, uint32_t m, uint32_t c) {
  uint64_t carry = c;
  for (int i = 0; i < a.n; i++) {
    uint64_t t = (uint64_t)a.at(i) * m + carry;
    a.at(i) = (uint32_t)t;
    carry = t >> 32;
  }
  if (carry) {
    if (a.n >= LIMBS) return false;
    a.at(a.n++) = (uint32_t)carry;
  }
  return true;
}

__device__ __forceinline__ bool big_mul_pow5(Big& a, long long k) {
  const uint32_t P13 = 1220703125u;  // 5^13
  while (k >= 13) {
    if (!big_mul_add(a, P13, 0)) return false;
    k -= 13;
  }
  uint32_t m = 1;
  while (k-- > 0) m *= 5;
  return m == 1 || big_mul_add(a, m, 0);
}

__device__ __forceinline__ long long big_bitlen(const Big& a) {
  if (a.n == 0) return 0;
  return 32ll * (a.n - 1) + (32 - __clz(a.at(a.n - 1)));
}

// dst = src * t (t < 2^64).
__device__ __forceinline__ bool big_mul_u64(Big& dst, const Big& src, uint64_t t) {
  const uint32_t tl = (uint32_t)t, th = (uint32_t)(t >> 32);
  if (src.n + 2 > LIMBS) return false;
  uint64_t carry = 0;
  for (int i = 0; i < src.n; i++) {
    uint64_t v = (uint64_t)src.at(i) * tl + carry;
    dst.at(i) = (uint32_t)v;
    carry = v >> 32;
  }
  dst.at(src.n) = (uint32_t)carry;
  dst.n = src.n + 1;
  if (th) {
    carry = 0;
    for (int i = 0; i < src.n; i++) {
      uint64_t v = (uint64_t)src.at(i) * th + dst.at(i + 1) + carry;
      dst.at(i + 1) = (uint32_t)v;
      carry = v >> 32;
    }
    dst.at(src.n + 1) = (uint32_t)carry;
    dst.n = src.n + 2;
  }
  while (dst.n && dst.at(dst.n - 1) == 0) dst.n--;
  return true;
}

__device__ __forceinline__ uint32_t limb_or0(const Big& a, long long i) {
  return (i >= 0 && i < a.n) ? a.at((int)i) : 0u;
}

// Compare X * 2^s with Y, given bitlen(X) + s == bitlen(Y) and s >= 0.
__device__ __forceinline__ int cmp_shifted(const Big& X, long long s, const Big& Y) {
  const long long ws = s >> 5;
  const int bs = (int)(s & 31);
  for (int i = Y.n - 1; i >= 0; i--) {
    uint32_t xi = limb_or0(X, i - ws) << bs;
    if (bs) xi |= limb_or0(X, i - ws - 1) >> (32 - bs);
    const uint32_t yi = Y.at(i);
    if (xi != yi) return xi < yi ? -1 : 1;
  }
  return 0;
}

// Sign of X * 2^sx - Y * 2^sy for nonzero X, Y.
__device__ __forceinline__ int cmp_scaled(const Big& X, long long sx, const Big& Y, long long sy) {
  const long long lx = big_bitlen(X) + sx, ly = big_bitlen(Y) + sy;
  if (lx != ly) return lx < ly ? -1 : 1;
  const long long d = sx - sy;
  if (d >= 0) return cmp_shifted(X, d, Y);
  return -cmp_shifted(Y, -d, X);
}

// M, e with value = M 2^e for a finite non-negative bit pattern of F.
template <class F>
__device__ __forceinline__ void float_parts(uint64_t x, uint64_t& M, int& e) {
  const uint64_t ef = x >> F::MBITS, fr = x & ((1ull << F::MBITS) - 1);
  if (ef == 0) {
    M = fr;
    e = 1 - F::BIAS - F::MBITS;  // the smallest subnormal's exponent
  } else {
    M = fr | (1ull << F::MBITS);
    e = (int)ef - F::BIAS - F::MBITS;
  }
}

struct LongResult {
  uint64_t bits;
  uint8_t status;
  uint8_t bignum;
  uint8_t error;
  uint8_t nl;  // the field ends at '\n' or at the end of the text (not at the delimiter)
};

__device__ __forceinline__ bool is_sep(uint32_t c, uint32_t delim) { return c == '\n' || c == delim; }

// Parse one field starting at f (at most lim bytes remain in the buffer).
template <class F>
__device__ LongResult parse_long_field(const uint8_t* f, unsigned long long lim, uint32_t delim,
                                       uint32_t grammar, bool need_nl, const Pow5& tab, Big D,
                                       Big P, Big B) {
  LongResult r;
  r.bignum = 0;
  r.error = 0;
  r.nl = 1;
  if (need_nl) {  // the terminator (only the column-major layout looks at it)
    unsigned long long t = 0;
    while (t < lim && !is_sep(f[t], delim)) t++;
    r.nl = t >= lim || f[t] == '\n';
  }
  // ---- 1. tokenize ---------------------------------------------------------
  unsigned long long i = 0;
  while (i < lim && is_ws(f[i])) i++;
  uint64_t sign = 0;
  if (i < lim && (f[i] == '-' || (f[i] == '+' && grammar != GRAMMAR_JSON))) {
    sign = f[i] == '-' ? F::SIGN : 0;
    i++;
  }
  if (grammar == GRAMMAR_HEX && i + 1 < lim && f[i] == '0' && (f[i + 1] | 0x20) == 'x') {
    // a long hexadecimal float: 16 significant hex digits, the rest into the
    // exponent (integer digits) or the sticky flag; exact without big numbers
    i += 2;
    uint64_t m = 0;
    int kept = 0;
    unsigned long long nd = 0;
    long long e2 = 0;
    bool sticky = false;
    for (int part = 0; part < 2; part++) {
      if (part == 1) {
        if (i < lim && f[i] == '.') i++;
        else break;
      }
      int dv;
      while (i < lim && (dv = hex_digit(f[i])) >= 0) {
        if (kept < 16) {
          if (m || dv) {
            m = m * 16 + (uint64_t)dv;
            kept++;
          }
          if (part == 1) e2 -= 4;
        } else {
          if (part == 0 && e2 < EXP_SAT) e2 += 4;
          sticky |= (dv != 0);
        }
        i++;
        nd++;
      }
    }
    bool ok = nd > 0;
    if (ok && i < lim && (f[i] | 0x20) == 'p') {
      i++;
      bool eneg = false;
      if (i < lim && (f[i] == '+' || f[i] == '-')) {
        eneg = f[i] == '-';
        i++;
      }
      unsigned long long ne = 0;
      long long ex = 0;
      while (i < lim && is_digit(f[i])) {
        if (ex < EXP_SAT) ex = ex * 10 + (f[i] - '0');
        if (ex > EXP_SAT) ex = EXP_SAT;
        i++;
        ne++;
      }
      ok = ne > 0;
      e2 += eneg ? -ex : ex;
    }
    while (i < lim && is_ws(f[i])) i++;
    ok = ok && (i == lim || is_sep(f[i], delim));
    if (!ok) {
      r.bits = F::QNAN;
      r.status = ST_INVALID;
      return r;
    }
    const uint64_t b = m ? hex_to_bits<F>(m, e2, sticky) : 0;
    r.bits = b | sign;
    r.status = m ? status_of<F>(b) : ST_OK;
    return r;
  }
  const unsigned long long int_start = i;
  while (i < lim && is_digit(f[i])) i++;
  const unsigned long long n_int = i - int_start;
  unsigned long long frac_start = i, n_frac = 0;
  if (i < lim && f[i] == '.') {
    i++;
    frac_start = i;
    while (i < lim && is_digit(f[i])) i++;
    n_frac = i - frac_start;
  }
  const unsigned long long ndig = n_int + n_frac;
  bool ok = ndig > 0;
  if (grammar == GRAMMAR_JSON) {
    // an integer part without leading zeros; digits after a point
    ok = ok && n_int > 0 && !(n_int > 1 && f[int_start] == '0') &&
         !(frac_start != int_start + n_int && n_frac == 0);
  }
  long long ex = 0;
  if (ok && i < lim && (f[i] | 0x20) == 'e') {
    i++;
    bool eneg = false;
    if (i < lim && (f[i] == '+' || f[i] == '-')) {
      eneg = f[i] == '-';
      i++;
    }
    unsigned long long ne = 0;
    while (i < lim && is_digit(f[i])) {
      if (ex < EXP_SAT) ex = ex * 10 + (f[i] - '0');
      if (ex > EXP_SAT) ex = EXP_SAT;
      i++;
      ne++;
    }
    ok = ne > 0;
    if (eneg) ex = -ex;
  }
  while (i < lim && is_ws(f[i])) i++;
  ok = ok && (i == lim || is_sep(f[i], delim));
  if (!ok) {
    r.bits = F::QNAN;
    r.status = ST_INVALID;
    return r;
  }
  auto digit = [&](unsigned long long k) -> uint32_t {
    return (k < n_int ? f[int_start + k] : f[frac_start + (k - n_int)]) - '0';
  };
  unsigned long long first = 0;
  while (first < ndig && digit(first) == 0) first++;
  if (first == ndig) {
    r.bits = sign;
    r.status = ST_OK;
    return r;
  }
  unsigned long long last = ndig - 1;
  while (digit(last) == 0) last--;
  const long long nsig = (long long)(last - first + 1);
  // value = (digits first..last) * 10^E
  const long long E = ex - (long long)n_frac + (long long)(ndig - 1 - last);
  // ---- quick exits: 10^(nsig-1+E) <= V < 10^(nsig+E) -------------------
  if (nsig - 1 + E >= F::DEC_OVF) {
    r.bits = F::INF | sign;
    r.status = ST_OVERFLOW;
    return r;
  }
  if (nsig + E <= F::DEC_UNF) {
    r.bits = sign;
    r.status = ST_UNDERFLOW;
    return r;
  }
  // ---- 19-digit prefix: Algorithm 1, then the w / w+1 check ---------------
  const int n19 = nsig < 19 ? (int)nsig : 19;
  uint64_t w = 0;
  for (int k = 0; k < n19; k++) w = w * 10 + digit(first + k);
  const long long q19 = E + (nsig - n19);
  const bool sticky19 = nsig > 19;
  ElResult a = convert_wq<F>(w, q19, tab, true);
  if (a.bits != EL_ABORT) {
    if (!sticky19) {
      r.bits = a.bits | sign;
      r.status = status_of<F>(a.bits);
      return r;
    }
    ElResult b = convert_wq<F>(w + 1, q19, tab, true);
    if (b.bits == a.bits) {
      r.bits = a.bits | sign;
      r.status = status_of<F>(a.bits);
      return r;
    }
  }
  // ---- 2. exact big-number comparison ------------------------------------
  r.bignum = 1;
  const long long nK = nsig < KMAX ? nsig : KMAX;
  long long ED = E + (nsig - nK);
  D.n = 0;
  for (long long k = 0; k < nK;) {
    uint32_t chunk = 0, mul = 1;
    for (int j = 0; j < 9 && k < nK; j++, k++) {
      chunk = chunk * 10 + digit(first + k);
      mul *= 10;
    }
    if (!big_mul_add(D, mul, chunk)) goto fail;
  }
  if (nsig > KMAX) {  // sticky digit
    if (!big_mul_add(D, 10, 1)) goto fail;
    ED -= 1;
  }
  {
    // V = D * 10^ED.  With ED >= 0 compare D 5^ED 2^ED against midpoints;
    // with ED < 0 compare D 2^ED against (2M+1) 5^-ED 2^(e-1).
    if (ED >= 0) {
      if (!big_mul_pow5(D, ED)) goto fail;
    } else {
      P.n = 1;
      P.at(0) = 1;
      if (!big_mul_pow5(P, -ED)) goto fail;
    }
    // ---- 3. candidate ------------------------------------------------------
    uint64_t x = convert_wq<F>(w, q19, tab, false).bits;
    // ---- 4. step to the nearest value of the format --------------------
    auto cmp_mid = [&](uint64_t lowbits, int& c) -> bool {
      // c = sign of V - midpoint(lowbits, lowbits + 1)
      uint64_t M;
      int e;
      float_parts<F>(lowbits, M, e);
      const uint64_t T = 2 * M + 1;
      if (ED >= 0) {
        B.n = 0;
        B.at(0) = (uint32_t)T;
        B.at(1) = (uint32_t)(T >> 32);
        B.n = B.at(1) ? 2 : 1;
        c = cmp_scaled(D, ED, B, (long long)e - 1);
      } else {
        if (!big_mul_u64(B, P, T)) return false;
        c = cmp_scaled(D, ED, B, (long long)e - 1);
      }
      return true;
    };
    for (int iter = 0; iter < 8; iter++) {
      int c;
      if (x < F::INF) {
        if (!cmp_mid(x, c)) goto fail;
        if (c > 0) {
          x += 1;
          continue;
        }
        if (c == 0) {
          x = (x & 1) ? x + 1 : x;
          goto done;
        }
      }
      if (x > 0) {
        if (!cmp_mid(x - 1, c)) goto fail;
        if (c < 0) {
          x -= 1;
          continue;
        }
        if (c == 0) {
          x = ((x - 1) & 1) ? x : x - 1;
          goto done;
        }
      }
      goto done;
    }
    goto fail;  // did not converge: an internal error
  done:
    r.bits = x | sign;
    r.status = status_of<F>(x);
    return r;
  }
fail:
  r.error = 1;
  r.bits = F::QNAN;
  r.status = ST_INVALID;
  return r;
}

template <class F>
__device__ __forceinline__ void resolve(const LaunchParams& p, unsigned long long oi, Big D, Big P,
                                        Big B, unsigned long long& n_items,
                                        unsigned long long& n_big) {
  const unsigned long long loc = p.loc[oi];
  const unsigned int dix = (unsigned int)(loc >> LOC_OFF_BITS);
  const unsigned long long off = loc & LOC_OFF_MASK;
  if (dix >= p.nbuf) {  // cannot happen for entries written by the parse kernel
    atomicCAS(&p.ctl->error, 0u, DERR_INTERNAL);
    return;
  }
  const BufDesc d = p.nbuf == 1 ? p.one : p.descs[dix];
  if (off >= d.len) {
    atomicCAS(&p.ctl->error, 0u, DERR_INTERNAL);
    return;
  }
  const uint8_t* f = d.base + d.o + off;
  const uint64_t* t = reinterpret_cast<const uint64_t*>(fp_pow5_table_dev);
  LongResult r = parse_long_field<F>(f, d.len - off, p.delim & 0xFFu, p.grammar, p.columns != 0,
                                     Pow5{t, 2, t + 1}, D, P, B);
  if (r.error) atomicCAS(&p.ctl->error, 0u, DERR_INTERNAL);
  unsigned long long dest = oi;
  if (p.columns) {  // column-major layout: oi is the field's index
    const unsigned long long row = oi / p.columns, col = oi - row * p.columns;
    dest = col * p.rows_cap + row;
    if ((bool)r.nl != (col == p.columns - 1)) r.status = ST_BAD_SHAPE;
  }
  reinterpret_cast<typename F::word*>(p.out_bits)[dest] = (typename F::word)r.bits;
  p.out_status[dest] = r.status;
  n_items++;
  n_big += r.bignum;
}

template <class F>
__global__ void __launch_bounds__(FB_NT) fallback_kernel(const LaunchParams p) {
  extern __shared__ __align__(16) uint32_t limbs[];
  const int tid = threadIdx.x;
  Big D{limbs + tid, 0}, P{limbs + LIMBS * FB_NT + tid, 0}, B{limbs + 2 * LIMBS * FB_NT + tid, 0};
  Ctl* ctl = p.ctl;
  const unsigned long long nq_all = *(volatile unsigned long long*)&ctl->qcount;
  const unsigned long long nq = nq_all < p.qcap ? nq_all : p.qcap;
  unsigned long long n_items = 0, n_big = 0, n_scan = 0;
  const unsigned long long gtid = (unsigned long long)blockIdx.x * FB_NT + tid;
  const unsigned long long gthreads = (unsigned long long)gridDim.x * FB_NT;
  for (unsigned long long i = gtid; i < nq; i += gthreads) {
    const unsigned long long oi = p.queue[i];
    resolve<F>(p, oi, D, P, B, n_items, n_big);
  }
  // Chunks whose pending fields did not fit the queue: one warp per chunk
  // scans its outputs for unlisted pending fields.
  const unsigned long long nov_all = *(volatile unsigned long long*)&ctl->ovf_count;
  const unsigned long long nov = nov_all < p.ovf_cap ? nov_all : p.ovf_cap;
  const int lane = tid & 31;
  const unsigned long long gwarp = gtid >> 5, gwarps = gthreads >> 5;
  for (unsigned long long c = gwarp; c < nov; c += gwarps) {
    const unsigned long long n = p.ovf[2 * c] & LOC_OFF_MASK;
    const unsigned long long ob = p.ovf[2 * c + 1];
    for (unsigned long long k = lane; k < n; k += 32) {
      unsigned long long sk = ob + k;  // the status slot of field ob + k
      if (p.columns) {
        const unsigned long long row = sk / p.columns;
        sk = (sk - row * p.columns) * p.rows_cap + row;
      }
      if (p.out_status[sk] == ST_PENDING_SCAN) {
        resolve<F>(p, ob + k, D, P, B, n_items, n_big);
        n_scan++;
      }
    }
  }
  // counters and end-of-launch reset
  __shared__ unsigned long long red[3];
  if (tid == 0) red[0] = red[1] = red[2] = 0;
  __syncthreads();
  if (n_items) atomicAdd(&red[0], n_items);
  if (n_big) atomicAdd(&red[1], n_big);
  if (n_scan) atomicAdd(&red[2], n_scan);
  __syncthreads();
  if (tid == 0) {
    if (red[0]) atomicAdd(&ctl->stats[CNT_FALLBACK], red[0]);
    if (red[1]) atomicAdd(&ctl->stats[CNT_FALLBACK_BIGNUM], red[1]);
    if (red[2]) atomicAdd(&ctl->stats[CNT_QUEUE_OVERFLOW], red[2]);
    __threadfence();
    const unsigned int prev = atomicAdd(&ctl->done_fallback, 1u);
    if (prev == gridDim.x - 1) {
      ctl->qcount = 0;
      ctl->ovf_count = 0;
      ctl->done_fallback = 0;
      __threadfence();
    }
  }
}

int fallback_smem_bytes() { return 3 * LIMBS * FB_NT * 4; }

template <class F>
static cudaError_t launch_fallback_f(const LaunchParams& p, int grid, cudaStream_t stream) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(fallback_kernel<F>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         fallback_smem_bytes());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  fallback_kernel<F><<<grid, FB_NT, fallback_smem_bytes(), stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fallback(const LaunchParams& p, int grid, cudaStream_t stream, bool f32) {
  return f32 ? launch_fallback_f<F32>(p, grid, stream) : launch_fallback_f<F64>(p, grid, stream);
}

template <class F>
static cudaError_t fallback_occupancy_f(int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(fallback_kernel<F>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       fallback_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fallback_kernel<F>, FB_NT,
                                                       fallback_smem_bytes());
}

cudaError_t fallback_occupancy(int* blocks_per_sm, bool f32) {
  return f32 ? fallback_occupancy_f<F32>(blocks_per_sm) : fallback_occupancy_f<F64>(blocks_per_sm);
}

}  // namespace fp
