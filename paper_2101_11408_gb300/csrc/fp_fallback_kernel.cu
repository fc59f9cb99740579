// fp_fallback_kernel.cu -- exact resolution of the fields the parse kernel
// could not settle (Section 11 "higher-precision approach"; the design here
// is this library's own: a big-number comparison against midpoints).
//
// A field arrives here when it is longer than the parse kernel's limit, when
// Algorithm 1 gave up (second product word all ones outside [-27, 55]), or
// when its 19-digit truncation w and w+1 round differently (Section 11).
//
// One warp per field, all lanes on the same field:
//   1. tokenize the whole field with 32-byte coalesced reads and ballots
//      (Section 4 grammar, or the JSON one): its end, sign, significand,
//      point, exponent; its significant digits go to shared memory;
//   2. Algorithm 1 on the 19-digit prefix w and on w+1 (one lane); equal
//      results settle the field;
//   3. otherwise D = the first 800 significant digits, with one extra digit 1
//      appended when there are more (the last one is nonzero).  Every
//      midpoint between adjacent floating-point values has at most 768
//      significant digits (Section 11), so D 10^E and the exact value lie on
//      the same side of every midpoint;
//   4. candidate x = the rounded truncated product of the prefix (within one
//      unit of the answer); compare D 10^E exactly with the midpoints above
//      and below x, as integers scaled by powers of two and five, and step x
//      until it is the nearest value; a tie picks the even one.
// The big naturals are limb arrays in shared memory with limb i on lane
// i mod 32: a multiply-add takes one 32-limb round per lane step, and its
// carries are resolved for all 32 limbs of a round at once by adding the
// round's generate and propagate ballots as integers.  Hexadecimal floats
// (exact from their digits) are decided by one lane.
#include <cuda_runtime.h>

#include "fp_device.cuh"
#include "fp_sync.cuh"
#include "fp_types.cuh"

namespace fp {

namespace {

constexpr int FB_WARPS = 4;           // warps per block
constexpr int FB_NT = 32 * FB_WARPS;  // threads per block
constexpr int LIMBS = 96;             // 32-bit limbs per big number: three rounds of 32
constexpr int KMAX = 800;             // significant digits kept before the sticky digit
constexpr int DIG_CAP = 832;          // digit bytes per warp (KMAX + 1, rounded up)
constexpr long long EXP_SAT = 1000000000000000ll;  // explicit exponent saturation
constexpr uint32_t FULL = 0xFFFFFFFFu;

// per warp: four big naturals and the digit buffer
struct WarpSmem {
  uint32_t D[LIMBS], P[LIMBS], B[LIMBS], Q[LIMBS];
  uint8_t dig[DIG_CAP];
};

// A big natural in shared memory; n (the number of limbs, top limb nonzero)
// is the same on every lane.
struct WBig {
  uint32_t* p;
  int n;
};

__device__ __forceinline__ uint32_t limb_at(const WBig& x, long long i) {
  return (i >= 0 && i < x.n) ? x.p[i] : 0u;
}

// Carries of one 32-limb round: this lane's partial limb r, whether its own
// sum overflowed (g), and cin, the carry into the round's first limb.  The
// carry into limb i is g(i-1) | (r(i-1) all ones & carry into i-1): with
// A = G | P and G as 32-bit integers, (A + G + cin) ^ A ^ G has bit i set
// exactly when a carry enters limb i.  Returns the finished limb; cin
// becomes the carry out of the round.
__device__ __forceinline__ uint32_t round_carries(uint32_t r, bool g, uint32_t& cin, int lane) {
  const uint32_t G = __ballot_sync(FULL, g);
  const uint32_t Pm = __ballot_sync(FULL, r == 0xFFFFFFFFu);
  const uint32_t A = G | Pm;
  const unsigned long long sum = (unsigned long long)A + G + cin;
  const uint32_t into = (uint32_t)sum ^ A ^ G;
  cin = (uint32_t)(sum >> 32);
  return r + ((into >> lane) & 1u);
}

// Set n from limb n0-1 downwards (limbs >= n0 are zero).
__device__ __forceinline__ void wb_trim(WBig& x, int n0) {
  int n = n0;
  while (n > 0 && x.p[n - 1] == 0) n--;
  x.n = n;
}

// y = x * m + c (y may be x).  False if the result needs more than LIMBS limbs.
__device__ bool wb_mul_add(WBig& y, const WBig& x, uint32_t m, uint32_t c, int lane) {
  const int n = x.n;
  if (n + 1 > LIMBS) return false;
  uint32_t hp_round = c, cin = 0;
  const int rounds = (n + 1 + 31) >> 5;  // limbs 0..n
  for (int j = 0; j < rounds; j++) {
    const int i = 32 * j + lane;
    const uint32_t xi = i < n ? x.p[i] : 0u;
    const unsigned long long prod = (unsigned long long)xi * m;
    const uint32_t lo = (uint32_t)prod, hi = (uint32_t)(prod >> 32);
    uint32_t hp = __shfl_up_sync(FULL, hi, 1);
    if (lane == 0) hp = hp_round;
    hp_round = __shfl_sync(FULL, hi, 31);
    const unsigned long long s = (unsigned long long)lo + hp;
    const uint32_t r = round_carries((uint32_t)s, (s >> 32) != 0, cin, lane);
    __syncwarp();
    if (i <= n) y.p[i] = r;
  }
  __syncwarp();
  wb_trim(y, n + 1);
  return true;
}

// y = y + x.
__device__ bool wb_add(WBig& y, const WBig& x, int lane) {
  const int n = y.n > x.n ? y.n : x.n;
  if (n + 1 > LIMBS) return false;
  uint32_t cin = 0;
  const int rounds = (n + 1 + 31) >> 5;
  for (int j = 0; j < rounds; j++) {
    const int i = 32 * j + lane;
    const uint32_t yi = i < y.n ? y.p[i] : 0u, xi = i < x.n ? x.p[i] : 0u;
    const unsigned long long s = (unsigned long long)yi + xi;
    const uint32_t r = round_carries((uint32_t)s, (s >> 32) != 0, cin, lane);
    __syncwarp();
    if (i <= n) y.p[i] = r;
  }
  __syncwarp();
  wb_trim(y, n + 1);
  return true;
}

// y = y * 2^32 (one limb up).
__device__ bool wb_shift_limb(WBig& y, int lane) {
  const int n = y.n;
  if (n == 0) return true;
  if (n + 1 > LIMBS) return false;
  uint32_t v[LIMBS / 32];
#pragma unroll
  for (int j = 0; j < LIMBS / 32; j++) {
    const int i = 32 * j + lane;
    v[j] = i < n ? y.p[i] : 0u;
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < LIMBS / 32; j++) {
    const int i = 32 * j + lane;
    if (i < n) y.p[i + 1] = v[j];
  }
  if (lane == 0) y.p[0] = 0;
  __syncwarp();
  y.n = n + 1;
  return true;
}

__device__ bool wb_mul_pow5(WBig& x, long long k, int lane) {
  const uint32_t P13 = 1220703125u;  // 5^13
  while (k >= 13) {
    if (!wb_mul_add(x, x, P13, 0, lane)) return false;
    k -= 13;
  }
  uint32_t m = 1;
  while (k-- > 0) m *= 5;
  return m == 1 || wb_mul_add(x, x, m, 0, lane);
}

__device__ __forceinline__ long long wb_bitlen(const WBig& x) {
  if (x.n == 0) return 0;
  return 32ll * (x.n - 1) + (32 - __clz(x.p[x.n - 1]));
}

// Sign of X * 2^s - Y, given bitlen(X) + s == bitlen(Y) and s >= 0: the
// highest limb where they differ decides.
__device__ int wb_cmp_shifted(const WBig& X, long long s, const WBig& Y, int lane) {
  const long long ws = s >> 5;
  const int bs = (int)(s & 31);
  for (int j = (Y.n - 1) >> 5; j >= 0; j--) {
    const int i = 32 * j + lane;
    uint32_t xi = 0, yi = 0;
    if (i < Y.n) {
      xi = limb_at(X, i - ws) << bs;
      if (bs) xi |= limb_at(X, i - ws - 1) >> (32 - bs);
      yi = Y.p[i];
    }
    const uint32_t diff = __ballot_sync(FULL, xi != yi);
    if (diff) {
      const int top = 31 - __clz(diff);
      const int lt = __shfl_sync(FULL, (int)(xi < yi), top);
      return lt ? -1 : 1;
    }
  }
  return 0;
}

// Sign of X * 2^sx - Y * 2^sy for nonzero X, Y.
__device__ int wb_cmp_scaled(const WBig& X, long long sx, const WBig& Y, long long sy, int lane) {
  const long long lx = wb_bitlen(X) + sx, ly = wb_bitlen(Y) + sy;
  if (lx != ly) return lx < ly ? -1 : 1;
  const long long d = sx - sy;
  if (d >= 0) return wb_cmp_shifted(X, d, Y, lane);
  return -wb_cmp_shifted(Y, -d, X, lane);
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

__device__ __forceinline__ bool is_sep(uint32_t c, uint32_t delim) { return c == '\n' || c == delim; }

struct LongResult {
  uint64_t bits;
  uint8_t status;
  uint8_t bignum;
  uint8_t error;
};

// A hexadecimal float (one lane): 16 significant hex digits, the rest into
// the exponent (integer digits) or the sticky flag; exact without big
// numbers.  i is the offset of the digits after "0x", fe the field's end.
template <class F>
__device__ LongResult hex_field(const uint8_t* f, unsigned long long i, unsigned long long fe,
                                uint64_t sign) {
  LongResult r;
  r.bignum = 0;
  r.error = 0;
  uint64_t m = 0;
  int kept = 0;
  unsigned long long nd = 0;
  long long e2 = 0;
  bool sticky = false;
  for (int part = 0; part < 2; part++) {
    if (part == 1) {
      if (i < fe && f[i] == '.') i++;
      else break;
    }
    int dv;
    while (i < fe && (dv = hex_digit(f[i])) >= 0) {
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
  if (ok && i < fe && (f[i] | 0x20) == 'p') {
    i++;
    bool eneg = false;
    if (i < fe && (f[i] == '+' || f[i] == '-')) {
      eneg = f[i] == '-';
      i++;
    }
    unsigned long long ne = 0;
    long long ex = 0;
    while (i < fe && is_digit(f[i])) {
      if (ex < EXP_SAT) ex = ex * 10 + (f[i] - '0');
      if (ex > EXP_SAT) ex = EXP_SAT;
      i++;
      ne++;
    }
    ok = ne > 0;
    e2 += eneg ? -ex : ex;
  }
  while (i < fe && is_ws(f[i])) i++;
  if (!ok || i != fe) {
    r.bits = F::QNAN;
    r.status = ST_INVALID;
    return r;
  }
  const uint64_t b = m ? hex_to_bits<F>(m, e2, sticky) : 0;
  r.bits = b | sign;
  r.status = m ? status_of<F>(b) : ST_OK;
  return r;
}

// One field starting at f (lim >= 1 bytes remain in the buffer), by the
// whole warp.  *nl: the field ends at '\n' or at the end of the text.
template <class F>
__device__ LongResult warp_field(const uint8_t* f, unsigned long long lim, uint32_t delim,
                                 uint32_t grammar, WarpSmem& sm, bool* nl, int lane) {
  LongResult r;
  r.bignum = 0;
  r.error = 0;
  const uint32_t lt_mask = (1u << lane) - 1;
  auto invalid = [&]() {
    r.bits = F::QNAN;
    r.status = ST_INVALID;
    return r;
  };
  // ---- the field's end, first and last non-blank byte ---------------------
  long long fe = (long long)lim;
  long long p0 = -1, p1 = 0;
  for (long long base = 0; base < (long long)lim; base += 32) {
    const long long i = base + lane;
    const uint32_t c = i < (long long)lim ? f[i] : '\n';
    const uint32_t S = __ballot_sync(FULL, is_sep(c, delim));
    const uint32_t valid = S ? ((S & (0u - S)) - 1) : FULL;  // lanes before the first separator
    const uint32_t nb = __ballot_sync(FULL, !is_ws(c)) & valid;
    if (nb) {
      if (p0 < 0) p0 = base + __ffs(nb) - 1;
      p1 = base + 32 - __clz(nb);
    }
    if (S) {
      fe = base + __ffs(S) - 1;
      break;
    }
  }
  *nl = fe >= (long long)lim || f[fe] == '\n';
  if (p0 < 0) return invalid();  // blank or empty
  // ---- sign -----------------------------------------------------------------
  const uint32_t c0 = f[p0];
  uint64_t sign = 0;
  long long s = p0;
  if (c0 == '-' || (c0 == '+' && grammar != GRAMMAR_JSON)) {
    sign = c0 == '-' ? F::SIGN : 0;
    s++;
  }
  if (grammar == GRAMMAR_HEX && s + 1 < p1 && f[s] == '0' && (f[s + 1] | 0x20) == 'x') {
    LongResult h;
    h.bits = 0;
    h.status = 0;
    if (lane == 0) h = hex_field<F>(f, s + 2, fe, sign);
    h.bits = __shfl_sync(FULL, h.bits, 0);
    h.status = (uint8_t)__shfl_sync(FULL, (uint32_t)h.status, 0);
    h.bignum = 0;
    h.error = 0;
    return h;
  }
  // ---- structure: the exponent marker, the point, the digits ---------------
  long long ep = p1;  // first 'e' / 'E' in [s, p1)
  long long dp = -1;  // the point
  long long ndot = 0, nbad = 0, ndig = 0;
  long long fz = -1, lz = -1;  // first and last nonzero digit of the significand
  for (long long base = s; base < p1; base += 32) {
    const long long i = base + lane;
    const bool in = i < p1;
    const uint32_t c = in ? f[i] : '0';
    const uint32_t E = __ballot_sync(FULL, in && (c | 0x20) == 'e');
    const uint32_t cut = E ? ((E & (0u - E)) - 1) : FULL;  // lanes before the marker
    const uint32_t inm = __ballot_sync(FULL, in) & cut;
    const uint32_t dots = __ballot_sync(FULL, c == '.') & inm;
    const uint32_t digs = __ballot_sync(FULL, is_digit(c)) & inm;
    const uint32_t nz = __ballot_sync(FULL, is_digit(c) && c != '0') & inm;
    nbad += __popc(inm & ~dots & ~digs);
    ndig += __popc(digs);
    if (dots) {
      ndot += __popc(dots);
      if (dp < 0) dp = base + __ffs(dots) - 1;
    }
    if (nz) {
      if (fz < 0) fz = base + __ffs(nz) - 1;
      lz = base + 31 - __clz(nz);
    }
    if (E) {
      ep = base + __ffs(E) - 1;
      break;
    }
  }
  if (nbad || ndot > 1 || ndig == 0) return invalid();
  if (grammar == GRAMMAR_JSON) {
    // an integer part without leading zeros; digits after a point
    const uint32_t a = f[s];
    if (a == '.') return invalid();
    if (a == '0' && s + 1 < ep && is_digit(f[s + 1])) return invalid();
    if (dp >= 0 && dp + 1 == ep) return invalid();
  }
  // ---- exponent ---------------------------------------------------------------
  long long ex = 0;
  if (ep < p1) {
    long long es = ep + 1;
    bool eneg = false;
    const uint32_t cs = es < p1 ? f[es] : 0u;
    if (cs == '+' || cs == '-') {
      eneg = cs == '-';
      es++;
    }
    if (es >= p1) return invalid();  // no exponent digits
    long long nonzero0 = -1, nondig = 0;
    for (long long base = es; base < p1; base += 32) {
      const long long i = base + lane;
      const uint32_t c = i < p1 ? f[i] : '0';
      nondig += __popc(__ballot_sync(FULL, !is_digit(c)));
      const uint32_t nzm = __ballot_sync(FULL, is_digit(c) && c != '0');
      if (nzm && nonzero0 < 0) nonzero0 = base + __ffs(nzm) - 1;
    }
    if (nondig) return invalid();
    if (nonzero0 >= 0) {
      if (p1 - nonzero0 > 16) {
        ex = EXP_SAT;  // at least 10^16
      } else {
        for (long long i = nonzero0; i < p1; i++) ex = ex * 10 + (f[i] - '0');
        if (ex > EXP_SAT) ex = EXP_SAT;
      }
    }
    if (eneg) ex = -ex;
  }
  if (fz < 0) {  // all digits zero
    r.bits = sign;
    r.status = ST_OK;
    return r;
  }
  // ---- significant digits to shared memory; the decimal exponent E ---------
  // the digits of [fz, lz] (the point skipped) in order; n_frac: digits after
  // the point; tz: the (zero) digits after lz
  long long nsig = 0, n_frac = 0, tz = 0;
  for (long long base = fz; base < ep; base += 32) {
    const long long i = base + lane;
    const uint32_t c = i < ep ? f[i] : '.';
    const bool dg = is_digit(c);
    const uint32_t sigm = __ballot_sync(FULL, dg && i <= lz);
    const long long rank = nsig + __popc(sigm & lt_mask);
    if (dg && i <= lz && rank < KMAX) sm.dig[rank] = (uint8_t)(c - '0');
    nsig += __popc(sigm);
    tz += __popc(__ballot_sync(FULL, dg && i > lz));
    if (dp >= 0) n_frac += __popc(__ballot_sync(FULL, dg && i > dp));
  }
  // zeros between the point and fz are fraction digits too
  if (dp >= 0 && dp < fz) n_frac += fz - dp - 1;
  __syncwarp();
  const long long E = ex - n_frac + tz;  // value = (digits fz..lz) * 10^E
  // ---- quick exits: 10^(nsig-1+E) <= V < 10^(nsig+E) ----------------------
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
  // ---- 19-digit prefix: Algorithm 1, then the w / w+1 check (one lane) ----
  const int n19 = nsig < 19 ? (int)nsig : 19;
  uint64_t w = 0;
  for (int k = 0; k < n19; k++) w = w * 10 + sm.dig[k];
  const long long q19 = E + (nsig - n19);
  const uint64_t* t = reinterpret_cast<const uint64_t*>(fp_pow5_table_dev);
  const Pow5 tab{t, 2, t + 1};
  uint64_t abits = 0;
  int settled = 0;
  if (lane == 0) {
    const ElResult a = convert_wq<F>(w, q19, tab, true);
    abits = a.bits;
    if (a.bits != EL_ABORT) {
      if (nsig <= 19) settled = 1;
      else settled = convert_wq<F>(w + 1, q19, tab, true).bits == a.bits;
    }
  }
  settled = __shfl_sync(FULL, settled, 0);
  if (settled) {
    abits = __shfl_sync(FULL, abits, 0);
    r.bits = abits | sign;
    r.status = status_of<F>(abits);
    return r;
  }
  // ---- exact big-number comparison --------------------------------------------
  r.bignum = 1;
  const long long nK = nsig < KMAX ? nsig : KMAX;
  long long ED = E + (nsig - nK);
  WBig D{sm.D, 0}, P{sm.P, 0}, B{sm.B, 0}, Q{sm.Q, 0};
  {
    // D from the digits, nine at a time: the chunks' values in parallel
    // (into Q), then one multiply-add per chunk
    const int nch = (int)((nK + 8) / 9);
    for (int c = lane; c < nch; c += 32) {
      uint32_t v = 0;
      const int k1 = 9 * c + 9 < nK ? 9 * c + 9 : (int)nK;
      for (int k = 9 * c; k < k1; k++) v = v * 10 + sm.dig[k];
      Q.p[c] = v;
    }
    __syncwarp();
    for (int c = 0; c < nch; c++) {
      const int len = 9 * c + 9 < nK ? 9 : (int)(nK - 9 * c);
      uint32_t p10 = 1;
      for (int k = 0; k < len; k++) p10 *= 10;
      if (!wb_mul_add(D, D, p10, Q.p[c], lane)) goto fail;
    }
    if (nsig > KMAX) {  // the sticky digit
      if (!wb_mul_add(D, D, 10, 1, lane)) goto fail;
      ED -= 1;
    }
  }
  {
    // V = D * 10^ED.  With ED >= 0 compare D 5^ED 2^ED against midpoints;
    // with ED < 0 compare D 2^ED against (2M+1) 5^-ED 2^(e-1).
    if (ED >= 0) {
      if (!wb_mul_pow5(D, ED, lane)) goto fail;
    } else {
      if (lane == 0) P.p[0] = 1;
      __syncwarp();
      P.n = 1;
      if (!wb_mul_pow5(P, -ED, lane)) goto fail;
    }
    // the candidate
    uint64_t x = 0;
    if (lane == 0) x = convert_wq<F>(w, q19, tab, false).bits;
    x = __shfl_sync(FULL, x, 0);
    // sign of V - midpoint(lowbits, lowbits + 1); false on a size error
    auto cmp_mid = [&](uint64_t lowbits, int& c) -> bool {
      uint64_t M;
      int e;
      float_parts<F>(lowbits, M, e);
      const uint64_t T = 2 * M + 1;  // < 2^55
      if (ED >= 0) {
        if (lane == 0) {
          B.p[0] = (uint32_t)T;
          B.p[1] = (uint32_t)(T >> 32);
        }
        __syncwarp();
        B.n = (T >> 32) ? 2 : 1;
      } else {
        const uint32_t th = (uint32_t)(T >> 32), tl = (uint32_t)T;
        if (th) {
          if (!wb_mul_add(B, P, th, 0, lane) || !wb_shift_limb(B, lane)) return false;
          if (!wb_mul_add(Q, P, tl, 0, lane) || !wb_add(B, Q, lane)) return false;
        } else {
          if (!wb_mul_add(B, P, tl, 0, lane)) return false;
        }
      }
      c = wb_cmp_scaled(D, ED, B, (long long)e - 1, lane);
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

// Decide pending field oi (its location in p.loc[oi]) with the whole warp.
template <class F>
__device__ void resolve(const LaunchParams& p, unsigned long long oi, WarpSmem& sm, int lane,
                        unsigned long long& n_items, unsigned long long& n_big) {
  const unsigned long long loc = p.loc[oi];
  const unsigned int dix = (unsigned int)(loc >> LOC_OFF_BITS);
  const unsigned long long off = loc & LOC_OFF_MASK;
  if (dix >= p.nbuf) {  // cannot happen for entries written by the parse kernel
    if (lane == 0) atomicCAS(&p.ctl->error, 0u, DERR_INTERNAL);
    return;
  }
  const BufDesc d = p.nbuf == 1 ? p.one : p.descs[dix];
  if (off >= d.len) {
    if (lane == 0) atomicCAS(&p.ctl->error, 0u, DERR_INTERNAL);
    return;
  }
  const uint8_t* f = d.base + d.o + off;
  bool nl = true;
  LongResult r = warp_field<F>(f, d.len - off, p.delim & 0xFFu, p.grammar, sm, &nl, lane);
  if (lane == 0) {
    if (r.error) atomicCAS(&p.ctl->error, 0u, DERR_INTERNAL);
    unsigned long long dest = oi;
    if (p.columns) {  // column-major layout: oi is the field's index
      const unsigned long long row = oi / p.columns, col = oi - row * p.columns;
      dest = col * p.rows_cap + row;
      if (nl != (col == p.columns - 1)) r.status = ST_BAD_SHAPE;
    }
    reinterpret_cast<typename F::word*>(p.out_bits)[dest] = (typename F::word)r.bits;
    p.out_status[dest] = r.status;
    n_items++;
    n_big += r.bignum;
  }
  __syncwarp();
}

template <class F>
__global__ void __launch_bounds__(FB_NT, 4) fallback_kernel(const LaunchParams p) {
  __shared__ WarpSmem smem[FB_WARPS];
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  WarpSmem& sm = smem[wib];
  Ctl* ctl = p.ctl;
  const unsigned long long nq_all = *(volatile unsigned long long*)&ctl->qcount;
  const unsigned long long nq = nq_all < p.qcap ? nq_all : p.qcap;
  unsigned long long n_items = 0, n_big = 0, n_scan = 0;
  const unsigned long long gwarp = (unsigned long long)blockIdx.x * FB_WARPS + wib;
  const unsigned long long gwarps = (unsigned long long)gridDim.x * FB_WARPS;
  for (unsigned long long i = gwarp; i < nq; i += gwarps)
    resolve<F>(p, p.queue[i], sm, lane, n_items, n_big);
  // Chunks whose pending fields did not fit the queue: one warp per chunk
  // finds them among its outputs and decides them one at a time.
  const unsigned long long nov_all = *(volatile unsigned long long*)&ctl->ovf_count;
  const unsigned long long nov = nov_all < p.ovf_cap ? nov_all : p.ovf_cap;
  for (unsigned long long c = gwarp; c < nov; c += gwarps) {
    const unsigned long long n = p.ovf[2 * c] & LOC_OFF_MASK;
    const unsigned long long ob = p.ovf[2 * c + 1];
    for (unsigned long long k0 = 0; k0 < n; k0 += 32) {
      const unsigned long long k = k0 + lane;
      bool pend = false;
      if (k < n) {
        unsigned long long sk = ob + k;  // the status slot of field ob + k
        if (p.columns) {
          const unsigned long long row = sk / p.columns;
          sk = (sk - row * p.columns) * p.rows_cap + row;
        }
        pend = p.out_status[sk] == ST_PENDING_SCAN;
      }
      uint32_t m = __ballot_sync(FULL, pend);
      while (m) {
        const int l = __ffs(m) - 1;
        m &= m - 1;
        resolve<F>(p, ob + k0 + l, sm, lane, n_items, n_big);
        if (lane == 0) n_scan++;
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

}  // namespace

int fallback_smem_bytes() { return 0; }  // static shared memory only

template <class F>
static cudaError_t launch_fallback_f(const LaunchParams& p, int grid, cudaStream_t stream) {
  fallback_kernel<F><<<grid, FB_NT, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fallback(const LaunchParams& p, int grid, cudaStream_t stream, bool f32) {
  return f32 ? launch_fallback_f<F32>(p, grid, stream) : launch_fallback_f<F64>(p, grid, stream);
}

template <class F>
static cudaError_t fallback_occupancy_f(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fallback_kernel<F>, FB_NT, 0);
}

cudaError_t fallback_occupancy(int* blocks_per_sm, bool f32) {
  return f32 ? fallback_occupancy_f<F32>(blocks_per_sm) : fallback_occupancy_f<F64>(blocks_per_sm);
}

}  // namespace fp
