// fp_fallback_kernel.cu -- exact resolution of the fields the parse kernel
// could not settle (Section 11 "higher-precision approach"; the design here
// is this library's own: a big-number comparison against midpoints).
//
// A field arrives here when it is longer than the parse kernel's limit, when
// Algorithm 1 gave up (second product word all ones outside [-27, 55]), or
// when its 19-digit truncation w and w+1 round differently (Section 11).
//
// One warp per field, all lanes on the same field:
//   1. tokenize the whole field (Section 4 grammar, or the JSON one): its end
//      from aligned 16-byte reads, 512 bytes per round; then one pass of
//      byte ballots, 64 bytes per round, that checks the grammar and finds
//      the exponent marker, the point and the first and last nonzero digit,
//      from which every digit count follows;
//   2. Algorithm 1 on the 19-digit prefix w (read from the text) and on w+1
//      (two lanes); equal results settle the field;
//   3. otherwise V = D 10^E with D the first 800 significant digits and one
//      extra digit 1 appended when there are more (the last one is nonzero),
//      copied from the text to shared memory by the lanes together.
//      Every midpoint between adjacent floating-point values has at most
//      768 significant digits (Section 11), so V and the exact value lie on
//      the same side of every midpoint;
//   4. when the two results of step 2 are adjacent values, V lies between
//      the two products and so on one side of the one midpoint between
//      them: one exact comparison decides (a tie picks the even one).  When
//      Algorithm 1 gave up, the candidate x = the rounded truncated product
//      of the prefix (within one unit of the answer) is stepped by exact
//      comparisons with the midpoints above and below it until it is the
//      nearest value.  A midpoint h = (2M+1) 2^(e-1) is written in base 10^9 --
//      (2M+1) 2^(e-1), or (2M+1) 5^(1-e) 10^(e-1) -- from a table power, a
//      small power and the factor 2M+1, and compared with V's digits
//      regrouped into the same base-10^9 chunks.
// The big naturals are base-10^9 limb arrays in shared memory with limb i on
// lane i mod 32: a multiply takes one 32-limb round per lane step, and its
// carries are resolved for all 32 limbs of a round at once by adding the
// round's generate and propagate ballots as integers.  Hexadecimal floats
// (exact from their digits) are decided by one lane.
#include <cuda_runtime.h>

#include "dec_tables.inc"
#include "fp_device.cuh"
#include "fp_launch.h"
#include "fp_sync.cuh"
#include "fp_types.cuh"

namespace fp {

namespace {

// Powers of five and two in base 10^9 (gen_dec_tables.py).
__device__ const uint32_t dec5_off[FP_DEC5_COUNT + 1] = {FP_DEC5_OFF_VALUES};
__device__ const uint32_t dec5_limbs[FP_DEC5_LIMBS] = {FP_DEC5_VALUES};
__device__ const uint32_t dec2_off[FP_DEC2_COUNT + 1] = {FP_DEC2_OFF_VALUES};
__device__ const uint32_t dec2_limbs[FP_DEC2_LIMBS] = {FP_DEC2_VALUES};
constexpr uint32_t DBASE = FP_DEC_BASE;
// 10^k, k < 19
__device__ const unsigned long long kPow10[19] = {
    1ull, 10ull, 100ull, 1000ull, 10000ull, 100000ull, 1000000ull, 10000000ull, 100000000ull,
    1000000000ull, 10000000000ull, 100000000000ull, 1000000000000ull, 10000000000000ull,
    100000000000000ull, 1000000000000000ull, 10000000000000000ull, 100000000000000000ull,
    1000000000000000000ull};

constexpr int FB_WARPS = 4;           // warps per block
constexpr int FB_NT = 32 * FB_WARPS;  // threads per block
constexpr int LIMBS = 96;             // base-10^9 limbs per big number: three rounds of 32
constexpr int KMAX = 800;             // significant digits kept before the sticky digit
constexpr int DIG_CAP = 832;          // digit bytes per warp (KMAX + 1, rounded up)
constexpr long long EXP_SAT = 1000000000000000ll;  // explicit exponent saturation
constexpr uint32_t FULL = 0xFFFFFFFFu;

// per warp: three big naturals and the digits of a field that needs them
struct WarpSmem {
  uint32_t P[LIMBS], B[LIMBS], Q[LIMBS];
  uint8_t dig[DIG_CAP];
};

// The significant digits of a field, read from its text: digit j (j = 0 is
// the first nonzero one) is the byte at fz + j, one further on from the
// point on (the digits of a valid significand are contiguous but for one
// point).  The first nreal digits are the text's (at most KMAX); a sticky
// digit 1 follows when the field has more (a nonzero digit lies beyond,
// since the last significant digit is nonzero); every later digit is 0.
struct DigitSrc {
  const uint8_t* f;
  long long fz;        // text offset of digit 0
  long long shift_at;  // first digit index after the point (or beyond all digits)
  long long nreal;
  bool sticky;
  __device__ __forceinline__ uint32_t at(long long j) const {
    if (j < nreal) return (uint32_t)f[fz + j + (j >= shift_at ? 1 : 0)] - '0';
    return (sticky && j == nreal) ? 1u : 0u;
  }
};

// A big natural in shared memory; n (the number of limbs, top limb nonzero)
// is the same on every lane.
struct WBig {
  uint32_t* p;
  int n;
};

// Set n from limb n0-1 downwards (limbs >= n0 are zero).
__device__ __forceinline__ void wb_trim(WBig& x, int n0) {
  int n = n0;
  while (n > 0 && x.p[n - 1] == 0) n--;
  x.n = n;
}

// ---- base 10^9 --------------------------------------------------------------
// Carries of one round in base 10^9: s is this lane's sum (< 2 * 10^9).
__device__ __forceinline__ uint32_t dec_round(uint32_t s, uint32_t& cin, int lane) {
  const bool g = s >= DBASE;
  if (g) s -= DBASE;
  const uint32_t G = __ballot_sync(FULL, g);
  const uint32_t Pm = __ballot_sync(FULL, s == DBASE - 1);
  const uint32_t A = G | Pm;
  const unsigned long long sum = (unsigned long long)A + G + cin;
  const uint32_t into = (uint32_t)sum ^ A ^ G;
  cin = (uint32_t)(sum >> 32);
  s += (into >> lane) & 1u;
  return s == DBASE ? 0u : s;
}

// y = x * m (m < 10^9), y != x.
__device__ __noinline__ bool dec_mul(WBig& y, const WBig& x, uint32_t m, int lane) {
  const int n = x.n;
  if (n + 1 > LIMBS) return false;
  uint32_t qp_round = 0, cin = 0;
  const int rounds = (n + 1 + 31) >> 5;
  for (int j = 0; j < rounds; j++) {
    const int i = 32 * j + lane;
    const unsigned long long prod = (unsigned long long)(i < n ? x.p[i] : 0u) * m;
    const uint32_t q = (uint32_t)(prod / DBASE), r = (uint32_t)(prod - (unsigned long long)q * DBASE);
    uint32_t qp = __shfl_up_sync(FULL, q, 1);
    if (lane == 0) qp = qp_round;
    qp_round = __shfl_sync(FULL, q, 31);
    const uint32_t v = dec_round(r + qp, cin, lane);
    if (i <= n) y.p[i] = v;
  }
  __syncwarp();
  wb_trim(y, n + 1);
  return true;
}

// y = y + x * 10^9 (x shifted one limb up), y != x.
__device__ __noinline__ bool dec_add_shifted(WBig& y, const WBig& x, int lane) {
  const int n = y.n > x.n + 1 ? y.n : x.n + 1;
  if (n + 1 > LIMBS) return false;
  uint32_t cin = 0;
  const int rounds = (n + 1 + 31) >> 5;
  for (int j = 0; j < rounds; j++) {
    const int i = 32 * j + lane;
    const uint32_t yi = i < y.n ? y.p[i] : 0u;
    const uint32_t xi = (i >= 1 && i - 1 < x.n) ? x.p[i - 1] : 0u;
    const uint32_t v = dec_round(yi + xi, cin, lane);
    __syncwarp();
    if (i <= n) y.p[i] = v;
  }
  __syncwarp();
  wb_trim(y, n + 1);
  return true;
}

// y = table entry [off[a], off[a+1]).
__device__ __noinline__ void dec_load(WBig& y, const uint32_t* limbs, const uint32_t* off, int a,
                                      int lane) {
  const int o0 = (int)off[a], n = (int)off[a + 1] - o0;
  for (int i = lane; i < n; i += 32) y.p[i] = limbs[o0 + i];
  __syncwarp();
  y.n = n;
}

__device__ __forceinline__ int dec_digits(uint32_t v) {  // decimal digits of 0 < v < 10^9
  int d = 1;
  for (uint32_t p = 10; d < 9 && v >= p; p *= 10) d++;
  return d;
}

// Sign of V - h, V = dig[0 .. nD) * 10^ED (dig[0] != 0), h = H * 10^Eh (H > 0
// in base 10^9): the leading digits' exponents, then V's digits regrouped
// into H's base-10^9 chunks (the first chunk as wide as H's top limb).
__device__ __noinline__ int dec_compare(const uint8_t* dig, long long nD, long long ED,
                                        const WBig& H, long long Eh, int lane) {
  const int nl = H.n;
  const int ltop = dec_digits(H.p[nl - 1]);
  const long long nH = ltop + 9ll * (nl - 1);
  const long long Lv = nD - 1 + ED, Lh = nH - 1 + Eh;
  if (Lv != Lh) return Lv < Lh ? -1 : 1;
  const long long vch = nD > ltop ? 1 + (nD - ltop + 8) / 9 : 1;
  const long long nch = vch > nl ? vch : nl;
  for (long long c0 = 0; c0 < nch; c0 += 32) {
    const long long c = c0 + lane;
    uint32_t hv = 0, vv = 0;
    if (c < nch) {
      hv = c < nl ? H.p[nl - 1 - c] : 0u;
      // chunk c holds digits [end - 9, end), end = ltop + 9c; digits before
      // 0 (in the first chunk) and from nD on are zeros
      const long long end = ltop + 9 * c;
#pragma unroll
      for (int k = 0; k < 9; k++) {
        const long long j = end - 9 + k;
        vv = vv * 10 + ((j >= 0 && j < nD) ? (uint32_t)dig[j] : 0u);
      }
    }
    const uint32_t diff = __ballot_sync(FULL, hv != vv);
    if (diff) {
      const int first = __ffs(diff) - 1;
      const int lt = __shfl_sync(FULL, (int)(vv < hv), first);
      return lt ? -1 : 1;
    }
  }
  return 0;
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


// The power part of a midpoint, 2^(e-1) or 5^(1-e) (times 10^Eh), for the
// exponent e of the last call: the midpoints on both sides of a candidate
// share it (unless they straddle a power of two), so it is formed once.
struct MidPower {
  bool valid;
  int e;
  long long Eh;
  WBig X;  // in sm.P or sm.Q
};

// Sign of V - h into c, V = sm.dig[0 .. nD) 10^ED and h the midpoint between
// the positive patterns lowbits and lowbits + 1 of F; false on a size error.
template <class F>
__device__ __noinline__ bool cmp_midpoint(uint64_t lowbits, WarpSmem& sm, long long nD,
                                          long long ED, int& c, int lane, MidPower& mp) {
  uint64_t M;
  int e;
  float_parts<F>(lowbits, M, e);
  const uint64_t T = 2 * M + 1;  // < 2^55 < 10^18
  if (!mp.valid || mp.e != e) {
    WBig X{sm.P, 0}, Y{sm.Q, 0};
    long long Eh;
    uint32_t m;  // the small power after the table's
    if (e >= 1) {  // h = T 2^(e-1)
      const int k = e - 1;
      dec_load(X, dec2_limbs, dec2_off, k / FP_DEC2_STEP, lane);
      m = 1u << (k % FP_DEC2_STEP);
      Eh = 0;
    } else {  // h = T 5^(1-e) 10^(e-1)
      const int j = 1 - e;
      dec_load(X, dec5_limbs, dec5_off, j / FP_DEC5_STEP, lane);
      m = 1;
      for (int b = j % FP_DEC5_STEP; b > 0; b--) m *= 5;
      Eh = e - 1;
    }
    if (m != 1) {
      if (!dec_mul(Y, X, m, lane)) return false;
      X = Y;  // the power now sits in sm.Q
    }
    mp.valid = true;
    mp.e = e;
    mp.Eh = Eh;
    mp.X = X;
  }
  const WBig X = mp.X;
  const long long Eh = mp.Eh;
  WBig A{sm.B, 0}, Y{X.p == sm.P ? sm.Q : sm.P, 0};  // the two buffers X does not use
  const uint32_t t0 = (uint32_t)(T % DBASE), t1 = (uint32_t)(T / DBASE);
  if (!dec_mul(A, X, t0, lane)) return false;
  if (t1) {
    if (!dec_mul(Y, X, t1, lane) || !dec_add_shifted(A, Y, lane)) return false;
  }
  c = dec_compare(sm.dig, nD, ED, A, Eh, lane);
  return true;
}

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
__device__ LongResult warp_field(const uint8_t* fg, unsigned long long lim, uint32_t delim,
                                 uint32_t grammar, WarpSmem& sm, bool* nl, int lane) {
  LongResult r;
  r.bignum = 0;
  r.error = 0;
  const uint8_t* f = fg;
  auto invalid = [&]() {
    r.bits = F::QNAN;
    r.status = ST_INVALID;
    return r;
  };
  // ---- the field's end, first and last non-blank byte ---------------------
  // 512 bytes per round: lane L tests the aligned 16-byte granule L of the
  // round with word-wide zero-byte tests.  A granule is read only if it
  // holds a byte of the text (x0 < lim), so no read leaves the 16-byte
  // granules of the buffer; bytes before the field are ignored and bytes at
  // or after lim act as separators.
  const uint8_t* fa = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(f) & ~(uintptr_t)15);
  const long long head = f - fa;
  long long fe = (long long)lim;
  long long p0 = -1, p1 = 0;
  for (long long r0 = 0;; r0 += 512) {
    const long long x0 = r0 + 16 * lane - head;  // field offset of this lane's first byte
    uint32_t sepm = 0xFFFFu, nbm = 0;           // bit b: byte x0 + b
    if (x0 < (long long)lim) {
      const uint4 v = *reinterpret_cast<const uint4*>(fa + r0 + 16 * lane);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
      uint32_t sz[4], wz[4];
      const uint32_t DLW = delim * 0x01010101u;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        sz[i] = zero_bytes(w4[i] ^ 0x0A0A0A0Au) | zero_bytes(w4[i] ^ DLW);
        wz[i] = zero_bytes(w4[i] ^ 0x20202020u) | zero_bytes(w4[i] ^ 0x09090909u) |
                zero_bytes(w4[i] ^ 0x0D0D0D0Du);
      }
      sepm = (flag_pair(sz[0], sz[1]) >> 7) | (flag_pair(sz[2], sz[3]) << 1);
      nbm = ~((flag_pair(wz[0], wz[1]) >> 7) | (flag_pair(wz[2], wz[3]) << 1)) & 0xFFFFu;
      if (x0 + 16 > (long long)lim) {  // bytes at or after lim: separators
        const uint32_t past = 0xFFFFu << (int)((long long)lim - x0);
        sepm |= past & 0xFFFFu;
        nbm &= ~past;
      }
      if (x0 < 0) {  // bytes before the field
        const uint32_t keep = 0xFFFFu << (int)(-x0);
        sepm &= keep;
        nbm &= keep;
      }
    }
    const uint32_t S = __ballot_sync(FULL, sepm != 0);
    int Ls = 32, bs = 0;
    if (S) {
      Ls = __ffs(S) - 1;
      bs = __ffs(__shfl_sync(FULL, sepm, Ls)) - 1;
      fe = r0 + 16 * Ls - head + bs;
    }
    // non-blank bytes before the first separator
    if (lane > Ls) nbm = 0;
    else if (lane == Ls) nbm &= (1u << bs) - 1u;
    const uint32_t NB = __ballot_sync(FULL, nbm != 0);
    if (NB) {
      const int L1 = 31 - __clz(NB);
      const uint32_t m1 = __shfl_sync(FULL, nbm, L1);
      if (p0 < 0) {
        const int L0 = __ffs(NB) - 1;
        const uint32_t m0 = __shfl_sync(FULL, nbm, L0);
        p0 = r0 + 16 * L0 - head + __ffs(m0) - 1;
      }
      p1 = r0 + 16 * L1 - head + (32 - __clz(m1));
    }
    if (S) break;
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
  // ---- structure: the exponent marker, the point, the nonzero digits -------
  // One pass over [s, the marker), 64 bytes per round (lane L takes bytes L
  // and 32 + L; 64-bit masks from pairs of ballots): the first marker ends
  // the significand; the first point, the first and the last nonzero digit
  // are located and any other byte flags the field.  A valid significand is
  // digits and at most one point, so every count below follows from these
  // positions, and its digits are read from the text where needed.  Each
  // round's bytes are read one round ahead, so that their loads overlap the
  // ballots of the round before.
  long long ep = p1;  // first 'e' / 'E' in [s, p1)
  long long dp = -1;  // the point
  long long fz = -1;  // first nonzero digit of the significand
  long long lz = -1;  // last nonzero digit of the significand
  long long ndot = 0;
  bool bad = false;
  auto pair = [&](bool lo, bool hi) -> unsigned long long {
    return ((unsigned long long)__ballot_sync(FULL, hi) << 32) | __ballot_sync(FULL, lo);
  };
  uint32_t cn0 = s + lane < p1 ? f[s + lane] : '0';
  uint32_t cn1 = s + 32 + lane < p1 ? f[s + 32 + lane] : '0';
  for (long long base = s; base < p1; base += 64) {
    const long long left = p1 - base;  // bytes of [s, p1) from this round on
    const unsigned long long inr = left >= 64 ? ~0ull : ((1ull << left) - 1ull);
    const uint32_t c0 = cn0, c1 = cn1;
    cn0 = base + 64 + lane < p1 ? f[base + 64 + lane] : '0';
    cn1 = base + 96 + lane < p1 ? f[base + 96 + lane] : '0';
    const bool d0 = is_digit(c0), d1 = is_digit(c1);
    const unsigned long long E = pair((c0 | 0x20) == 'e', (c1 | 0x20) == 'e') & inr;
    const unsigned long long inm = inr & (E ? ((E & (0ull - E)) - 1ull) : ~0ull);  // before the marker
    const unsigned long long dots = pair(c0 == '.', c1 == '.') & inm;
    const unsigned long long other = pair(!d0 && c0 != '.', !d1 && c1 != '.') & inm;
    const unsigned long long nz = pair(d0 && c0 != '0', d1 && c1 != '0') & inm;
    bad |= other != 0;
    if (dots) {
      ndot += __popcll(dots);
      if (dp < 0) dp = base + __ffsll((long long)dots) - 1;
    }
    if (nz) {
      if (fz < 0) fz = base + __ffsll((long long)nz) - 1;
      lz = base + 63 - __clzll((long long)nz);
    }
    if (E) {
      ep = base + __ffsll((long long)E) - 1;
      break;
    }
  }
  // [s, ep) holds ep - s - ndot digits
  if (bad || ndot > 1 || ep - s - ndot == 0) return invalid();
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
      const long long ne = p1 - nonzero0;  // digits from the first nonzero one
      if (ne > 16) {
        ex = EXP_SAT;  // at least 10^16
      } else {
        // lane k < ne weighs digit k by 10^(ne-1-k); a butterfly adds them
        uint64_t term = lane < ne ? (uint64_t)(f[nonzero0 + lane] - '0') * kPow10[ne - 1 - lane] : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) term += __shfl_xor_sync(FULL, term, off);
        ex = (long long)term;
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
  // ---- the decimal exponent E ----------------------------------------------
  // significant digits fz .. lz and the zeros after them (the point
  // excluded); digits after the point
  const long long nsig = lz - fz + 1 - ((dp > fz && dp < lz) ? 1 : 0);
  const long long nst = ep - fz - (dp > fz ? 1 : 0);
  const long long n_frac = dp >= 0 ? ep - dp - 1 : 0;
  const long long tz = nst - nsig;  // the zero digits after the last nonzero one
  const long long E = ex - n_frac + tz;  // value = (digits fz..lz) * 10^E
  const DigitSrc src{f, fz, dp > fz ? dp - fz : (long long)(1ll << 62), nsig < KMAX ? nsig : KMAX,
                     nsig > KMAX};
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
  // w = the first n19 digits: lane k < n19 weighs digit k by 10^(n19-1-k),
  // and a butterfly adds the terms
  uint64_t w = lane < n19 ? (uint64_t)src.at(lane) * kPow10[n19 - 1 - lane] : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(FULL, w, off);
  const long long q19 = E + (nsig - n19);
  const uint64_t* t = reinterpret_cast<const uint64_t*>(fp_pow5_table_dev);
  const Pow5 tab{t, 2, t + 1};
  // Algorithm 1 on w (lane 0) and, for more than 19 digits, on w + 1 (lane 1)
  uint64_t mine = EL_ABORT;
  if (lane == 0 || (lane == 1 && nsig > 19)) mine = convert_wq<F>(w + lane, q19, tab, true).bits;
  const uint64_t abits = __shfl_sync(FULL, mine, 0);
  const uint64_t bbits = __shfl_sync(FULL, mine, 1);
  const bool settled = abits != EL_ABORT && (nsig <= 19 || bbits == abits);
  if (settled) {
    r.bits = abits | sign;
    r.status = status_of<F>(abits);
    return r;
  }
  // ---- exact comparison with midpoints, in decimal --------------------------
  r.bignum = 1;
  {
    // the first KMAX digits and, for more, a sticky digit 1 one place below,
    // to shared memory (lanes take digits j = lane mod 32)
    const long long nD = src.nreal + (src.sticky ? 1 : 0);
    const long long ED = E + (nsig - src.nreal) - (src.sticky ? 1 : 0);
#pragma unroll 4
    for (long long j = lane; j < nD; j += 32) sm.dig[j] = (uint8_t)src.at(j);
    __syncwarp();
    MidPower mp;
    mp.valid = false;
    mp.e = 0;
    mp.Eh = 0;
    mp.X = WBig{sm.P, 0};
    auto cmp_mid = [&](uint64_t lowbits, int& c) -> bool {
      return cmp_midpoint<F>(lowbits, sm, nD, ED, c, lane, mp);
    };
    uint64_t x = 0;
    if (abits != EL_ABORT && bbits != EL_ABORT && bbits == abits + 1) {
      // V lies in [w, w+1) 10^q19, whose products round to abits and
      // abits + 1 (Algorithm 1 is exact on them): that interval, of relative
      // width at most 10^-18, holds one midpoint, the one above abits, and
      // one comparison with it decides
      int c;
      if (!cmp_mid(abits, c)) goto fail;
      x = c > 0 ? abits + 1 : (c < 0 ? abits : ((abits & 1) ? abits + 1 : abits));
      goto done;
    }
    // the candidate (Algorithm 1 gave up on w or w + 1): the rounded
    // truncated product, within one unit of the answer, stepped below
    if (lane == 0) x = convert_wq<F>(w, q19, tab, false).bits;
    x = __shfl_sync(FULL, x, 0);
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

// Two builds (MINB, the blocks per SM the registers must allow): 5 (96
// registers) for a launch that is expected to find nothing queued, 8 (64
// registers, a few spilled) for a stream with fallback work.  The wider one
// decided the hard-case mix 3% faster (2.53 against 2.61 ms), but used for
// every call it made the bulk step 3.7 us longer.
template <class F, int MINB>
__global__ void __launch_bounds__(FB_NT, MINB) fallback_kernel(const LaunchParams p) {
  __shared__ WarpSmem smem[FB_WARPS];
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  WarpSmem& sm = smem[wib];
  Ctl* ctl = p.ctl;
  // The next call's parse kernel (a programmatic dependent launch) may be
  // set up now; it waits on the device until this grid has completed.
  grid_launch_dependents();
  // the parse grid this launch depends on has completed, its writes visible
  grid_dependency_wait();
  const unsigned long long nq_all = *(volatile unsigned long long*)&ctl->qcount;
  const unsigned long long nov_all = *(volatile unsigned long long*)&ctl->ovf_count;
  // Nothing pending (the usual case): nothing to decide and nothing to
  // reset.  Every block sees the same two words (the parse kernel has ended
  // and the reset below happens only when one of them is nonzero, after
  // every block has read them), so either all blocks leave here or none.
  if ((nq_all | nov_all) == 0) {
    if (blockIdx.x == 0 && tid == 0 && p.pending_out) *p.pending_out = 0;
    return;
  }
  const unsigned long long nq = nq_all < p.qcap ? nq_all : p.qcap;
  unsigned long long n_items = 0, n_big = 0, n_scan = 0;
  const unsigned long long gwarp = (unsigned long long)blockIdx.x * FB_WARPS + wib;
  const unsigned long long gwarps = (unsigned long long)gridDim.x * FB_WARPS;
  for (unsigned long long i = gwarp; i < nq; i += gwarps)
    resolve<F>(p, p.queue[i], sm, lane, n_items, n_big);
  // Chunks whose pending fields did not fit the queue: one warp per chunk
  // finds them among its outputs and decides them one at a time.
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
      // every block's errors were made visible before its count above
      if (p.err_out) *p.err_out = *(volatile unsigned int*)&ctl->error;
      if (p.pending_out) *p.pending_out = nq_all + nov_all;
    }
  }
}

}  // namespace

// A programmatic dependent launch: the parse kernel releases it as it starts,
// so this launch's set-up overlaps the parse; its blocks wait on the device
// (griddepcontrol.wait) until the parse grid has completed and its writes
// are visible.  On a workload with nothing pending they then return at once,
// and the call pays little more than the parse.  It releases the next call's
// parse kernel in turn, so that launch's set-up overlaps this one.
template <class F>
static cudaError_t launch_fallback_f(const LaunchParams& p, int grid, cudaStream_t stream,
                                     bool busy) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(FB_NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return busy ? cudaLaunchKernelEx(&cfg, fallback_kernel<F, FB_BUSY_BLOCKS>, p)
              : cudaLaunchKernelEx(&cfg, fallback_kernel<F, FB_IDLE_BLOCKS>, p);
}

// One block that does nothing, queued between a parse kernel and the
// fallback kernel when the stream's calls have fallback work.  Launched
// right behind the parse kernel, the fallback kernel's blocks run in the
// parse kernel's division of each SM's on-chip memory (212 KB of shared
// memory, little L1 cache) and the fallback, which reads its fields' text
// again and again through L1, took 8.6% longer (2.83 against 2.61 ms on the
// hard-case mix); behind this launch it runs in its own (large L1) division.
__global__ void fallback_separator_kernel() {}

cudaError_t launch_fallback_separator(cudaStream_t stream) {
  fallback_separator_kernel<<<1, 32, 0, stream>>>();
  return cudaGetLastError();
}

cudaError_t launch_fallback(const LaunchParams& p, int grid, cudaStream_t stream, bool f32,
                            bool busy) {
  return f32 ? launch_fallback_f<F32>(p, grid, stream, busy)
             : launch_fallback_f<F64>(p, grid, stream, busy);
}

template <class F>
static cudaError_t fallback_occupancy_f(int* blocks_per_sm, bool busy) {
  return busy ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    blocks_per_sm, fallback_kernel<F, FB_BUSY_BLOCKS>, FB_NT, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    blocks_per_sm, fallback_kernel<F, FB_IDLE_BLOCKS>, FB_NT, 0);
}

cudaError_t fallback_occupancy(int* blocks_per_sm, bool f32, bool busy) {
  return f32 ? fallback_occupancy_f<F32>(blocks_per_sm, busy)
             : fallback_occupancy_f<F64>(blocks_per_sm, busy);
}

}  // namespace fp
