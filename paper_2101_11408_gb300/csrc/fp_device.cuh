// fp_device.cuh -- device-side building blocks of the parser (sm_103a).
//
// Algorithm 1 of the paper (Section 5; its steps are justified in Sections 6-10) on a decimal significand w < 2^64
// and exponent q, against the 128-bit power-of-five table; the field
// grammar of Section 4; the 19-digit truncation check of Section 11.
#pragma once
#include <cstdint>

#include "pow5_table.inc"

// The arithmetic below is plain integer code; FP_HD lets a host build of the
// same functions exist for development checks.
#ifdef __CUDACC__
#define FP_HD __host__ __device__ __forceinline__
#else
#define FP_HD inline
#endif

namespace fp {

// ---------------------------------------------------------------------------
// status and sentinels
// ---------------------------------------------------------------------------
enum : uint8_t {
  ST_OK = 0,
  ST_INVALID = 1,
  ST_OVERFLOW = 2,
  ST_UNDERFLOW = 3,
  ST_BAD_SHAPE = 4,          // columnar output: the field's terminator disagrees with its column
  ST_PENDING = 0xFF,         // internal result of the short-field parser
  ST_PENDING_QUEUED = 0xFE,  // stored status: pending, listed in the fallback queue
  ST_PENDING_SCAN = 0xFF,    // stored status: pending, found by scanning its chunk
  ST_GENERAL = 0xFD,         // staged only: the general tokenizer must decide
};

constexpr uint64_t QNAN_BITS = 0x7FF8000000000000ull;
constexpr uint64_t INF_BITS = 0x7FF0000000000000ull;
constexpr uint64_t SIGN_BIT = 0x8000000000000000ull;
constexpr uint64_t EL_ABORT = ~0ull;  // never a positive binary64 or binary32 pattern

// The two output formats (Section 2) as Algorithm 1 sees them: MBITS
// stored significand bits, the bias, SHIFT = 64 - (MBITS + 3) so that
// hi >> (u + SHIFT) keeps MBITS + 2 bits (one for rounding), the ties range
// of q (Sections 6, 8.1, 9.1), the decimal-magnitude range exits of the
// exact fallback, and the patterns of infinity, quiet NaN and the sign.
struct F64 {
  using word = unsigned long long;
  static constexpr int MBITS = 52, BIAS = 1023, EMAX_FIELD = 2047, SHIFT = 9;
  static constexpr int TIE_QMIN = -4, TIE_QMAX = 23;
  static constexpr int DEC_OVF = 309, DEC_UNF = -324;  // 1e309 > 2^1024, 1e-324 < 2^-1075
  static constexpr uint64_t INF = INF_BITS, QNAN = QNAN_BITS, SIGN = SIGN_BIT;
};
struct F32 {
  using word = unsigned int;
  static constexpr int MBITS = 23, BIAS = 127, EMAX_FIELD = 255, SHIFT = 38;
  static constexpr int TIE_QMIN = -17, TIE_QMAX = 10;
  static constexpr int DEC_OVF = 39, DEC_UNF = -46;  // 1e39 > 2^128, 1e-46 < 2^-150
  static constexpr uint64_t INF = 0x7F800000ull, QNAN = 0x7FC00000ull, SIGN = 0x80000000ull;
};

// Field grammars (the readings of include/fpparse.h): the decimal one, that
// or a hexadecimal float (Appendix C), or the JSON number grammar.
enum : uint32_t { GRAMMAR_DECIMAL = 0, GRAMMAR_HEX = 1, GRAMMAR_JSON = 2 };

// Fields longer than this many bytes are handed to the fallback kernel.
constexpr int LMAX = 64;

// Device error codes (mirrors fp_err_t values).
constexpr uint32_t DERR_TIMEOUT = 5;
constexpr uint32_t DERR_INTERNAL = 6;

// Counters kept per CTA and added to the stream's totals.
enum {
  CNT_FIELDS = 0,
  CNT_EL,       // fields settled by the window tokenizer and Algorithm 1 at once
  CNT_TWO_MUL,
  CNT_LONG,
  CNT_LONG_SETTLED,
  CNT_FALLBACK,
  CNT_FALLBACK_BIGNUM,
  CNT_QUEUE_OVERFLOW,
  CNT_SLOW,     // fields that needed the general tokenizer
  CNT_NOT_FAST, // fields the window tokenizer and Algorithm 1 did not settle at once
  CNT_NUM
};

#ifdef __CUDACC__
// The table in global memory (read once per CTA into shared memory).
__device__ const unsigned long long fp_pow5_table_dev[2 * FP_POW5_ENTRIES] = {
    FP_POW5_TABLE_VALUES};
#endif

FP_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}
FP_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// ---------------------------------------------------------------------------
// Algorithm 1
// ---------------------------------------------------------------------------
// The power-of-five table as the kernels see it: the high words, possibly a
// dense copy in shared memory (hi_stride 1) or the interleaved table itself
// (hi_stride 2), and the low words read from the interleaved table (only
// needed for the second product, Sections 7-8).
struct Pow5 {
  const uint64_t* hi;
  int hi_stride;
  const uint64_t* lo;  // &table[1]: the low word of entry i is lo[2 i]
};

FP_HD uint64_t load_lo(const uint64_t* p) {
#ifdef __CUDA_ARCH__
  return __ldg(reinterpret_cast<const unsigned long long*>(p));
#else
  return *p;
#endif
}

struct ElResult {
  uint64_t bits;  // positive pattern of the format, or EL_ABORT
  int two_mul;    // 1 if the second 64x64 product was needed
  // ST_OK, ST_UNDERFLOW (a zero result) or ST_OVERFLOW (infinity), decided
  // where the result is (ST_GENERAL when Algorithm 1 gave up)
  uint8_t status;
};

// w in [1, 2^64), q in [FP_POW5_QMIN, FP_POW5_QMAX]; tab points at the table
// (shared memory).  allow_abort = false returns the rounded truncated
// product even where Algorithm 1 would give up; that value is then within
// one unit in the last place of the correct result (the fallback kernel
// uses it as its first candidate).
template <class F = F64>
FP_HD ElResult eisel_lemire(uint64_t w, int q, const Pow5& tab, bool allow_abort) {
  ElResult r;
  r.two_mul = 0;
  r.status = ST_OK;
  // Normalise the decimal significand into [2^63, 2^64) (Algorithm 1).
  int l = clz64(w);
  w <<= l;
  const uint64_t thi = tab.hi[(q - FP_POW5_QMIN) * tab.hi_stride];
  // z = (T[q] * w) / 2^64, truncated: first the product with the high word.
  uint64_t lo = w * thi;
  uint64_t hi = mulhi64(w, thi);
  // Unless the low SHIFT bits of the high word are all ones, the top
  // MBITS + 3 bits (55 for binary64, 26 for binary32) are exact and one
  // product suffices (Algorithm 1; Sections 8 and 9).
  constexpr uint64_t LOWMASK = (1ull << F::SHIFT) - 1;
  if ((hi & LOWMASK) == LOWMASK) {
    const uint64_t tlo = load_lo(tab.lo + 2 * (q - FP_POW5_QMIN));
    uint64_t h2 = mulhi64(w, tlo);
    lo += h2;
    hi += (lo < h2);
    r.two_mul = 1;
  }
  // The second word all ones outside [-27, 55]: a third product could
  // still carry into the top word, so give up (Algorithm 1).
  if (allow_abort && lo == ~0ull && (q < -27 || q > 55)) {
    r.bits = EL_ABORT;
    r.status = ST_GENERAL;
    return r;
  }
  // MBITS + 2 significant bits (the significand plus one rounding bit)
  // below a possible leading zero bit u of the 128-bit product.
  const int u = (int)(hi >> 63);
  uint64_t m = hi >> (u + F::SHIFT);
  // Biased binary exponent: floor(log2 10^q) = (217706 q) >> 16 for
  // q in (-400, 350) (Section 10), plus 63 - l + u, plus the bias.
  int E = ((217706 * q) >> 16) + 63 - l + u + F::BIAS;
  if (E <= 0) {
    // Subnormal (Section 9.3): m sits 2-E places above the grid of the
    // smallest subnormal; shift by 1-E, then round on the last bit.  No ties
    // are possible here (Section 6).  Rounding up to 2^MBITS yields the
    // smallest normal number, whose bit pattern is that same integer.
    if (E <= -63) {
      r.bits = 0;
      r.status = ST_UNDERFLOW;
      return r;
    }
    m >>= (1 - E);
    m += (m & 1);
    m >>= 1;
    r.bits = m;
    r.status = m ? ST_OK : ST_UNDERFLOW;
    return r;
  }
  // Ties to even (Sections 8.1 and 9.1): only for q in [TIE_QMIN,
  // TIE_QMAX] ([-4, 23] for binary64, [-17, 10] for binary32), when the
  // product below m's lowest bit is zero (second word <= 1 and the bits of
  // the high word under m all zero) and m ends in binary 01: clear the
  // rounding bit so that the round step does not go up.
  if (lo <= 1 && q >= F::TIE_QMIN && q <= F::TIE_QMAX && (m & 3) == 1 &&
      (m << (u + F::SHIFT)) == hi)
    m &= ~1ull;
  // round to nearest on the last bit: (m + (m & 1)) >> 1 is (m + 1) >> 1
  m = (m + 1) >> 1;
  // Pack with the significand's leading bit added into the exponent field:
  // (E - 1) + 1 = E, and a rounding carry to 2^(MBITS+1) adds one more (the
  // significand field then being zero), as Algorithm 1's carry step does.
  // A field of EMAX_FIELD or more is infinity.
  const uint64_t bits = ((uint64_t)(E - 1) << F::MBITS) + m;
  const bool ovf = bits >= F::INF;
  r.bits = ovf ? F::INF : bits;
  r.status = ovf ? ST_OVERFLOW : ST_OK;
  return r;
}

// Quick exits of Algorithm 1 plus the product, for w != 0.  The product is
// formed with q clamped to the table's range and the exits applied after,
// so that the code has no data-dependent branch around the table access.
template <class F = F64>
FP_HD ElResult convert_wq(uint64_t w, int64_t q, const Pow5& tab, bool allow_abort) {
  const int qc = q < FP_POW5_QMIN ? FP_POW5_QMIN : (q > FP_POW5_QMAX ? FP_POW5_QMAX : (int)q);
  ElResult r = eisel_lemire<F>(w, qc, tab, allow_abort);
  if (q < FP_POW5_QMIN) {
    r.bits = 0;
    r.status = ST_UNDERFLOW;
  }
  if (q > FP_POW5_QMAX) {
    r.bits = F::INF;
    r.status = ST_OVERFLOW;
  }
  return r;
}

template <class F = F64>
FP_HD uint8_t status_of(uint64_t pos_bits) {
  if (pos_bits == 0) return ST_UNDERFLOW;  // nonzero text, zero result
  if (pos_bits == F::INF) return ST_OVERFLOW;
  return ST_OK;
}

// Nearest positive pattern of F to (m + d) 2^e2, where 0 <= d < 1 and d > 0
// exactly when `sticky` (hexadecimal floats are dyadic: the digits give the
// bits, so rounding needs no table and no big numbers).  m != 0.
template <class F>
FP_HD uint64_t hex_to_bits(uint64_t m, int64_t e2, bool sticky) {
  const int l = clz64(m);
  m <<= l;
  e2 -= l;  // value in [2^(e2+63), 2^(e2+64))
  const int64_t E = e2 + 63 + F::BIAS;  // biased exponent if normal
  if (E >= F::EMAX_FIELD) return F::INF;
  // bits of m below the last place kept: 63 - MBITS when normal, more when
  // subnormal (the last place is fixed at 2^(1 - BIAS - MBITS))
  const int64_t sh = (63 - F::MBITS) + (E < 1 ? 1 - E : 0);
  if (sh > 64) return 0;  // below half the smallest subnormal
  uint64_t q, rem, half;
  if (sh == 64) {
    q = 0;
    rem = m;
    half = 1ull << 63;
  } else {
    q = m >> sh;
    rem = m & ((1ull << sh) - 1);
    half = 1ull << (sh - 1);
  }
  if (rem > half || (rem == half && (sticky || (q & 1)))) q += 1;
  if (E < 1) return q;  // subnormal (reaching 2^MBITS gives the smallest normal)
  uint64_t Ef = (uint64_t)E;
  if (q >> (F::MBITS + 1)) {  // rounding carried into a new bit
    q >>= 1;
    Ef += 1;
    if (Ef >= (uint64_t)F::EMAX_FIELD) return F::INF;
  }
  return (Ef << F::MBITS) | (q & ((1ull << F::MBITS) - 1));
}

FP_HD int hex_digit(uint32_t c) {
  if (c - '0' < 10u) return (int)(c - '0');
  const uint32_t l = c | 0x20u;
  if (l - 'a' < 6u) return (int)(l - 'a' + 10);
  return -1;
}

FP_HD bool is_digit(uint32_t c) { return (c - '0') < 10u; }
FP_HD bool is_ws(uint32_t c) { return c == ' ' || c == '\t' || c == '\r'; }

// ---------------------------------------------------------------------------
// Field tokenizer for short fields held in shared memory (Section 4)
// ---------------------------------------------------------------------------
struct FieldResult {
  uint64_t bits;   // signed result pattern (valid unless pending)
  uint8_t status;  // ST_* or ST_PENDING
  uint8_t two_mul;
  uint8_t is_long;
  uint8_t long_settled;
};

// Parse s[0, n) (n <= LMAX) completely.  Up to 19 significant digits are
// accumulated into w; later digits only move the exponent (integer part)
// and feed a sticky flag.  With a nonzero sticky flag the value lies in
// (w 10^q, (w+1) 10^q), and if both ends round to the same double that is
// the answer (Section 11); otherwise the field is left pending.
template <class F = F64>
FP_HD FieldResult parse_short_field(const uint8_t* s, int n, const Pow5& tab,
                                    uint32_t grammar = GRAMMAR_DECIMAL) {
  FieldResult r;
  r.two_mul = 0;
  r.is_long = 0;
  r.long_settled = 0;
  int i = 0;
  while (i < n && is_ws(s[i])) i++;
  uint64_t sign = 0;
  if (i < n && (s[i] == '-' || (s[i] == '+' && grammar != GRAMMAR_JSON))) {
    sign = (s[i] == '-') ? F::SIGN : 0;
    i++;
  }
  if (grammar == GRAMMAR_HEX && i + 1 < n && s[i] == '0' && (s[i + 1] | 0x20) == 'x') {
    // hexadecimal float: up to 16 significant hex digits in m, the rest into
    // the exponent (integer digits) or the sticky flag
    i += 2;
    uint64_t m = 0;
    int kept = 0, nd = 0;
    int64_t e2 = 0;
    bool sticky = false;
    for (int part = 0; part < 2; part++) {
      if (part == 1) {
        if (i < n && s[i] == '.') i++;
        else break;
      }
      int d;
      while (i < n && (d = hex_digit(s[i])) >= 0) {
        if (kept < 16) {
          if (m || d) {
            m = m * 16 + (uint64_t)d;
            kept++;
          }
          if (part == 1) e2 -= 4;
        } else {
          if (part == 0) e2 += 4;
          sticky |= (d != 0);
        }
        i++;
        nd++;
      }
    }
    bool ok = nd > 0;
    if (ok && i < n && (s[i] | 0x20) == 'p') {
      i++;
      bool eneg = false;
      if (i < n && (s[i] == '+' || s[i] == '-')) {
        eneg = (s[i] == '-');
        i++;
      }
      int ne = 0;
      int64_t ex = 0;
      while (i < n && is_digit(s[i])) {
        if (ex < 100000000) ex = ex * 10 + (s[i] - '0');
        i++;
        ne++;
      }
      ok = ne > 0;
      e2 += eneg ? -ex : ex;
    }
    while (i < n && is_ws(s[i])) i++;
    if (!ok || i != n) {
      r.bits = F::QNAN;
      r.status = ST_INVALID;
      return r;
    }
    const uint64_t b = m ? hex_to_bits<F>(m, e2, sticky) : 0;
    r.bits = b | sign;
    r.status = m ? status_of<F>(b) : ST_OK;
    return r;
  }
  const int int_start = i;
  uint64_t w = 0;
  int nsig = 0;        // significant digits kept in w (<= 19)
  int exp_adj = 0;     // + integer digits dropped, - fraction digits kept
  bool sticky = false; // a nonzero digit was dropped
  int ndig = 0;
  while (i < n && is_digit(s[i])) {
    uint32_t d = s[i] - '0';
    if (nsig < 19) {
      if (nsig > 0 || d != 0) {
        w = w * 10 + d;
        nsig++;
      }
    } else {
      exp_adj++;
      sticky |= (d != 0);
    }
    i++;
    ndig++;
  }
  const int nint = ndig;
  bool point = false;
  if (i < n && s[i] == '.') {
    i++;
    point = true;
    while (i < n && is_digit(s[i])) {
      uint32_t d = s[i] - '0';
      if (nsig < 19) {
        if (nsig > 0 || d != 0) {
          w = w * 10 + d;
          nsig++;
        }
        exp_adj--;
      } else {
        sticky |= (d != 0);
      }
      i++;
      ndig++;
    }
  }
  bool ok = ndig > 0;
  if (grammar == GRAMMAR_JSON) {
    // an integer part without leading zeros; digits after a point
    ok = ok && nint > 0 && !(nint > 1 && s[int_start] == '0') && !(point && ndig == nint);
  }
  int64_t ex = 0;
  if (ok && i < n && (s[i] | 0x20) == 'e') {
    i++;
    bool eneg = false;
    if (i < n && (s[i] == '+' || s[i] == '-')) {
      eneg = (s[i] == '-');
      i++;
    }
    int ne = 0;
    while (i < n && is_digit(s[i])) {
      if (ex < 100000000) ex = ex * 10 + (s[i] - '0');
      i++;
      ne++;
    }
    ok = ne > 0;
    if (eneg) ex = -ex;
  }
  while (i < n && is_ws(s[i])) i++;
  ok = ok && (i == n);
  if (!ok) {
    r.bits = F::QNAN;
    r.status = ST_INVALID;
    return r;
  }
  if (w == 0) {
    r.bits = sign;
    r.status = ST_OK;
    return r;
  }
  const int64_t q = ex + exp_adj;
  ElResult a = convert_wq<F>(w, q, tab, true);
  r.two_mul = (uint8_t)a.two_mul;
  if (sticky) {
    r.is_long = 1;
    ElResult b = convert_wq<F>(w + 1, q, tab, true);
    r.two_mul |= (uint8_t)b.two_mul;
    if (a.bits == EL_ABORT || b.bits != a.bits) {
      r.status = ST_PENDING;
      r.bits = 0;
      return r;
    }
    r.long_settled = 1;
  } else if (a.bits == EL_ABORT) {
    r.status = ST_PENDING;
    r.bits = 0;
    return r;
  }
  r.bits = a.bits | sign;
  r.status = status_of<F>(a.bits);
  return r;
}


// ---------------------------------------------------------------------------
// SWAR fast path (Section 4; eight digits at a time as in Appendix D's
// string functions, with GPU byte-dot-product instructions for the values)
// ---------------------------------------------------------------------------

// (hi:lo) >> sh for sh in [0, 31].
FP_HD uint32_t fshr(uint32_t lo, uint32_t hi, uint32_t sh) {
#ifdef __CUDA_ARCH__
  return __funnelshift_r(lo, hi, sh);
#else
  return (uint32_t)((((uint64_t)hi << 32) | lo) >> (sh & 31));
#endif
}

FP_HD int ctz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __ffs(x) - 1;
#else
  return __builtin_ctz(x);
#endif
}

FP_HD int ctz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __ffsll((long long)x) - 1;
#else
  return __builtin_ctzll(x);
#endif
}

// Value of four ASCII digits, the first byte (lowest address) most
// significant: 1000 b0 + 100 b1 + 10 b2 + b3 - 1111 * '0'.
FP_HD uint32_t dig4(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __dp2a_hi(0x0001000Au, x, __dp2a_lo(0x006403E8u, x, 0u - 53328u));
#else
  return 1000u * (x & 0xFF) + 100u * ((x >> 8) & 0xFF) + 10u * ((x >> 16) & 0xFF) + (x >> 24) -
         53328u;
#endif
}

FP_HD uint32_t dig8(uint32_t a, uint32_t b) { return dig4(a) * 10000u + dig4(b); }

// Byte permute: byte i of the result is byte ((sel >> 4i) & 7) of (y:x).
FP_HD uint32_t byte_perm(uint32_t x, uint32_t y, uint32_t sel) {
#ifdef __CUDA_ARCH__
  return __byte_perm(x, y, sel);
#else
  const uint64_t v = ((uint64_t)y << 32) | x;
  uint32_t r = 0;
  for (int i = 0; i < 4; i++) r |= (uint32_t)((v >> (8 * ((sel >> (4 * i)) & 7))) & 0xFF) << (8 * i);
  return r;
#endif
}

FP_HD int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz(x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

// Sum of the four unsigned byte products of a and b, plus c.
FP_HD uint32_t dp4a_u(uint32_t a, uint32_t b, uint32_t c) {
#ifdef __CUDA_ARCH__
  return __dp4a(a, b, c);
#else
  for (int i = 0; i < 4; i++) c += ((a >> (8 * i)) & 0xFF) * ((b >> (8 * i)) & 0xFF);
  return c;
#endif
}

// Two words of flag bytes (each 0x80 or 0) to 128 times an 8-bit mask, plus
// c: bit b for byte b of w0, bit 4 + b for byte b of w1 (a byte dot product
// weighs each flag by 2^b or 2^(4+b)).
FP_HD uint32_t flag_pair(uint32_t w0, uint32_t w1, uint32_t c = 0u) {
  return dp4a_u(w1, 0x80402010u, dp4a_u(w0, 0x08040201u, c));
}

// 0x80 in every byte of t that is zero, exactly.
FP_HD uint32_t zero_bytes(uint32_t t) {
  return ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u;
}

// 0x80 in every byte of w equal to the byte repeated in pat, exactly, for a
// pattern byte below 0x80: zero_bytes(w ^ pat), where the final test can use
// w's own bit 7 (pat's is clear), so the XOR costs nothing extra.
FP_HD uint32_t sep_flags_one(uint32_t w, uint32_t pat) {
  return ~((((w ^ pat) & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
}

// The same for bytes equal to either of two patterns (both below 0x80).
FP_HD uint32_t sep_flags_two(uint32_t w, uint32_t p1, uint32_t p2) {
  const uint32_t s1 = ((w ^ p1) & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
  const uint32_t s2 = ((w ^ p2) & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
  return ~((s1 & s2) | w) & 0x80808080u;
}

struct FastToken {
  uint64_t w;     // decimal significand (< 10^19)
  int q;          // decimal exponent
  uint64_t sign;
  // where the significand starts and ends and where its point is (-1: none);
  // used by the JSON check, dead code otherwise
  int s1, send, dot;
};

// 0x80 in every byte of x that is not an ASCII digit, exactly: for a byte b
// below 0x80, (b ^ '0') is below 10 exactly for '0'..'9', and adding 0x76
// sets bit 7 exactly when it is not (the sum stays below 0x100, so nothing
// carries into the next byte); bytes from 0x80 up have bit 7 already.
FP_HD uint32_t nondigit_exact(uint32_t x) {
  const uint32_t t = (x ^ 0x30303030u) & 0x7F7F7F7Fu;
  return ((t + 0x76767676u) | x) & 0x80808080u;
}

// Shared-memory tables of the window tokenizer (1,664 bytes), so that the
// per-field byte moves are table lookups instead of computed masks:
//   sel[j][d]        byte-permute selector of window word j that moves the
//                    bytes at or before window position d (a point) one place
//                    toward the end, over the point (d = 24: no point, the
//                    identity);
//   keep_from[j][l]  mask of the bytes of word j at window positions >= l;
//   keep_below[j-4][m-16]  masks of words 4 and 5 for the positions below m
//                    (an exponent marker at m >= 16).
// The position is the inner index and rows are 32 words, so the lanes of a
// warp, each looking up its own field's position in the same row, read 32
// different banks (no shared-memory bank conflicts).
struct WindowTables {
  uint32_t sel[6][32];
  uint32_t keep_from[6][32];
  uint32_t keep_below[2][16];
};
constexpr int WINDOW_TABLE_WORDS = (int)(sizeof(WindowTables) / 4);

// Word i of the tables (in the struct's order).
FP_HD uint32_t window_table_word(int i) {
  if (i < 6 * 32) {  // sel[j][d]
    const int j = i >> 5, d = i & 31;
    if (d >= 24) return 0x7654u;
    int c = d + 1 - 4 * j;  // bytes of word j at or before the point
    c = c < 0 ? 0 : (c > 4 ? 4 : c);
    const uint32_t m = 0xFFFFu >> (16 - 4 * c);
    return (0x6543u & m) | (0x7654u & ~m & 0xFFFFu);
  }
  i -= 6 * 32;
  if (i < 6 * 32) {  // keep_from[j][l]
    const int j = i >> 5, l = i & 31;
    uint32_t m = 0;
    for (int b = 0; b < 4; b++)
      if (4 * j + b >= l) m |= 0xFFu << (8 * b);
    return m;
  }
  i -= 6 * 32;
  const int j = 4 + (i >> 4), mk = 16 + (i & 15);  // keep_below[j-4][mk-16]
  uint32_t m = 0;
  for (int b = 0; b < 4; b++)
    if (4 * j + b < mk) m |= 0xFFu << (8 * b);
  return m;
}

// Straight-line tokenizer for the common field shape (Section 4)
//     [+-] digits-with-at-most-one-'.' [ [eE] [+-] d{1,4} ]
// with at most 24 bytes after the sign and a value of the significand
// below 10^19 when the exponent part's bytes count as trailing zero digits.
// s is the field's first byte and e its terminator (tile offsets; the bytes
// in [s, e) are text).  The 24 bytes that end at e are read as one window;
// exact per-byte non-digit flags locate the point and the exponent marker;
// the bytes up to the point move one place over it (table selectors), the
// bytes before the significand and the exponent part become '0' (table
// masks), and the 20 low digits are converted four at a time.  Every field
// of this shape runs the same instructions.  Returns false for anything
// else; the general tokenizer then decides (with identical results for the
// shapes accepted here).  tile is 4-byte aligned; reads may touch up to 28
// bytes before e and 4 after it, and those bytes never change the result.
FP_HD bool parse_window(const uint8_t* tile, const WindowTables& wt, int s, int e, FastToken& t) {
  const int L = e - s;
  if (L < 1 || L > 25) return false;
  const uint32_t c0 = tile[s];
  const int sg = (c0 == '-') | (c0 == '+');
  t.sign = (c0 == '-') ? SIGN_BIT : 0;
  const int s1 = s + sg;
  const int tsig = 24 - (e - s1);  // window position of the first byte after the sign
  if (tsig < 0) return false;
  // the window [e - 24, e)
  const int w0 = e - 24;
  const uint32_t* t32 = reinterpret_cast<const uint32_t*>(tile);
  const int i0 = w0 >> 2;  // floor, also for negative w0
  const uint32_t sh = (uint32_t)(w0 & 3) * 8;
  uint32_t x[6];
  {
    uint32_t W[7];
#pragma unroll
    for (int j = 0; j < 7; j++) W[j] = t32[i0 + j];
#pragma unroll
    for (int j = 0; j < 6; j++) x[j] = fshr(W[j], W[j + 1], sh);
  }
  // bit i: window byte i is not a digit (bytes before the field cleared)
  uint32_t M;
  {
    uint32_t f[6];
#pragma unroll
    for (int j = 0; j < 6; j++) f[j] = nondigit_exact(x[j]);
    // 128 M, the higher pairs carried in the dot products' accumulator (128 M
    // < 2^31)
    uint32_t t = flag_pair(f[4], f[5]);
    t = flag_pair(f[2], f[3], t << 8);
    M = flag_pair(f[0], f[1], t << 8) >> 7;
    M &= 0xFFFFFFFFu << tsig;
  }
  // An exponent: the last non-digit is an 'e' or 'E', or a sign right after
  // one, and 1 to 4 digits follow.  em: where the significand ends.
  const int hb = 31 - clz32(M);  // -1 when M == 0
  int em = 24, ex = 0;
  if (hb >= 19 && hb <= 22) {
    const uint32_t ch = tile[w0 + hb];
    const int hs = (ch == '+') | (ch == '-');
    const int m = hb - hs;
    if ((tile[w0 + m] | 0x20u) == 'e' && m > tsig) {
      em = m;
      const uint32_t keep = 0xFFFFFFFFu << (8 * (hb - 19));  // the 23 - hb exponent digits
      ex = (int)dig4((x[5] & keep) | (0x30303030u & ~keep));
      if (ch == '-') ex = -ex;
    }
  }
  // the significand: digits and at most one non-digit, which is the point
  const uint32_t Ms = M & ((1u << em) - 1u);
  if (Ms & (Ms - 1u)) return false;
  const int hp = Ms != 0;
  const int dpos = hp ? ctz32(Ms) : 24;
  if (hp && tile[w0 + dpos] != '.') return false;
  const int lo = tsig + hp;  // the first digit's position once the point is gone
  if (em - lo < 1) return false;  // no digit at all
  {
    uint32_t prev = 0x30303030u;
#pragma unroll
    for (int j = 0; j < 6; j++) {
      const uint32_t xj = x[j];
      x[j] = byte_perm(prev, xj, wt.sel[j][dpos]);
      prev = xj;
    }
    uint32_t k[6];
#pragma unroll
    for (int j = 0; j < 6; j++) k[j] = wt.keep_from[j][lo];
    k[4] &= wt.keep_below[0][em - 16];
    k[5] &= wt.keep_below[1][em - 16];
#pragma unroll
    for (int j = 0; j < 6; j++) x[j] = (x[j] & k[j]) | (0x30303030u & ~k[j]);
  }
  // the five high positions zero, so that the value is below 10^19
  if (x[0] != 0x30303030u || (x[1] & 0xFFu) != 0x30u) return false;
  // two 8-digit halves in 32-bit arithmetic, then two 64-bit steps
  t.w = ((uint64_t)dig4(x[1]) * 100000000u + dig8(x[2], x[3])) * 100000000ull + dig8(x[4], x[5]);
  // the last digit sits at window position 23 once the exponent part is
  // zeros: with a point, 23 - dpos of the digits follow it
  t.q = ex + (hp ? dpos - 23 : em - 24);
  t.s1 = s1;
  t.send = w0 + em;
  t.dot = hp ? w0 + dpos : -1;
  return true;
}

// The JSON number grammar on a field parse_window accepted: no '+', a digit
// before the point, a digit after it, and no leading zero before another
// digit.
FP_HD bool json_ok_fast(const uint8_t* tile, int s, const FastToken& t) {
  const uint32_t a = tile[t.s1];
  bool bad = tile[s] == '+';
  bad |= a == '.';
  bad |= t.dot >= 0 && t.dot + 1 == t.send;
  bad |= a == '0' && t.s1 + 1 < t.send && tile[t.s1 + 1] != '.';
  return !bad;
}


// Value of four hexadecimal digit values (bytes 0-15), the first byte most
// significant: 4096 v0 + 256 v1 + 16 v2 + v3.
FP_HD uint32_t hex4(uint32_t v) {
#ifdef __CUDA_ARCH__
  return __dp2a_hi(0x00010010u, v, __dp2a_lo(0x01001000u, v, 0u));
#else
  return 4096u * (v & 0xFF) + 256u * ((v >> 8) & 0xFF) + 16u * ((v >> 16) & 0xFF) + (v >> 24);
#endif
}

// Straight-line tokenizer for the common shape of a hexadecimal float
// (Appendix C's %a form, Python's float.hex()):
//     [+-] 0 (x|X) hexdigits-with-at-most-one-'.' (p|P) [+-] d{1,4}
// with at most 24 bytes after the sign and a significand below 2^64 (at
// most 16 hexadecimal digits from the first nonzero one).  The same window
// as parse_window: the 24 bytes ending at the terminator e.  Exact per-byte
// flags mark the bytes that are not hexadecimal digits (and, in the last
// two words, not decimal digits: the exponent's); the point is moved out
// and the bytes outside the significand set to '0' with parse_window's
// tables; four digit values per byte-dot-product pair give the 96-bit
// window, which is shifted right by the exponent part's length.  The value
// is exactly significand x 2^(exponent - 4 x fraction digits), rounded
// once (hex_to_bits).  Returns false for any other shape; the general
// tokenizer then decides (with identical results for the shapes accepted
// here).  Reads as parse_window does.
template <class F>
FP_HD bool parse_hex_window(const uint8_t* tile, const WindowTables& wt, int s, int e,
                            uint64_t& bits, uint8_t& status) {
  const int L = e - s;
  if (L < 5 || L > 25) return false;
  const uint32_t c0 = tile[s];
  const int sg = (c0 == '-') | (c0 == '+');
  const int s1 = s + sg;
  const int tsig = 24 - (e - s1);  // window position of the "0x"
  if (tsig < 0 || tile[s1] != '0' || (tile[s1 + 1] | 0x20u) != 'x') return false;
  const int w0 = e - 24;
  const uint32_t* t32 = reinterpret_cast<const uint32_t*>(tile);
  const int i0 = w0 >> 2;
  const uint32_t sh = (uint32_t)(w0 & 3) * 8;
  uint32_t x[6];
  {
    uint32_t W[7];
#pragma unroll
    for (int j = 0; j < 7; j++) W[j] = t32[i0 + j];
#pragma unroll
    for (int j = 0; j < 6; j++) x[j] = fshr(W[j], W[j + 1], sh);
  }
  // per byte (bit 7 of a flag byte): nd = not a decimal digit (exact, as
  // nondigit_exact); nl = not a letter a-f or A-F: with the case bit set,
  // (byte ^ 0x60) & 0x7F lies in [1, 6] exactly for those letters
  uint32_t fh[6];  // not a hexadecimal digit
  uint32_t fd4 = 0, fd5 = 0;
#pragma unroll
  for (int j = 0; j < 6; j++) {
    const uint32_t t1 = (x[j] ^ 0x30303030u) & 0x7F7F7F7Fu;
    const uint32_t nd = (t1 + 0x76767676u) | x[j];
    const uint32_t t2 = ((x[j] | 0x20202020u) ^ 0x60606060u) & 0x7F7F7F7Fu;
    const uint32_t nl = (t2 + 0x79797979u) | ~(t2 + 0x7F7F7F7Fu) | x[j];
    fh[j] = nd & nl & 0x80808080u;
    if (j == 4) fd4 = nd & 0x80808080u;
    if (j == 5) fd5 = nd & 0x80808080u;
  }
  const int m0 = tsig + 2;  // first byte after the "0x"
  uint32_t MH;              // bit i: window byte i is not a hexadecimal digit
  {
    uint32_t t = flag_pair(fh[4], fh[5]);
    t = flag_pair(fh[2], fh[3], t << 8);
    MH = (flag_pair(fh[0], fh[1], t << 8) >> 7) & (0xFFFFFFFFu << m0);
  }
  // The exponent: the last byte that is not a hexadecimal digit is a 'p'
  // or a sign right after one, and 1 to 4 decimal digits follow it.
  const int hb = 31 - clz32(MH);
  if (hb < 19 || hb > 22) return false;
  const uint32_t MD = ((flag_pair(fd4, fd5) >> 7) << 16) & (0xFFFFFFFFu << (hb + 1));
  if (MD != 0) return false;  // a letter among the exponent digits
  const uint32_t ch = tile[w0 + hb];
  const int hs = (ch == '+') | (ch == '-');
  const int pp = hb - hs;  // the marker's position
  if ((tile[w0 + pp] | 0x20u) != 'p' || pp <= m0) return false;
  const uint32_t keep_e = 0xFFFFFFFFu << (8 * (hb - 19));  // the 23 - hb exponent digits
  int ex = (int)dig4((x[5] & keep_e) | (0x30303030u & ~keep_e));
  if (ch == '-') ex = -ex;
  // the significand [m0, pp): hexadecimal digits and at most one point
  const uint32_t Mp = MH & ((1u << pp) - 1u);
  if (Mp & (Mp - 1u)) return false;
  const int hp = Mp != 0;
  const int dpos = hp ? ctz32(Mp) : 24;
  if (hp && tile[w0 + dpos] != '.') return false;
  const int lo = m0 + hp;  // the first digit's position once the point is gone
  if (pp - lo < 1) return false;  // no digit at all
  {
    uint32_t prev = 0x30303030u;
#pragma unroll
    for (int j = 0; j < 6; j++) {
      const uint32_t xj = x[j];
      x[j] = byte_perm(prev, xj, wt.sel[j][dpos]);
      prev = xj;
    }
    uint32_t k[6];
#pragma unroll
    for (int j = 0; j < 6; j++) k[j] = wt.keep_from[j][lo];
    k[4] &= wt.keep_below[0][pp - 16];
    k[5] &= wt.keep_below[1][pp - 16];
#pragma unroll
    for (int j = 0; j < 6; j++) x[j] = (x[j] & k[j]) | (0x30303030u & ~k[j]);
  }
  // digit values (letters have bit 6 set: their low nibble + 9), four per
  // 16-bit group, the window as three 32-bit words
  uint32_t N[6];
#pragma unroll
  for (int j = 0; j < 6; j++)
    N[j] = hex4((x[j] & 0x0F0F0F0Fu) + 9u * ((x[j] >> 6) & 0x01010101u));
  const uint32_t v_hi = (N[0] << 16) | N[1], v_mid = (N[2] << 16) | N[3], v_lo = (N[4] << 16) | N[5];
  // the 24 - pp zero digits from the exponent part shifted out
  const uint32_t zs = 4u * (uint32_t)(24 - pp);  // 8..24
  if (v_hi >> zs) return false;  // more than 64 bits of significand
  const uint64_t m = ((uint64_t)fshr(v_mid, v_hi, zs) << 32) | fshr(v_lo, v_mid, zs);
  const int64_t e2 = (int64_t)ex - 4 * (hp ? pp - 1 - dpos : 0);
  const uint64_t b = m ? hex_to_bits<F>(m, e2, false) : 0;
  bits = b | (c0 == '-' ? F::SIGN : 0);
  status = m ? status_of<F>(b) : (uint8_t)ST_OK;
  return true;
}

}  // namespace fp
