// fp_device.cuh -- device-side building blocks of the parser (sm_103a).
//
// Algorithm 1 of the paper (Sections 6-9) on a decimal significand w < 2^64
// and exponent q, against the 128-bit power-of-five table; the field
// grammar of Section 4; the 19-digit truncation check of Section 10.
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
  ST_PENDING = 0xFF,         // internal result of the short-field parser
  ST_PENDING_QUEUED = 0xFE,  // stored status: pending, listed in the fallback queue
  ST_PENDING_SCAN = 0xFF,    // stored status: pending, found by scanning its chunk
};

constexpr uint64_t QNAN_BITS = 0x7FF8000000000000ull;
constexpr uint64_t INF_BITS = 0x7FF0000000000000ull;
constexpr uint64_t SIGN_BIT = 0x8000000000000000ull;
constexpr uint64_t EL_ABORT = ~0ull;  // never a positive binary64 pattern

// Fields longer than this many bytes are handed to the fallback kernel.
constexpr int LMAX = 64;

// Device error codes (mirrors fp_err_t values).
constexpr uint32_t DERR_TIMEOUT = 5;
constexpr uint32_t DERR_INTERNAL = 6;

// Counters kept per CTA and added to the stream's totals.
enum {
  CNT_FIELDS = 0,
  CNT_ONE_MUL,
  CNT_TWO_MUL,
  CNT_LONG,
  CNT_LONG_SETTLED,
  CNT_FALLBACK,
  CNT_FALLBACK_BIGNUM,
  CNT_QUEUE_OVERFLOW,
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
struct ElResult {
  uint64_t bits;  // positive binary64 pattern, or EL_ABORT
  int two_mul;    // 1 if the second 64x64 product was needed
};

// w in [1, 2^64), q in [FP_POW5_QMIN, FP_POW5_QMAX]; tab points at the table
// (shared memory).  allow_abort = false returns the rounded truncated
// product even where Algorithm 1 would give up; that value is then within
// one unit in the last place of the correct result (the fallback kernel
// uses it as its first candidate).
FP_HD ElResult eisel_lemire(uint64_t w, int q, const uint64_t* tab,
                                                 bool allow_abort) {
  ElResult r;
  r.two_mul = 0;
  // Normalise the decimal significand into [2^63, 2^64) (Section 7).
  int l = clz64(w);
  w <<= l;
  const uint64_t thi = tab[2 * (q - FP_POW5_QMIN)];
  // z = (T[q] * w) / 2^64, truncated: first the product with the high word.
  uint64_t lo = w * thi;
  uint64_t hi = mulhi64(w, thi);
  // Unless the low 9 bits of the high word are all ones, the top 55 bits
  // are exact and one product suffices (Sections 7 and 8).
  if ((hi & 0x1FF) == 0x1FF) {
    const uint64_t tlo = tab[2 * (q - FP_POW5_QMIN) + 1];
    uint64_t h2 = mulhi64(w, tlo);
    lo += h2;
    hi += (lo < h2);
    r.two_mul = 1;
  }
  // The second word all ones outside [-27, 55]: a third product could
  // still carry into the top word, so give up (Algorithm 1).
  if (allow_abort && lo == ~0ull && (q < -27 || q > 55)) {
    r.bits = EL_ABORT;
    return r;
  }
  // 54 significant bits (53 plus one rounding bit) below a possible
  // leading zero bit u of the 128-bit product.
  const int u = (int)(hi >> 63);
  uint64_t m = hi >> (u + 9);
  // Biased binary exponent: floor(log2 10^q) = (217706 q) >> 16 for
  // q in (-400, 350) (Section 9), plus 63 - l + u, plus the bias 1023.
  int E = ((217706 * q) >> 16) + 63 - l + u + 1023;
  if (E <= 0) {
    // Subnormal (Section 8.3): the 54-bit m sits 2-E places above the
    // 2^-1074 grid; shift by 1-E, then round on the last bit.  No ties are
    // possible here (Section 5).  Rounding up to 2^52 yields the smallest
    // normal number, whose bit pattern is that same integer.
    if (E <= -63) {
      r.bits = 0;
      return r;
    }
    m >>= (1 - E);
    m += (m & 1);
    m >>= 1;
    r.bits = m;
    return r;
  }
  // Ties to even (Sections 7.1 and 8.1): only for q in [-4, 23], when the
  // product below m's lowest bit is zero (second word <= 1 and the bits of
  // the high word under m all zero) and m ends in binary 01: clear the
  // rounding bit so that the round step does not go up.
  if (lo <= 1 && q >= -4 && q <= 23 && (m & 3) == 1 && (m << (u + 9)) == hi) m &= ~1ull;
  m += (m & 1);
  m >>= 1;
  if (m >= (1ull << 53)) {  // rounding carried into a new bit
    m = 1ull << 52;
    E += 1;
  }
  if (E >= 2047) {
    r.bits = INF_BITS;
    return r;
  }
  r.bits = ((uint64_t)E << 52) | (m & ((1ull << 52) - 1));
  return r;
}

// Quick exits of Algorithm 1 plus the product, for w != 0.
FP_HD ElResult convert_wq(uint64_t w, int64_t q, const uint64_t* tab,
                                               bool allow_abort) {
  ElResult r;
  r.two_mul = 0;
  if (q < FP_POW5_QMIN) {
    r.bits = 0;
    return r;
  }
  if (q > FP_POW5_QMAX) {
    r.bits = INF_BITS;
    return r;
  }
  return eisel_lemire(w, (int)q, tab, allow_abort);
}

FP_HD uint8_t status_of(uint64_t pos_bits) {
  if (pos_bits == 0) return ST_UNDERFLOW;  // nonzero text, zero result
  if (pos_bits == INF_BITS) return ST_OVERFLOW;
  return ST_OK;
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
// the answer (Section 10); otherwise the field is left pending.
FP_HD FieldResult parse_short_field(const uint8_t* s, int n,
                                                         const uint64_t* tab) {
  FieldResult r;
  r.two_mul = 0;
  r.is_long = 0;
  r.long_settled = 0;
  int i = 0;
  while (i < n && is_ws(s[i])) i++;
  uint64_t sign = 0;
  if (i < n && (s[i] == '+' || s[i] == '-')) {
    sign = (s[i] == '-') ? SIGN_BIT : 0;
    i++;
  }
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
  if (i < n && s[i] == '.') {
    i++;
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
    r.bits = QNAN_BITS;
    r.status = ST_INVALID;
    return r;
  }
  if (w == 0) {
    r.bits = sign;
    r.status = ST_OK;
    return r;
  }
  const int64_t q = ex + exp_adj;
  ElResult a = convert_wq(w, q, tab, true);
  r.two_mul = (uint8_t)a.two_mul;
  if (sticky) {
    r.is_long = 1;
    ElResult b = convert_wq(w + 1, q, tab, true);
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
  r.status = status_of(a.bits);
  return r;
}

}  // namespace fp
