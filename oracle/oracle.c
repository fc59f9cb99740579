/*
 * oracle.c -- exact decimal text -> nearest IEEE-754 binary64 or binary32
 * (ties to even).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle for the GPU path:
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with
 * the CUDA library, and the CUDA library never calls it.
 *
 * What it computes is the plain definition of the problem (Section 1 and
 * Section 2 of the paper): the binary64 (or binary32, Section 2's other
 * format) value nearest to the exact rational value of the decimal string,
 * with ties broken toward the even significand,
 * signed zero and signed infinity kept (the sign is applied last, Algorithm 1
 * handles negatives by flipping the sign bit).  No table, no truncated
 * product, no fast path: the decimal value is held as an exact ratio of two
 * arbitrary-precision naturals and rounded by integer division.
 *
 * Grammar of one field (Section 4 lists the choices; this is the reading
 * taken here):
 *     [ \t\r]*  [+-]?  ( d+ ( '.' d* )? | '.' d+ )  ( [eE] [+-]? d+ )?  [ \t\r]*
 * A field that does not match as a whole is INVALID (value = quiet NaN).
 * An explicit exponent whose magnitude exceeds 10^15 saturates at 10^15
 * (Section 4 allows stopping the update above a threshold); this is exact
 * for every field shorter than about 10^15 bytes.
 *
 * Status byte: 0 OK, 1 INVALID, 2 OVERFLOW (finite text, |value| rounds to
 * infinity), 3 UNDERFLOW (nonzero text, value rounds to zero).
 *
 * Buffers: fields are the byte runs between separators {delim, '\n'}.  A
 * buffer that ends in a separator has no trailing empty field; an empty
 * field elsewhere is INVALID.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

enum { OR_OK = 0, OR_INVALID = 1, OR_OVERFLOW = 2, OR_UNDERFLOW = 3 };

#define OR_EXP_SAT 1000000000000000LL /* 10^15 */
#define OR_QNAN_BITS 0x7FF8000000000000ULL
#define OR_INF_BITS 0x7FF0000000000000ULL

/* An IEEE-754 binary format (Section 2): p significand bits (the leading
 * one included), normal exponents emin..emax, and the decimal-magnitude
 * limits of the cheap range exits in convert_exact.                        */
typedef struct {
    int p;
    int emin, emax;
    int dec_ovf; /* nd-1+E >= dec_ovf  =>  V >= 10^dec_ovf, beyond the largest finite */
    int dec_unf; /* nd+E <= dec_unf    =>  V < 10^dec_unf, below half the smallest subnormal */
    uint64_t inf_bits, qnan_bits, sign_bit;
} fmt;
/* 1e309 > 2^1024 and 1e-324 < 2^-1075; 1e39 > 2^128 and 1e-46 < 2^-150. */
static const fmt FMT64 = {53, -1022, 1023, 309, -324, OR_INF_BITS, OR_QNAN_BITS,
                          0x8000000000000000ULL};
static const fmt FMT32 = {24, -126, 127, 39, -46, 0x7F800000ULL, 0x7FC00000ULL, 0x80000000ULL};

/* ------------------------------------------------------------------------ */
/* Arbitrary-precision naturals: little-endian base-2^32 limbs, normalised   */
/* so that the top limb is nonzero (n == 0 means the value 0).               */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t *d;
    size_t n;
    size_t cap;
} big;

static int big_reserve(big *a, size_t cap) {
    if (cap <= a->cap) return 0;
    size_t nc = a->cap ? a->cap : 8;
    while (nc < cap) nc *= 2;
    uint32_t *p = (uint32_t *)realloc(a->d, nc * sizeof(uint32_t));
    if (!p) return -1;
    a->d = p;
    a->cap = nc;
    return 0;
}

static void big_free(big *a) {
    free(a->d);
    a->d = NULL;
    a->n = a->cap = 0;
}

static void big_trim(big *a) {
    while (a->n && a->d[a->n - 1] == 0) a->n--;
}

static int big_set_u64(big *a, uint64_t v) {
    if (big_reserve(a, 2)) return -1;
    a->d[0] = (uint32_t)v;
    a->d[1] = (uint32_t)(v >> 32);
    a->n = 2;
    big_trim(a);
    return 0;
}

static int big_copy(big *dst, const big *src) {
    if (big_reserve(dst, src->n + 1)) return -1;
    if (src->n) memcpy(dst->d, src->d, src->n * sizeof(uint32_t));
    dst->n = src->n;
    return 0;
}

/* a = a * m + c */
static int big_mul_add_small(big *a, uint32_t m, uint32_t c) {
    uint64_t carry = c;
    for (size_t i = 0; i < a->n; i++) {
        uint64_t t = (uint64_t)a->d[i] * m + carry;
        a->d[i] = (uint32_t)t;
        carry = t >> 32;
    }
    if (carry) {
        if (big_reserve(a, a->n + 1)) return -1;
        a->d[a->n++] = (uint32_t)carry;
    }
    big_trim(a);
    return 0;
}

/* a = a * 10^k */
static int big_mul_pow10(big *a, int64_t k) {
    while (k >= 9) {
        if (big_mul_add_small(a, 1000000000u, 0)) return -1;
        k -= 9;
    }
    uint32_t p = 1;
    while (k-- > 0) p *= 10;
    if (p != 1 && big_mul_add_small(a, p, 0)) return -1;
    return 0;
}

/* a = a * 2^s */
static int big_shl(big *a, uint64_t s) {
    if (a->n == 0 || s == 0) return 0;
    size_t w = (size_t)(s / 32);
    unsigned b = (unsigned)(s % 32);
    if (big_reserve(a, a->n + w + 1)) return -1;
    size_t n = a->n;
    a->d[n + w] = 0;
    for (size_t i = n; i-- > 0;) {
        uint32_t v = a->d[i];
        if (b) {
            a->d[i + w + 1] |= v >> (32 - b);
            a->d[i + w] = v << b;
        } else {
            a->d[i + w] = v;
        }
    }
    for (size_t i = 0; i < w; i++) a->d[i] = 0;
    a->n = n + w + 1;
    big_trim(a);
    return 0;
}

/* a = floor(a / 2) */
static void big_shr1(big *a) {
    for (size_t i = 0; i < a->n; i++) {
        uint32_t hi = (i + 1 < a->n) ? a->d[i + 1] : 0;
        a->d[i] = (a->d[i] >> 1) | (hi << 31);
    }
    big_trim(a);
}

static int big_cmp(const big *a, const big *b) {
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (size_t i = a->n; i-- > 0;) {
        if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
    }
    return 0;
}

/* a = a - b, requires a >= b */
static void big_sub(big *a, const big *b) {
    int64_t borrow = 0;
    for (size_t i = 0; i < a->n; i++) {
        int64_t t = (int64_t)a->d[i] - (i < b->n ? (int64_t)b->d[i] : 0) - borrow;
        borrow = t < 0;
        a->d[i] = (uint32_t)(t + (borrow ? ((int64_t)1 << 32) : 0));
    }
    big_trim(a);
}

static uint64_t big_bitlen(const big *a) {
    if (a->n == 0) return 0;
    uint32_t top = a->d[a->n - 1];
    unsigned bits = 0;
    while (top) {
        bits++;
        top >>= 1;
    }
    return (uint64_t)(a->n - 1) * 32 + bits;
}

/* ------------------------------------------------------------------------ */
/* Tokenizer                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int negative;
    int hex; /* hexadecimal significand, binary exponent */
    /* the digit characters of the significand, possibly split by one '.' */
    const char *int_digits;
    size_t n_int;
    const char *frac_digits;
    size_t n_frac;
    int64_t exp10; /* explicit exponent (of 10, or of 2 when hex), saturated */
} token;

/* Field grammars (the library's readings):
 *   OR_GRAMMAR_DEFAULT  the decimal grammar in the header comment;
 *   OR_GRAMMAR_HEX      that, or a hexadecimal float (Appendix C's form as
 *                       printed by %a; the binary exponent is optional, as
 *                       strtod reads it):
 *                         [ \t\r]* [+-]? 0[xX] ( h+ ( '.' h* )? | '.' h+ )
 *                         ( [pP] [+-]? d+ )? [ \t\r]*
 *   OR_GRAMMAR_JSON     the JSON number grammar, with blanks around it:
 *                         [ \t\r]* '-'? ( '0' | [1-9] d* ) ( '.' d+ )?
 *                         ( [eE] [+-]? d+ )? [ \t\r]*                       */
enum { OR_GRAMMAR_DEFAULT = 0, OR_GRAMMAR_HEX = 1, OR_GRAMMAR_JSON = 2 };

static int is_ws(char c) { return c == ' ' || c == '\t' || c == '\r'; }
static int is_digit(char c) { return c >= '0' && c <= '9'; }

/* returns 0 on a whole-field match, -1 otherwise */
static int hex_value(char c) {
    if (c >= '0' && c <= '9') return c - '0';
    if (c >= 'a' && c <= 'f') return c - 'a' + 10;
    if (c >= 'A' && c <= 'F') return c - 'A' + 10;
    return -1;
}

/* The exponent part after 'e'/'p' at s[*pi]: [+-]? d+, saturated. */
static int read_exponent(const char *s, size_t n, size_t *pi, int64_t *out) {
    size_t i = *pi;
    int eneg = 0;
    if (i < n && (s[i] == '+' || s[i] == '-')) {
        eneg = (s[i] == '-');
        i++;
    }
    size_t nd = 0;
    int64_t e = 0;
    while (i < n && is_digit(s[i])) {
        if (e < OR_EXP_SAT) e = e * 10 + (s[i] - '0');
        if (e > OR_EXP_SAT) e = OR_EXP_SAT;
        i++;
        nd++;
    }
    if (nd == 0) return -1; /* the exponent needs digits */
    *out = eneg ? -e : e;
    *pi = i;
    return 0;
}

static int tokenize(const char *s, size_t n, int grammar, token *t) {
    size_t i = 0;
    memset(t, 0, sizeof(*t));
    while (i < n && is_ws(s[i])) i++;
    if (i < n && (s[i] == '-' || (s[i] == '+' && grammar != OR_GRAMMAR_JSON))) {
        t->negative = (s[i] == '-');
        i++;
    }
    if (grammar == OR_GRAMMAR_HEX && i + 1 < n && s[i] == '0' && (s[i + 1] | 0x20) == 'x') {
        t->hex = 1;
        i += 2;
        t->int_digits = s + i;
        while (i < n && hex_value(s[i]) >= 0) {
            i++;
            t->n_int++;
        }
        if (i < n && s[i] == '.') {
            i++;
            t->frac_digits = s + i;
            while (i < n && hex_value(s[i]) >= 0) {
                i++;
                t->n_frac++;
            }
        }
        if (t->n_int + t->n_frac == 0) return -1;
        if (i < n && (s[i] | 0x20) == 'p') {
            i++;
            if (read_exponent(s, n, &i, &t->exp10)) return -1;
        }
    } else {
        t->int_digits = s + i;
        while (i < n && is_digit(s[i])) {
            i++;
            t->n_int++;
        }
        if (grammar == OR_GRAMMAR_JSON) {
            /* an integer part is required, without leading zeros */
            if (t->n_int == 0) return -1;
            if (t->n_int > 1 && t->int_digits[0] == '0') return -1;
        }
        if (i < n && s[i] == '.') {
            i++;
            t->frac_digits = s + i;
            while (i < n && is_digit(s[i])) {
                i++;
                t->n_frac++;
            }
            if (grammar == OR_GRAMMAR_JSON && t->n_frac == 0) return -1;
        }
        if (t->n_int + t->n_frac == 0) return -1; /* needs at least one digit */
        if (i < n && (s[i] == 'e' || s[i] == 'E')) {
            i++;
            if (read_exponent(s, n, &i, &t->exp10)) return -1;
        }
    }
    while (i < n && is_ws(s[i])) i++;
    return i == n ? 0 : -1;
}

/* digit k (0-based) of the concatenated significand digit string */
static int digit_at(const token *t, size_t k) {
    const char c = k < t->n_int ? t->int_digits[k] : t->frac_digits[k - t->n_int];
    return t->hex ? hex_value(c) : c - '0';
}

/* ------------------------------------------------------------------------ */
/* Exact conversion                                                         */
/* ------------------------------------------------------------------------ */

/*
 * Nearest value of format f to V = N / D (N, D > 0): k = floor(log2 V)
 * exactly, then Q = floor(V / 2^e) with e = max(k, emin) - (p-1) by binary
 * long division, rounded half to even on the remainder.  Returns the
 * unsigned bit pattern and writes the status; frees N and D.
 */
static uint64_t round_ratio(big *Np, big *Dp, const fmt *f, uint8_t *status, int *err) {
    big N = *Np, D = *Dp, num = {0}, den = {0}, tmp = {0};
    uint64_t bits = 0;
    /* k = floor(log2 V).  With bn, bd the bit lengths,
     * V lies in (2^(bn-1-bd), 2^(bn-bd+1)), so k is bn-bd or bn-bd-1:
     * it is bn-bd exactly when N >= D * 2^(bn-bd).                          */
    int64_t k = (int64_t)big_bitlen(&N) - (int64_t)big_bitlen(&D);
    if (big_copy(&num, &N) || big_copy(&den, &D)) goto oom;
    if (k >= 0) {
        if (big_shl(&den, (uint64_t)k)) goto oom;
    } else {
        if (big_shl(&num, (uint64_t)(-k))) goto oom;
    }
    if (big_cmp(&num, &den) < 0) k -= 1;

    /* Unit in the last place of the result: 2^e with e = max(k,emin) - (p-1).
     * Q = floor(V / 2^e) < 2^p and R is the remainder of that division.     */
    const int pm1 = f->p - 1;
    int64_t e = (k > f->emin ? k : f->emin) - pm1;
    if (big_copy(&num, &N) || big_copy(&den, &D)) goto oom;
    if (e >= 0) {
        if (big_shl(&den, (uint64_t)e)) goto oom;
    } else {
        if (big_shl(&num, (uint64_t)(-e))) goto oom;
    }
    /* Binary long division, p quotient bits (Q < 2^p). */
    uint64_t Q = 0;
    if (big_copy(&tmp, &den) || big_shl(&tmp, (uint64_t)pm1)) goto oom;
    for (int i = pm1; i >= 0; i--) {
        if (big_cmp(&num, &tmp) >= 0) {
            big_sub(&num, &tmp);
            Q |= (uint64_t)1 << i;
        }
        big_shr1(&tmp);
    }
    /* num now holds R.  Round half to even: compare 2R with den. */
    if (big_shl(&num, 1)) goto oom;
    int c = big_cmp(&num, &den);
    if (c > 0 || (c == 0 && (Q & 1))) Q += 1;
    if (Q == ((uint64_t)1 << f->p)) {
        Q >>= 1;
        e += 1;
    }
    if (e > f->emax - pm1) {
        *status = OR_OVERFLOW;
        bits = f->inf_bits;
    } else if (Q == 0) {
        *status = OR_UNDERFLOW;
        bits = 0;
    } else if (Q < ((uint64_t)1 << pm1)) {
        /* subnormal: exponent field 0, e == emin - (p-1) */
        *status = OR_OK;
        bits = Q;
    } else {
        /* biased exponent field = e + (p-1) + emax */
        *status = OR_OK;
        bits = ((uint64_t)(e + pm1 + f->emax) << pm1) | (Q - ((uint64_t)1 << pm1));
    }
    big_free(&N);
    big_free(&D);
    big_free(&num);
    big_free(&den);
    big_free(&tmp);
    return bits;
oom:
    big_free(&N);
    big_free(&D);
    big_free(&num);
    big_free(&den);
    big_free(&tmp);
    *err = 1;
    *status = OR_INVALID;
    return f->qnan_bits;
}

/*
 * Nearest value of format f to D * 10^E for a natural D given by its
 * significant digits [first, last] of the token (first digit nonzero, last
 * digit nonzero).  Returns the unsigned bit pattern; writes the status.
 */
static uint64_t convert_exact(const token *t, size_t first, size_t last, int64_t E,
                              const fmt *f, uint8_t *status, int *err) {
    size_t nd = last - first + 1;
    /* Cheap range exits, each by a wide margin:
     *   10^(nd-1+E) <= V < 10^(nd+E).
     *   nd-1+E >= dec_ovf  =>  V >= 10^dec_ovf > 2^(emax+1): rounds to infinity.
     *   nd+E <= dec_unf    =>  V < 10^dec_unf < 2^(emin-p): rounds to zero.  */
    if ((int64_t)nd - 1 + E >= f->dec_ovf) {
        *status = OR_OVERFLOW;
        return f->inf_bits;
    }
    if ((int64_t)nd + E <= f->dec_unf) {
        *status = OR_UNDERFLOW;
        return 0;
    }

    big N = {0}, D = {0};
    *err = 0;

    /* N = digits * 10^max(E,0),  D = 10^max(-E,0)  so that V = N / D. */
    if (big_set_u64(&N, 0)) goto oom;
    {
        size_t k = first;
        while (k <= last) {
            uint32_t chunk = 0, mul = 1;
            for (int j = 0; j < 9 && k <= last; j++, k++) {
                chunk = chunk * 10 + (uint32_t)digit_at(t, k);
                mul *= 10;
            }
            if (big_mul_add_small(&N, mul, chunk)) goto oom;
        }
    }
    if (big_set_u64(&D, 1)) goto oom;
    if (E >= 0) {
        if (big_mul_pow10(&N, E)) goto oom;
    } else {
        if (big_mul_pow10(&D, -E)) goto oom;
    }
    return round_ratio(&N, &D, f, status, err);
oom:
    big_free(&N);
    big_free(&D);
    *err = 1;
    *status = OR_INVALID;
    return f->qnan_bits;
}

/*
 * Nearest value of format f to H * 2^E2 for the natural H given by the
 * significant hexadecimal digits [first, last] of the token (first and last
 * digit nonzero).  A hexadecimal float is a dyadic rational, so the same
 * exact rounding applies with D a power of two.
 */
static uint64_t convert_hex(const token *t, size_t first, size_t last, int64_t E2, const fmt *f,
                            uint8_t *status, int *err) {
    size_t nd = last - first + 1;
    int top = digit_at(t, first), tb = 0;
    while (top) {
        tb++;
        top >>= 1;
    }
    /* 2^(bl-1) <= H < 2^bl with bl = 4 (nd-1) + bits of the first digit.
     *   bl-1+E2 >= emax+1  =>  V >= 2^(emax+1): rounds to infinity.
     *   bl+E2 <= emin-p    =>  V < 2^(emin-p), half the smallest subnormal: 0. */
    const int64_t bl = 4 * (int64_t)(nd - 1) + tb;
    *err = 0;
    if (bl - 1 + E2 >= f->emax + 1) {
        *status = OR_OVERFLOW;
        return f->inf_bits;
    }
    if (bl + E2 <= f->emin - f->p) {
        *status = OR_UNDERFLOW;
        return 0;
    }
    big N = {0}, D = {0};
    if (big_set_u64(&N, 0)) goto oom;
    for (size_t k = first; k <= last; k++)
        if (big_mul_add_small(&N, 16, (uint32_t)digit_at(t, k))) goto oom;
    if (big_set_u64(&D, 1)) goto oom;
    if (E2 >= 0) {
        if (big_shl(&N, (uint64_t)E2)) goto oom;
    } else {
        if (big_shl(&D, (uint64_t)(-E2))) goto oom;
    }
    return round_ratio(&N, &D, f, status, err);
oom:
    big_free(&N);
    big_free(&D);
    *err = 1;
    *status = OR_INVALID;
    return f->qnan_bits;
}

/* One field in format f under a grammar.  Returns 0, or -1 if memory ran out. */
static int parse_field_fmt(const char *s, size_t n, const fmt *f, int grammar, uint64_t *out_bits,
                           uint8_t *status) {
    token t;
    if (tokenize(s, n, grammar, &t) != 0) {
        *out_bits = f->qnan_bits;
        *status = OR_INVALID;
        return 0;
    }
    size_t total = t.n_int + t.n_frac;
    /* strip leading zeros */
    size_t first = 0;
    while (first < total && digit_at(&t, first) == 0) first++;
    uint64_t sign = t.negative ? f->sign_bit : 0;
    if (first == total) { /* the value is zero */
        *out_bits = sign;
        *status = OR_OK;
        return 0;
    }
    /* strip trailing zeros; each one folds into the exponent */
    size_t last = total - 1;
    while (digit_at(&t, last) == 0) last--;
    /* V = (digits first..last) * 10^E,
     * E = explicit exponent - fraction digits + stripped trailing zeros;
     * for a hexadecimal float V = (hex digits first..last) * 2^E with four
     * binary places per hexadecimal digit.                                 */
    int err = 0;
    uint64_t bits;
    if (t.hex) {
        int64_t E2 = t.exp10 - 4 * (int64_t)t.n_frac + 4 * (int64_t)(total - 1 - last);
        bits = convert_hex(&t, first, last, E2, f, status, &err);
    } else {
        int64_t E = t.exp10 - (int64_t)t.n_frac + (int64_t)(total - 1 - last);
        bits = convert_exact(&t, first, last, E, f, status, &err);
    }
    *out_bits = bits | sign;
    if (bits == f->qnan_bits) *out_bits = bits;
    return err ? -1 : 0;
}

/* One field -> binary64.  Returns 0, or -1 if memory ran out. */
int oracle_parse_field(const char *s, size_t n, uint64_t *out_bits, uint8_t *status) {
    return parse_field_fmt(s, n, &FMT64, OR_GRAMMAR_DEFAULT, out_bits, status);
}

/* One field -> binary32 (the pattern in the low 32 bits). */
int oracle_parse_field_f32(const char *s, size_t n, uint32_t *out_bits, uint8_t *status) {
    uint64_t b = 0;
    int rc = parse_field_fmt(s, n, &FMT32, OR_GRAMMAR_DEFAULT, &b, status);
    *out_bits = (uint32_t)b;
    return rc;
}

/* One field, format (0 binary64, 1 binary32) and grammar (OR_GRAMMAR_*)
 * chosen; the pattern is in the low bits of *out_bits. */
int oracle_parse_field_ex(const char *s, size_t n, int f32, int grammar, uint64_t *out_bits,
                          uint8_t *status) {
    return parse_field_fmt(s, n, f32 ? &FMT32 : &FMT64, grammar, out_bits, status);
}

/* ------------------------------------------------------------------------ */
/* Buffers                                                                  */
/* ------------------------------------------------------------------------ */
static int is_sep(char c, char delim) { return c == '\n' || c == delim; }

/* Number of fields in text[0, len) under the buffer rule above. */
uint64_t oracle_count_fields(const char *text, size_t len, char delim) {
    if (len == 0) return 0;
    uint64_t n = 1;
    for (size_t i = 0; i + 1 < len; i++) n += is_sep(text[i], delim);
    return n;
}

typedef struct {
    const char *text;
    size_t len;
    char delim;
    size_t lo, hi; /* this worker parses fields whose first byte is in [lo,hi) */
    uint64_t first_index;
    uint64_t *out_bits;   /* binary64 results, or */
    uint32_t *out_bits32; /* binary32 results */
    uint8_t *status;
    int grammar;
    int err;
} work;

/* is position p the first byte of a field? */
static int starts_field(const char *text, size_t len, char delim, size_t p) {
    return p < len && (p == 0 || is_sep(text[p - 1], delim));
}

static uint64_t count_starts(const char *text, size_t len, char delim, size_t lo, size_t hi) {
    uint64_t n = 0;
    for (size_t p = lo; p < hi; p++) n += starts_field(text, len, delim, p);
    return n;
}

static void *worker(void *arg) {
    work *w = (work *)arg;
    uint64_t idx = w->first_index;
    for (size_t p = w->lo; p < w->hi; p++) {
        if (!starts_field(w->text, w->len, w->delim, p)) continue;
        size_t q = p;
        while (q < w->len && !is_sep(w->text[q], w->delim)) q++;
        int rc;
        if (w->out_bits32) {
            uint64_t b = 0;
            rc = parse_field_fmt(w->text + p, q - p, &FMT32, w->grammar, &b, &w->status[idx]);
            w->out_bits32[idx] = (uint32_t)b;
        } else {
            rc = parse_field_fmt(w->text + p, q - p, &FMT64, w->grammar, &w->out_bits[idx],
                                 &w->status[idx]);
        }
        if (rc) w->err = 1;
        idx++;
        p = q; /* the loop increment steps over the separator */
    }
    return NULL;
}

/*
 * Parse every field of text[0,len).  out_bits/status must hold `cap`
 * entries; the number of fields is written to *count.  Returns 0, -1 on a
 * capacity or memory error.  nthreads <= 1 runs on the calling thread.
 */
static int parse_buffer(const char *text, size_t len, char delim, uint64_t *out_bits,
                        uint32_t *out_bits32, uint8_t *status, uint64_t cap, uint64_t *count,
                        int nthreads, int grammar) {
    uint64_t total = oracle_count_fields(text, len, delim);
    *count = total;
    if (total > cap) return -1;
    if (nthreads < 1) nthreads = 1;
    if ((size_t)nthreads > len / 4096 + 1) nthreads = (int)(len / 4096 + 1);
    work *ws = (work *)calloc((size_t)nthreads, sizeof(work));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!ws || !th) {
        free(ws);
        free(th);
        return -1;
    }
    uint64_t before = 0;
    for (int i = 0; i < nthreads; i++) {
        ws[i].text = text;
        ws[i].len = len;
        ws[i].delim = delim;
        ws[i].lo = (size_t)((unsigned __int128)len * (unsigned)i / (unsigned)nthreads);
        ws[i].hi = (size_t)((unsigned __int128)len * (unsigned)(i + 1) / (unsigned)nthreads);
        ws[i].out_bits = out_bits;
        ws[i].out_bits32 = out_bits32;
        ws[i].status = status;
        ws[i].grammar = grammar;
        ws[i].first_index = before;
        before += count_starts(text, len, delim, ws[i].lo, ws[i].hi);
    }
    int rc = 0;
    if (nthreads == 1) {
        worker(&ws[0]);
    } else {
        for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, worker, &ws[i]);
        for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    }
    for (int i = 0; i < nthreads; i++) rc |= ws[i].err;
    free(ws);
    free(th);
    return rc ? -1 : 0;
}

int oracle_parse_buffer(const char *text, size_t len, char delim, uint64_t *out_bits,
                        uint8_t *status, uint64_t cap, uint64_t *count, int nthreads) {
    return parse_buffer(text, len, delim, out_bits, NULL, status, cap, count, nthreads,
                        OR_GRAMMAR_DEFAULT);
}

/* As oracle_parse_buffer, to binary32. */
int oracle_parse_buffer_f32(const char *text, size_t len, char delim, uint32_t *out_bits,
                            uint8_t *status, uint64_t cap, uint64_t *count, int nthreads) {
    return parse_buffer(text, len, delim, NULL, out_bits, status, cap, count, nthreads,
                        OR_GRAMMAR_DEFAULT);
}

/* Either format (binary32 patterns are stored as uint32), any grammar. */
int oracle_parse_buffer_ex(const char *text, size_t len, char delim, int f32, int grammar,
                           void *out_bits, uint8_t *status, uint64_t cap, uint64_t *count,
                           int nthreads) {
    return parse_buffer(text, len, delim, f32 ? NULL : (uint64_t *)out_bits,
                        f32 ? (uint32_t *)out_bits : NULL, status, cap, count, nthreads, grammar);
}
