"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and prints them as text; it holds none
of the parsing arithmetic, and both the oracle and the GPU path consume its
output.  The paper measures on the "canada" coordinate file, a "uniform"
[0,1) set and an "integer" set (Section 12); those files are not available,
so the generators below stand in for them:

* ``uniform_text``  -- %.17g of U[0,1) doubles, newline-separated (the
  uniform set at 17 significant digits).
* ``bulk_mixed_text`` -- 40% uniform %.17g, 30% coordinates (latitude in
  [-90,90] or longitude in [-180,180], 12..16 fractional digits; stands in
  for canada), 20% integers in [0,2^63), 10% ``d.ddddE+xxx`` with exponents
  in [-340,320] (subnormals, underflow, overflow).
* ``hard_case_text`` -- long significands (20..800 significant digits),
  exact midpoints between adjacent doubles printed in full (exact, +1 and
  -1 in the last digit), and subnormal / near-DBL_MAX values with 17..25
  digits including rounded half-ulp boundaries.
* ``batch_buffers`` -- many independent buffers with lognormal sizes whose
  content is uniform %.17g text.
* ``csv_request`` -- CSV blocks of 8 comma-separated uniform columns.

Every generator takes a seed; the default seeds are fixed so that runs are
reproducible.
"""
from __future__ import annotations

import hashlib
import os
from fractions import Fraction

import numpy as np

SEED_BASE = 0x210111408


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _cache_path(name: str) -> str | None:
    d = os.environ.get("FP_WORKLOAD_CACHE")
    if not d:
        return None
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, hashlib.sha1(name.encode()).hexdigest()[:16] + ".bin")


def _cached(name: str, make):
    p = _cache_path(name)
    if p and os.path.exists(p):
        with open(p, "rb") as f:
            return f.read()
    data = make()
    if p:
        tmp = p + ".%d.tmp" % os.getpid()
        with open(tmp, "wb") as f:
            f.write(data)
        os.replace(tmp, p)
    return data


def _uniform_doubles(rng: np.random.Generator, n: int) -> np.ndarray:
    # 53 random bits -> a double in [0,1)
    return (rng.integers(0, 1 << 53, size=n, dtype=np.int64).astype(np.float64)
            * (1.0 / (1 << 53)))


def _fmt_g17(xs) -> list[str]:
    return ["%.17g" % x for x in xs.tolist()]


def uniform_lines(n: int, seed: int) -> list[str]:
    return _fmt_g17(_uniform_doubles(_rng(seed), n))


def uniform_text(n: int = 10_000, seed: int = SEED_BASE + 1) -> bytes:
    """n values %.17g of U[0,1), newline-separated (about 19 B per value)."""
    return _cached("uniform:%d:%d" % (n, seed),
                   lambda: "\n".join(uniform_lines(n, seed)).encode())


def bulk_mixed_lines(n: int, seed: int) -> list[str]:
    rng = _rng(seed)
    cat = rng.choice(4, size=n, p=[0.4, 0.3, 0.2, 0.1])
    out = [None] * n
    idx = [np.nonzero(cat == c)[0] for c in range(4)]
    # 0: uniform [0,1) at 17 significant digits
    for i, s in zip(idx[0].tolist(), _fmt_g17(_uniform_doubles(rng, idx[0].size))):
        out[i] = s
    # 1: coordinates, latitude or longitude, 12..16 fractional digits
    k = idx[1].size
    is_lon = rng.integers(0, 2, size=k).astype(bool)
    u = _uniform_doubles(rng, k)
    val = np.where(is_lon, u * 360.0 - 180.0, u * 180.0 - 90.0)
    prec = rng.integers(12, 17, size=k)
    for i, v, p in zip(idx[1].tolist(), val.tolist(), prec.tolist()):
        out[i] = "%.*f" % (p, v)
    # 2: integers uniform in [0, 2^63)
    ints = rng.integers(0, np.iinfo(np.int64).max, size=idx[2].size, dtype=np.int64,
                        endpoint=True)
    for i, v in zip(idx[2].tolist(), ints.tolist()):
        out[i] = str(v)
    # 3: scientific d.ddddE+xxx, exponent uniform in [-340, 320]
    k = idx[3].size
    lead = rng.integers(1, 10, size=k)
    frac = rng.integers(0, 10000, size=k)
    ex = rng.integers(-340, 321, size=k)
    for i, a, b, e in zip(idx[3].tolist(), lead.tolist(), frac.tolist(), ex.tolist()):
        out[i] = "%d.%04dE%s%03d" % (a, b, "-" if e < 0 else "+", abs(e))
    return out


def bulk_mixed_text(n: int = 10_000_000, seed: int = SEED_BASE + 2) -> bytes:
    """The bulk mixed workload: n newline-separated numbers (about 18.8 B each)."""
    return _cached("bulk:%d:%d" % (n, seed),
                   lambda: "\n".join(bulk_mixed_lines(n, seed)).encode())


# ---------------------------------------------------------------------------
# hard cases
# ---------------------------------------------------------------------------

def _exact_decimal(num: int, den_pow2: int) -> tuple[str, int]:
    """num / 2^den_pow2 (or num * 2^-den_pow2 for negative) as (digits, exp10)
    with value = int(digits) * 10^exp10 exactly, no trailing zeros."""
    if den_pow2 <= 0:
        v, e = num << (-den_pow2), 0
    else:
        v, e = num * 5 ** den_pow2, -den_pow2
    s = str(v)
    t = s.rstrip("0")
    e += len(s) - len(t)
    return t, e


def _sci(digits: str, exp10: int) -> str:
    """digits * 10^exp10 written as d.ddd...E+x."""
    e = exp10 + len(digits) - 1
    body = digits[0] + ("." + digits[1:] if len(digits) > 1 else "")
    return "%sE%+d" % (body, e)


def _double_parts(bits: int) -> tuple[int, int]:
    """(M, e) with value = M * 2^e for a finite non-negative binary64."""
    ef = bits >> 52
    frac = bits & ((1 << 52) - 1)
    if ef == 0:
        return frac, -1074
    return frac | (1 << 52), ef - 1075


def midpoint_decimal(bits: int) -> tuple[str, int]:
    """Exact decimal (digits, exp10) of the midpoint between the non-negative
    binary64 with this bit pattern and its successor (2^1024 after DBL_MAX)."""
    M, e = _double_parts(bits)
    return _exact_decimal(2 * M + 1, -(e - 1))


def _round_sig(x: Fraction, p: int) -> tuple[str, int]:
    """x > 0 rounded to p significant decimal digits (half up)."""
    e = len(str(x.numerator // x.denominator)) - 1 if x >= 1 else -len(
        str(x.denominator // x.numerator))
    # adjust e so that 10^e <= x < 10^(e+1)
    while Fraction(10) ** e > x:
        e -= 1
    while Fraction(10) ** (e + 1) <= x:
        e += 1
    scaled = x / Fraction(10) ** (e - p + 1)
    d = (scaled.numerator * 2 + scaled.denominator) // (2 * scaled.denominator)
    s = str(d)
    exp10 = e - p + 1
    if len(s) > p:
        s, exp10 = s[:-1], exp10 + 1
    return s, exp10


def hard_case_lines(n: int, seed: int) -> list[str]:
    rng = _rng(seed)
    cat = rng.choice(3, size=n, p=[0.5, 0.3, 0.2])
    out = [None] * n
    # 0: 20..800 significant digits, random '.', magnitude 10^[-330, 300]
    idx = np.nonzero(cat == 0)[0]
    lens = rng.integers(20, 801, size=idx.size)
    allbytes = rng.integers(ord("0"), ord("9") + 1, size=int(lens.sum()), dtype=np.uint8)
    leads = rng.integers(ord("1"), ord("9") + 1, size=idx.size, dtype=np.uint8)
    dots = rng.integers(0, 2, size=idx.size)
    mags = rng.integers(-330, 301, size=idx.size)
    dotpos = rng.random(idx.size)
    off = 0
    raw = allbytes.tobytes()
    for j, i in enumerate(idx.tolist()):
        L = int(lens[j])
        s = chr(leads[j]) + raw[off + 1: off + L].decode()
        off += L
        if dots[j]:
            p = 1 + int(dotpos[j] * (L - 1))  # digits before the point
            s = s[:p] + "." + s[p:]
        else:
            p = L
        ex = int(mags[j]) - (p - 1)
        out[i] = "%se%d" % (s, ex)
    # 1: exact midpoints between adjacent doubles, exact / +1 / -1 in the last digit
    idx = np.nonzero(cat == 1)[0]
    bits = rng.integers(0, 0x7FEFFFFFFFFFFFFF, size=idx.size, dtype=np.int64,
                        endpoint=True)
    which = rng.integers(0, 3, size=idx.size)
    for j, i in enumerate(idx.tolist()):
        digits, e10 = midpoint_decimal(int(bits[j]))
        v = int(digits) + (0, 1, -1)[int(which[j])]
        ds = str(v)
        out[i] = _sci(ds, e10 + 0) if len(ds) == len(digits) else _sci(ds, e10)
    # 2: subnormal range and near DBL_MAX with 17..25 significant digits,
    #    including half-ulp boundaries rounded to that many digits
    idx = np.nonzero(cat == 2)[0]
    sub = rng.integers(0, 2, size=idx.size).astype(bool)
    half = rng.integers(0, 3, size=idx.size)
    prec = rng.integers(17, 26, size=idx.size)
    sb = rng.integers(1, 1 << 52, size=idx.size, dtype=np.int64)
    hb = rng.integers(0x7FEFFFFF00000000, 0x7FEFFFFFFFFFFFFF, size=idx.size,
                      dtype=np.int64, endpoint=True)
    for j, i in enumerate(idx.tolist()):
        b = int(sb[j]) if sub[j] else int(hb[j])
        M, e = _double_parts(b)
        if half[j] == 0:
            x = Fraction(M) * Fraction(2) ** e
        else:
            x = Fraction(2 * M + 1) * Fraction(2) ** (e - 1)
        digits, e10 = _round_sig(x, int(prec[j]))
        out[i] = _sci(digits, e10)
    return out


def hard_case_text(n: int = 1_000_000, seed: int = SEED_BASE + 3) -> bytes:
    return _cached("hard:%d:%d" % (n, seed),
                   lambda: "\n".join(hard_case_lines(n, seed)).encode())


# ---------------------------------------------------------------------------
# the other grammars and the columnar layout
# ---------------------------------------------------------------------------

def hex_float_lines(n: int, seed: int) -> list[str]:
    """n hexadecimal floats (Python's float.hex, e.g. 0x1.921fb54442d18p+1):
    half of uniform [0,1) doubles, half of random finite binary64 bit
    patterns of either sign (subnormals and zeros included)."""
    rng = _rng(seed)
    k = n // 2
    u = _uniform_doubles(rng, k)
    bits = rng.integers(0, 0x7FF0000000000000, size=n - k, dtype=np.int64)
    sign = rng.integers(0, 2, size=n - k).astype(np.int64) << 63
    r = (bits | sign).view(np.float64)
    vals = np.concatenate([u, r])
    order = rng.permutation(n)
    return [float(x).hex() for x in vals[order].tolist()]


def hex_float_text(n: int = 10_000_000, seed: int = SEED_BASE + 6) -> bytes:
    """The hexadecimal-float workload: n newline-separated values (about 21 B each)."""
    return _cached("hex:%d:%d" % (n, seed), lambda: "\n".join(hex_float_lines(n, seed)).encode())


def csv_columns_text(rows: int, cols: int = 8, seed: int = SEED_BASE + 7) -> bytes:
    """rows lines of `cols` comma-separated uniform [0,1) %.17g values (the
    served requests' content), for the column-major layout."""
    def make():
        vals = uniform_lines(rows * cols, seed)
        return "\n".join(",".join(vals[r * cols:(r + 1) * cols]) for r in range(rows)).encode()
    return _cached("csvcols:%d:%d:%d" % (rows, cols, seed), make)


# ---------------------------------------------------------------------------
# batched and served
# ---------------------------------------------------------------------------

def _pool_text(nbytes: int, seed: int, sep: bytes = b"\n", cols: int = 1) -> bytes:
    """About nbytes of uniform [0,1) %.17g values (the 10,000-number
    workload's content), one per line, or `cols` comma-separated per row."""
    n = nbytes // 19 + 16
    vals = uniform_lines(n, seed)
    if cols == 1:
        return "\n".join(vals).encode()
    rows = [",".join(vals[r * cols:(r + 1) * cols]) for r in range(n // cols)]
    return "\n".join(rows).encode()


def _cut(pool: bytes, start: int, size: int) -> bytes:
    """size bytes of the pool (wrapping) starting at the line after `start`,
    trimmed back to end at a line break."""
    start = pool.find(b"\n", start % len(pool)) + 1
    out = bytearray()
    while len(out) < size:
        take = pool[start:start + size - len(out)]
        out += take
        start = 0
        if len(out) < size:
            out += b"\n"
    cut = out.rfind(b"\n", 0, size)
    return bytes(out[:cut] if cut > 0 else out[:size])


def lognormal_sizes(count: int, total: int, lo: int, hi: int, sigma: float,
                    seed: int) -> list[int]:
    """count sizes clip(lognormal(mu, sigma), lo, hi) with mu bisected so the
    sum is close to total."""
    z = _rng(seed).standard_normal(count)

    def tot(mu):
        return np.clip(np.exp(mu + sigma * z), lo, hi).sum()

    a, b = np.log(lo) - 5 * sigma, np.log(hi) + 5 * sigma
    for _ in range(100):
        m = 0.5 * (a + b)
        if tot(m) < total:
            a = m
        else:
            b = m
    return [int(s) for s in np.clip(np.exp(0.5 * (a + b) + sigma * z), lo, hi)]


def batch_buffers(count: int = 4096, total: int = 2 << 30, lo: int = 1 << 10,
                  hi: int = 64 << 20, seed: int = SEED_BASE + 4,
                  pool_bytes: int = 64 << 20) -> list[bytes]:
    """count independent newline-separated buffers, lognormal sizes
    (sigma 2.0) in [lo, hi] summing to about `total` bytes.  Content is cut
    from a pool of uniform %.17g text."""
    sizes = lognormal_sizes(count, total, lo, hi, 2.0, seed)
    pool = _cached("pool:%d:%d" % (pool_bytes, seed),
                   lambda: _pool_text(pool_bytes, seed + 1))
    starts = _rng(seed + 2).integers(0, len(pool), size=count)
    return [_cut(pool, int(s), z) for s, z in zip(starts.tolist(), sizes)]


def csv_request(size: int, seed: int, pool: bytes | None = None) -> bytes:
    """One CSV block of 8 comma-separated uniform columns, '\\n' rows, about
    `size` bytes, ending at a row break."""
    if pool is None:
        pool = csv_pool()
    start = int(_rng(seed).integers(0, len(pool)))
    return _cut(pool, start, size)


def csv_pool(pool_bytes: int = 64 << 20, seed: int = SEED_BASE + 5) -> bytes:
    return _cached("csvpool:%d:%d" % (pool_bytes, seed),
                   lambda: _pool_text(pool_bytes, seed, cols=8))


def pack_buffers(texts: list[bytes], skew: bool = True) -> tuple[np.ndarray, list[int]]:
    """Lay many buffers out in one byte array, as a caller holding them in one
    allocation would: each starts on a 16-byte boundary plus (index mod 16)
    bytes when `skew` (so every start alignment occurs), with 16 bytes of
    digits between neighbours.  Returns (array, start offsets)."""
    starts, pos = [], 0
    for b, t in enumerate(texts):
        pos = (pos + 15) & ~15
        if skew:
            pos += b % 16
        starts.append(pos)
        pos += len(t) + 16
    arr = np.full(pos + 16, ord("7"), dtype=np.uint8)
    for s, t in zip(starts, texts):
        if t:
            arr[s:s + len(t)] = np.frombuffer(t, dtype=np.uint8)
    return arr, starts


def integer_lines(n: int, seed: int) -> list[str]:
    """Plain integers, the shape of the paper's integer file (Section 12):
    mostly uniform 32-bit values, plus signs, leading zeros, values around
    2^53 (odd ones above it round to even) and up to 19 digits."""
    r = _rng(seed)
    kinds = r.integers(0, 10, size=n)
    out = []
    for k, a, b in zip(kinds.tolist(), r.integers(0, 1 << 32, size=n).tolist(),
                       r.integers(0, 1 << 62, size=n).tolist()):
        if k < 6:
            out.append(str(a))
        elif k == 6:
            out.append("-" + str(a))
        elif k == 7:
            out.append("+" + "0" * (a % 5) + str(a % 100000))
        elif k == 8:
            out.append(str((1 << 53) + (a % 4096)))
        else:
            out.append(str(b * 2 + (a & 1)))  # up to 19 digits
    return out


def integer_text(n: int, seed: int) -> bytes:
    return "\n".join(integer_lines(n, seed)).encode()
