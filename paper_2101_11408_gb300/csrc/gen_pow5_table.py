"""Generate pow5_table.inc: the 651 x 128-bit power-of-five table T[q].

T[q] for q in [-342, 308] (Appendix "Table Generation Script" defines the
three regimes; Sections 8 and 9 derive them):

* q >= 0 (Section 8): 5^q scaled by a power of two into [2^127, 2^128),
  truncated (bits below the top 128 dropped).
* -27 <= q <= -1 (Section 9.1): the rounded-up reciprocal
  ceil(2^b / 5^-q) with b = 127 + ceil(log2 5^-q); it lies in [2^127, 2^128).
* q < -27 (Section 9.2): the top 128 bits of ceil(2^(2b) / 5^-q) with
  b = 64 + ceil(log2 5^-q).

Each entry is stored as two 64-bit words, the more significant first, at
index 2*(q+342).  Run as a script to rewrite the include file next to it.
"""
from __future__ import annotations

import os

Q_MIN, Q_MAX = -342, 308


def ceil_log2(n: int) -> int:
    """Smallest z with 2^z >= n, for n >= 1."""
    return (n - 1).bit_length()


def table_entry(q: int) -> int:
    """The 128-bit value T[q]."""
    if q >= 0:
        v = 5 ** q
        shift = 128 - v.bit_length()
        return v << shift if shift >= 0 else v >> (-shift)
    d = 5 ** (-q)
    if q >= -27:
        b = 127 + ceil_log2(d)
        c = -((-(1 << b)) // d)  # ceil(2^b / d)
        assert (1 << 127) <= c < (1 << 128)
        return c
    b = 64 + ceil_log2(d)
    c = -((-(1 << (2 * b))) // d)  # ceil(2^(2b) / d)
    return c >> (c.bit_length() - 128)


def table() -> list[tuple[int, int]]:
    out = []
    for q in range(Q_MIN, Q_MAX + 1):
        v = table_entry(q)
        out.append((v >> 64, v & ((1 << 64) - 1)))
    return out


def render() -> str:
    lines = [
        "/* Generated by gen_pow5_table.py -- do not edit.",
        " * T[q], q in [-342, 308]: word 2*(q+342) is the high 64 bits, word",
        " * 2*(q+342)+1 the low 64 bits (Appendix B; Sections 8-9).",
        " * Use as:  const unsigned long long t[2 * FP_POW5_ENTRIES] = { FP_POW5_TABLE_VALUES }; */",
        "#define FP_POW5_QMIN (-342)",
        "#define FP_POW5_QMAX 308",
        "#define FP_POW5_ENTRIES 651",
        "#define FP_POW5_TABLE_VALUES \\",
    ]
    for i, (hi, lo) in enumerate(table()):
        lines.append("    0x%016xULL, 0x%016xULL, /* q = %d */ \\" % (hi, lo, Q_MIN + i))
    lines.append("    /* end */")
    return "\n".join(lines) + "\n"


def main() -> None:
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pow5_table.inc")
    text = render()
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
