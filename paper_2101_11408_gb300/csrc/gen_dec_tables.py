"""Generate dec_tables.inc: powers of five and of two in base 10^9.

The fallback kernel decides a field by comparing its decimal digits with
the midpoint h = (2M + 1) 2^(e - 1) between two adjacent floating-point
values, written in base 10^9 (Section 11: such midpoints have at most 768
significant digits).  With e - 1 >= 0, h = T 2^(e-1); with e - 1 < 0,
h = T 5^(1-e) 10^(e-1).  The kernel starts from a table entry and
multiplies by the remaining small power and by T:

* FP_DEC5: 5^(13 a) for a = 0 .. FP_DEC5_COUNT - 1 (5^(13 a) reaches past
  5^1075, the largest power a binary64 midpoint needs);
* FP_DEC2: 2^(28 a) for a = 0 .. FP_DEC2_COUNT - 1 (past 2^970).

Entry a occupies limbs [OFF[a], OFF[a+1]) of its array, least significant
limb first.  Run as a script to rewrite the include file next to it.
"""
from __future__ import annotations

import os

DEC5_STEP, DEC5_COUNT = 13, 83   # 13 * 82 = 1066 <= 1075 < 13 * 83
DEC2_STEP, DEC2_COUNT = 28, 35   # 28 * 34 = 952 <= 970 < 28 * 35
BASE = 10 ** 9


def limbs(v: int) -> list[int]:
    out = []
    while True:
        out.append(v % BASE)
        v //= BASE
        if v == 0:
            return out


def table(base: int, step: int, count: int) -> tuple[list[int], list[int]]:
    offs, data = [0], []
    for a in range(count):
        data += limbs(base ** (step * a))
        offs.append(len(data))
    return offs, data


def render() -> str:
    lines = ["/* Generated by gen_dec_tables.py: powers of five and two in base 10^9,",
             " * least significant limb first; entry a is limbs [OFF[a], OFF[a+1]). */",
             "#define FP_DEC_BASE 1000000000u"]
    for name, base, step, count in (("DEC5", 5, DEC5_STEP, DEC5_COUNT),
                                    ("DEC2", 2, DEC2_STEP, DEC2_COUNT)):
        offs, data = table(base, step, count)
        lines.append("#define FP_%s_STEP %d" % (name, step))
        lines.append("#define FP_%s_COUNT %d" % (name, count))
        lines.append("#define FP_%s_LIMBS %d" % (name, len(data)))
        lines.append("#define FP_%s_OFF_VALUES \\" % name)
        for i in range(0, len(offs), 16):
            lines.append("  " + ", ".join(str(v) for v in offs[i:i + 16]) + ", \\")
        lines.append("  /* end */")
        lines.append("#define FP_%s_VALUES \\" % name)
        for i in range(0, len(data), 8):
            lines.append("  " + ", ".join("%du" % v for v in data[i:i + 8]) + ", \\")
        lines.append("  /* end */")
    return "\n".join(lines) + "\n"


def main() -> None:
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dec_tables.inc")
    text = render()
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
