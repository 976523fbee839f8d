"""Exact rational rounding used to pin the oracle's emulated arithmetic.

Independent of the oracle: values are converted to ``fractions.Fraction``,
combined exactly, and rounded to nearest-even at the target format by integer
arithmetic, following the IEEE 754 definition of roundTiesToEven with gradual
underflow.
"""
from __future__ import annotations

import math
from fractions import Fraction

FORMATS = {           # (significand bits incl. hidden, emin, emax)
    "fp32": (24, -126, 127),
    "fp16": (11, -14, 15),
    "bf16": (8, -126, 127),
}


def rn(q: Fraction, fmt: str, zero_sign: float = 1.0) -> float:
    """Round the exact rational ``q`` to ``fmt``; an exact zero gets
    ``zero_sign``'s sign."""
    p, emin, emax = FORMATS[fmt]
    if q == 0:
        return math.copysign(0.0, zero_sign)
    sign = -1.0 if q < 0 else 1.0
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, emin)
    quantum = Fraction(2) ** (e - p + 1)
    n = a / quantum
    fl = n.numerator // n.denominator
    rem = n - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    r = fl * quantum
    maxv = (2 - Fraction(2) ** (1 - p)) * Fraction(2) ** emax
    if r > maxv:
        return sign * math.inf
    if r == 0:
        return math.copysign(0.0, sign)
    return sign * float(r)


def exact_fma(a: float, b: float, c: float, fmt: str) -> float:
    """IEEE fma(a, b, c) in ``fmt`` for finite operands of that format."""
    q = Fraction(a) * Fraction(b) + Fraction(c)
    if q == 0:
        # exact zero: +0 unless both the product and the addend are -0 / negative zero sum
        prod_neg = (math.copysign(1.0, a) * math.copysign(1.0, b)) < 0
        prod_zero = a == 0 or b == 0
        if prod_zero and c == 0:
            neg = prod_neg and math.copysign(1.0, c) < 0
            return -0.0 if neg else 0.0
        return 0.0
    return rn(q, fmt)
