"""Exact rational arithmetic on FP64 / FP64x2 values, for pinning the oracle.

Every finite double is an integer multiple of 2^-1074, so a value is held as
the Python integer N with value = N * 2^-1074 (a product as N * 2^-2148).
Nothing here shares code with the oracle or with the CUDA path."""
from __future__ import annotations

from fractions import Fraction

import numpy as np

SHIFT = 1074


def fixed(x: float) -> int:
    """x == fixed(x) * 2^-1074 exactly."""
    num, den = float(x).as_integer_ratio()
    return num << (SHIFT - (den.bit_length() - 1))


def dd_fixed(hi: float, lo: float) -> int:
    return fixed(hi) + fixed(lo)


def exact_dot(a_hi, a_lo, b_hi, b_lo) -> int:
    """sum_l (a_hi[l] + a_lo[l]) (b_hi[l] + b_lo[l]) exactly, scaled by 2^2148."""
    s = 0
    for ah, al, bh, bl in zip(a_hi.tolist(), a_lo.tolist(), b_hi.tolist(), b_lo.tolist()):
        s += dd_fixed(ah, al) * dd_fixed(bh, bl)
    return s


def err_vs_exact(c_hi: float, c_lo: float, exact_scaled: int) -> float:
    """|c_hi + c_lo - exact| as a float, exact given scaled by 2^2148."""
    got = dd_fixed(c_hi, c_lo) << SHIFT
    return float(Fraction(abs(got - exact_scaled), 1 << (2 * SHIFT)))


def abs_product(a_hi, b_hi):
    """(|A| |B|) from the hi parts, in float64 (a bound's scale, not a value)."""
    return np.abs(a_hi) @ np.abs(b_hi)


def dd_is_normalised(hi, lo) -> bool:
    """hi == fl(hi + lo): |lo| <= ulp(hi)/2 (round-to-nearest-even)."""
    hi = np.asarray(hi)
    lo = np.asarray(lo)
    return bool(np.all(hi + lo == hi))
