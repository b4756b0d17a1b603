"""Ill-conditioned products, after the paper's accuracy experiments (Sec.
"Accuracy experiments", "Ill-conditioned experiments"): A = Q with
orthonormal rows, C with entries of magnitude (t, 10 t) and random signs and
one entry 1 per column, B = Q^T C computed beyond FP64x2, then A and B rounded
to FP64x2.  Then (A B)_ij ~ C_ij while |A| |B| ~ 1: most entries of the
product are dot products with condition number ~ 1 / t.

The paper takes Q from an FP128 Householder QR of a random matrix.  Here Q is
exactly orthogonal instead: a product of a few Householder reflections
H = I - 2 v v^T / (v^T v) with integer vectors v, carried in exact integer
arithmetic (a common denominator per matrix), and B = Q^T C is exact too;
only the final rounding to FP64x2 is inexact.  Test and study data only: no
arithmetic of the method lives here.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

SHIFT = 1074  # every double is an integer multiple of 2^-1074


def _fixed(x: float) -> int:
    num, den = float(x).as_integer_ratio()
    return num << (SHIFT - (den.bit_length() - 1))


def _reflect(x: list, v: list, vv: int) -> list:
    """(v^T v) H x = (v^T v) x - 2 v (v^T x), exactly, for integer x and v."""
    d = sum(a * b for a, b in zip(v, x))
    return [vv * xi - 2 * vi * d for xi, vi in zip(x, v)]


def _to_dd(num: int, den: int):
    """The FP64x2 (hi, lo) nearest to num / den: hi = fl(num/den),
    lo = fl(num/den - hi), both correctly rounded."""
    q = Fraction(num, den)
    hi = float(q)
    lo = float(q - Fraction(hi))
    return hi, lo


def illcond_inputs(n: int, t: float, seed: int = 0, reflections: int = 4, vbits: int = 12):
    """A (n x n) and B (n x n) as FP64x2 (hi, lo) arrays with A B ~ C.

    Draw order from default_rng(seed): the reflection vectors, then C's
    magnitudes, signs and the row of each column's 1."""
    rng = np.random.default_rng(seed)
    vs = [[int(x) for x in rng.integers(-(2 ** vbits), 2 ** vbits + 1, n)] for _ in range(reflections)]
    vvs = [sum(x * x for x in v) for v in vs]
    den_q = 1
    for vv in vvs:
        den_q *= vv
    # Q = H_1 H_2 ... H_r: column j is H_1 (H_2 (... (H_r e_j)))
    a_hi = np.zeros((n, n))
    a_lo = np.zeros((n, n))
    for j in range(n):
        x = [0] * n
        x[j] = 1
        for v, vv in zip(reversed(vs), reversed(vvs)):
            x = _reflect(x, v, vv)
        for i in range(n):
            a_hi[i, j], a_lo[i, j] = _to_dd(x[i], den_q)
    # C: entries +-U(t, 10 t), one entry 1 per column
    mag = rng.uniform(t, 10.0 * t, size=(n, n))
    sgn = np.where(rng.integers(0, 2, size=(n, n)) == 0, -1.0, 1.0)
    c = mag * sgn
    c[rng.integers(0, n, size=n), np.arange(n)] = 1.0
    # B = Q^T C = H_r (... (H_1 C)) exactly, column by column
    b_hi = np.zeros((n, n))
    b_lo = np.zeros((n, n))
    den_b = den_q << SHIFT
    for j in range(n):
        x = [_fixed(c[i, j]) for i in range(n)]
        for v, vv in zip(vs, vvs):
            x = _reflect(x, v, vv)
        for i in range(n):
            b_hi[i, j], b_lo[i, j] = _to_dd(x[i], den_b)
    return a_hi, a_lo, b_hi, b_lo, c
