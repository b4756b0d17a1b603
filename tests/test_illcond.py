"""The ill-conditioned products of the paper's accuracy experiments (Sec.
"Accuracy experiments", "Ill-conditioned experiments"), workloads/illcond.py.

Generator: Q is an exact product of Householder reflections, so the rounded
A = fl_dd(Q) has A A^T = I up to FP64x2 rounding, and A B reproduces C up to
it; the dot products have condition ~ 1/t.

Claim: the paper finds the cascade more accurate than the FP64x2 triple loop
on these products ("vastly superior", since the highest-order bits are
computed error-free whatever the condition number).  Checked here on the CPU
restatement against exact rationals."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import cascade as cs
from oracle import dd
from tests import exact
from workloads.illcond import illcond_inputs


def rel_errors(c_hi, c_lo, a, rows, cols):
    out = []
    for i, j in zip(rows, cols):
        ex = exact.exact_dot(a[0][i], a[1][i], a[2][:, j], a[3][:, j])
        val = abs(Fraction(ex, 1 << (2 * exact.SHIFT)))
        out.append(exact.err_vs_exact(c_hi[i, j], c_lo[i, j], ex) / float(val))
    return np.array(out)


def test_generator_orthogonal_and_conditioned():
    n, t = 24, 1e-14
    a_hi, a_lo, b_hi, b_lo, c = illcond_inputs(n, t, seed=3)
    for i in range(n):
        for j in range(n):
            s = exact.exact_dot(a_hi[i], a_lo[i], a_hi[j], a_lo[j])      # (A A^T)_ij
            want = 1 << (2 * exact.SHIFT) if i == j else 0
            assert abs(Fraction(s - want, 1 << (2 * exact.SHIFT))) <= 2.0 ** -100
    rng = np.random.default_rng(0)
    for i, j in zip(rng.integers(0, n, 40), rng.integers(0, n, 40)):
        ab = Fraction(exact.exact_dot(a_hi[i], a_lo[i], b_hi[:, j], b_lo[:, j]),
                      1 << (2 * exact.SHIFT))
        assert abs(ab - Fraction(c[i, j])) <= 2.0 ** -100
        cond = (np.linalg.norm(a_hi[i]) * np.linalg.norm(b_hi[:, j])) / abs(float(ab))
        assert cond >= 0.99 or abs(c[i, j]) == 1.0
        assert abs(c[i, j]) == 1.0 or cond > 1.0 / (11 * t)


@pytest.mark.parametrize("n,t", [(64, 1e-14), (96, 1e-19)])
def test_cascade_more_accurate_than_fp64x2_loop(n, t):
    a = illcond_inputs(n, t, seed=n)[:4]
    rng = np.random.default_rng(1)
    rows, cols = rng.integers(0, n, 50), rng.integers(0, n, 50)
    c_hi, c_lo = cs.cascade_ddgemm(*a)
    o_hi, o_lo = dd.ddgemm(*a)
    e_casc = rel_errors(c_hi, c_lo, a, rows, cols)
    e_dd = rel_errors(o_hi, o_lo, a, rows, cols)
    assert e_casc.max() * 10 < e_dd.max()


@pytest.mark.parametrize("n,t", [(64, 1e-14), (96, 1e-19)])
def test_int8_eight_bit_pieces_more_accurate_than_fp64x2_loop(n, t):
    """The INT8 form with 15 eight-bit pieces (F = 118 fraction bits below
    the block scale) also beats the FP64x2 triple loop on these products;
    the seven-bit form with 16 pieces (F = 111) does not have that margin."""
    from oracle import cascade_int8 as c8
    a = illcond_inputs(n, t, seed=n)[:4]
    rng = np.random.default_rng(1)
    rows, cols = rng.integers(0, n, 50), rng.integers(0, n, 50)
    c_hi, c_lo = c8.cascade_int8_ddgemm(*a, s=15)
    o_hi, o_lo = dd.ddgemm(*a)
    assert rel_errors(c_hi, c_lo, a, rows, cols).max() * 3 < rel_errors(o_hi, o_lo, a, rows, cols).max()
