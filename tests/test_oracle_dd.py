"""Pins for the double-double GEMM oracle (oracle/dd_oracle.c).

The oracle is checked against things other than itself: exact rational
arithmetic (brute force on small inputs), exact integer products, identity
and permutation matrices, the normalisation invariant and the FP64x2 dot
product error bound |fl(x^T y) - x^T y| <= gamma_k |x|^T |y| with
gamma_k ~ k 2^-106 (Sec. "Forward Error Analysis", eq. fp64x2)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import dd
from tests import exact
from workloads import gemm_inputs, integer_inputs

EPS_DD = 2.0 ** -106


def test_two_sum_exact():
    rng = np.random.default_rng(1)
    vals = list(rng.standard_normal(200) * np.exp2(rng.integers(-60, 60, 200)))
    vals += [1.0, 2.0 ** -60, -1.0, 0.0, 2.0 ** 53, 0.5, 3.0 * 2.0 ** -54]
    for a, b in zip(vals, vals[::-1]):
        s, e = dd.two_sum(a, b)
        assert exact.fixed(s) + exact.fixed(e) == exact.fixed(a) + exact.fixed(b)
        assert s == a + b


def test_two_prod_exact():
    rng = np.random.default_rng(2)
    a = rng.standard_normal(300) * np.exp2(rng.integers(-100, 100, 300))
    b = rng.standard_normal(300) * np.exp2(rng.integers(-100, 100, 300))
    for x, y in zip(a, b):
        p, e = dd.two_prod(float(x), float(y))
        assert (exact.fixed(p) + exact.fixed(e)) << exact.SHIFT == exact.fixed(x) * exact.fixed(y)


def test_dd_add_and_mul_error():
    rng = np.random.default_rng(3)
    for _ in range(300):
        ah = float(rng.standard_normal())
        al = ah * 2.0 ** -53 * float(rng.uniform(-1, 1))
        bh = float(rng.standard_normal()) * 2.0 ** float(rng.integers(-30, 30))
        bl = bh * 2.0 ** -53 * float(rng.uniform(-1, 1))
        rh, rl = dd.dd_add(ah, al, bh, bl)
        true = exact.dd_fixed(ah, al) + exact.dd_fixed(bh, bl)
        err = abs(exact.dd_fixed(rh, rl) - true)
        assert (err << 106) <= 4 * abs(true) + (1 << 106), (ah, al, bh, bl)
        assert rh + rl == rh
        ph, pl = dd.dd_mul(ah, al, bh, bl)
        truep = exact.dd_fixed(ah, al) * exact.dd_fixed(bh, bl)
        errp = abs((exact.dd_fixed(ph, pl) << exact.SHIFT) - truep)
        assert (errp << 106) <= 8 * abs(truep) + (1 << 106)
        assert ph + pl == ph


@pytest.mark.parametrize("m,n,k", [(3, 5, 7), (8, 8, 33), (4, 6, 300)])
@pytest.mark.parametrize("kind", ["uniform", "wide"])
def test_ddgemm_vs_exact_rationals(m, n, k, kind):
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind=kind, seed=m * 100 + k)
    c_hi, c_lo = dd.ddgemm(a_hi, a_lo, b_hi, b_lo)
    assert exact.dd_is_normalised(c_hi, c_lo)
    absab = exact.abs_product(a_hi, b_hi)
    for i in range(m):
        for j in range(n):
            ex = exact.exact_dot(a_hi[i], a_lo[i], b_hi[:, j], b_lo[:, j])
            err = exact.err_vs_exact(c_hi[i, j], c_lo[i, j], ex)
            # gamma_k |x|^T |y| for FP64x2 arithmetic, with a small constant
            # for the product's own rounding
            assert err <= 4 * (k + 2) * EPS_DD * absab[i, j] * (1 + 2.0 ** -40)


def test_ddgemm_lo_parts_matter():
    """Each cross term a_hi b_lo and a_lo b_hi is ~2^-53 relative: an oracle
    that dropped either would miss the exact result by far more than the
    FP64x2 bound.  Also a non-square, non-symmetric case so a transposed
    operand cannot pass."""
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(5, 3, 9, seed=7)
    c_hi, c_lo = dd.ddgemm(a_hi, a_lo, b_hi, b_lo)
    for i in range(5):
        for j in range(3):
            ex = exact.exact_dot(a_hi[i], a_lo[i], b_hi[:, j], b_lo[:, j])
            no_lo = exact.exact_dot(a_hi[i], np.zeros(9), b_hi[:, j], np.zeros(9))
            gap = float(Fraction(abs(ex - no_lo), 1 << (2 * exact.SHIFT)))
            err = exact.err_vs_exact(c_hi[i, j], c_lo[i, j], ex)
            assert gap > 1e6 * err  # the lo parts are well above the oracle's error


def test_ddgemm_integers_exact():
    a_hi, a_lo, b_hi, b_lo = integer_inputs(9, 11, 600, bits=10, seed=4)
    c_hi, c_lo = dd.ddgemm(a_hi, a_lo, b_hi, b_lo)
    ref = a_hi.astype(np.int64) @ b_hi.astype(np.int64)
    assert np.array_equal(c_hi, ref.astype(np.float64))
    assert np.all(c_lo == 0)


def test_ddgemm_identity_and_permutation():
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(1, 12, 12, seed=5)
    eye = np.eye(12)
    # the generator's lo may reach ulp(hi), so the oracle may return another
    # (normalised) hi/lo split of the same value: compare exact values
    def same_values(ch, cl, bh, bl):
        return all(exact.dd_fixed(x, y) == exact.dd_fixed(u, v)
                   for x, y, u, v in zip(ch.ravel(), cl.ravel(), bh.ravel(), bl.ravel()))

    c_hi, c_lo = dd.ddgemm(eye, np.zeros_like(eye), b_hi, b_lo)
    assert same_values(c_hi, c_lo, b_hi, b_lo) and exact.dd_is_normalised(c_hi, c_lo)
    perm = np.random.default_rng(6).permutation(12)
    p = eye[perm]
    c_hi, c_lo = dd.ddgemm(p, np.zeros_like(p), b_hi, b_lo)
    assert same_values(c_hi, c_lo, b_hi[perm], b_lo[perm])


def test_ddgemm_empty_and_k0():
    a = np.zeros((3, 0))
    b = np.zeros((0, 4))
    c_hi, c_lo = dd.ddgemm(a, a, b, b)
    assert c_hi.shape == (3, 4) and not c_hi.any() and not c_lo.any()
    c_hi, c_lo = dd.ddgemm(np.zeros((0, 5)), np.zeros((0, 5)), np.ones((5, 2)), np.zeros((5, 2)))
    assert c_hi.shape == (0, 2)


def test_entries_match_full():
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(7, 9, 40, kind="wide", seed=8)
    c_hi, c_lo = dd.ddgemm(a_hi, a_lo, b_hi, b_lo)
    rows = np.array([0, 6, 3, 3])
    cols = np.array([8, 0, 4, 5])
    eh, el = dd.ddgemm_entries(a_hi, a_lo, b_hi, b_lo, rows, cols)
    assert np.array_equal(eh, c_hi[rows, cols]) and np.array_equal(el, c_lo[rows, cols])


def test_dd_add_relative_error_under_cancellation():
    """The accurate FP64x2 addition (two TwoSums, Sec. "FP64 and FP64x2
    numbers") errs by at most a few 2^-106 of |a + b| even when a + b
    cancels most of a and b; the one-TwoSum ("sloppy") addition does not
    (its error is relative to |a| + |b|), so this pins which one the
    oracle uses."""
    rng = np.random.default_rng(7)
    for _ in range(400):
        ah = float(rng.standard_normal())
        al = ah * 2.0 ** -53 * float(rng.uniform(-1, 1))
        # b = -a plus a small relative change, in both words
        d = 2.0 ** -float(rng.integers(1, 50))
        bh = -ah * (1.0 + d * float(rng.uniform(-1, 1)))
        bl = -al * float(rng.uniform(0.0, 2.0))
        rh, rl = dd.dd_add(ah, al, bh, bl)
        true = exact.dd_fixed(ah, al) + exact.dd_fixed(bh, bl)
        err = abs(exact.dd_fixed(rh, rl) - true)
        assert (err << 104) <= abs(true) + 1, (ah, al, bh, bl)
