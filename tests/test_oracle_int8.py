"""Pins for the INT8 restatement (oracle/cascade_int8.py).

  * rne_scaled equals round-half-even of the exact rational x 2^sh;
  * the digits reconstruct X exactly and lie in [-128, 127], the first in
    [-65, 65] (they fit INT8);
  * the fixed-point value is within 2^-F sigma of the FP64x2 entry;
  * diagonal sums equal brute-force integer dot products;
  * the whole INT8 cascade meets the error bound derived below against
    exact rationals, integer matrices come out exact, and the worked example
    of Sec. "Forward Error Analysis" gives fl_FP64(eps) like the FP64 form;
  * planted mistakes (a dropped diagonal, a digit off by one position, the
    wrong rounding) fail a pin.

Bound (per entry, per k-block p with scales sigma_p, tau_p and length k_p):
  conversion  2 k_p sigma tau 2^-F               (|delta x| <= 2^-F sigma)
  dropped     4.02 (s-1) k_p 2^-8s sigma tau     (diagonals i+j >= s, |digit| <= 128)
  assembly    4 s 2^-106 k_p sigma tau, and 4 K_B 2^-106 |A||B| across blocks."""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import cascade_int8 as c8
from oracle import dd
from tests import exact
from workloads import gemm_inputs, integer_inputs


def int8_bound(a_hi, b_hi, s, kb=None, bits=c8.BITS):
    """Per-entry bound of the INT8 form with s pieces of `bits` bits: the
    dropped-diagonal term is (s-1) k 2^(2 bits - 14) (1 + 2^(1-bits))
    2^(-bits s) sigma tau (|digit| <= 2^(bits-1)): 4.02 (s-1) k 2^-8s for
    eight bits, 1.01 (s-1) k 2^-7s for seven."""
    kb = kb or c8.kblock(bits)
    m, k = a_hi.shape
    n = b_hi.shape[1]
    e_a = c8.block_exponents(a_hi, kb)
    e_b = c8.block_exponents(np.ascontiguousarray(b_hi.T), kb)
    f = c8.frac_bits(s, bits)
    dropped = (s - 1) * 2.0 ** (2 * bits - 14) * (1 + 2.0 ** (1 - bits)) * 2.0 ** (-bits * s)
    tot = np.zeros((m, n))
    for p in range(e_a.shape[1]):
        kp = min(kb, k - p * kb)
        st = np.exp2(e_a[:, p][:, None] + e_b[:, p][None, :])
        tot += kp * st * (2.0 ** (1 - f) + dropped + 4 * s * 2.0 ** -106)
    return tot + 4 * e_a.shape[1] * 2.0 ** -106 * (np.abs(a_hi) @ np.abs(b_hi))


def test_rne_scaled_is_round_half_even():
    rng = np.random.default_rng(0)
    xs = list(rng.standard_normal(400) * np.exp2(rng.integers(-40, 40, 400)))
    xs += [0.5, 1.5, 2.5, -0.5, -1.5, 3 * 2.0 ** -10, 2.0 ** -1074, -(2.0 ** -60)]
    for x in xs:
        for sh in (-5, 0, 3, 60, 111):
            assert c8.rne_scaled(x, sh) == round(Fraction(x) * Fraction(2) ** sh)


@pytest.mark.parametrize("s,bits", [(8, 8), (12, 8), (15, 8), (12, 7), (16, 7)])
def test_digits_reconstruct_and_fit_int8(s, bits):
    """Every X the conversion produces (|X| <= 2^F + 1) has digits that fit
    INT8: balanced base 2^bits, the first within [-65, 65]."""
    rnd = random.Random(s)
    f = c8.frac_bits(s, bits)
    base, half = 1 << bits, 1 << (bits - 1)
    xs = [rnd.randint(-(2 ** f) - 1, 2 ** f + 1) >> rnd.randint(0, f) for _ in range(500)]
    xs += [2 ** f + 1, -(2 ** f) - 1, 2 ** f, -(2 ** f), 0, 1, -1, half, -half, half - 1,
           -half - 1, base - 1]
    for x in xs:
        ds = c8.digits(x, s, bits)
        assert all(-half <= d < half for d in ds[1:]) and -65 <= ds[0] <= 65, (x, ds)
        assert sum(d * base ** (s - 1 - i) for i, d in enumerate(ds)) == x


def test_fixed_point_conversion_error():
    a_hi, a_lo, _, _ = gemm_inputs(6, 1, 300, kind="wide", seed=2)
    e = c8.block_exponents(a_hi)
    s = 15
    f = c8.frac_bits(s)
    for i in range(6):
        assert 2.0 ** (e[i, 0] - 1) <= np.abs(a_hi[i]).max() < 2.0 ** e[i, 0]
        for l in range(300):
            x = c8.to_fixed(a_hi[i, l], a_lo[i, l], int(e[i, 0]), s)
            exact_scaled = (Fraction(a_hi[i, l]) + Fraction(a_lo[i, l])) * Fraction(2) ** (f - int(e[i, 0]))
            assert abs(x - exact_scaled) <= 1
            assert abs(x) <= 2 ** f


def test_diagonal_sums_brute_force():
    rng = np.random.default_rng(3)
    s, m, n, k = 5, 3, 4, 7
    da = rng.integers(-128, 128, (s, m, k))
    db = rng.integers(-128, 128, (s, n, k))
    got = c8.diagonal_sums(da, db, s)
    for t in range(s):
        for i in range(m):
            for j in range(n):
                want = sum(int(da[u, i, l]) * int(db[t - u, j, l]) for u in range(t + 1)
                           for l in range(k))
                assert got[t, i, j] == want


def max_ratio(fn, m, n, k, kind, seed, s, bits=c8.BITS):
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind=kind, seed=seed)
    c_hi, c_lo = fn(a_hi, a_lo, b_hi, b_lo, s=s)
    bound = int8_bound(a_hi, b_hi, s, bits=bits)
    worst = 0.0
    for i in range(m):
        for j in range(n):
            ex = exact.exact_dot(a_hi[i], a_lo[i], b_hi[:, j], b_lo[:, j])
            worst = max(worst, exact.err_vs_exact(c_hi[i, j], c_lo[i, j], ex) / bound[i, j])
    return worst


@pytest.mark.parametrize("m,n,k,kind,s,bits", [(5, 6, 200, "uniform", 15, 8),
                                               (4, 5, 300, "wide", 15, 8),
                                               (3, 3, 64, "uniform", 12, 8),
                                               (4, 4, 100, "wide", 13, 8),
                                               (4, 4, 120, "wide", 14, 8),
                                               (4, 5, 300, "wide", 16, 7),
                                               (3, 4, 90, "uniform", 14, 7)])
def test_int8_cascade_meets_bound(m, n, k, kind, s, bits):
    def fn(*a, s):
        return c8.cascade_int8_ddgemm(*a, s=s, bits=bits)
    assert max_ratio(fn, m, n, k, kind, k, s, bits) <= 1.0


def test_int8_cascade_near_fp64x2_on_uniform():
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(8, 8, 256, seed=4)
    c_hi, c_lo = c8.cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=15)
    o_hi, o_lo = dd.ddgemm(a_hi, a_lo, b_hi, b_lo)
    assert np.all(np.abs((c_hi - o_hi) + (c_lo - o_lo)) <= 1e-28 * (np.abs(a_hi) @ np.abs(b_hi)))
    assert exact.dd_is_normalised(c_hi, c_lo)


def test_int8_integers_exact():
    a_hi, a_lo, b_hi, b_lo = integer_inputs(5, 4, 120, bits=10, seed=5)
    c_hi, c_lo = c8.cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=6)
    ref = a_hi.astype(np.int64) @ b_hi.astype(np.int64)
    assert np.array_equal(c_hi, ref.astype(np.float64)) and np.all(c_lo == 0)


def test_int8_worked_example():
    eps_hi, eps_lo = 1.5 * 2.0 ** -71, 2.0 ** -130
    c_hi, c_lo = c8.cascade_int8_ddgemm(np.array([[1.0, eps_hi]]), np.array([[0.0, eps_lo]]),
                                        np.array([[0.0], [1.0]]), np.zeros((2, 1)), s=15)
    assert c_hi[0, 0] == eps_hi and c_lo[0, 0] == 0.0


# ---- exact assembly (the tensor-core form) ---------------------------------

def is_nearest(x: Fraction, v: float) -> bool:
    """v is a round-to-nearest-even double of x: no neighbour of v is
    closer, and an exact tie picks the even significand."""
    if v == 0.0:
        return abs(x) <= Fraction(2.0 ** -1075)
    up, down = math.nextafter(v, math.inf), math.nextafter(v, -math.inf)
    d = abs(x - Fraction(v))
    if d > abs(x - Fraction(up)) or d > abs(x - Fraction(down)):
        return False
    if d == abs(x - Fraction(up)) or d == abs(x - Fraction(down)):
        return (Fraction(v) / Fraction(math.ulp(v))).numerator % 2 == 0
    return True


def hard_block_values():
    """Exact integers T (and exponents) with ties and near-ties at both
    roundings, carries across 2^53, cancellation, and full-width values."""
    rnd = random.Random(9)
    out = []
    for _ in range(300):
        bits = rnd.randint(1, 143)
        out.append((rnd.choice((-1, 1)) * rnd.getrandbits(bits), rnd.randint(-140, 10)))
    for top in (2 ** 52 + 1, 2 ** 53 - 1, 2 ** 52, 3):
        for sh in (1, 2, 30, 53, 60, 64, 83, 90):
            half = 1 << (sh - 1)
            for rem in (half, half - 1, half + 1, 0):
                t = (top << sh) + rem
                out += [(t, -117), (-t, -50)]
                # a tie in the second rounding: lo = 2^54 + 1 then half an ulp
                t2 = (top << (sh + 56)) + (((1 << 54) + 1) << 2) + 2
                t3 = (top << (sh + 64)) + (((1 << 54) + 1) << 9) + (1 << 8)
                out += [(t2, -200), (t3, -230)]
    return out


def test_round_dd_is_the_nearest_fp64x2():
    for t, e in hard_block_values():
        hi, lo = c8.round_dd(t, e)
        x = Fraction(t) * Fraction(2) ** e
        assert is_nearest(x, hi), (t, e)
        assert is_nearest(x - Fraction(hi), lo), (t, e)


@pytest.mark.parametrize("s,bits", [(15, 8), (16, 7)])
def test_exact_assembly_brute_force(s, bits):
    """Block value of random diagonal sums against the exact rational sum of
    S_t 2^(-12-bits t) 2^scale, entry by entry."""
    rng = np.random.default_rng(11)
    diag = rng.integers(-(2 ** 31) + 1, 2 ** 31, (s, 3, 4))
    diag[:, 0, 0] = 0
    diag[5:, 1, 1] = 0                       # short expansions
    diag[0, 2, 3] = 15 * 2 ** 27             # the largest sum a k-block allows
    scale = rng.integers(-30, 30, (3, 4))
    h, l = c8.assemble_exact(diag, s, scale, bits)
    for i in range(3):
        for j in range(4):
            x = sum(Fraction(int(diag[t, i, j])) * Fraction(2) ** (-12 - bits * t)
                    for t in range(s))
            x *= Fraction(2) ** int(scale[i, j])
            assert is_nearest(x, h[i, j]) and is_nearest(x - Fraction(h[i, j]), l[i, j])


@pytest.mark.parametrize("m,n,k,kind,s,bits", [(5, 6, 200, "uniform", 15, 8),
                                               (4, 5, 300, "wide", 14, 8),
                                               (3, 3, 64, "uniform", 12, 8),
                                               (4, 5, 300, "wide", 16, 7)])
def test_exact_assembly_meets_bound(m, n, k, kind, s, bits):
    def fn(*a, s):
        return c8.cascade_int8_ddgemm(*a, s=s, assembly="exact", bits=bits)
    assert max_ratio(fn, m, n, k, kind, k + 1, s, bits) <= 1.0


def test_exact_assembly_integers_and_worked_example():
    a_hi, a_lo, b_hi, b_lo = integer_inputs(5, 4, 120, bits=10, seed=5)
    c_hi, c_lo = c8.cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=6, assembly="exact")
    ref = a_hi.astype(np.int64) @ b_hi.astype(np.int64)
    assert np.array_equal(c_hi, ref.astype(np.float64)) and np.all(c_lo == 0)
    eps_hi, eps_lo = 1.5 * 2.0 ** -71, 2.0 ** -130
    c_hi, c_lo = c8.cascade_int8_ddgemm(np.array([[1.0, eps_hi]]), np.array([[0.0, eps_lo]]),
                                        np.array([[0.0], [1.0]]), np.zeros((2, 1)), s=15,
                                        assembly="exact")
    assert c_hi[0, 0] == eps_hi and c_lo[0, 0] == 0.0


def test_exact_and_fp64x2_assembly_agree_closely():
    """Same diagonal sums, two assemblies: they differ by the FP64x2
    roundings of the smallest-first sum only."""
    a = gemm_inputs(6, 7, 500, kind="wide", seed=12)
    x_hi, x_lo = c8.cascade_int8_ddgemm(*a, s=15, assembly="exact")
    y_hi, y_lo = c8.cascade_int8_ddgemm(*a, s=15)
    diff = np.abs((x_hi - y_hi) + (x_lo - y_lo))
    assert np.all(diff <= 4 * 15 * 2.0 ** -106 * (np.abs(a[0]) @ np.abs(a[2])))


# ---- planted mistakes ------------------------------------------------------

def test_planted_exact_assembly_rounding_is_caught(monkeypatch):
    def truncating(num, exp2):
        # hi as it should be, lo rounded toward zero at 40 bits
        x = Fraction(num) * Fraction(2) ** exp2
        hi = float(x)
        lo = float(x - Fraction(hi))
        if lo:
            e = math.frexp(lo)[1]
            lo = math.ldexp(math.trunc(math.ldexp(lo, 40 - e)), e - 40)
        return hi, lo
    monkeypatch.setattr(c8, "round_dd", truncating)
    with pytest.raises(AssertionError):
        test_round_dd_is_the_nearest_fp64x2()


def test_planted_exact_assembly_weight_is_caught(monkeypatch):
    real = c8.round_dd
    monkeypatch.setattr(c8, "round_dd", lambda num, e: real(num, e + 1))
    with pytest.raises(AssertionError):
        test_exact_assembly_brute_force(15, 8)


def test_planted_dropped_diagonal_is_caught(monkeypatch):
    real = c8.diagonal_sums

    def drop_two(da, db, s):
        out = real(da, db, s)
        out[2] = 0
        return out
    monkeypatch.setattr(c8, "diagonal_sums", drop_two)
    assert max_ratio(c8.cascade_int8_ddgemm, 4, 4, 100, "uniform", 6, 15) > 1.0


def test_planted_digit_weight_is_caught(monkeypatch):
    real = c8.digits

    def shifted(x, s, bits=8):
        d = real(x, s, bits)
        return d[1:] + [0]      # every digit one place too high
    monkeypatch.setattr(c8, "digits", shifted)
    with pytest.raises(AssertionError):
        test_digits_reconstruct_and_fit_int8(15, 8)


def test_planted_rounding_is_caught(monkeypatch):
    monkeypatch.setattr(c8, "rne_scaled", lambda x, sh: math.floor(Fraction(x) * Fraction(2) ** sh))
    with pytest.raises(AssertionError):
        test_rne_scaled_is_round_half_even()


def test_first_block_add_into_zero_is_the_pair_itself():
    """The first k-block's FP64x2 add into C = (0, 0) (Sec. "Simple": the
    blocks are accumulated into C in FP64x2) returns the exactly rounded
    pair (RN(x), RN(x - RN(x))) unchanged, bit for bit, ties included: the
    tcgen05 kernels store that pair without an FP64 operation."""
    from oracle import cascade as cs
    rng = random.Random(12)
    cases = []
    for _ in range(3000):
        bits = rng.randrange(1, 140)
        num = rng.getrandbits(bits) * rng.choice((-1, 1))
        cases.append((num, rng.randrange(-200, 60)))
    for _ in range(500):                  # ties at the first rounding (x = hi + ulp/2)
        m = rng.getrandbits(53) | (1 << 52)
        sh = rng.randrange(1, 80)
        cases.append(((m << sh) + (1 << (sh - 1)), rng.randrange(-150, 0)))
        cases.append((-((m << sh) + (1 << (sh - 1))), rng.randrange(-150, 0)))
    for _ in range(500):                  # just below a power of two
        p = rng.randrange(54, 130)
        cases.append(((1 << p) - rng.randrange(1, 1 << 20), rng.randrange(-150, 0)))
    his, los = zip(*(c8.round_dd(num, e) for num, e in cases))
    h = np.array(his)
    lo = np.array(los)
    zh, zl = cs.dd_add(np.zeros_like(h), np.zeros_like(lo), h, lo)
    assert np.array_equal(zh.view(np.int64), h.view(np.int64))
    assert np.array_equal(zl.view(np.int64), lo.view(np.int64))
    assert not np.any((lo == 0) & np.signbit(lo))      # no -0 low word
