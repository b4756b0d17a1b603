"""Pins for the numpy restatement of the cascade (oracle/cascade.py).

Each property comes from the paper or from plain mathematics, not from the
code under test:
  * digit budget c = (22, 21, 21) from the inequalities of Sec. "Cascading
    vectors and dot products" at k = 256, eps_casc = 2^-117;
  * Appendix A's add/subtract trick rounds to a grid (checked against integer
    rounding);
  * a single FP64 splits exactly, pieces on their grids with |piece| <= 1;
    an FP64x2 splits within |delta x| sigma <= 2 eps_casc ||x||_inf
    (eq. sigma) and exactly when hi's leading bit is >= 2^-11 sigma;
  * bins 0-2 equal integer dot products of the integerised pieces (the
    "computed exactly" claim of Sec. "Cascading vectors and dot products");
  * the whole cascade meets eq. (cascerr) of Sec. "Forward error", summed
    over k-blocks, against exact rational products;
  * the worked example of Sec. "Forward Error Analysis" (golden file);
  * integer matrices come out exact; identity reproduces B.
The last tests plant plausible mistakes in the oracle and check that one of
these pins fails."""
import math
import os

import numpy as np
import pytest

from oracle import cascade as cs
from oracle import dd
from tests import exact
from tests.bounds import paper_bound
from workloads import gemm_inputs, integer_inputs

EPS_DD = 2.0 ** -106
EPS_CASC = 2.0 ** -117
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_digit_budget_for_short_blocks():
    """Sec. "Cascading vectors and dot products": "if k = 64 ... we allow
    c0 = 23"; every block length satisfies the four inequalities with equality
    or one to spare, and no digit could be wider."""
    assert cs.digit_budget(64)[0] == 23
    assert cs.digit_budget(256) == (22, 21, 21)
    for n in range(1, 257):
        c0, c1, c2 = cs.digit_budget(n)
        L = math.ceil(math.log2(n)) if n > 1 else 0
        assert 2 * c0 + L <= 53 < 2 * (c0 + 1) + L
        assert c0 + c1 + L + 1 <= 53 and 2 * c1 + L + 2 <= 53
        assert c0 + c1 + 1 + L + 1 > 53 or 2 * (c1 + 1) + L + 2 > 53
        assert c0 + c2 + L + 2 <= 53 < c0 + c2 + 1 + L + 2


def test_digit_budget_from_paper_inequalities():
    k = 256
    lg = int(math.log2(k))
    c0 = max(c for c in range(60) if 2 * c + lg <= 53)
    c1 = max(c for c in range(60) if c0 + c + lg + 1 <= 53 and 2 * c + lg + 2 <= 53)
    c2 = max(c for c in range(60) if c0 + c + lg + 2 <= 53)
    assert (c0, c1, c2) == (cs.C0, cs.C1, cs.C2) == (22, 21, 21)
    d0, d1, d2 = c0, c0 + c1, c0 + c1 + c2
    assert (cs.SIGMA1, cs.SIGMA2, cs.SIGMA3) == (2.0 ** -d0, 2.0 ** -d1, 2.0 ** -d2)
    assert d2 + 53 == 117  # eps_casc = 2^-(D2 + D)
    assert cs.KC == 256


@pytest.mark.parametrize("d", [21, 22])
def test_round_digits_is_grid_rounding(d):
    rng = np.random.default_rng(d)
    x = np.concatenate([rng.uniform(-1, 1, 4000),
                        rng.uniform(-1, 1, 1000) * np.exp2(-rng.integers(0, 60, 1000)),
                        [0.0, 2.0 ** -d, -(2.0 ** -d), 3 * 2.0 ** -d, 1 - 2.0 ** -53]])
    r = cs.round_digits(x, d)
    unit = 2.0 ** (1 - d)
    for xv, rv in zip(x.tolist(), r.tolist()):
        # nearest multiple of 2^(1-d), ties to even multiple
        q = xv / unit
        fl = math.floor(q)
        frac = q - fl
        want = fl + (1 if frac > 0.5 or (frac == 0.5 and fl % 2 == 1) else 0)
        assert rv == want * unit, (xv, rv)


def test_split_single_fp64_exact():
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, 3000) * np.exp2(-rng.integers(0, 80, 3000))
    x0, x1, x2, x3, *_ = cs.split_fp64(x)
    grid = [2.0 ** 21, 2.0 ** 20, 2.0 ** 20]
    for piece, g in zip((x0, x1, x2), grid):
        assert np.all(np.abs(piece) <= 1)
        assert np.all(piece * g == np.round(piece * g))
    assert np.all(np.abs(x3) <= 1)
    for v, a, b, c, d in zip(x, x0, x1, x2, x3):
        rec = (exact.fixed(a) << 64) + (exact.fixed(b) << 42) + (exact.fixed(c) << 21) + exact.fixed(d)
        assert rec == exact.fixed(v) << 64


@pytest.mark.parametrize("kind", ["uniform", "wide"])
def test_split_fp64x2_conversion_bound(kind):
    a_hi, a_lo, _, _ = gemm_inputs(16, 1, 256, kind=kind, seed=3)
    e = cs.block_exponents_rows(a_hi)
    assert e.shape == (16, 1)
    sig = np.exp2(e[:, 0])
    mx = np.abs(a_hi).max(axis=1)
    assert np.all((mx < sig) & (sig <= 2 * mx))  # ||x||_inf < sigma <= 2 ||x||_inf
    (x0, x1, x2, x3), _ = cs.cascade_entries(a_hi, a_lo, e)
    n_exact = 0
    for i in range(16):
        for l in range(256):
            rec = ((exact.fixed(x0[i, l]) << 64) + (exact.fixed(x1[i, l]) << 42)
                   + (exact.fixed(x2[i, l]) << 21) + exact.fixed(x3[i, l]))
            true = (exact.dd_fixed(a_hi[i, l], a_lo[i, l]) << 64) >> int(e[i, 0]) if e[i, 0] >= 0 \
                else (exact.dd_fixed(a_hi[i, l], a_lo[i, l]) << (64 - int(e[i, 0])))
            # both in units of 2^-(1074+64) of the scaled value x / sigma
            err = abs(rec - true)
            # eq. (sigma): |delta x| sigma <= 2 eps_casc ||x||_inf, i.e. in
            # units of sigma at most 2^-116
            assert err <= (1 << (1074 + 64)) >> 116
            lead = math.frexp(abs(a_hi[i, l]))[1] if a_hi[i, l] else -10 ** 9
            if lead - 1 >= int(e[i, 0]) - 11:
                assert err == 0
                n_exact += 1
    assert n_exact > 0


def test_tails_b4_b5_b6_within_one_rounding():
    _, _, b_hi, b_lo = gemm_inputs(1, 24, 256, kind="wide", seed=5)
    e = cs.block_exponents_cols(b_hi)
    b0, b1, b2, b3, b4, b5, b6 = cs.cascade_b(b_hi, b_lo, e, 0)
    s1, s2, s3 = cs.SIGMA1, cs.SIGMA2, cs.SIGMA3
    # undo the sigma factors of eq. (Gemm10) (exact powers of two)
    B0, B1, B2, B3 = b0, b1 / s1, b2 / s2, b3 / s3
    B4, B5 = b4 / s2, b5 / s1
    for l in range(256):
        for j in range(24):
            f = lambda v: exact.fixed(v)
            # B4 = B2 + B3 s3/s2, B5 = B1 + B2 s2/s1 + B3 s3/s1, B6 = B0 + s1 B1 + s2 B2 + s3 B3
            want4 = (f(B2[l, j]) << 21) + f(B3[l, j])
            want5 = (f(B1[l, j]) << 42) + (f(B2[l, j]) << 21) + f(B3[l, j])
            want6 = (f(B0[l, j]) << 64) + (f(B1[l, j]) << 42) + (f(B2[l, j]) << 21) + f(B3[l, j])
            for got, want, sh in ((B4[l, j], want4, 21), (B5[l, j], want5, 42), (b6[l, j], want6, 64)):
                g = f(got) << sh
                ulp = math.ulp(got) if got else 2.0 ** -1074
                # one rounding of the tail, plus the one rounding of chunk 3
                assert abs(g - want) <= (exact.fixed(ulp) << sh) + (exact.fixed(math.ulp(1.0)) << 0)


@pytest.mark.parametrize("kind", ["uniform", "wide"])
@pytest.mark.parametrize("k", [256, 100, 64, 3])
def test_bins_0_to_2_are_exact_integer_dots(kind, k):
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(12, 10, k, kind=kind, seed=21)
    e_a = cs.block_exponents_rows(a_hi)
    e_b = cs.block_exponents_cols(b_hi)
    As = cs.cascade_a(a_hi, a_lo, e_a, 0)
    Bs = cs.cascade_b(b_hi, b_lo, e_b, 0)
    bin0, bin1, bin2, _ = cs.ten_products(As, Bs)

    def ints(x, unit_exp):
        y = np.ldexp(x, unit_exp)
        assert np.all(y == np.round(y))
        return [[int(v) for v in row] for row in y.tolist()]

    # scaled panels: A0 on the grid 2^(1-c0), s1 A1 on 2^(1-c0-c1), s2 A2 on
    # 2^(1-c0-c1-c2) (2^-21, 2^-42, 2^-63 for a full block); B likewise
    c0, c1, c2 = cs.digit_budget(k)
    g0, g1, g2 = c0 - 1, c0 + c1 - 1, c0 + c1 + c2 - 1
    A0, A1, A2 = ints(As[0], g0), ints(As[1], g1), ints(As[2], g2)
    B0, B1, B2 = (ints(Bs[0].T, g0), ints(Bs[1].T, g1), ints(Bs[2].T, g2))

    def dot(x, y):
        return sum(p * q for p, q in zip(x, y))

    for i in range(12):
        for j in range(10):
            b0 = dot(A0[i], B0[j])                                  # units 2^-(2 g0)
            b1 = dot(A0[i], B1[j]) + dot(A1[i], B0[j])              # units 2^-(g0 + g1)
            assert abs(b0) < 2 ** 53 and abs(b1) < 2 ** 53
            assert bin0[i, j] == math.ldexp(b0, -2 * g0)
            assert bin1[i, j] == math.ldexp(b1, -(g0 + g1))
            # A0 B2 and A2 B0 are on 2^-(g0 + g2), A1 B1 on 2^-(2 g1): common unit
            u = max(g0 + g2, 2 * g1)
            b2u = ((dot(A0[i], B2[j]) + dot(A2[i], B0[j])) << (u - g0 - g2)) + \
                (dot(A1[i], B1[j]) << (u - 2 * g1))
            assert abs(b2u) < 2 ** 53
            assert bin2[i, j] == math.ldexp(b2u, -u)


def max_bound_ratio(fn, m, n, k, kind, seed):
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind=kind, seed=seed)
    c_hi, c_lo = fn(a_hi, a_lo, b_hi, b_lo)
    bound = paper_bound(a_hi, b_hi)
    worst = 0.0
    for i in range(m):
        for j in range(n):
            ex = exact.exact_dot(a_hi[i], a_lo[i], b_hi[:, j], b_lo[:, j])
            worst = max(worst, exact.err_vs_exact(c_hi[i, j], c_lo[i, j], ex) / bound[i, j])
    return worst


@pytest.mark.parametrize("m,n,k,kind", [(6, 7, 200, "uniform"), (5, 6, 530, "wide"),
                                        (4, 4, 1, "uniform"), (3, 5, 257, "wide")])
def test_cascade_meets_paper_bound(m, n, k, kind):
    assert max_bound_ratio(cs.cascade_ddgemm, m, n, k, kind, seed=k) <= 1.0


def test_cascade_vs_dd_oracle_contract():
    """The accuracy contract |C - C_dd| <= 1e-28 (|A||B|) holds for the
    cascade restated on the CPU (uniform and wide inputs)."""
    for kind in ("uniform", "wide"):
        a_hi, a_lo, b_hi, b_lo = gemm_inputs(40, 48, 600, kind=kind, seed=9)
        c_hi, c_lo = cs.cascade_ddgemm(a_hi, a_lo, b_hi, b_lo)
        o_hi, o_lo = dd.ddgemm(a_hi, a_lo, b_hi, b_lo)
        diff = np.abs((c_hi - o_hi) + (c_lo - o_lo))
        assert np.all(diff <= 1e-28 * exact.abs_product(a_hi, b_hi))
        assert exact.dd_is_normalised(c_hi, c_lo)


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals[key] = np.array([float.fromhex(t) if key != "pad_to" else int(t) for t in rest])
    return vals


def worked_example_vectors():
    """x, y of the worked example, zero-padded to the fixture's pad_to."""
    g = _read_golden("worked_example.txt")
    k = int(g["pad_to"][0])
    out = {}
    for key in ("x_hi", "x_lo", "y_hi", "y_lo"):
        v = np.zeros(k)
        v[:g[key].size] = g[key]
        out[key] = v
    return g, out


def test_worked_example_golden():
    g, v = worked_example_vectors()
    a_hi, a_lo = v["x_hi"][None, :], v["x_lo"][None, :]
    b_hi, b_lo = v["y_hi"][:, None], v["y_lo"][:, None]
    c_hi, c_lo = cs.cascade_ddgemm(a_hi, a_lo, b_hi, b_lo)
    assert c_hi[0, 0] == g["cascade_hi"][0] and c_lo[0, 0] == g["cascade_lo"][0]
    o_hi, o_lo = dd.ddgemm(a_hi, a_lo, b_hi, b_lo)
    assert o_hi[0, 0] == g["fp64x2_hi"][0] and o_lo[0, 0] == g["fp64x2_lo"][0]


@pytest.mark.parametrize("k", [100, 256, 700])
def test_integers_exact(k):
    a_hi, a_lo, b_hi, b_lo = integer_inputs(9, 7, k, bits=10, seed=k)
    c_hi, c_lo = cs.cascade_ddgemm(a_hi, a_lo, b_hi, b_lo)
    ref = a_hi.astype(np.int64) @ b_hi.astype(np.int64)
    assert np.array_equal(c_hi, ref.astype(np.float64)) and np.all(c_lo == 0)


def test_identity_reproduces_b():
    _, _, b_hi, b_lo = gemm_inputs(1, 20, 300, seed=12)
    eye = np.eye(300)
    c_hi, c_lo = cs.cascade_ddgemm(eye, np.zeros_like(eye), b_hi, b_lo)
    for x, y, u, v in zip(c_hi.ravel(), c_lo.ravel(), b_hi.ravel(), b_lo.ravel()):
        err = abs(exact.dd_fixed(x, y) - exact.dd_fixed(u, v))
        assert err <= exact.fixed(abs(u)) >> 104


def test_empty_shapes():
    c_hi, c_lo = cs.cascade_ddgemm(np.zeros((3, 0)), np.zeros((3, 0)), np.zeros((0, 2)), np.zeros((0, 2)))
    assert c_hi.shape == (3, 2) and not c_hi.any() and not c_lo.any()
    c_hi, _ = cs.cascade_ddgemm(np.zeros((0, 4)), np.zeros((0, 4)), np.ones((4, 2)), np.zeros((4, 2)))
    assert c_hi.shape == (0, 2)


# ---- planted mistakes: each must make a pin above fail --------------------

def _planted(monkeypatch, name, fn):
    monkeypatch.setattr(cs, name, fn)


def test_planted_dropped_product_is_caught(monkeypatch):
    real = cs.ten_products

    def drop_a3b6(As, Bs):
        b0, b1, b2, b36 = real(As, Bs)
        return b0, b1, b2, b36 - As[3] @ Bs[6]
    _planted(monkeypatch, "ten_products", drop_a3b6)
    assert max_bound_ratio(cs.cascade_ddgemm, 5, 6, 300, "uniform", seed=1) > 1.0


def test_planted_wrong_sigma_is_caught(monkeypatch):
    real_a = cs.cascade_a

    def swapped(a_hi, a_lo, e_a, p, kc=cs.KC):
        a0, a1, a2, a3 = real_a(a_hi, a_lo, e_a, p, kc)
        return a0, a1 * 2.0, a2, a3       # sigma_1 off by one bit
    _planted(monkeypatch, "cascade_a", swapped)
    assert max_bound_ratio(cs.cascade_ddgemm, 5, 6, 300, "uniform", seed=2) > 1.0


def test_planted_transposed_tail_is_caught(monkeypatch):
    real_b = cs.cascade_b

    def wrong_tails(b_hi, b_lo, e_b, p, kc=cs.KC):
        b = list(real_b(b_hi, b_lo, e_b, p, kc))
        b[4], b[5] = b[5] * (cs.SIGMA2 / cs.SIGMA1), b[4] * (cs.SIGMA1 / cs.SIGMA2)  # B4 <-> B5
        return tuple(b)
    _planted(monkeypatch, "cascade_b", wrong_tails)
    assert max_bound_ratio(cs.cascade_ddgemm, 5, 6, 300, "wide", seed=3) > 1.0


def test_planted_sign_error_in_two_sum_is_caught(monkeypatch):
    def bad_two_sum(a, b):
        s = a + b
        bv = s - a
        av = s - bv
        return s, (a - av) - (b - bv)
    _planted(monkeypatch, "two_sum", bad_two_sum)
    assert max_bound_ratio(cs.cascade_ddgemm, 5, 6, 300, "uniform", seed=4) > 1.0


def test_planted_rounding_constant_is_caught(monkeypatch):
    _planted(monkeypatch, "_round_const", lambda d: 2.0 ** (53 - d))  # the "2^{53-d}" only
    with pytest.raises(AssertionError):
        test_round_digits_is_grid_rounding(22)


def test_planted_scale_exponent_is_caught(monkeypatch):
    real = cs.block_exponents_rows

    def off_by_one(x_hi, kc=cs.KC):
        return real(x_hi, kc) - 1          # sigma no longer above max |x|
    _planted(monkeypatch, "block_exponents_rows", off_by_one)
    with pytest.raises(AssertionError):
        test_split_fp64x2_conversion_bound("uniform")


@pytest.mark.parametrize("kind", ["uniform", "wide"])
def test_folding_bins_3_to_6_is_not_dropping_them(kind):
    """Sec. "Cascading matrices and GEMM": folding bins 3-6 into four
    products (eq. Gemm10) is not the same as dropping bins 4-6, though both
    give ten products.  Against exact rationals the folded form matches all
    sixteen products of eq. (Gemm16) to within FP64x2 rounding, while
    dropping bins 4-6 is orders of magnitude worse."""
    a = gemm_inputs(10, 10, 300, kind=kind, seed=77)
    absab = exact.abs_product(a[0], a[2])
    worst = {}
    for mode in ("gemm10", "gemm16", "drop456"):
        h, l = cs.cascade_ddgemm(*a, products=mode)
        w = 0.0
        for i in range(10):
            for j in range(10):
                ex = exact.exact_dot(a[0][i], a[1][i], a[2][:, j], a[3][:, j])
                w = max(w, exact.err_vs_exact(h[i, j], l[i, j], ex) / absab[i, j])
        worst[mode] = w
    assert worst["gemm10"] <= 4 * worst["gemm16"] + 2.0 ** -104
    assert worst["gemm16"] <= 4 * worst["gemm10"] + 2.0 ** -104
    assert worst["drop456"] > 1e3 * worst["gemm10"]
    assert max_bound_ratio(lambda *x: cs.cascade_ddgemm(*x, products="gemm16"),
                           5, 6, 300, kind, seed=8) <= 1.0
