"""The cascading GEMM's own steps, written plainly in numpy FP64.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA product path, and it never imports that path.

Source: Parikh, van de Geijn, Henry, "Cascading GEMM: High Precision from Low
Precision" (arXiv 2303.04353).  Each function cites the passage it follows.
The definition of the *target* quantity (the double-double GEMM itself) is
the C oracle in ``dd_oracle.c``; this module restates the approximation
the paper builds, step by step and in the paper's order:

  1. scales sigma, tau per row of A / column of B and per k-block
     (Sec. "Cascading vectors and dot products"; Appendix A),
  2. the split of every FP64x2 entry into four FP64 pieces
     (Appendix A, "Cascading a FP64x2: technical details"),
  3. the combined panels B4, B5, B6 (Sec. "Cascading matrices and GEMM"),
  4. the ten FP64 products of eq. (Gemm10) accumulated into four bins,
  5. the sum across bins from bin 3-6 up to bin 0 in FP64x2, the Sigma/T
     scaling, and FP64x2 accumulation over k-blocks
     (Sec. "Simple: FP64x2 GEMM via ten FP64 GEMMs").

Readings where the paper is silent or garbled:
  * sigma = 2**e with e the frexp exponent of max |hi| over the block, i.e.
    the smallest power of two strictly above the largest magnitude; an
    all-zero block gets sigma = 1.
  * Scales are per (row, k-block of K_C = 256) for A and per (k-block,
    column) for B: the exactness argument is made for dot products of
    length k <= K_C, and the paper cascades per packed K_C panel.
  * The rounding constant of Appendix A is used literally,
    M_d = 2**(53-d) + 2**(52-d), one add then one subtract; chunks are then
    multiples of 2**(1-d) with |chunk| <= 1.  (The appendix's "2^{53-c-1}"
    in the second stage is read as 2^{53-c_1}.)
  * c follows the digit budget of the block's own length L = ceil(log2 len)
    (the paper widens the splits for small k): (22, 21, 21) for full
    256-entry blocks, (23, 22, 22) for 64, (26, 25, 25) for one entry.
  * B4, B5, B6 are the FP64 roundings of the exact remainders the split
    already holds (one rounding each), equal in exact arithmetic to the
    paper's B2 + B3 s3/s2, B1 + B2 s2/s1 + B3 s3/s1, B0 + s1 B1 + s2 B2 +
    s3 B3.
  * Within a bin, products are added in FP64; bin 3-6 is summed as
    ((A0 B3 + A1 B4) + A2 B5) + A3 B6.
"""
from __future__ import annotations

import numpy as np

# K_C: the k-block the exactness argument is made for (Sec. "Blocking for
# the k dimension"; Sec. "Simple", k_C = 256).
KC = 256
# Digits per fixed-width split at k = 256 (Sec. "Cascading vectors and dot
# products": 2 c0 + log2 k <= 53 etc. gives c0 = 22, c1 = 21, c2 = 21).
C0, C1, C2 = 22, 21, 21
# sigma_1 = 2^-D0, sigma_2 = 2^-D1, sigma_3 = 2^-D2 with D0 = c0,
# D1 = c0 + c1, D2 = c0 + c1 + c2 (glossary; Sec. "Cascading scalars").
SIGMA1 = 2.0 ** -C0
SIGMA2 = 2.0 ** -(C0 + C1)
SIGMA3 = 2.0 ** -(C0 + C1 + C2)


def digit_budget(block_len: int):
    """(c0, c1, c2) for a k-block of `block_len` entries, from the
    inequalities of Sec. "Cascading vectors and dot products" with
    L = ceil(log2 block_len): 2 c0 + L <= 53 (bin 0); c0 + c1 + L + 1 <= 53
    and 2 c1 + L + 2 <= 53 (bins 1 and 2); c0 + c2 + L + 2 <= 53 (bin 2).
    The paper allows wider splits when k is smaller ("if k = 64 ... c0 = 23")."""
    L = max(0, (int(block_len) - 1).bit_length())
    c0 = (53 - L) // 2
    c1 = min(53 - c0 - L - 1, (53 - L - 2) // 2)
    c2 = 53 - c0 - L - 2
    return c0, c1, c2


def sigmas(c):
    """sigma_1 = 2^-D0, sigma_2 = 2^-D1, sigma_3 = 2^-D2 for digits c."""
    c0, c1, c2 = c
    return 2.0 ** -c0, 2.0 ** -(c0 + c1), 2.0 ** -(c0 + c1 + c2)


def _round_const(d: int) -> float:
    """Appendix A, second observation: 2^(53-d) + 2^(53-d-1), precomputed."""
    return 2.0 ** (53 - d) + 2.0 ** (52 - d)


def round_digits(x: np.ndarray, d: int) -> np.ndarray:
    """Appendix A: add then subtract 2^(53-d) + 2^(53-d-1) in FP64.

    For |x| < 1 the sum stays in [2^(53-d), 2^(54-d)), whose spacing is
    2^(1-d), so the result is x rounded to a multiple of 2^(1-d)."""
    m = _round_const(d)
    x = np.asarray(x, dtype=np.float64)
    return (x + m) - m


def block_exponents_rows(x_hi: np.ndarray, kc: int = KC) -> np.ndarray:
    """e[i, p] with sigma = 2^e > max_{l in block p} |x_hi[i, l]|.

    Sec. "Cascading vectors and dot products": divide a vector by the
    smallest power of two greater than its largest element; Appendix A:
    sigma_0 = 2^e, e the exponent of the largest element.  Rows of A are the
    vectors x; each K_C-wide block of columns is cascaded on its own."""
    m, k = x_hi.shape
    kb = (k + kc - 1) // kc
    e = np.zeros((m, kb), dtype=np.int64)
    for p in range(kb):
        blk = np.abs(x_hi[:, p * kc:(p + 1) * kc])
        mx = blk.max(axis=1) if blk.shape[1] else np.zeros(m)
        e[:, p] = np.frexp(mx)[1]          # frexp(0) gives exponent 0
    return e


def block_exponents_cols(y_hi: np.ndarray, kc: int = KC) -> np.ndarray:
    """e[p, j] for the columns of B (the vectors y), per k-block p."""
    return block_exponents_rows(np.ascontiguousarray(y_hi.T), kc).T.copy()


def split_fp64(x: np.ndarray, c=(C0, C1, C2)):
    """Appendix A for one FP64 array already scaled by 2^-e.

    Returns (x0, x1, x2, x3, r0, r1, r2): the four splits and the running
    values the appendix holds before each rounding stage (r0 = the scaled
    input, r1 after removing x0 and shifting by 2^c0, r2 after removing x1
    and shifting by 2^c1).  Every subtraction and shift here is exact."""
    c0, c1, c2 = c
    r0 = np.asarray(x, dtype=np.float64)
    x0 = round_digits(r0, c0)
    r1 = (r0 - x0) * 2.0 ** c0
    x1 = round_digits(r1, c1)
    r2 = (r1 - x1) * 2.0 ** c1
    x2 = round_digits(r2, c2)
    x3 = (r2 - x2) * 2.0 ** c2
    return x0, x1, x2, x3, r0, r1, r2


def cascade_entries(hi: np.ndarray, lo: np.ndarray, e: np.ndarray, c=(C0, C1, C2)):
    """Appendix A: scale hi and lo by 2^-e, split each, add the splits.

    chi_i = chi_hi,i + chi_lo,i (exact for i <= 2; one rounding for i = 3).
    Also returns the FP64 roundings of the exact tails used for B4, B5, B6:
    t1 = fl(r1_hi + r1_lo), t2 = fl(r2_hi + r2_lo), t0 = fl(r0_hi + r0_lo)."""
    h = split_fp64(np.ldexp(hi, -e), c)
    l = split_fp64(np.ldexp(lo, -e), c)
    chunks = tuple(h[i] + l[i] for i in range(4))
    t0, t1, t2 = (h[4] + l[4], h[5] + l[5], h[6] + l[6])
    return chunks, (t0, t1, t2)


def block_digits(k, p, kc=KC):
    """Digits of k-block p: the budget of its length."""
    return digit_budget(min(kc, k - p * kc))


def cascade_a(a_hi, a_lo, e_a, p, kc=KC):
    """Row panel p of A -> [A0; s1 A1; s2 A2; s3 A3] (left factor of Gemm10)."""
    sl = slice(p * kc, (p + 1) * kc)
    e = e_a[:, p:p + 1]
    c = block_digits(a_hi.shape[1], p, kc)
    s1, s2, s3 = sigmas(c)
    (a0, a1, a2, a3), _ = cascade_entries(a_hi[:, sl], a_lo[:, sl], e, c)
    return a0, s1 * a1, s2 * a2, s3 * a3


def cascade_b(b_hi, b_lo, e_b, p, kc=KC):
    """Row panel p of B -> [B0 | s1 B1 | s2 B2 | s3 B3 || s2 B4 | s1 B5 | B6].

    Sec. "Cascading matrices and GEMM": B4 = B2 + B3 s3/s2,
    B5 = B1 + B2 s2/s1 + B3 s3/s1, B6 = B0 + s1 B1 + s2 B2 + s3 B3; in exact
    arithmetic these are the tails t2, t1, t0 the split already holds."""
    sl = slice(p * kc, (p + 1) * kc)
    e = e_b[p:p + 1, :]
    c = block_digits(b_hi.shape[0], p, kc)
    s1, s2, s3 = sigmas(c)
    (b0, b1, b2, b3), (t0, t1, t2) = cascade_entries(b_hi[sl, :], b_lo[sl, :], e, c)
    b4, b5, b6 = t2, t1, t0
    return b0, s1 * b1, s2 * b2, s3 * b3, s2 * b4, s1 * b5, b6


def ten_products(As, Bs):
    """Eq. (Gemm10): the ten FP64 products, added within their bins in FP64.

    bin 0   = A0 B0
    bin 1   = s1 A0 B1 + s1 A1 B0
    bin 2   = s2 A0 B2 + s1^2 A1 B1 + s2 A2 B0
    bin 3-6 = s3 A0 B3 + s1 s2 A1 B4 + s2 s1 A2 B5 + s3 A3 B6
    (the sigma factors are already inside the scaled panels)."""
    a0, a1, a2, a3 = As
    b0, b1, b2, b3, b4, b5, b6 = Bs
    bin0 = a0 @ b0
    bin1 = a0 @ b1 + a1 @ b0
    bin2 = (a0 @ b2 + a1 @ b1) + a2 @ b0
    bin36 = ((a0 @ b3 + a1 @ b4) + a2 @ b5) + a3 @ b6
    return bin0, bin1, bin2, bin36


def sixteen_products(As, Bs):
    """Eq. (Gemm16): all sixteen products; bins 0-2 as in eq. (Gemm10), and
    every lower product (bins 3-6) summed in FP64 in the order of the
    equation's rows: s3 A0 B3; s1 s2 A1 B2, s1 s3 A1 B3; s2 s1 A2 B1,
    s2^2 A2 B2, s2 s3 A2 B3; s3 A3 B0, s3 s1 A3 B1, s3 s2 A3 B2, s3^2 A3 B3.
    (Accuracy ablation; the method itself is ten_products.)"""
    a0, a1, a2, a3 = As
    b0, b1, b2, b3 = Bs[:4]
    bin0 = a0 @ b0
    bin1 = a0 @ b1 + a1 @ b0
    bin2 = (a0 @ b2 + a1 @ b1) + a2 @ b0
    lower = [a0 @ b3, a1 @ b2, a1 @ b3, a2 @ b1, a2 @ b2, a2 @ b3, a3 @ b0, a3 @ b1, a3 @ b2,
             a3 @ b3]
    bin36 = lower[0]
    for t in lower[1:]:
        bin36 = bin36 + t
    return bin0, bin1, bin2, bin36


def dropped_products(As, Bs):
    """Ten products by dropping bins 4-6 altogether: bins 0-3 of eq. (Gemm16)
    only (the alternative the paper contrasts with folding bins 3-6 into
    four products).  Accuracy ablation."""
    a0, a1, a2, a3 = As
    b0, b1, b2, b3 = Bs[:4]
    bin0 = a0 @ b0
    bin1 = a0 @ b1 + a1 @ b0
    bin2 = (a0 @ b2 + a1 @ b1) + a2 @ b0
    bin3 = ((a0 @ b3 + a1 @ b2) + a2 @ b1) + a3 @ b0
    return bin0, bin1, bin2, bin3


PRODUCT_RULES = {"gemm10": "ten_products", "gemm16": "sixteen_products",
                 "drop456": "dropped_products"}


def two_sum(a, b):
    """Knuth TwoSum, element-wise: s + e == a + b exactly."""
    s = a + b
    bv = s - a
    av = s - bv
    return s, (a - av) + (b - bv)


def fast_two_sum(a, b):
    """Dekker's quick-two-sum (Sec. "Cascading vectors and dot products"
    cites it for adding across bins 0-2); needs |a| >= |b|."""
    s = a + b
    return s, b - (s - a)


def dd_add_d(h, l, b):
    """FP64x2 (h, l) + FP64 b."""
    s, e = two_sum(h, b)
    e = e + l
    return fast_two_sum(s, e)


def dd_add(ah, al, bh, bl):
    """FP64x2 + FP64x2 (two TwoSums, two renormalisations)."""
    s, e = two_sum(ah, bh)
    t, f = two_sum(al, bl)
    e = e + t
    s, e = fast_two_sum(s, e)
    e = e + f
    return fast_two_sum(s, e)


def assemble_bins(bin0, bin1, bin2, bin36):
    """Sec. "Simple": add bin 3-6, then bin 2, bin 1, bin 0, in FP64x2, so
    that the likely lower-order terms go in first."""
    h, l = two_sum(bin2, bin36)
    h, l = dd_add_d(h, l, bin1)
    h, l = dd_add_d(h, l, bin0)
    return h, l


def cascade_ddgemm(a_hi, a_lo, b_hi, b_lo, kc=KC, return_bins=False, products="gemm10"):
    """C := A B approximated by the ten-GEMM cascade, k staged by K_C.

    Sec. "Simple": C is built as a sequence of rank-K_C updates; each update
    is cascaded, computed as ten FP64 products into four bins, assembled in
    FP64x2, scaled by Sigma and T (exact powers of two), and added into C in
    FP64x2.  Row-major float64 inputs; returns (C_hi, C_lo).  `products`
    selects eq. (Gemm10) (the method), eq. (Gemm16) or dropping bins 4-6."""
    a_hi = np.asarray(a_hi, np.float64)
    a_lo = np.asarray(a_lo, np.float64)
    b_hi = np.asarray(b_hi, np.float64)
    b_lo = np.asarray(b_lo, np.float64)
    m, k = a_hi.shape
    n = b_hi.shape[1]
    c_hi = np.zeros((m, n))
    c_lo = np.zeros((m, n))
    e_a = block_exponents_rows(a_hi, kc)
    e_b = block_exponents_cols(b_hi, kc)
    bins = []
    for p in range((k + kc - 1) // kc):
        As = cascade_a(a_hi, a_lo, e_a, p, kc)
        Bs = cascade_b(b_hi, b_lo, e_b, p, kc)
        b4 = globals()[PRODUCT_RULES[products]](As, Bs)
        if return_bins:
            bins.append(b4)
        h, l = assemble_bins(*b4)
        scale = e_a[:, p][:, None] + e_b[p, :][None, :]
        h, l = np.ldexp(h, scale), np.ldexp(l, scale)
        c_hi, c_lo = dd_add(c_hi, c_lo, h, l)
    if return_bins:
        return c_hi, c_lo, bins, (e_a, e_b)
    return c_hi, c_lo
