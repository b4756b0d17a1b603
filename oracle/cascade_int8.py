"""The cascade re-sliced into INT8 pieces, step by step (plain Python ints
and numpy int64; exact).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper sketches this form in Sec. "FP64x2 in terms of INT8": convert each
operand to fixed point, store it as about 15 INT8 pieces, compute the
pair-products that matter (the triangle i + j <= s - 1, Sec. "Safely dropping
lower order bins") with 32-bit integer accumulation, and add the results
across bins in FP64x2.  The paper gives no further detail; the readings
below fill it in.

  * Scale: sigma = 2^e per (row of A, k-block) and per (k-block, column of
    B), e the frexp exponent of max |hi| in the block, as in the FP64 form.
    The k-block is KB8 = 8192 entries: the longest power of two whose
    diagonal sums stay inside int32 for up to 15 pieces (|digit| <= 128:
    15 * 8192 * 2^14 < 2^31).
  * Fixed point: X = rne(x_hi 2^(F-e)) + rne(x_lo 2^(F-e)), an integer,
    with F = 6 + 8 (s - 1) fraction bits (rne = round to nearest, ties to
    even); |X| <= 2^F + 1 fits a signed 128-bit integer for s <= 15.
  * Pieces: the balanced base-2^8 digits of X, most significant first:
    X = sum_i d_i 256^(s-1-i), d_i in [-128, 127] (the first one in
    [-65, 65]), so x / sigma ~ sum_i d_i 2^(-6-8i).  Each piece fits INT8:
    the paper's "about 15 INT8 pieces" of eight bits each.
  * Products: for every diagonal t = i + j <= s - 1 the integer sum
    S_t = sum_{i+j=t} sum_l dA_i[l] dB_j[l] (exact in int32).
  * Assembly: for t = s-1 down to 0 (smallest first), v = S_t 2^(-12-8t)
    (exact in FP64) is added into an FP64x2 sum (TwoSum, add lo,
    FastTwoSum); the block result is scaled by sigma tau and added into C
    with the FP64x2 add, as in the FP64 form.
  * Exact assembly (assembly="exact"; the tensor-core form of the library
    uses it): the diagonal sums are integers, so the block value
    sum_t S_t 2^(-12-8t) sigma tau is formed exactly and rounded once to the
    nearest FP64x2 (hi = RN(x), lo = RN(x - hi)); the blocks are then added
    into C with the FP64x2 add as above.
  * Digit width (bits): the mma.sync form takes eight-bit pieces; the
    tcgen05 form takes seven-bit pieces (balanced base 128, d in [-64, 64],
    F = 6 + 7 (s - 1), k-blocks of 16384, s up to 16), whose products its FP32
    accumulators sum exactly over 256 entries instead of 64.  Every formula
    above holds with 8 replaced by bits.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import cascade as _fp64

BITS = 8                      # digit width of the INT8 form (mma.sync)
BITS_TC = 7                   # digit width of its tcgen05 form (see below)


def kblock(bits: int = BITS) -> int:
    """Longest power-of-two k-block whose int32 diagonal sums stay exact:
    8192 for eight-bit pieces (15 * 8192 * 2^14 < 2^31), 16384 for seven-bit
    ones (up to 18 pieces: 18 * 16384 * 2^12 < 2^31)."""
    return 8192 if bits == 8 else 16384


KB8 = kblock(BITS)
SLICES = {8: (12, 13, 14, 15), 7: (12, 13, 14, 15, 16)}   # F + 2 <= 127 bits


def frac_bits(s: int, bits: int = BITS) -> int:
    return 6 + bits * (s - 1)


def rne_scaled(x: float, sh: int) -> int:
    """round-half-even(x * 2^sh) as a Python int (exact)."""
    num, den = float(x).as_integer_ratio()     # den is a power of two
    p = sh - (den.bit_length() - 1)
    if p >= 0:
        return num << p
    q, r = divmod(num, 1 << -p)                # floor division, 0 <= r < 2^-p
    half = 1 << (-p - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return q


def to_fixed(hi: float, lo: float, e: int, s: int, bits: int = BITS) -> int:
    f = frac_bits(s, bits)
    return rne_scaled(hi, f - e) + rne_scaled(lo, f - e)


def digits(x: int, s: int, bits: int = BITS) -> list[int]:
    """Balanced base-2^bits digits of x, most significant first."""
    base, half = 1 << bits, 1 << (bits - 1)
    out = [0] * s
    for i in range(s - 1, 0, -1):
        d = ((x + half) & (base - 1)) - half
        out[i] = d
        x = (x - d) >> bits
    out[0] = x
    return out


def block_exponents(x_hi: np.ndarray, kb: int = KB8) -> np.ndarray:
    """e[v, p] for vectors along the rows of x_hi (reuses the FP64 form's
    rule; only the block length differs)."""
    return _fp64.block_exponents_rows(x_hi, kb)


def digit_planes(x_hi, x_lo, e, s, kb=KB8, bits=BITS):
    """Pieces of every row of x (vectors along rows): int64 [s][rows][k]."""
    rows, k = x_hi.shape
    out = np.zeros((s, rows, k), dtype=np.int64)
    for v in range(rows):
        for l in range(k):
            ds = digits(to_fixed(x_hi[v, l], x_lo[v, l], int(e[v, l // kb]), s, bits), s, bits)
            out[:, v, l] = ds
    return out


def diagonal_sums(da: np.ndarray, db: np.ndarray, s: int) -> np.ndarray:
    """S_t = sum_{i+j=t} dA_i dB_j^T for t = 0..s-1 (int64, exact).
    da: [s][m][k], db: [s][n][k]."""
    m, n = da.shape[1], db.shape[1]
    out = np.zeros((s, m, n), dtype=np.int64)
    for i in range(s):
        for j in range(s - i):
            out[i + j] += da[i] @ db[j].T
    return out


def assemble(diag: np.ndarray, s: int, bits: int = BITS):
    """Add v_t = S_t 2^(-12-bits t) for t = s-1 .. 0 into an FP64x2 sum."""
    h = np.zeros(diag.shape[1:])
    l = np.zeros(diag.shape[1:])
    for t in range(s - 1, -1, -1):
        v = np.ldexp(diag[t].astype(np.float64), -12 - bits * t)
        h, l = _fp64.dd_add_d(h, l, v)
    return h, l


def round_dd(num: int, exp2: int):
    """The nearest FP64x2 to the exact x = num 2^exp2: hi = RN(x) and
    lo = RN(x - hi), round to nearest, ties to even (Python's int / int and
    Fraction -> float conversions round correctly)."""
    x = Fraction(num) * Fraction(2) ** exp2
    hi = float(x)
    lo = float(x - Fraction(hi))
    return hi, lo


def assemble_exact(diag: np.ndarray, s: int, scale: np.ndarray, bits: int = BITS):
    """The block value sum_t S_t 2^(-12-bits t) 2^scale of every entry,
    formed exactly from the integer diagonal sums and rounded once to
    FP64x2."""
    m, n = diag.shape[1:]
    h = np.zeros((m, n))
    l = np.zeros((m, n))
    for i in range(m):
        for j in range(n):
            t_sum = 0
            for t in range(s):
                t_sum += int(diag[t, i, j]) << (bits * (s - 1 - t))
            h[i, j], l[i, j] = round_dd(t_sum, int(scale[i, j]) - 12 - bits * (s - 1))
    return h, l


def cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=15, kb=None, return_parts=False,
                        assembly="fp64x2", bits=BITS):
    """C := A B through s INT8 pieces of `bits` bits per entry.  Returns
    (C_hi, C_lo).  kb: the k-block (default kblock(bits)).  assembly:
    "fp64x2" (diagonals added smallest first in FP64x2) or "exact" (the
    exact block value rounded once)."""
    if assembly not in ("fp64x2", "exact"):
        raise ValueError(assembly)
    if kb is None:
        kb = kblock(bits)
    a_hi = np.asarray(a_hi, np.float64)
    a_lo = np.asarray(a_lo, np.float64)
    bt_hi = np.ascontiguousarray(np.asarray(b_hi, np.float64).T)   # columns of B as rows
    bt_lo = np.ascontiguousarray(np.asarray(b_lo, np.float64).T)
    m, k = a_hi.shape
    n = bt_hi.shape[0]
    e_a = block_exponents(a_hi, kb)
    e_b = block_exponents(bt_hi, kb)
    c_hi = np.zeros((m, n))
    c_lo = np.zeros((m, n))
    parts = []
    for p in range((k + kb - 1) // kb):
        sl = slice(p * kb, (p + 1) * kb)
        da = digit_planes(a_hi[:, sl], a_lo[:, sl], e_a[:, p:p + 1], s, kb=k + 1, bits=bits)
        db = digit_planes(bt_hi[:, sl], bt_lo[:, sl], e_b[:, p:p + 1], s, kb=k + 1, bits=bits)
        diag = diagonal_sums(da, db, s)
        sc = e_a[:, p][:, None] + e_b[:, p][None, :]
        if assembly == "exact":
            h, l = assemble_exact(diag, s, sc, bits)
        else:
            h, l = assemble(diag, s, bits)
            h, l = np.ldexp(h, sc), np.ldexp(l, sc)
        c_hi, c_lo = _fp64.dd_add(c_hi, c_lo, h, l)
        if return_parts:
            parts.append((da, db, diag))
    if return_parts:
        return c_hi, c_lo, parts, (e_a, e_b)
    return c_hi, c_lo


def cascade_int8_tc_ddgemm(a_hi, a_lo, b_hi, b_lo, s=16):
    """The tcgen05 form's product: seven-bit pieces (k-blocks of 16384) and
    the exact assembly."""
    return cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=s, assembly="exact", bits=BITS_TC)


def cascade_int8_tc8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=15):
    """The tcgen05 form with the mma.sync form's eight-bit pieces (k-blocks
    of 8192) and the exact assembly."""
    return cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=s, assembly="exact", bits=BITS)
