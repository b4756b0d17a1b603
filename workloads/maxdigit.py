"""Seeded inputs whose cascade pieces sit next to their largest magnitude
(test data only).

The exactness of the method rests on bounds: the FP64 form's bins 0-2 stay
below 2^53 units of their grid, the INT8 form's int32 diagonal sums below
2^31, and the tcgen05 form's FP32 partial sums below 2^24 per chunk.  Random
entries pass far from those bounds.  These generators compose every entry
from chosen pieces of (nearly) the largest magnitude and one sign, so that
every product of a bin or a diagonal has the same sign and the sums come
within a few per cent of the bound.  Each piece is drawn next to its
extreme (not at it) so that the products carry odd low-order bits: a sum
that went past its bound would then lose them.

The values are put together in exact integer arithmetic; nothing here
computes any step of the method.  Every generator also returns the pieces
it composed, so that a test can compare a split against them.  Row r of A
is scaled by 2^ra[r] and column c of B by 2^rb[c] (exact), with the scale
exponents returned too.
"""
from __future__ import annotations

import numpy as np


def _scales(rng, count, spread):
    return rng.integers(-spread, spread + 1, size=count) if spread else np.zeros(count, np.int64)


def fp64_max_pieces(m, n, k, seed=0, spread=20):
    """A (m x k) and B (k x n) for the FP64 form with full 256-entry
    k-blocks (22, 21, 21 digits).  Every entry is one double,
        x = 2^r (x0 + 2^-22 x1 + 2^-43 x2),  lo = 0, with
        x0 = X0 2^-21, X0 = 2^21 - u0,                 u0 in [0, 2^10)
        x1 = X1 2^-20, X1 = -(2^20 - u1),              u1 in [0, 2^9)
        x2 = X2 2^-20, X2 = 2^20 - (1 + u2) 2^10,      u2 in [0, 2^6)
    so x0 is next to 1, x1 next to -1 and x2 next to 1 (53 significant bits
    from 2^-1 to 2^-53), and 1 - 2^-22 < x / 2^r < 1.  Returns
    (a_hi, a_lo, b_hi, b_lo, pa, pb, ra, rb) with pa[i] (i = 0, 1, 2) the
    integers X_i of A (m x k), pb[i] those of B (k x n), ra the row scale
    exponents of A and rb the column ones of B."""
    if k % 256:
        raise ValueError("k must be a multiple of 256 (full k-blocks)")
    rng = np.random.default_rng(seed)

    def pieces(shape):
        x0 = (1 << 21) - rng.integers(0, 1 << 10, size=shape)
        x1 = -((1 << 20) - rng.integers(0, 1 << 9, size=shape))
        x2 = (1 << 20) - (1 + rng.integers(0, 1 << 6, size=shape)) * (1 << 10)
        return np.stack([x0, x1, x2]).astype(np.int64)

    def compose(p):
        # x in units of 2^-63: X0 2^42 + X1 2^21 + X2, 53 bits from 2^62 to 2^10
        n_int = (p[0].astype(object) << 42) + (p[1].astype(object) << 21) + p[2].astype(object)
        return np.vectorize(lambda v: float(v) * 2.0 ** -63, otypes=[np.float64])(n_int)

    pa, pb = pieces((m, k)), pieces((k, n))
    ra, rb = _scales(rng, m, spread), _scales(rng, n, spread)
    a_hi = np.ldexp(compose(pa), ra[:, None])
    b_hi = np.ldexp(compose(pb), rb[None, :])
    return a_hi, np.zeros_like(a_hi), b_hi, np.zeros_like(b_hi), pa, pb, ra, rb


def int8_max_digits(m, n, k, bits, slices, seed=0, spread=20):
    """A (m x k) and B (k x n) for the INT8 forms with `slices` pieces of
    `bits` bits (8: balanced base 256; 7: base 128).  Every entry is
        x = 2^r X 2^-F,  F = 6 + bits (slices - 1),
        X = sum_i d_i 2^(bits (slices - 1 - i)),
    with d_0 in [-60, -56] and every lower digit in [-2^(bits-1),
    -2^(bits-1) + 4], except that X must fit the 106 bits of an FP64x2 pair
    (its lowest set bit at 2^max(0, F - 105)): digits below that are 0, and
    the digit across it takes the most negative value that keeps only the
    bits above it.  So -1 < x / 2^r < -1/2, and the normalised pair (hi, lo)
    holds X exactly: hi 2^F and lo 2^F are integers that add up to X.
    Returns (a_hi, a_lo, b_hi, b_lo, da, db, ra, rb): da [s][m][k] and
    db [s][n][k] the digits of A's rows and B's columns, ra and rb the scale
    exponents."""
    rng = np.random.default_rng(seed)
    s = slices
    f = 6 + bits * (s - 1)
    w = max(0, f - 105)                      # lowest bit the pair can hold
    half = 1 << (bits - 1)

    def digits(shape):
        d = np.empty((s,) + shape, dtype=np.int64)
        d[0] = rng.integers(-60, -55, size=shape)
        for i in range(1, s):
            weight = bits * (s - 1 - i)
            if weight >= w:
                d[i] = -half + rng.integers(0, 5, size=shape)
            elif weight + bits > w:
                # a multiple of 2^(w - weight), which -half is: -half or the next one up
                d[i] = -half + (1 << (w - weight)) * rng.integers(0, 2, size=shape)
            else:
                d[i] = 0
        return d

    def compose(d):
        x = np.zeros(d.shape[1:], dtype=object)
        for i in range(s):
            x = x + (d[i].astype(object) << (bits * (s - 1 - i)))
        # hi = X rounded to 53 bits (Python's int -> float rounds correctly),
        # lo = the rest, exact: X spans at most 106 bits
        hi = np.vectorize(lambda v: float(v) * 2.0 ** -f, otypes=[np.float64])(x)
        lo = np.vectorize(lambda v: float(v - int(float(v))) * 2.0 ** -f, otypes=[np.float64])(x)
        return hi, lo

    da, db = digits((m, k)), digits((n, k))
    ra, rb = _scales(rng, m, spread), _scales(rng, n, spread)
    a_hi, a_lo = compose(da)
    bt_hi, bt_lo = compose(db)
    a_hi, a_lo = np.ldexp(a_hi, ra[:, None]), np.ldexp(a_lo, ra[:, None])
    b_hi = np.ldexp(np.ascontiguousarray(bt_hi.T), rb[None, :])
    b_lo = np.ldexp(np.ascontiguousarray(bt_lo.T), rb[None, :])
    return a_hi, a_lo, b_hi, b_lo, da, db, ra, rb
