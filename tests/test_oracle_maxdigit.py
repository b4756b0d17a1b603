"""Pins of the CPU restatements on inputs whose pieces sit next to their
largest magnitude (workloads/maxdigit.py), where the exactness arguments of
the method are tight.

* FP64 form (Sec. "Cascading vectors and dot products": a bin of products
  of fixed-point pieces over one k-block of K_C = 256 is exact while it
  stays below 2^53 units of its grid): the split recovers the composed
  pieces exactly, bins 0-2 equal the exact integer dot products of the
  pieces and reach 97 % of their largest possible magnitude (2^50, 2^50
  and 2.5 2^49 units for (22, 21, 21) digits).
* INT8 form (Sec. "FP64x2 in terms of INT8": int32 accumulation of
  products of eight-bit pieces): the digits are the composed ones, the
  diagonal sums equal brute-force integer sums, and over a full k-block of
  8192 entries the largest one reaches 70 % of 2^31 while staying below it.
* The tcgen05 form's FP32 accumulation (exact for integers up to 2^24):
  within a chunk of 256 entries (seven-bit pieces) or 64 (eight-bit) every
  partial sum of a diagonal stays at or below 2^24 and the largest reaches
  85 % (seven-bit) or 75 % (eight-bit) of it; summed in FP32 the chunk is
  exact.  A chunk twice as long (a planted mistake) passes 2^24 and FP32
  then loses bits, so these inputs tell the right chunk from a wrong one."""
import numpy as np
import pytest

from oracle import cascade as cs
from oracle import cascade_int8 as c8
from workloads.maxdigit import fp64_max_pieces, int8_max_digits


def test_fp64_split_recovers_the_composed_pieces():
    a_hi, a_lo, b_hi, b_lo, pa, pb, ra, rb = fp64_max_pieces(9, 7, 512, seed=1)
    e_a = cs.block_exponents_rows(a_hi)
    e_b = cs.block_exponents_cols(b_hi)
    assert np.array_equal(e_a, np.repeat(ra[:, None], 2, axis=1))
    assert np.array_equal(e_b, np.repeat(rb[None, :], 2, axis=0))
    for p in range(2):
        sl = slice(256 * p, 256 * (p + 1))
        a = cs.cascade_a(a_hi, a_lo, e_a, p)
        b = cs.cascade_b(b_hi, b_lo, e_b, p)
        assert np.array_equal(a[0], np.ldexp(pa[0][:, sl].astype(float), -21))
        assert np.array_equal(a[1], np.ldexp(pa[1][:, sl].astype(float), -42))
        assert np.array_equal(a[2], np.ldexp(pa[2][:, sl].astype(float), -63))
        assert not a[3].any()
        assert np.array_equal(b[0], np.ldexp(pb[0][sl].astype(float), -21))
        assert np.array_equal(b[1], np.ldexp(pb[1][sl].astype(float), -42))
        assert np.array_equal(b[2], np.ldexp(pb[2][sl].astype(float), -63))


def exact_bins(pa, pb):
    """Bins 0-2 of one block as exact integers in their units 2^-42, 2^-63,
    2^-84: the integer dot products of the pieces."""
    x0a, x1a, x2a = pa
    x0b, x1b, x2b = pb
    return (x0a @ x0b, x0a @ x1b + x1a @ x0b, x0a @ x2b + x1a @ x1b + x2a @ x0b)


def test_fp64_bins_are_exact_at_their_bound():
    a_hi, a_lo, b_hi, b_lo, pa, pb, _, _ = fp64_max_pieces(6, 5, 256, seed=2)
    _, _, bins, _ = cs.cascade_ddgemm(a_hi, a_lo, b_hi, b_lo, return_bins=True)
    b0, b1, b2, _ = bins[0]
    w0, w1, w2 = exact_bins(pa, pb)
    assert np.array_equal(b0, np.ldexp(w0.astype(float), -42))
    assert np.array_equal(b1, np.ldexp(w1.astype(float), -63))
    assert np.array_equal(b2, np.ldexp(w2.astype(float), -84))
    # the largest magnitudes the digits allow (|piece| <= 1 on its grid)
    assert np.all(w0 >= 0.97 * 2 ** 50) and np.all(w0 <= 2 ** 50)
    assert np.all(-w1 >= 0.97 * 2 ** 50) and np.all(-w1 <= 2 ** 50)
    assert np.all(w2 >= 0.97 * 2.5 * 2 ** 49) and np.all(w2 <= 2.5 * 2 ** 49)


@pytest.mark.parametrize("bits,s", [(8, 15), (7, 16), (8, 12), (7, 13)])
def test_int8_digits_are_the_composed_ones(bits, s):
    a_hi, a_lo, b_hi, b_lo, da, db, ra, rb = int8_max_digits(4, 3, 300, bits, s, seed=bits + s)
    kb = c8.kblock(bits)
    e_a = c8.block_exponents(a_hi, kb)
    bt_hi, bt_lo = np.ascontiguousarray(b_hi.T), np.ascontiguousarray(b_lo.T)
    e_b = c8.block_exponents(bt_hi, kb)
    assert np.array_equal(e_a[:, 0], ra) and np.array_equal(e_b[:, 0], rb)
    assert np.array_equal(c8.digit_planes(a_hi, a_lo, e_a, s, kb=kb, bits=bits), da)
    assert np.array_equal(c8.digit_planes(bt_hi, bt_lo, e_b, s, kb=kb, bits=bits), db)
    assert np.all(a_hi + a_lo == a_hi)          # normalised pairs


def brute_diagonals(da, db, s):
    """S_t[i][j] = sum over i' + j' = t and l of da[i'][i][l] db[j'][j][l],
    in Python integers."""
    m, n = da.shape[1], db.shape[1]
    out = np.zeros((s, m, n), dtype=object)
    for t in range(s):
        for i in range(m):
            for j in range(n):
                out[t, i, j] = sum(int(x) * int(y) for p in range(t + 1)
                                   for x, y in zip(da[p, i], db[t - p, j]))
    return out


def test_int8_diagonal_sums_at_the_int32_bound():
    """Eight-bit pieces over one full k-block of 8192 entries: the
    restatement's diagonal sums are the brute-force integers, the largest
    within 70 % of 2^31 and below it."""
    s, bits = 15, 8
    _, _, _, _, da, db, _, _ = int8_max_digits(2, 2, 8192, bits, s, seed=4, spread=0)
    diag = c8.diagonal_sums(da, db, s)
    assert np.abs(diag).max() < 2 ** 31
    assert np.abs(diag).max() >= 0.7 * 2 ** 31
    small = (da[:, :, :40], db[:, :, :40])
    assert np.array_equal(c8.diagonal_sums(*small, s), brute_diagonals(*small, s).astype(np.int64))


@pytest.mark.parametrize("bits,s,chunk,reach", [(7, 16, 256, 0.85), (8, 15, 64, 0.75)])
def test_fp32_chunk_sums_at_the_2_24_bound(bits, s, chunk, reach):
    """The tcgen05 form's FP32 accumulators: per entry a diagonal t adds
    t + 1 digit products; over a chunk every partial sum stays <= 2^24 (the
    largest within `reach` of it: the first digit and the lowest ones an
    FP64x2 pair can hold are smaller) and FP32 adds the chunk exactly, while
    a chunk of twice the length goes past 2^24 and FP32 rounds."""
    _, _, _, _, da, db, _, _ = int8_max_digits(1, 1, 2 * chunk, bits, s, seed=7, spread=0)
    sums = [sum(da[p, 0] * db[t - p, 0] for p in range(t + 1)) for t in range(s)]  # int64
    t = int(np.argmax([x[:chunk].sum() for x in sums]))
    per_entry = sums[t]
    prefix = np.cumsum(per_entry)
    assert np.all(per_entry > 0)
    assert prefix[chunk - 1] <= 2 ** 24 and prefix[chunk - 1] >= reach * 2 ** 24

    def fp32_sum(vals):
        acc = np.float32(0)
        for v in vals:
            acc = np.float32(acc + np.float32(v))
        return int(acc)
    assert fp32_sum(per_entry[:chunk]) == int(prefix[chunk - 1])
    # planted mistake: one chunk of twice the length
    assert prefix[-1] > 2 ** 24
    assert fp32_sum(per_entry) != int(prefix[-1])
