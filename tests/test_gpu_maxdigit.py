"""The CUDA path at the bounds its exactness rests on (inputs from
workloads/maxdigit.py, whose pieces sit next to their largest magnitude, all
products of a bin or diagonal of one sign; the CPU pins of the same inputs
are in test_oracle_maxdigit.py).

* FP64 form, one full k-block: bins 0-2 reach 97 % of 2^50, 2^50 and
  2.5 2^49 units (Sec. "Cascading vectors and dot products") and must equal
  the exact integer dot products of the composed pieces bit for bit; C over
  two k-blocks is within the contract of the double-double oracle.
* mma.sync INT8 form: int32 diagonal sums at 70 % of 2^31 over a full
  k-block of 8192 entries, one and two k-blocks: C bit for bit equal to the
  restatement's assembly of the composed digits' diagonal sums.
* tcgen05 forms: FP32 partial sums at 85 % (seven-bit, chunks of 256) and
  75 % (eight-bit, chunks of 64) of 2^24, over several chunks and ragged
  tiles: C bit for bit equal to the exact assembly of the same sums.
A chunk, k-block, diagonal placement or group fold that went wrong only
near these bounds would change bits here."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cascade as cs  # noqa: E402
from oracle import cascade_int8 as c8  # noqa: E402
from oracle import dd  # noqa: E402
from workloads.maxdigit import fp64_max_pieces, int8_max_digits  # noqa: E402

pytestmark = pytest.mark.gpu

CONTRACT = 1e-28


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04353_gb300 import ops as _ops
    return _ops


def dev(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def host(*tensors):
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in tensors]


def same(x, y):
    return x.shape == y.shape and np.array_equal(x.view(np.int64), y.view(np.int64))


@pytest.mark.parametrize("m,n", [(70, 40), (130, 65)])
def test_fp64_bins_exact_at_their_bound(ops, m, n):
    a_hi, a_lo, b_hi, b_lo, pa, pb, _, _ = fp64_max_pieces(m, n, 256, seed=m + n)
    (got,) = host(ops.bins(*dev(a_hi, a_lo, b_hi, b_lo)))
    x0a, x1a, x2a = pa
    x0b, x1b, x2b = pb
    w0 = x0a @ x0b
    w1 = x0a @ x1b + x1a @ x0b
    w2 = x0a @ x2b + x1a @ x1b + x2a @ x0b
    assert np.all(w0 >= 0.97 * 2 ** 50) and np.all(-w1 >= 0.97 * 2 ** 50)
    assert same(got[0], np.ldexp(w0.astype(float), -42))
    assert same(got[1], np.ldexp(w1.astype(float), -63))
    assert same(got[2], np.ldexp(w2.astype(float), -84))


def test_fp64_product_at_the_bound_within_contract(ops):
    m, n, k = 70, 40, 512
    a_hi, a_lo, b_hi, b_lo, _, _, ra, rb = fp64_max_pieces(m, n, k, seed=3)
    a = (a_hi, a_lo, b_hi, b_lo)
    c_hi, c_lo = host(*ops.ddgemm(*dev(*a), split_k=1))
    oh, ol = dd.ddgemm(*a)
    absab = np.abs(a_hi) @ np.abs(b_hi)
    assert np.max(np.abs((c_hi - oh) + (c_lo - ol)) / absab) <= CONTRACT
    # and the cascade restatement up to bin 3-6's summation order (at most
    # 2^-92 sigma tau per k-block) and the FP64x2 roundings after it
    rh, rl = cs.cascade_ddgemm(*a)
    tol = 2 * np.ldexp(2.0 ** -92, ra[:, None] + rb[None, :]) + 16 * 2.0 ** -106 * np.abs(rh)
    assert np.all(np.abs((c_hi - rh) + (c_lo - rl)) <= tol)


def expected_int8(da, db, ra, rb, k, s, bits, exact):
    """C from the composed digits by the restatement's own steps
    (oracle/cascade_int8.py: diagonal sums per k-block, their assembly, the
    scale 2^(e_a + e_b) and the FP64x2 add into C).  The digits are the ones
    the restatement's split gives for these inputs (test_oracle_maxdigit.py)."""
    kb = c8.kblock(bits)
    m, n = da.shape[1], db.shape[1]
    c_hi, c_lo = np.zeros((m, n)), np.zeros((m, n))
    sc = ra[:, None] + rb[None, :]
    for p in range((k + kb - 1) // kb):
        sl = slice(p * kb, (p + 1) * kb)
        diag = c8.diagonal_sums(da[:, :, sl], db[:, :, sl], s)
        if exact:
            h, l = c8.assemble_exact(diag, s, sc, bits)
        else:
            h, l = c8.assemble(diag, s, bits)
            h, l = np.ldexp(h, sc), np.ldexp(l, sc)
        c_hi, c_lo = cs.dd_add(c_hi, c_lo, h, l)
    return c_hi, c_lo


@pytest.mark.parametrize("k", [8192, 16384])
def test_int8_mma_sync_at_the_int32_bound(ops, k):
    s, bits = 15, 8
    m, n = 40, 36
    a_hi, a_lo, b_hi, b_lo, da, db, ra, rb = int8_max_digits(m, n, k, bits, s, seed=k)
    want = expected_int8(da, db, ra, rb, k, s, bits, exact=False)
    got = host(*ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=1, int8_slices=s))
    assert same(got[0], want[0]) and same(got[1], want[1])


@pytest.mark.parametrize("variant,bits,s,m,n,k", [
    (4, 7, 16, 130, 20, 768),     # three chunks of 256
    (4, 7, 16, 200, 33, 300),     # a ragged chunk
    (4, 7, 12, 64, 16, 512),
    (5, 8, 15, 130, 20, 320),     # five chunks of 64
    (5, 8, 15, 70, 17, 8200),     # two k-blocks of 8192
])
def test_tcgen05_at_the_fp32_bound(ops, variant, bits, s, m, n, k):
    a_hi, a_lo, b_hi, b_lo, da, db, ra, rb = int8_max_digits(m, n, k, bits, s, seed=m + k)
    want = expected_int8(da, db, ra, rb, k, s, bits, exact=True)
    got = host(*ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=variant, int8_slices=s))
    assert same(got[0], want[0]) and same(got[1], want[1])
