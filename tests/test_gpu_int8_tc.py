"""Parity of the tensor-core INT8 form (C ABI, variant DDGEMM_VARIANT_INT8_TC)
with its CPU restatement (oracle/cascade_int8.py, assembly="exact").

The digits, the exponents and the diagonal sums are the INT8 form's, exact
integers; the tcgen05 products are exact (bf16 digits, FP32 sums below
2^24 per 256-entry chunk); the assembly rounds the exact block value once
to the nearest FP64x2, and the blocks are added into C by the same FP64x2
add as the restatement.  So C must be bit-identical to the restatement.
The assembly step alone is checked bit for bit on hard cases (ties at both
roundings, cancellation, the largest sums)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cascade_int8 as c8  # noqa: E402
from oracle import dd  # noqa: E402
from tests import exact  # noqa: E402
from tests.test_oracle_int8 import hard_block_values  # noqa: E402
from workloads import gemm_inputs, integer_inputs  # noqa: E402

pytestmark = pytest.mark.gpu
CONTRACT = 1e-28
TC = 4


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


def same(a, b):
    return np.array_equal(a, b) and np.array_equal(np.signbit(a), np.signbit(b))


# ---- the assembly step ----------------------------------------------------

def diag_for(t_val, s):
    """Diagonal sums whose block value is exactly t_val 2^(-12-7(s-1)):
    balanced base-128 digits of t_val, the top one taking what is left."""
    out = [0] * s
    x = t_val
    for i in range(s - 1, 0, -1):
        d = ((x + 64) & 127) - 64
        out[i] = d
        x = (x - d) >> 7
    out[0] = x
    return out


@pytest.mark.parametrize("s", [16, 12, 13, 15])
def test_assemble_bitwise_on_hard_values(ops, s):
    cases = []
    for t_val, e in hard_block_values():
        ds = diag_for(t_val, s)
        if abs(ds[0]) < 2 ** 30:
            cases.append((ds, e))
    rng = np.random.default_rng(s)
    for _ in range(400):      # full-range sums: every diagonal up to 2^30
        cases.append((list(rng.integers(-(2 ** 31), 2 ** 31, s)), int(rng.integers(-150, 20))))
    cases.append(([2 ** 31 - 1] * s, 0))
    cases.append(([-(2 ** 31)] * s, -40))
    cases.append(([2 ** 30] * s, 3))
    cases.append(([0] * s, 0))
    diag = np.array([c[0] for c in cases], dtype=np.int64).T
    scale = np.array([c[1] for c in cases], dtype=np.int64)
    hi, lo = host(*ops.assemble_int8(torch.from_numpy(diag.astype(np.int32)).cuda(),
                                     torch.from_numpy(scale.astype(np.int32)).cuda()))
    for i in range(len(cases)):
        t_val = sum(int(diag[t, i]) << (7 * (s - 1 - t)) for t in range(s))
        want = c8.round_dd(t_val, int(scale[i]) - 12 - 7 * (s - 1))
        assert hi[i] == want[0] and lo[i] == want[1], (i, cases[i])
        assert not np.signbit(lo[i]) or lo[i] != 0.0


# ---- the whole form -----------------------------------------------------

def tc(ops, a_hi, a_lo, b_hi, b_lo, s=16, **kw):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    c_hi, c_lo = ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=TC, int8_slices=s,
                            status=status, **kw)
    c_hi, c_lo, st = host(c_hi, c_lo, status)
    assert st[0] == 0
    return c_hi, c_lo


@pytest.mark.parametrize("m,n,k", [(128, 16, 256), (1, 1, 1), (130, 20, 300), (200, 50, 1000),
                                   (129, 17, 16), (70, 100, 513)])
@pytest.mark.parametrize("kind", ["uniform", "wide"])
def test_tc_bitwise_vs_restatement(ops, m, n, k, kind):
    a = gemm_inputs(m, n, k, kind=kind, seed=m + 3 * n + k)
    c_hi, c_lo = tc(ops, *a)
    w_hi, w_lo = c8.cascade_int8_tc_ddgemm(*a, s=16)
    assert same(c_hi, w_hi) and same(c_lo, w_lo)


@pytest.mark.parametrize("s", [12, 14, 15])
def test_tc_other_piece_counts(ops, s):
    a = gemm_inputs(150, 40, 700, kind="wide", seed=s)
    c_hi, c_lo = tc(ops, *a, s=s)
    w_hi, w_lo = c8.cascade_int8_tc_ddgemm(*a, s=s)
    assert same(c_hi, w_hi) and same(c_lo, w_lo)


def test_tc_two_k_blocks(ops):
    """k > 16384: two k-blocks with their own exponents, added in FP64x2."""
    a = gemm_inputs(5, 3, 17000, kind="wide", seed=21)
    c_hi, c_lo = tc(ops, *a)
    w_hi, w_lo = c8.cascade_int8_tc_ddgemm(*a, s=16)
    assert same(c_hi, w_hi) and same(c_lo, w_lo)


@pytest.mark.parametrize("ta,tb", [(True, False), (False, True), (True, True)])
def test_tc_transposed(ops, ta, tb):
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(90, 40, 400, kind="wide", seed=7)
    sa = (a_hi.T, a_lo.T) if ta else (a_hi, a_lo)
    sb = (b_hi.T, b_lo.T) if tb else (b_hi, b_lo)
    c_hi, c_lo = tc(ops, *sa, *sb, trans_a=ta, trans_b=tb)
    w_hi, w_lo = c8.cascade_int8_tc_ddgemm(a_hi, a_lo, b_hi, b_lo, s=16)
    assert same(c_hi, w_hi) and same(c_lo, w_lo)


def test_tc_integers_exact_and_contract(ops):
    a_hi, a_lo, b_hi, b_lo = integer_inputs(160, 48, 2000, bits=10, seed=3)
    c_hi, c_lo = tc(ops, a_hi, a_lo, b_hi, b_lo)
    ref = a_hi.astype(np.int64) @ b_hi.astype(np.int64)
    assert np.array_equal(c_hi, ref.astype(np.float64)) and np.all(c_lo == 0)
    a = gemm_inputs(300, 64, 3000, kind="uniform", seed=4)
    c_hi, c_lo = tc(ops, *a)
    rng = np.random.default_rng(0)
    rows, cols = rng.integers(0, 300, 64), rng.integers(0, 64, 64)
    o_hi, o_lo = dd.ddgemm_entries(*a, rows, cols)
    absab = np.array([np.abs(a[0][i]) @ np.abs(a[2][:, j]) for i, j in zip(rows, cols)])
    err = np.abs((c_hi[rows, cols] - o_hi) + (c_lo[rows, cols] - o_lo))
    assert np.all(err <= CONTRACT * absab)
    assert exact.dd_is_normalised(c_hi, c_lo)


def test_tc_close_to_int8_form(ops):
    """The mma.sync INT8 form (15 eight-bit pieces) and this one (16
    seven-bit pieces) are two approximations of the same product: they agree
    within the sum of their two INT8 bounds."""
    from tests.test_oracle_int8 import int8_bound
    a = gemm_inputs(256, 80, 1200, kind="wide", seed=5)
    c_hi, c_lo = tc(ops, *a)
    i_hi, i_lo = host(*ops.ddgemm(*dev(*a), variant=1))
    diff = np.abs((c_hi - i_hi) + (c_lo - i_lo))
    bound = int8_bound(a[0], a[2], 16, bits=7) + int8_bound(a[0], a[2], 15, bits=8)
    assert np.all(diff <= bound)


def test_tc_nonfinite_sets_status(ops):
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(20, 20, 40, seed=3)
    a_hi[3, 5] = np.inf
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=TC, status=status)
    (st,) = host(status)
    assert st[0] & 0x1 and not st[0] & 0x2


@pytest.mark.parametrize("m", [2048, 4096, 8192])
def test_tc_full_size_sampled(ops, m):
    """The sweep's size and the benchmark workloads (4096^3, 8192^3, wide
    entries), in the bench's launch configuration: sampled entries within
    1e-28 (|A||B|) of the double-double oracle, a few within the INT8 bound
    of exact rationals."""
    from tests.test_oracle_int8 import int8_bound
    n = k = m
    a = gemm_inputs(m, n, k, kind="wide", seed=0)
    c_hi, c_lo = tc(ops, *a)
    rng = np.random.default_rng(1)
    rows, cols = rng.integers(0, m, 48), rng.integers(0, n, 48)
    o_hi, o_lo = dd.ddgemm_entries(*a, rows, cols)
    absab = np.array([np.abs(a[0][i]) @ np.abs(a[2][:, j]) for i, j in zip(rows, cols)])
    err = np.abs((c_hi[rows, cols] - o_hi) + (c_lo[rows, cols] - o_lo))
    assert np.all(err <= CONTRACT * absab)
    for t in range(3):
        i, j = rows[t], cols[t]
        ex = exact.exact_dot(a[0][i], a[1][i], a[2][:, j], a[3][:, j])
        bound = int8_bound(a[0][i:i + 1], a[2][:, j:j + 1], 16, bits=7)[0, 0]
        assert exact.err_vs_exact(c_hi[i, j], c_lo[i, j], ex) <= bound


def test_tc_k_zero_empty_and_worked_example(ops):
    a = torch.zeros((5, 0), dtype=torch.float64, device="cuda")
    b = torch.zeros((0, 7), dtype=torch.float64, device="cuda")
    out = (torch.full((5, 7), 3.0, dtype=torch.float64, device="cuda"),
           torch.full((5, 7), 3.0, dtype=torch.float64, device="cuda"))
    c_hi, c_lo = host(*ops.ddgemm(a, a, b, b, out=out, variant=TC))
    assert not c_hi.any() and not c_lo.any()
    e = torch.zeros((0, 4), dtype=torch.float64, device="cuda")
    bb = torch.ones((4, 3), dtype=torch.float64, device="cuda")
    c_hi, _ = ops.ddgemm(e, e, bb, bb * 0, variant=TC)
    assert tuple(c_hi.shape) == (0, 3)
    # Sec. "Forward Error Analysis": x = (1, eps), y = (0, 1) gives eps exactly
    eps_hi, eps_lo = 1.5 * 2.0 ** -71, 2.0 ** -130
    c_hi, c_lo = tc(ops, np.array([[1.0, eps_hi]]), np.array([[0.0, eps_lo]]),
                    np.array([[0.0], [1.0]]), np.zeros((2, 1)))
    assert c_hi[0, 0] == eps_hi and c_lo[0, 0] == 0.0


def test_tc_noalloc_matches_tc_ddgemm(ops):
    from paper_2303_04353_gb300 import _lib
    m, n, k = 120, 90, 300
    a = gemm_inputs(m, n, k, kind="wide", seed=53)
    t = dev(*a)
    c = [torch.empty((m, n), dtype=torch.float64, device="cuda") for _ in range(2)]
    _lib.ddgemm_noalloc(m, n, k, t[0].data_ptr(), t[1].data_ptr(), k, t[2].data_ptr(),
                        t[3].data_ptr(), n, c[0].data_ptr(), c[1].data_ptr(), n,
                        torch.cuda.current_stream().cuda_stream, _lib.make_opts(variant=TC))
    got = host(*c)
    want = c8.cascade_int8_tc_ddgemm(*a, s=16)
    assert same(got[0], want[0]) and same(got[1], want[1])


# ---- the eight-bit tcgen05 form (DDGEMM_VARIANT_INT8_TC8) -----------------

TC8 = 5


def tc8(ops, a_hi, a_lo, b_hi, b_lo, s=15, **kw):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    c_hi, c_lo = ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=TC8, int8_slices=s,
                            status=status, **kw)
    c_hi, c_lo, st = host(c_hi, c_lo, status)
    assert st[0] == 0
    return c_hi, c_lo


@pytest.mark.parametrize("m,n,k", [(128, 16, 256), (1, 1, 1), (130, 20, 300), (200, 50, 1000),
                                   (129, 17, 16), (70, 100, 65)])
@pytest.mark.parametrize("kind", ["uniform", "wide"])
def test_tc8_bitwise_vs_restatement(ops, m, n, k, kind):
    """Eight-bit pieces on tcgen05, read out every 64 entries (k = 65: a
    chunk and one entry): bit-identical to the restatement with the
    mma.sync form's pieces and the exact assembly."""
    a = gemm_inputs(m, n, k, kind=kind, seed=m + 5 * n + k)
    c_hi, c_lo = tc8(ops, *a)
    w_hi, w_lo = c8.cascade_int8_tc8_ddgemm(*a, s=15)
    assert same(c_hi, w_hi) and same(c_lo, w_lo)


@pytest.mark.parametrize("s", [12, 13, 14])
def test_tc8_other_piece_counts(ops, s):
    a = gemm_inputs(150, 40, 700, kind="wide", seed=s + 40)
    c_hi, c_lo = tc8(ops, *a, s=s)
    w_hi, w_lo = c8.cascade_int8_tc8_ddgemm(*a, s=s)
    assert same(c_hi, w_hi) and same(c_lo, w_lo)


def test_tc8_two_k_blocks_and_transposes(ops):
    """k > 8192: two k-blocks with their own exponents; transposed storage."""
    a = gemm_inputs(5, 3, 8300, kind="wide", seed=22)
    c_hi, c_lo = tc8(ops, *a)
    w_hi, w_lo = c8.cascade_int8_tc8_ddgemm(*a, s=15)
    assert same(c_hi, w_hi) and same(c_lo, w_lo)
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(90, 40, 400, kind="wide", seed=8)
    c_hi, c_lo = tc8(ops, a_hi.T, a_lo.T, b_hi.T, b_lo.T, trans_a=True, trans_b=True)
    w_hi, w_lo = c8.cascade_int8_tc8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=15)
    assert same(c_hi, w_hi) and same(c_lo, w_lo)


def test_tc8_matches_int8_form_assembly_bound(ops):
    """Same pieces and products as the mma.sync form, only the assembly
    differs (one rounding against s): within 4 s 2^-106 |A||B| of it."""
    a = gemm_inputs(256, 80, 1200, kind="wide", seed=6)
    c_hi, c_lo = tc8(ops, *a)
    i_hi, i_lo = host(*ops.ddgemm(*dev(*a), variant=1))
    absab = np.abs(a[0]) @ np.abs(a[2])
    diff = np.abs((c_hi - i_hi) + (c_lo - i_lo))
    assert np.all(diff <= 4 * 15 * 2.0 ** -106 * absab)


def test_tc8_full_size_sampled(ops):
    """4096^3, wide entries: sampled entries within 1e-28 (|A||B|) of the
    double-double oracle."""
    m = n = k = 4096
    a = gemm_inputs(m, n, k, kind="wide", seed=0)
    c_hi, c_lo = tc8(ops, *a)
    rng = np.random.default_rng(1)
    rows, cols = rng.integers(0, m, 48), rng.integers(0, n, 48)
    o_hi, o_lo = dd.ddgemm_entries(*a, rows, cols)
    absab = np.array([np.abs(a[0][i]) @ np.abs(a[2][:, j]) for i, j in zip(rows, cols)])
    err = np.abs((c_hi[rows, cols] - o_hi) + (c_lo[rows, cols] - o_lo))
    assert np.all(err <= CONTRACT * absab)


def test_tc8_illconditioned_beats_fp64x2_loop(ops):
    """On the ill-conditioned products of the accuracy study the eight-bit
    pieces (118 fraction bits) beat the FP64x2 triple loop, as the mma.sync
    form does; bit-identical to the restatement."""
    from workloads.illcond import illcond_inputs
    from tests.test_illcond import rel_errors
    n = 128
    a = illcond_inputs(n, 1e-19, seed=n)[:4]
    c_hi, c_lo = tc8(ops, *a)
    w_hi, w_lo = c8.cascade_int8_tc8_ddgemm(*a, s=15)
    assert same(c_hi, w_hi) and same(c_lo, w_lo)
    rng = np.random.default_rng(2)
    rows, cols = rng.integers(0, n, 40), rng.integers(0, n, 40)
    o_hi, o_lo = dd.ddgemm(*a)
    assert rel_errors(c_hi, c_lo, a, rows, cols).max() * 3 < rel_errors(o_hi, o_lo, a, rows, cols).max()


def test_tc_block_rounding_ties_and_carries(ops):
    """The epilogue's exact rounding of a block value to FP64x2 (hi = RN(x),
    lo = RN(x - hi)) on values that land on ties, on the next power of two
    and on wide remainders: C = A B with k = 1, A's column the chosen
    integers (exact FP64x2 pairs) and B's row signed powers of two, so every
    C entry is a known integer; C must be its correctly rounded pair, both
    forms (seven- and eight-bit pieces)."""
    import random
    rng = random.Random(5)
    vals = []
    for _ in range(48):                          # ties at hi's rounding
        sh = rng.randrange(1, 50)
        m = rng.getrandbits(53) | (1 << 52)
        vals.append((m << sh) + (1 << (sh - 1)))
    for _ in range(40):                          # just below a power of two
        vals.append((1 << rng.randrange(54, 100)) - rng.randrange(1, 1 << 12))
    for _ in range(40):                          # wide values (lo carries many bits)
        vals.append(rng.getrandbits(rng.randrange(54, 100)) | 1)
    vals = [v if rng.random() < 0.5 else -v for v in vals]
    m, n = len(vals), 16
    a_hi = np.array([float(v) for v in vals])[:, None]
    a_lo = np.array([float(v - int(float(v))) for v in vals])[:, None]
    pw = [rng.randrange(0, 30) for _ in range(n)]
    sg = [rng.choice((-1, 1)) for _ in range(n)]
    b_hi = np.array([[s * 2.0 ** p for s, p in zip(sg, pw)]])
    b_lo = np.zeros_like(b_hi)
    want_hi = np.array([[float(v * s << p) for s, p in zip(sg, pw)] for v in vals])
    want_lo = np.array([[float((v * s << p) - int(float(v * s << p))) for s, p in zip(sg, pw)]
                        for v in vals])
    for variant in (TC, 5):
        c = ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=variant)
        c_hi, c_lo = host(*c)
        assert same(c_hi, want_hi) and same(c_lo, want_lo), variant
