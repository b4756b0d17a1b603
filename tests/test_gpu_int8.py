"""Parity of the INT8 form (C ABI, variant DDGEMM_VARIANT_INT8) with its
CPU restatement (oracle/cascade_int8.py) and with the double-double oracle.

Everything in the INT8 form up to the FP64x2 assembly is integer and exact,
and the assembly is one fixed sequence of FP64 operations, so the CUDA
result must be bit-identical to the restatement: digits, exponents and C."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cascade_int8 as c8  # noqa: E402
from oracle import dd  # noqa: E402
from tests import exact  # noqa: E402
from tests.test_oracle_int8 import int8_bound  # noqa: E402
from workloads import gemm_inputs, integer_inputs  # noqa: E402

pytestmark = pytest.mark.gpu
CONTRACT = 1e-28
INT8 = 1


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


@pytest.mark.parametrize("nvec,k", [(37, 300), (64, 64), (5, 1), (33, 130), (3, 8200)])
@pytest.mark.parametrize("kind", ["uniform", "wide"])
@pytest.mark.parametrize("as_b,trans", [(False, False), (False, True), (True, False), (True, True)])
@pytest.mark.parametrize("s", [12, 14, 15])
def test_split_int8_bitwise(ops, nvec, k, kind, as_b, trans, s):
    x_hi, x_lo, _, _ = gemm_inputs(nvec, 1, k, kind=kind, seed=nvec + k)   # vectors as rows
    e = c8.block_exponents(x_hi)
    want = c8.digit_planes(x_hi, x_lo, e, s)
    if as_b:   # B = x^T (k x nvec); stored transposed when trans
        src = (x_hi, x_lo) if trans else (x_hi.T, x_lo.T)
    else:      # A = x (nvec x k); stored transposed when trans
        src = (x_hi.T, x_lo.T) if trans else (x_hi, x_lo)
    d, ex = ops.split_int8(*dev(*src), as_b=as_b, trans=trans, slices=s)
    d, ex = host(d, ex)
    assert np.array_equal(ex, e.T)
    assert np.array_equal(d.astype(np.int64), want)


@pytest.mark.parametrize("m,n,k", [(64, 64, 256), (37, 45, 300), (1, 1, 1), (70, 33, 100)])
@pytest.mark.parametrize("kind", ["uniform", "wide"])
@pytest.mark.parametrize("s", [12, 13, 15])
def test_int8_ddgemm_bit_identical(ops, m, n, k, kind, s):
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind=kind, seed=m * 7 + n + k)
    want_hi, want_lo = c8.cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=s)
    c_hi, c_lo = host(*ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=INT8, int8_slices=s))
    assert np.array_equal(c_hi, want_hi) and np.array_equal(c_lo, want_lo)


@pytest.mark.parametrize("ta,tb", [(True, False), (False, True), (True, True)])
def test_int8_transposed(ops, ta, tb):
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(40, 50, 90, kind="wide", seed=3)
    want_hi, want_lo = c8.cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=15)
    sa = (a_hi.T, a_lo.T) if ta else (a_hi, a_lo)
    sb = (b_hi.T, b_lo.T) if tb else (b_hi, b_lo)
    c_hi, c_lo = host(*ops.ddgemm(*dev(*sa), *dev(*sb), trans_a=ta, trans_b=tb, variant=INT8))
    assert np.array_equal(c_hi, want_hi) and np.array_equal(c_lo, want_lo)


def test_int8_two_k_blocks(ops):
    """k > 16384: two INT8 k-blocks with their own scales."""
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(4, 6, 17000, kind="wide", seed=4)
    want_hi, want_lo = c8.cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=15)
    c_hi, c_lo = host(*ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=INT8))
    assert np.array_equal(c_hi, want_hi) and np.array_equal(c_lo, want_lo)


def test_int8_integers_and_worked_example(ops):
    a_hi, a_lo, b_hi, b_lo = integer_inputs(64, 48, 700, bits=10, seed=5)
    c_hi, c_lo = host(*ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=INT8))
    ref = a_hi.astype(np.int64) @ b_hi.astype(np.int64)
    assert np.array_equal(c_hi, ref.astype(np.float64)) and np.all(c_lo == 0)
    x_hi, x_lo = np.array([[1.0, 1.5 * 2.0 ** -71]]), np.array([[0.0, 2.0 ** -130]])
    c_hi, c_lo = host(*ops.ddgemm(*dev(x_hi, x_lo, np.array([[0.0], [1.0]]), np.zeros((2, 1))),
                                  variant=INT8))
    assert c_hi[0, 0] == 1.5 * 2.0 ** -71 and c_lo[0, 0] == 0.0


@pytest.mark.parametrize("m,n,k,kind", [(4096, 4096, 4096, "wide"), (8192, 8192, 8192, "wide")])
def test_int8_full_size_sampled(ops, m, n, k, kind):
    """The INT8 workloads on sampled entries: within 1e-28 (|A||B|) of the
    double-double oracle and within the INT8 bound of exact rationals."""
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind=kind, seed=0)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    c_hi, c_lo, st = host(*ops.ddgemm(*dev(a_hi, a_lo, b_hi, b_lo), variant=INT8, status=status),
                          status)
    assert st[0] == 0
    rng = np.random.default_rng(9)
    rows, cols = rng.integers(0, m, 64), rng.integers(0, n, 64)
    o_hi, o_lo = dd.ddgemm_entries(a_hi, a_lo, b_hi, b_lo, rows, cols)
    absab = np.array([np.abs(a_hi[i]) @ np.abs(b_hi[:, j]) for i, j in zip(rows, cols)])
    diff = np.abs((c_hi[rows, cols] - o_hi) + (c_lo[rows, cols] - o_lo))
    assert np.all(diff <= CONTRACT * absab)
    for t in range(4):
        i, j = rows[t], cols[t]
        ex = exact.exact_dot(a_hi[i], a_lo[i], b_hi[:, j], b_lo[:, j])
        bound = int8_bound(a_hi[i:i + 1], b_hi[:, j:j + 1], 15)[0, 0]
        assert exact.err_vs_exact(c_hi[i, j], c_lo[i, j], ex) <= bound


def test_int8_backward_matches_int8_forward_products(ops):
    """ddgemm_backward with the INT8 variant: dA = W B^T and dB = A^T W are
    the INT8 form's products of those operands, bit for bit."""
    from paper_2303_04353_gb300 import _lib
    m, n, k = 40, 30, 90
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind="wide", seed=50)
    w_hi, w_lo = gemm_inputs(m, 1, n, seed=51)[0:2]          # an m x n FP64x2 matrix
    ta = dev(a_hi, a_lo, b_hi, b_lo, w_hi, w_lo)
    opts = _lib.make_opts(variant=INT8)
    ws = torch.empty(_lib.ddgemm_backward_workspace_size(m, n, k, opts), dtype=torch.uint8,
                     device="cuda")
    da = [torch.empty((m, k), dtype=torch.float64, device="cuda") for _ in range(2)]
    db = [torch.empty((k, n), dtype=torch.float64, device="cuda") for _ in range(2)]
    _lib.ddgemm_backward(m, n, k, ta[0].data_ptr(), ta[1].data_ptr(), k, ta[2].data_ptr(),
                         ta[3].data_ptr(), n, ta[4].data_ptr(), ta[5].data_ptr(), n,
                         da[0].data_ptr(), da[1].data_ptr(), k, db[0].data_ptr(),
                         db[1].data_ptr(), n, ws.data_ptr(), ws.numel(),
                         torch.cuda.current_stream().cuda_stream, opts)
    da_hi, da_lo, db_hi, db_lo = host(*da, *db)
    want = c8.cascade_int8_ddgemm(w_hi, w_lo, b_hi.T, b_lo.T, s=15)
    assert np.array_equal(da_hi, want[0]) and np.array_equal(da_lo, want[1])
    want = c8.cascade_int8_ddgemm(a_hi.T, a_lo.T, w_hi, w_lo, s=15)
    assert np.array_equal(db_hi, want[0]) and np.array_equal(db_lo, want[1])


def test_int8_noalloc_matches_int8_ddgemm(ops):
    from paper_2303_04353_gb300 import _lib
    m, n, k = 120, 90, 300
    a = gemm_inputs(m, n, k, kind="wide", seed=52)
    t = dev(*a)
    c = [torch.empty((m, n), dtype=torch.float64, device="cuda") for _ in range(2)]
    _lib.ddgemm_noalloc(m, n, k, t[0].data_ptr(), t[1].data_ptr(), k, t[2].data_ptr(),
                        t[3].data_ptr(), n, c[0].data_ptr(), c[1].data_ptr(), n,
                        torch.cuda.current_stream().cuda_stream, _lib.make_opts(variant=INT8))
    got = host(*c)
    want = c8.cascade_int8_ddgemm(*a, s=15)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
