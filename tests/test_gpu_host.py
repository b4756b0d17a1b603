"""ddgemm_host: the cascade on host operands, with the copies in and out run
by the library's own streams so that they overlap the kernels (row chunks of
op(A); include/ddgemm.h).

* Multi-chunk shapes: C is bit-identical to ddgemm() on device copies of the
  operands (split_k = 1 for the FP64 form), agrees element by element with
  the cascade restatement of the oracle within the FP64 summation-order
  tolerance, and on sampled entries with the double-double oracle within
  the 1e-28 |A||B| contract.
* Both INT8 forms on multi-chunk shapes: bit-identical to ddgemm() of the
  same form, and to the form's restatement on the rows at every chunk
  boundary.
* Transposed storage, leading dimensions above the width, pageable host
  memory, k = 0, empty m, buffer reuse by back-to-back calls on one stream,
  non-finite input.

The chunk counts of these shapes are pinned on the CPU
(tests/test_abi.py::test_host_buffer_size)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cascade as cs  # noqa: E402
from oracle import cascade_int8 as c8  # noqa: E402
from oracle import dd  # noqa: E402
from tests import exact  # noqa: E402
from workloads import gemm_inputs  # noqa: E402

pytestmark = pytest.mark.gpu

CONTRACT = 1e-28
FP64, INT8, INT8_TC, INT8_TC8 = 0, 1, 4, 5


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04353_gb300 import ops as _ops
    return _ops


def pinned(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrays]


def dev(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def np_of(*tensors):
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in tensors]


def run_host(ops, a, b, trans_a=False, trans_b=False, **kw):
    """ddgemm_host on pinned copies of (a_hi, a_lo) and (b_hi, b_lo), given in
    their mathematical shapes and stored transposed when asked."""
    sa = (a[0].T, a[1].T) if trans_a else a
    sb = (b[0].T, b[1].T) if trans_b else b
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # the host operands stay referenced until the copies are done
    ins = pinned(*sa) + pinned(*sb)
    c = ops.ddgemm_host(*ins, trans_a=trans_a, trans_b=trans_b, status=status, **kw)
    torch.cuda.synchronize()
    del ins
    assert int(status.item()) == 0
    return c[0].numpy().copy(), c[1].numpy().copy()


def run_device(ops, a, b, trans_a=False, trans_b=False, **kw):
    sa = (a[0].T, a[1].T) if trans_a else a
    sb = (b[0].T, b[1].T) if trans_b else b
    return np_of(*ops.ddgemm(*dev(*sa), *dev(*sb), trans_a=trans_a, trans_b=trans_b, **kw))


def cascade_tolerance(a_hi, b_hi, c_ref):
    """|C_gpu - C_cascade_oracle| for the FP64 form: bin 3-6's FP64
    summation order (<= 2^-92 sigma tau per k-block) and the FP64x2
    roundings that follow (a few 2^-106 |C| per block)."""
    e_a = cs.block_exponents_rows(a_hi)
    e_b = cs.block_exponents_cols(b_hi)
    tol = np.zeros((a_hi.shape[0], b_hi.shape[1]))
    for p in range(e_a.shape[1]):
        tol += np.ldexp(2.0 ** -92, e_a[:, p][:, None] + e_b[p, :][None, :])
    return tol + 8 * e_a.shape[1] * 2.0 ** -106 * np.abs(c_ref)


def check_sampled_contract(a_hi, a_lo, b_hi, b_lo, c_hi, c_lo, seed=0, count=64):
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, a_hi.shape[0], count)
    cols = rng.integers(0, b_hi.shape[1], count)
    o_hi, o_lo = dd.ddgemm_entries(a_hi, a_lo, b_hi, b_lo, rows, cols)
    absab = np.array([np.abs(a_hi[i]) @ np.abs(b_hi[:, j]) for i, j in zip(rows, cols)])
    err = np.abs((c_hi[rows, cols] - o_hi) + (c_lo[rows, cols] - o_lo))
    assert np.all(err <= CONTRACT * absab), float(np.max(err / absab))


@pytest.mark.parametrize("ta,tb", [(False, False), (True, True), (True, False)])
def test_host_fp64_four_chunks(ops, ta, tb):
    """2100 x 8192 x 300: chunks of 640, 640, 640 and 180 rows of op(A)."""
    m, n, k = 2100, 8192, 300
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind="uniform", seed=11)
    c_hi, c_lo = run_host(ops, (a_hi, a_lo), (b_hi, b_lo), ta, tb, split_k=1)
    d_hi, d_lo = run_device(ops, (a_hi, a_lo), (b_hi, b_lo), ta, tb, split_k=1)
    assert np.array_equal(c_hi, d_hi) and np.array_equal(c_lo, d_lo)
    assert exact.dd_is_normalised(c_hi, c_lo)
    s_hi, s_lo = cs.cascade_ddgemm(a_hi, a_lo, b_hi, b_lo)
    assert np.all(np.abs((c_hi - s_hi) + (c_lo - s_lo)) <= cascade_tolerance(a_hi, b_hi, s_hi))
    check_sampled_contract(a_hi, a_lo, b_hi, b_lo, c_hi, c_lo)


@pytest.mark.parametrize("ta,tb", [(False, False), (True, True), (False, True)])
def test_host_fp64_first_chunk_by_parts_of_b(ops, ta, tb):
    """2100 x 2048 x 1100: two chunks of op(A)'s rows (2048 and 52); B comes
    in parts of 512, 512 and 76 entries of k, and the first chunk is
    multiplied part by part, each part added into C.  With split_k = 1 the
    k-blocks reach C in the same order as one launch: C is bit-identical to
    ddgemm(), and the second chunk (B split whole) too."""
    m, n, k = 2100, 2048, 1100
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind="wide", seed=13)
    c_hi, c_lo = run_host(ops, (a_hi, a_lo), (b_hi, b_lo), ta, tb, split_k=1)
    d_hi, d_lo = run_device(ops, (a_hi, a_lo), (b_hi, b_lo), ta, tb, split_k=1)
    assert np.array_equal(c_hi, d_hi) and np.array_equal(c_lo, d_lo)
    check_sampled_contract(a_hi, a_lo, b_hi, b_lo, c_hi, c_lo, seed=3)


def test_host_fp64_split_k_chunks(ops):
    """The default split-k choice per chunk: within the reordering the FP64x2
    sum of k-block groups allows (8 (K_B + g) 2^-106 |A||B|, g <= 16)."""
    m, n, k = 2100, 8192, 1100
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind="wide", seed=12)
    c_hi, c_lo = run_host(ops, (a_hi, a_lo), (b_hi, b_lo))
    d_hi, d_lo = run_device(ops, (a_hi, a_lo), (b_hi, b_lo), split_k=1)
    absab = np.abs(a_hi) @ np.abs(b_hi)
    kb = -(-k // 256)
    assert np.all(np.abs((c_hi - d_hi) + (c_lo - d_lo)) <= 8 * (kb + 16) * 2.0 ** -106 * absab)
    check_sampled_contract(a_hi, a_lo, b_hi, b_lo, c_hi, c_lo, seed=1)


def sample_rows_cols(m, n, mc, seed):
    """Rows on both sides of every chunk boundary (chunks of mc rows) and
    random ones; random columns and both edges."""
    rng = np.random.default_rng(seed)
    edges = {0, m - 1}
    for r0 in range(mc, m, mc):
        edges |= {r0 - 1, r0}
    rows = np.array(sorted(edges | set(rng.integers(0, m, 10).tolist())))
    cols = np.array(sorted({0, n - 1} | set(rng.integers(0, n, 40).tolist())))
    return rows, cols


@pytest.mark.parametrize("variant,m,n,mc,s,ta", [(INT8, 2500, 2048, 640, 15, False),
                                                (INT8, 2500, 2048, 640, 13, True),
                                                (INT8_TC, 4200, 2048, 1152, 16, False),
                                                (INT8_TC, 4200, 2048, 1152, 14, True),
                                                (INT8_TC8, 4200, 2048, 1152, 15, False)])
def test_host_int8_forms(ops, variant, m, n, mc, s, ta):
    """Four chunks of op(A)'s rows (640/640/640/580 for mma.sync,
    1152/1152/1152/744 for tcgen05): C is bit-identical to ddgemm() of the same
    form, and on the rows at every chunk boundary (and random ones) by 42
    columns bit-identical to the form's restatement.  Rows and columns of C
    are independent in the method (per-row and per-column scales), so the
    restatement of the sampled rows of A against the sampled columns of B
    gives exactly those entries."""
    k = 300
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind="wide", seed=21 + s)
    c_hi, c_lo = run_host(ops, (a_hi, a_lo), (b_hi, b_lo), ta, False, variant=variant,
                          int8_slices=s)
    d_hi, d_lo = run_device(ops, (a_hi, a_lo), (b_hi, b_lo), ta, False, variant=variant,
                            int8_slices=s)
    assert np.array_equal(c_hi, d_hi) and np.array_equal(c_lo, d_lo)
    rows, cols = sample_rows_cols(m, n, mc, seed=s)
    sub = (a_hi[rows], a_lo[rows], b_hi[:, cols], b_lo[:, cols])
    if variant == INT8:
        w_hi, w_lo = c8.cascade_int8_ddgemm(*sub, s=s)
    elif variant == INT8_TC8:
        w_hi, w_lo = c8.cascade_int8_tc8_ddgemm(*sub, s=s)
    else:
        w_hi, w_lo = c8.cascade_int8_tc_ddgemm(*sub, s=s)
    assert np.array_equal(c_hi[np.ix_(rows, cols)], w_hi)
    assert np.array_equal(c_lo[np.ix_(rows, cols)], w_lo)
    if s == (16 if variant == INT8_TC else 15):
        # the default piece counts meet the contract on this workload; fewer
        # pieces trade accuracy for speed (their error is 2^(bits (15 - s))
        # or so larger)
        check_sampled_contract(a_hi, a_lo, b_hi, b_lo, c_hi, c_lo, seed=2)


def test_host_strided_pageable_and_small(ops):
    """Leading dimensions above the width (views of wider host arrays),
    pageable (not pinned) memory, a single chunk."""
    m, n, k = 70, 90, 300
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind="wide", seed=5)
    wide = [np.zeros((r, c + 13)) for r, c in ((m, k), (m, k), (k, n), (k, n))]
    for w, x in zip(wide, (a_hi, a_lo, b_hi, b_lo)):
        w[:, :x.shape[1]] = x
    views = [torch.from_numpy(w)[:, :x.shape[1]] for w, x in zip(wide, (a_hi, a_lo, b_hi, b_lo))]
    out_store = [torch.full((m, n + 7), np.nan, dtype=torch.float64) for _ in range(2)]
    out = tuple(o[:, :n] for o in out_store)
    ops.ddgemm_host(*views, out=out)
    torch.cuda.synchronize()
    d_hi, d_lo = run_device(ops, (a_hi, a_lo), (b_hi, b_lo))
    assert np.array_equal(out[0].numpy(), d_hi) and np.array_equal(out[1].numpy(), d_lo)
    assert np.all(np.isnan(out_store[0].numpy()[:, n:]))       # padding untouched
    s_hi, s_lo = cs.cascade_ddgemm(a_hi, a_lo, b_hi, b_lo)
    assert np.all(np.abs((d_hi - s_hi) + (d_lo - s_lo)) <= cascade_tolerance(a_hi, b_hi, s_hi))


def test_host_k0_and_empty(ops):
    z = torch.zeros((5, 0), dtype=torch.float64).pin_memory()
    zb = torch.zeros((0, 4), dtype=torch.float64).pin_memory()
    out = (torch.full((5, 4), np.nan, dtype=torch.float64), torch.full((5, 4), np.nan,
                                                                        dtype=torch.float64))
    ops.ddgemm_host(z, z, zb, zb, out=out)
    torch.cuda.synchronize()
    assert np.all(out[0].numpy() == 0) and np.all(out[1].numpy() == 0)
    e = torch.zeros((0, 3), dtype=torch.float64)
    b = torch.zeros((3, 4), dtype=torch.float64)
    c = ops.ddgemm_host(e, e, b, b)
    assert tuple(c[0].shape) == (0, 4)


def test_host_back_to_back_calls_share_a_buffer(ops):
    """Two calls on one stream with one buffer and no synchronisation
    between them: the second's copies wait for the first's kernels."""
    m, n, k = 2100, 8192, 300
    x = gemm_inputs(m, n, k, kind="uniform", seed=31)
    y = gemm_inputs(m, n, k, kind="wide", seed=32)
    buf = torch.empty(ops.host_buffer_bytes(m, n, k, split_k=1), dtype=torch.uint8,
                      device="cuda")
    # both calls' host operands stay referenced until the stream is done: a
    # pinned tensor freed earlier could be handed out again by PyTorch's
    # pinned-memory cache while a copy still reads it
    px, py = pinned(*x), pinned(*y)
    cx = ops.ddgemm_host(*px, buffer=buf, split_k=1)
    cy = ops.ddgemm_host(*py, buffer=buf, split_k=1)
    torch.cuda.synchronize()
    for c, inp in ((cx, x), (cy, y)):
        d_hi, d_lo = run_device(ops, inp[:2], inp[2:], split_k=1)
        assert np.array_equal(c[0].numpy(), d_hi) and np.array_equal(c[1].numpy(), d_lo)


def test_host_nonfinite_sets_status(ops):
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(40, 30, 50, kind="uniform", seed=3)
    a_hi[3, 7] = np.inf
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ins = pinned(a_hi, a_lo, b_hi, b_lo)
    ops.ddgemm_host(*ins, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & 0x1
