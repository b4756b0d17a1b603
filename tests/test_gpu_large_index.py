"""Operands of more than 2^31 entries: the 64-bit index paths of every form.

Four cases, each with one operand of 65539 x 32808 = 2.15e9 entries (ragged
in the long dimension; k a multiple of 8 but not of 256): A of m x k =
65539 x 32808 with n = 40, or B of k x n = 32808 x 65539 with m = 40, each
stored as is or transposed, so that the long operand goes through both the
contiguous and the strided split kernels.  The skinny side leaves a grid of
1025 FP64 tiles, so the FP64 form also takes its split-k path.  Inputs
follow the uniform workload's law and are drawn on the device
(workloads.device_uniform_dd); 10 sampled entries, among them the first and
last row and column, come back to the host:
* the FP64 form within 1e-28 (|A||B|) of the double-double oracle and
  within the summation-order tolerance of the cascade restatement;
* the three INT8 forms bit for bit against their CPU restatements
  (oracle/cascade_int8.py), which need only the sampled rows of A and
  columns of B (every scale is per row or column and k-block).
Each case holds 100-160 GB on the device; it skips where less is free."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cascade as cs  # noqa: E402
from oracle import cascade_int8 as c8  # noqa: E402
from oracle import dd  # noqa: E402
from tests import exact  # noqa: E402
from tests.bounds import paper_bound  # noqa: E402
from workloads import device_uniform_dd  # noqa: E402

pytestmark = pytest.mark.gpu

CONTRACT = 1e-28
SAMPLES = 10
# (variant, slices, assembly, bits) of the INT8 forms' restatements
INT8_FORMS = ((1, 15, "fp64x2", 8), (4, 16, "exact", 7), (5, 15, "exact", 8))


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04353_gb300 import ops as _ops
    return _ops


def sample_indices(m, n, seed):
    rng = np.random.default_rng(seed)
    rows = np.concatenate([[0, m - 1], rng.integers(0, m, SAMPLES - 2)])
    cols = np.concatenate([[n - 1, 0], rng.integers(0, n, SAMPLES - 2)])
    return rows, cols


def to_host(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("large,trans_a,trans_b", [("a", False, False), ("a", True, False),
                                                   ("b", False, False), ("b", False, True)])
def test_operands_past_2_pow_31_entries(ops, large, trans_a, trans_b):
    from tests.test_gpu_parity import cascade_tolerance, split_groups, split_tolerance
    from paper_2303_04353_gb300 import _lib

    m, n, k = (65539, 40, 32808) if large == "a" else (40, 65539, 32808)
    assert max(m, n) * k > 2 ** 31
    variants = [_lib.DDGEMM_VARIANT_FP64] + [f[0] for f in INT8_FORMS]
    inputs = 2 * 8 * (m * k + k * n)
    need = inputs + max(ops.workspace_bytes(m, n, k, variant=v) for v in variants) + (4 << 30)
    free, _ = torch.cuda.mem_get_info()
    if free < need:
        pytest.skip(f"needs {need / 2**30:.0f} GiB of device memory, {free / 2**30:.0f} free")

    # op(A) is m x k, stored k x m when transposed; op(B) likewise
    a_hi, a_lo = device_uniform_dd((k, m) if trans_a else (m, k), seed=71)
    b_hi, b_lo = device_uniform_dd((n, k) if trans_b else (k, n), seed=72)
    rows, cols = sample_indices(m, n, seed=73)
    ri = torch.from_numpy(rows).cuda()
    ci = torch.from_numpy(cols).cuda()
    # the sampled rows of op(A) (10 x k) and columns of op(B) (k x 10)
    if trans_a:
        sa_hi, sa_lo = to_host(a_hi[:, ri]).T.copy(), to_host(a_lo[:, ri]).T.copy()
    else:
        sa_hi, sa_lo = to_host(a_hi[ri]), to_host(a_lo[ri])
    if trans_b:
        sb_hi, sb_lo = to_host(b_hi[ci]).T.copy(), to_host(b_lo[ci]).T.copy()
    else:
        sb_hi, sb_lo = to_host(b_hi[:, ci]), to_host(b_lo[:, ci])
    diag = np.arange(SAMPLES)

    # FP64 form
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    c_hi, c_lo = ops.ddgemm(a_hi, a_lo, b_hi, b_lo, trans_a=trans_a, trans_b=trans_b,
                            status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got_hi, got_lo = to_host(c_hi[ri, ci]), to_host(c_lo[ri, ci])
    assert bool(torch.isfinite(c_hi).all()) and bool(torch.isfinite(c_lo).all())
    del c_hi, c_lo
    torch.cuda.empty_cache()
    assert exact.dd_is_normalised(got_hi, got_lo)
    o_hi, o_lo = dd.ddgemm_entries(sa_hi, sa_lo, sb_hi, sb_lo, diag, diag)
    absab = np.abs(sa_hi) @ np.abs(sb_hi)
    diff = np.abs((got_hi - o_hi) + (got_lo - o_lo))
    bound = np.diag(paper_bound(sa_hi, sb_hi)) + 4 * (k + 2) * 2.0 ** -106 * np.diag(absab)
    assert np.all(diff <= bound)
    assert np.all(diff <= CONTRACT * np.diag(absab))
    s_hi, s_lo = cs.cascade_ddgemm(sa_hi, sa_lo, sb_hi, sb_lo)
    dcs = np.abs((got_hi - np.diag(s_hi)) + (got_lo - np.diag(s_lo)))
    groups = split_groups(m, n, k)
    tol = cascade_tolerance(sa_hi, sb_hi, s_hi) + split_tolerance(sa_hi, sb_hi, groups)
    assert np.all(dcs <= np.diag(np.broadcast_to(tol, s_hi.shape)))

    # INT8 forms, bit for bit on the sampled entries
    for variant, s, assembly, bits in INT8_FORMS:
        status.zero_()
        c_hi, c_lo = ops.ddgemm(a_hi, a_lo, b_hi, b_lo, trans_a=trans_a, trans_b=trans_b,
                                variant=variant, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got_hi, got_lo = to_host(c_hi[ri, ci]), to_host(c_lo[ri, ci])
        del c_hi, c_lo
        torch.cuda.empty_cache()
        w_hi, w_lo = c8.cascade_int8_ddgemm(sa_hi, sa_lo, sb_hi, sb_lo, s=s, assembly=assembly,
                                            bits=bits)
        assert np.array_equal(got_hi, np.diag(w_hi)), variant
        assert np.array_equal(got_lo, np.diag(w_lo)), variant
