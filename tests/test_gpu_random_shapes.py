"""Randomized shapes through all three forms (seeded, reproducible): m, n,
k drawn in [1, 300] with ragged tiles, both value kinds, random
transposition of either operand.

* the INT8 form on mma.sync and on tcgen05 (seven- and eight-bit pieces):
  bit-identical to their CPU restatements (oracle/cascade_int8.py);
* the FP64 form: within the paper's bound of the double-double oracle and
  within the summation-order tolerance of the cascade restatement
  (tests/test_gpu_parity.py's check)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cascade_int8 as c8  # noqa: E402
from workloads import gemm_inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04353_gb300 import ops as _ops
    return _ops


def cases(count=40, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for c in range(count):
        m, n, k = (int(x) for x in rng.integers(1, 301, 3))
        out.append((c, m, n, k, "wide" if c % 2 else "uniform", bool(rng.integers(0, 2)),
                    bool(rng.integers(0, 2))))
    return out


def dev(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


@pytest.mark.parametrize("c,m,n,k,kind,ta,tb", cases())
def test_random_shape_all_forms(ops, c, m, n, k, kind, ta, tb):
    from tests.test_gpu_parity import check_against_oracles
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind=kind, seed=500 + c)
    sa = (a_hi.T, a_lo.T) if ta else (a_hi, a_lo)
    sb = (b_hi.T, b_lo.T) if tb else (b_hi, b_lo)
    # FP64 form (automatic split-k included)
    check_against_oracles(ops, a_hi, a_lo, b_hi, b_lo, trans_a=ta, trans_b=tb,
                          contract=kind == "uniform")
    # INT8 forms, bit for bit
    for variant, s, assembly, bits in ((1, 15, "fp64x2", 8), (4, 16, "exact", 7),
                                       (5, 15, "exact", 8)):
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        c_hi, c_lo = ops.ddgemm(*dev(*sa), *dev(*sb), trans_a=ta, trans_b=tb, variant=variant,
                                status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        w_hi, w_lo = c8.cascade_int8_ddgemm(a_hi, a_lo, b_hi, b_lo, s=s, assembly=assembly,
                                            bits=bits)
        assert np.array_equal(c_hi.cpu().numpy(), w_hi), (variant, m, n, k)
        assert np.array_equal(c_lo.cpu().numpy(), w_lo), (variant, m, n, k)
