"""The cascade kernels' own timeout path, driven without any fault.

`ddgemm_diag_withheld_copy` runs a form's real cascade kernel with one copy
of one CTA never issued: the mbarrier that copy would complete never does,
so that CTA's waits run out after the given limit (20 ms here).  The CTA
must then set DDGEMM_DEV_TIMEOUT, let its other copies land, release its
tensor memory (tcgen05 forms) and return, and the call must end long before
the default ~2 s limit.  The same context must afterwards compute every form
bit for bit as before: a CTA that kept its tensor memory or left copies in
flight would break the next tcgen05 launch on its SM."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import gemm_inputs  # noqa: E402

pytestmark = pytest.mark.gpu

LIMIT_NS = 20_000_000   # 20 ms
TIMEOUT = 0x2
FP64, INT8, TC, TC8 = 0, 1, 4, 5
SLICES = {FP64: 0, INT8: 15, TC: 16, TC8: 15}


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04353_gb300 import ops as _ops
    return _ops


def dev(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def same(x, y):
    return x.shape == y.shape and np.array_equal(x.view(np.int64), y.view(np.int64))


def withheld_call(ops, t, m, n, k, variant, cta, step, split_k=0):
    """One ddgemm with the copy of ring step `step` of CTA `cta` withheld;
    returns (status word, seconds, C)."""
    from paper_2303_04353_gb300 import _lib
    s8 = SLICES[variant]
    ws = ops.alloc_workspace(m, n, k, "cuda", variant, s8, split_k=split_k)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    c = [torch.zeros((m, n), dtype=torch.float64, device="cuda") for _ in range(2)]
    opts = _lib.make_opts(variant=variant, int8_slices=s8, status_dev=status.data_ptr(),
                          split_k=split_k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _lib.ddgemm_diag_withheld_copy(m, n, k, t[0].data_ptr(), t[1].data_ptr(), k, t[2].data_ptr(),
                                   t[3].data_ptr(), n, c[0].data_ptr(), c[1].data_ptr(), n,
                                   ws.data_ptr(), ws.numel(),
                                   torch.cuda.current_stream().cuda_stream, opts, cta, step,
                                   LIMIT_NS)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return int(status.item()), dt, [x.cpu().numpy() for x in c]


def reference(ops, t, variant, split_k=0):
    out = ops.ddgemm(*t, variant=variant, int8_slices=SLICES[variant], split_k=split_k)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in out]


# (m, n, k, step): for the tcgen05 forms the second case gives CTA 0 a
# second tile (160 tiles of 128 x 16 on 152 SMs) and withholds a stage of it
CASES = {
    FP64: [(300, 200, 700, 0), (300, 200, 700, 5)],
    INT8: [(300, 200, 700, 0), (300, 200, 700, 5)],
    TC: [(300, 200, 700, 0), (640, 512, 300, 25)],
    TC8: [(300, 200, 700, 3), (640, 512, 300, 25)],
}


@pytest.mark.parametrize("variant,case", [(v, c) for v, cs in CASES.items() for c in cs])
def test_withheld_copy_times_out_and_context_survives(ops, variant, case):
    m, n, k, step = case
    a = gemm_inputs(m, n, k, kind="wide", seed=m + step)
    t = dev(*a)
    before = {v: reference(ops, t, v) for v in SLICES}
    st, dt, c = withheld_call(ops, t, m, n, k, variant, cta=0, step=step)
    assert st & TIMEOUT, f"status {st:#x}"
    assert dt < 1.0, f"the call took {dt:.2f} s"
    if variant == FP64:
        # CTA 0 owns the first 64 x 64 tile: NaN, not a plausible partial sum
        assert np.isnan(c[0][:64, :64]).all() and np.isnan(c[1][:64, :64]).all()
        assert np.isfinite(c[0][64:, :]).all()
    # the context is intact: every form again bit for bit
    for v, want in before.items():
        got = reference(ops, t, v)
        assert same(got[0], want[0]) and same(got[1], want[1]), v


def test_withheld_copy_of_a_split_k_group_poisons_its_tile(ops):
    """Split-k: a group whose wait runs out writes NaN into its partial
    tile, so the fix-up makes that tile of C NaN instead of adding stale
    partial sums; every other tile is the normal result bit for bit."""
    m, n, k = 128, 128, 2048          # 4 tiles of 64 x 64, 8 k-blocks
    a = gemm_inputs(m, n, k, kind="uniform", seed=5)
    t = dev(*a)
    want = reference(ops, t, FP64, split_k=4)
    # CTA index = group * tiles + tile: CTA 5 is group 1 of tile 1
    st, dt, c = withheld_call(ops, t, m, n, k, FP64, cta=5, step=0, split_k=4)
    assert st & TIMEOUT and dt < 1.0
    tile = np.zeros((m, n), dtype=bool)
    tile[:64, 64:] = True               # tile 1 in the grouped tile order
    if not np.isnan(c[0][tile]).all():  # locate the poisoned tile whatever the order
        nan = np.isnan(c[0])
        assert nan.sum() == 64 * 64
        tile = nan
    assert np.isnan(c[0][tile]).all() and np.isnan(c[1][tile]).all()
    assert same(c[0][~tile], want[0][~tile]) and same(c[1][~tile], want[1][~tile])
    got = reference(ops, t, FP64, split_k=4)
    assert same(got[0], want[0]) and same(got[1], want[1])


@pytest.mark.parametrize("variant", [TC, TC8])
def test_batched_tc_withheld_copy(ops, variant):
    """The persistent batched tcgen05 kernel: CTA 0 gives up on its withheld
    stage within the limit, the status reports it, and the batch then runs
    again bit-identically to its first run."""
    from paper_2303_04353_gb300 import _lib
    rng = np.random.default_rng(3)
    probs, host = [], []
    for i in range(24):
        m, n, k = (int(x) for x in rng.integers(40, 400, 3))
        a = gemm_inputs(m, n, k, kind="uniform", seed=100 + i)
        t = dev(*a)
        probs.append((*t, torch.empty((m, n), dtype=torch.float64, device="cuda"),
                      torch.empty((m, n), dtype=torch.float64, device="cuda")))
        host.append(a)
    batch = ops.Batch(probs, variant=variant)
    batch.run()
    torch.cuda.synchronize()
    want = [(p[4].cpu().numpy().copy(), p[5].cpu().numpy().copy()) for p in probs]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    opts = _lib.make_opts(variant=variant, status_dev=status.data_ptr())
    t0 = time.perf_counter()
    _lib.ddgemm_diag_batched_withheld_copy(batch.count, batch.host, batch.dev.data_ptr(),
                                           batch.workspace.data_ptr(), batch.workspace.numel(),
                                           torch.cuda.current_stream().cuda_stream, opts, 0, 3,
                                           LIMIT_NS)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(status.item()) & TIMEOUT and dt < 1.0
    batch.run()
    torch.cuda.synchronize()
    for p, (h, lo) in zip(probs, want):
        assert same(p[4].cpu().numpy(), h) and same(p[5].cpu().numpy(), lo)
