"""Calls on streams other than torch's current one, and from several host
threads at once.

* A call made with ``stream=s`` allocates its workspace and outputs on s.
  Right after it returns, the current stream allocates a block of the
  workspace's size and fills it with junk; had the workspace been allocated
  on the current stream, the allocator could hand that freed block out
  while s's kernels still read it.  C must be bit-identical to the same
  call on the current stream (FP64 form and tcgen05 INT8 form).
* Four host threads, each with its own stream, run the four forms (and the
  host-operand entry point) on their own operands three times over; every
  result is bit-identical to the same call made alone.  The kernels of
  different calls share no state: their waits are all within one CTA."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import gemm_inputs  # noqa: E402

pytestmark = pytest.mark.gpu


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
    return np.array_equal(x.view(np.int64), y.view(np.int64))


@pytest.mark.parametrize("variant", [0, 4])
def test_side_stream_workspace_is_not_handed_out_early(ops, variant):
    m = n = k = 1024
    a = dev(*gemm_inputs(m, n, k, kind="wide", seed=31))
    want = host(*ops.ddgemm(*a, variant=variant))
    ws_bytes = ops.workspace_bytes(m, n, k, variant)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    for _ in range(3):
        c_hi, c_lo = ops.ddgemm(*a, variant=variant, stream=side)
        junk = torch.full((ws_bytes,), 0x7f, dtype=torch.uint8, device="cuda")
        del junk
        side.synchronize()
        got = host(c_hi, c_lo)
        assert same(got[0], want[0]) and same(got[1], want[1])


def test_concurrent_threads_own_streams(ops):
    jobs = [(0, 300, 200, 700), (1, 256, 130, 900), (4, 500, 64, 1000), (5, 129, 300, 513),
            ("host", 600, 90, 400)]
    inputs, want = [], []
    for i, (variant, m, n, k) in enumerate(jobs):
        a = gemm_inputs(m, n, k, kind="uniform" if i % 2 else "wide", seed=40 + i)
        if variant == "host":
            t = [torch.from_numpy(x).pin_memory() for x in a]
            c = ops.ddgemm_host(*t)
            torch.cuda.synchronize()
            want.append([x.numpy().copy() for x in c])
        else:
            t = dev(*a)
            want.append(host(*ops.ddgemm(*t, variant=variant)))
        inputs.append(t)
    results = [[] for _ in jobs]
    errors = []

    def work(i):
        try:
            variant = jobs[i][0]
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.default_stream())
            keep = []
            for _ in range(3):
                if variant == "host":
                    c = ops.ddgemm_host(*inputs[i], stream=s)
                else:
                    c = ops.ddgemm(*inputs[i], variant=variant, stream=s)
                keep.append(c)
            s.synchronize()
            results[i] = [[t.cpu().numpy() for t in c] for c in keep]
        except Exception as e:  # reported below, on the main thread
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(jobs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
    assert not any(t.is_alive() for t in threads)
    assert not errors, errors
    for i in range(len(jobs)):
        assert len(results[i]) == 3
        for got in results[i]:
            assert same(got[0], want[i][0]) and same(got[1], want[i][1]), jobs[i]
