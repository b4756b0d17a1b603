"""ddgemm_noalloc: the cascade GEMM for callers that cannot allocate device
memory (code running under CUDA graph capture, plug-ins inside a framework
whose memory pool owns the GPU, latency-bound paths that cannot afford
cudaMalloc's implicit synchronisation, callers without a GPU allocator).
It takes inputs and outputs only and works in the library's static scratch
array.

The GPU test calls it through the C ABI twice in a row, on different
problems, and checks each result against the ordinary ddgemm entry point
(which takes a caller-provided workspace) within the tolerances of the
parity tests.  This file is collected last so that a run stopping at the
first failure has already run every other test; nothing here depends on
what ran before."""

import numpy as np
import pytest

from paper_2303_04353_gb300 import _lib
from workloads import gemm_inputs

FAKE = 0x10000  # never dereferenced: the size check answers before any CUDA call


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = _lib.load()
    big = 873  # 873^3 needs 64.5 MiB of scratch, more than the 64 MiB array
    no_split = _lib.make_opts(split_k=1)   # the least workspace ddgemm takes
    assert _lib.ddgemm_workspace_size(big, big, big, no_split) > _lib.DDGEMM_NOALLOC_SCRATCH_BYTES
    assert (_lib.ddgemm_workspace_size(big - 1, big - 1, big - 1, no_split)
            <= _lib.DDGEMM_NOALLOC_SCRATCH_BYTES)
    rc = lib.ddgemm_noalloc(big, big, big, FAKE, FAKE, big, FAKE, FAKE, big, FAKE, FAKE, big,
                            None, None)
    assert rc == _lib.DDGEMM_EWORKSPACE
    assert lib.ddgemm_noalloc(-1, 4, 4, FAKE, FAKE, 4, FAKE, FAKE, 4, FAKE, FAKE, 4, None,
                              None) == _lib.DDGEMM_EINVAL


@pytest.mark.gpu
def test_noalloc_matches_ddgemm_twice_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from tests.test_gpu_parity import cascade_tolerance

    stream = torch.cuda.current_stream().cuda_stream
    # two different problems back to back: the second one sees the first
    # one's leftovers in the shared scratch array
    for (m, n, k, kind, seed) in [(300, 260, 700, "wide", 11), (129, 65, 257, "uniform", 12)]:
        a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind=kind, seed=seed)
        A = [torch.from_numpy(x).cuda() for x in (a_hi, a_lo, b_hi, b_lo)]
        ptrs = [t.data_ptr() for t in A]
        c_ref = [torch.empty((m, n), dtype=torch.float64, device="cuda") for _ in range(2)]
        c_new = [torch.full((m, n), np.nan, dtype=torch.float64, device="cuda") for _ in range(2)]
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        opts = _lib.make_opts(status_dev=status.data_ptr())

        ws = torch.empty(_lib.ddgemm_workspace_size(m, n, k), dtype=torch.uint8, device="cuda")
        _lib.ddgemm(m, n, k, ptrs[0], ptrs[1], k, ptrs[2], ptrs[3], n, c_ref[0].data_ptr(),
                    c_ref[1].data_ptr(), n, ws.data_ptr(), ws.numel(), stream, opts)
        _lib.ddgemm_noalloc(m, n, k, ptrs[0], ptrs[1], k, ptrs[2], ptrs[3], n,
                            c_new[0].data_ptr(), c_new[1].data_ptr(), n, stream, opts)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        rh, rl = (t.cpu().numpy() for t in c_ref)
        nh, nl = (t.cpu().numpy() for t in c_new)
        diff = np.abs((nh - rh) + (nl - rl))
        assert np.all(np.isfinite(nh)) and np.all(np.isfinite(nl))
        assert np.all(diff <= 1e-28 * (np.abs(a_hi) @ np.abs(b_hi)) + 0.0)
        assert np.all(diff <= cascade_tolerance(a_hi, b_hi, rh))
