"""PyTorch-facing wrappers of the C ABI.  PyTorch supplies device memory
(outputs, workspace) and the stream; every step of the computation runs in
libddgemm's kernels.  Inputs must be float64 CUDA tensors with unit stride
in their last dimension; a (hi, lo) pair must share shape and strides."""
from __future__ import annotations

import contextlib
import ctypes
import functools

import torch

from . import _lib


def _check_pair(hi: torch.Tensor, lo: torch.Tensor, name: str) -> int:
    if hi.dtype != torch.float64 or lo.dtype != torch.float64:
        raise TypeError(f"{name}: hi and lo must be float64")
    if not (hi.is_cuda and lo.is_cuda):
        raise ValueError(f"{name}: hi and lo must be CUDA tensors (there is no CPU path)")
    if hi.dim() != 2 or hi.shape != lo.shape or hi.stride() != lo.stride():
        raise ValueError(f"{name}: hi and lo must be 2-D with equal shape and strides")
    if hi.numel() > 0 and hi.shape[1] > 1 and hi.stride(1) != 1:
        raise ValueError(f"{name}: the last dimension must be contiguous")
    return max(hi.stride(0), hi.shape[1], 1)


def current_stream_ptr(stream: torch.cuda.Stream | None = None) -> int:
    return (stream if stream is not None else torch.cuda.current_stream()).cuda_stream


def _cuda_devices(args, kwargs, stream):
    """The CUDA devices of the tensors among a call's arguments (one level
    of tuples and lists included) and of its stream."""
    devs = set()
    for a in list(args) + list(kwargs.values()):
        for t in (a if isinstance(a, (tuple, list)) else (a,)):
            if isinstance(t, torch.Tensor) and t.is_cuda:
                devs.add(t.device)
    if stream is not None:
        devs.add(stream.device)
    return devs


def _on_call_stream(fn):
    """Runs a wrapper on the device of its CUDA tensors (all on one device,
    else ValueError: the library launches on the current device), with its
    `stream` argument as torch's current stream, so that its outputs and
    temporaries are allocated (and zero-filled) on the stream its kernels
    use.  The caching allocator ties every block to the stream it was
    allocated on: a workspace freed when the call returns is then not
    handed out to another stream while those kernels may still run."""
    @functools.wraps(fn)
    def call(*args, stream=None, **kwargs):
        devs = _cuda_devices(args, kwargs, stream)
        if len(devs) > 1:
            raise ValueError(f"tensors and stream on different devices: {sorted(map(str, devs))}")
        with contextlib.ExitStack() as scope:
            if devs:
                scope.enter_context(torch.cuda.device(devs.pop()))
            if stream is not None:
                scope.enter_context(torch.cuda.stream(stream))
            return fn(*args, stream=stream, **kwargs)
    return call


def workspace_bytes(m: int, n: int, k: int, variant: int = _lib.DDGEMM_VARIANT_FP64,
                    int8_slices: int = 0, split_k: int = 0) -> int:
    return _lib.ddgemm_workspace_size(m, n, k, _lib.make_opts(
        variant=variant, int8_slices=int8_slices, split_k=split_k))


def split_groups(m: int, n: int, k: int, device=None, ws_bytes: int | None = None,
                 variant: int = _lib.DDGEMM_VARIANT_FP64, split_k: int = 0) -> int:
    """Split-k groups ddgemm() launches on `device` with a workspace of
    ws_bytes (default: workspace_bytes())."""
    opts = _lib.make_opts(variant=variant, split_k=split_k)
    if ws_bytes is None:
        ws_bytes = _lib.ddgemm_workspace_size(m, n, k, opts)
    sms = torch.cuda.get_device_properties(device or torch.cuda.current_device()).multi_processor_count
    return _lib.load().ddgemm_split_groups(m, n, k, sms, ws_bytes, ctypes.byref(opts))


def alloc_workspace(m: int, n: int, k: int, device=None, variant: int = _lib.DDGEMM_VARIANT_FP64,
                    int8_slices: int = 0, split_k: int = 0) -> torch.Tensor:
    nbytes = workspace_bytes(m, n, k, variant, int8_slices, split_k)
    # torch's caching allocator hands out 512-byte aligned blocks
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device or "cuda")


@_on_call_stream
def ddgemm(a_hi, a_lo, b_hi, b_lo, *, trans_a=False, trans_b=False, out=None, workspace=None,
           status=None, flags=None, stream=None, phase_events=None,
           variant=_lib.DDGEMM_VARIANT_FP64, int8_slices=0, split_k=0):
    """C := op(A) op(B) in FP64x2 by the ten-GEMM cascade.  Returns (c_hi, c_lo).

    trans_a: A is stored k x m and op(A) = A^T (likewise trans_b: B stored n x k).
    out: optional (c_hi, c_lo) float64 tensors, m x n, unit last stride.
    status: optional int32 CUDA tensor of one element; DDGEMM_DEV_* bits are OR-ed in.
    flags: optional int32 CUDA tensor (m x n, contiguous) for cancellation counts.
    phase_events: optional three recorded torch.cuda.Event objects; the library
    re-records them around the split and the cascade kernel on the stream.
    variant: DDGEMM_VARIANT_FP64 (ten FP64 products) or DDGEMM_VARIANT_INT8
    (int8_slices INT8 pieces per entry, 0 = 15).
    split_k: 0 = automatic split-k for small grids, 1 = never, 2-16 = forced."""
    lda = _check_pair(a_hi, a_lo, "A")
    ldb = _check_pair(b_hi, b_lo, "B")
    m, k = (a_hi.shape[1], a_hi.shape[0]) if trans_a else tuple(a_hi.shape)
    kb, n = (b_hi.shape[1], b_hi.shape[0]) if trans_b else tuple(b_hi.shape)
    if k != kb:
        raise ValueError(f"inner dimensions differ: {k} vs {kb}")
    dev = a_hi.device
    if out is None:
        c_hi = torch.empty((m, n), dtype=torch.float64, device=dev)
        c_lo = torch.empty((m, n), dtype=torch.float64, device=dev)
    else:
        c_hi, c_lo = out
        if tuple(c_hi.shape) != (m, n):
            raise ValueError("out has the wrong shape")
    ldc = _check_pair(c_hi, c_lo, "C")
    if workspace is None:
        workspace = alloc_workspace(m, n, k, dev, variant, int8_slices, split_k)
    if status is not None and (status.dtype != torch.int32 or not status.is_cuda):
        raise TypeError("status must be an int32 CUDA tensor")
    if flags is not None and (flags.dtype != torch.int32 or not flags.is_contiguous()
                              or flags.numel() < m * n):
        raise TypeError("flags must be a contiguous int32 CUDA tensor with m*n entries")
    evs = None
    if phase_events is not None:
        if len(phase_events) != 3 or not all(e.cuda_event for e in phase_events):
            raise ValueError("phase_events: three torch.cuda.Event, each recorded once")
        evs = (ctypes.c_void_p * 3)(*[e.cuda_event for e in phase_events])
    opts = _lib.make_opts(trans_a, trans_b, variant,
                          status.data_ptr() if status is not None else 0,
                          flags.data_ptr() if flags is not None else 0, evs, int8_slices, split_k)
    _lib.ddgemm(m, n, k, a_hi.data_ptr(), a_lo.data_ptr(), lda, b_hi.data_ptr(),
                b_lo.data_ptr(), ldb, c_hi.data_ptr(), c_lo.data_ptr(), ldc,
                workspace.data_ptr(), workspace.numel(), current_stream_ptr(stream), opts)
    return c_hi, c_lo


def _check_host_pair(hi: torch.Tensor, lo: torch.Tensor, name: str) -> int:
    if hi.dtype != torch.float64 or lo.dtype != torch.float64:
        raise TypeError(f"{name}: hi and lo must be float64")
    if hi.is_cuda or lo.is_cuda:
        raise ValueError(f"{name}: ddgemm_host takes host (CPU) tensors")
    if hi.dim() != 2 or hi.shape != lo.shape or hi.stride() != lo.stride():
        raise ValueError(f"{name}: hi and lo must be 2-D with equal shape and strides")
    if hi.numel() > 0 and hi.shape[1] > 1 and hi.stride(1) != 1:
        raise ValueError(f"{name}: the last dimension must be contiguous")
    return max(hi.stride(0), hi.shape[1], 1)


def host_buffer_bytes(m: int, n: int, k: int, variant: int = _lib.DDGEMM_VARIANT_FP64,
                      int8_slices: int = 0, split_k: int = 0, trans_a=False,
                      trans_b=False) -> int:
    return _lib.ddgemm_host_buffer_size(m, n, k, _lib.make_opts(
        trans_a, trans_b, variant, int8_slices=int8_slices, split_k=split_k))


@_on_call_stream
def ddgemm_host(a_hi, a_lo, b_hi, b_lo, *, trans_a=False, trans_b=False, out=None, buffer=None,
                device=None, status=None, stream=None, variant=_lib.DDGEMM_VARIANT_FP64,
                int8_slices=0, split_k=0):
    """C := op(A) op(B) on HOST (CPU) float64 tensors through ddgemm_host:
    the library copies the operands in and C out on streams of its own,
    overlapping the cascade on `stream`.  Use pinned tensors
    (``pin_memory()``) for asynchronous copies.  Returns (c_hi, c_lo), host
    tensors that hold C once `stream` has been synchronised.  Keep the input
    tensors referenced and unchanged until then: PyTorch's pinned-memory
    cache can hand a freed pinned block out again while the library's copy
    still reads it.

    buffer: optional device uint8 tensor of >= host_buffer_bytes() bytes
    (allocated on `device`, default the current CUDA device, when None)."""
    lda = _check_host_pair(a_hi, a_lo, "A")
    ldb = _check_host_pair(b_hi, b_lo, "B")
    m, k = (a_hi.shape[1], a_hi.shape[0]) if trans_a else tuple(a_hi.shape)
    kb, n = (b_hi.shape[1], b_hi.shape[0]) if trans_b else tuple(b_hi.shape)
    if k != kb:
        raise ValueError(f"inner dimensions differ: {k} vs {kb}")
    if out is None:
        pin = a_hi.is_pinned()
        c_hi = torch.empty((m, n), dtype=torch.float64, pin_memory=pin)
        c_lo = torch.empty((m, n), dtype=torch.float64, pin_memory=pin)
    else:
        c_hi, c_lo = out
        if tuple(c_hi.shape) != (m, n):
            raise ValueError("out has the wrong shape")
    ldc = _check_host_pair(c_hi, c_lo, "C")
    if buffer is None:
        nbytes = host_buffer_bytes(m, n, k, variant, int8_slices, split_k, trans_a, trans_b)
        buffer = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device or "cuda")
    if status is not None and (status.dtype != torch.int32 or not status.is_cuda):
        raise TypeError("status must be an int32 CUDA tensor")
    opts = _lib.make_opts(trans_a, trans_b, variant,
                          status.data_ptr() if status is not None else 0,
                          int8_slices=int8_slices, split_k=split_k)
    _lib.ddgemm_host(m, n, k, a_hi.data_ptr(), a_lo.data_ptr(), lda, b_hi.data_ptr(),
                     b_lo.data_ptr(), ldb, c_hi.data_ptr(), c_lo.data_ptr(), ldc,
                     buffer.data_ptr(), buffer.numel(), current_stream_ptr(stream), opts)
    return c_hi, c_lo


@_on_call_stream
def assemble_int8(diag: torch.Tensor, scale: torch.Tensor, *, stream=None):
    """The exact assembly of the tensor-core INT8 form on the device: for
    diag [s, count] int32 and scale [count] int32, returns (hi, lo), the
    FP64x2 nearest to sum_t diag[t] 2^(-12-7t) 2^scale."""
    if diag.dtype != torch.int32 or scale.dtype != torch.int32 or not diag.is_cuda:
        raise TypeError("diag and scale must be int32 CUDA tensors")
    s, count = diag.shape
    diag = diag.contiguous()
    scale = scale.contiguous()
    hi = torch.empty(count, dtype=torch.float64, device=diag.device)
    lo = torch.empty(count, dtype=torch.float64, device=diag.device)
    _lib.ddgemm_assemble_int8(count, s, diag.data_ptr(), scale.data_ptr(), hi.data_ptr(),
                              lo.data_ptr(), current_stream_ptr(stream))
    return hi, lo


@_on_call_stream
def split_a(a_hi, a_lo, *, trans_a=False, stream=None, status=None):
    """The split step for A: returns (slices [4, m, k], exps [ceil(k/256), m])."""
    lda = _check_pair(a_hi, a_lo, "A")
    m, k = (a_hi.shape[1], a_hi.shape[0]) if trans_a else tuple(a_hi.shape)
    slices = torch.zeros((4, m, k), dtype=torch.float64, device=a_hi.device)
    exps = torch.zeros(((k + 255) // 256, m), dtype=torch.int32, device=a_hi.device)
    _lib.ddgemm_split_a(m, k, a_hi.data_ptr(), a_lo.data_ptr(), lda, trans_a,
                        slices.data_ptr(), max(k, 1), exps.data_ptr(),
                        status.data_ptr() if status is not None else 0,
                        current_stream_ptr(stream))
    return slices, exps


@_on_call_stream
def split_b(b_hi, b_lo, *, trans_b=False, stream=None, status=None):
    """The split step for B: returns (panels [7, k, n], exps [ceil(k/256), n])."""
    ldb = _check_pair(b_hi, b_lo, "B")
    k, n = (b_hi.shape[1], b_hi.shape[0]) if trans_b else tuple(b_hi.shape)
    slices = torch.zeros((7, k, n), dtype=torch.float64, device=b_hi.device)
    exps = torch.zeros(((k + 255) // 256, n), dtype=torch.int32, device=b_hi.device)
    _lib.ddgemm_split_b(k, n, b_hi.data_ptr(), b_lo.data_ptr(), ldb, trans_b,
                        slices.data_ptr(), max(n, 1), exps.data_ptr(),
                        status.data_ptr() if status is not None else 0,
                        current_stream_ptr(stream))
    return slices, exps


@_on_call_stream
def bins(a_hi, a_lo, b_hi, b_lo, *, stream=None):
    """The four bins of the single k-block (k <= 256), shape [4, m, n]."""
    lda = _check_pair(a_hi, a_lo, "A")
    ldb = _check_pair(b_hi, b_lo, "B")
    m, k = a_hi.shape
    n = b_hi.shape[1]
    out = torch.empty((4, m, n), dtype=torch.float64, device=a_hi.device)
    ws = alloc_workspace(m, n, k, a_hi.device)
    _lib.ddgemm_bins(m, n, k, a_hi.data_ptr(), a_lo.data_ptr(), lda, b_hi.data_ptr(),
                     b_lo.data_ptr(), ldb, out.data_ptr(), ws.data_ptr(), ws.numel(),
                     current_stream_ptr(stream), None)
    return out


@_on_call_stream
def ddgemm_backward(a_hi, a_lo, b_hi, b_lo, dc_hi, dc_lo, *, trans_a=False, trans_b=False,
                    workspace=None, status=None, stream=None,
                    variant=_lib.DDGEMM_VARIANT_FP64, int8_slices=0):
    """dA = dC op(B)^T and dB = op(A)^T dC through the cascade (variant: the
    FP64 form or one of the INT8 forms); returns (dA_hi, dA_lo, dB_hi,
    dB_lo) in the storage shapes of A and B."""
    lda = _check_pair(a_hi, a_lo, "A")
    ldb = _check_pair(b_hi, b_lo, "B")
    lddc = _check_pair(dc_hi, dc_lo, "dC")
    m, k = (a_hi.shape[1], a_hi.shape[0]) if trans_a else tuple(a_hi.shape)
    kb, n = (b_hi.shape[1], b_hi.shape[0]) if trans_b else tuple(b_hi.shape)
    if k != kb or tuple(dc_hi.shape) != (m, n):
        raise ValueError("shapes of A, B and dC do not match")
    dev = a_hi.device
    da = [torch.empty(a_hi.shape, dtype=torch.float64, device=dev) for _ in range(2)]
    db = [torch.empty(b_hi.shape, dtype=torch.float64, device=dev) for _ in range(2)]
    opts = _lib.make_opts(trans_a, trans_b, variant,
                          status.data_ptr() if status is not None else 0,
                          int8_slices=int8_slices)
    if workspace is None:
        nbytes = _lib.ddgemm_backward_workspace_size(m, n, k, opts)
        workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    _lib.ddgemm_backward(m, n, k, a_hi.data_ptr(), a_lo.data_ptr(), lda, b_hi.data_ptr(),
                         b_lo.data_ptr(), ldb, dc_hi.data_ptr(), dc_lo.data_ptr(), lddc,
                         da[0].data_ptr(), da[1].data_ptr(), max(da[0].shape[1], 1),
                         db[0].data_ptr(), db[1].data_ptr(), max(db[0].shape[1], 1),
                         workspace.data_ptr(), workspace.numel(), current_stream_ptr(stream),
                         opts)
    return da[0], da[1], db[0], db[1]


@_on_call_stream
def split_int8(x_hi, x_lo, *, as_b=False, trans=False, slices=15, stream=None, status=None):
    """The INT8 split of A (as_b=False; vectors = rows of op(A)) or of B
    (as_b=True; vectors = columns of op(B)).  Returns (digits [s, nvec, k]
    int8, exps [ceil(k/8192), nvec] int32)."""
    ld = _check_pair(x_hi, x_lo, "X")
    if not as_b:
        nvec, k = (x_hi.shape[1], x_hi.shape[0]) if trans else tuple(x_hi.shape)
    else:
        k, nvec = (x_hi.shape[1], x_hi.shape[0]) if trans else tuple(x_hi.shape)
    ldd = max(16, (k + 15) // 16 * 16)
    digits = torch.zeros((slices, nvec, ldd), dtype=torch.int8, device=x_hi.device)
    exps = torch.zeros(((k + 8191) // 8192, nvec), dtype=torch.int32, device=x_hi.device)
    fn = _lib.ddgemm_split_int8_b if as_b else _lib.ddgemm_split_int8_a
    if as_b:
        fn(k, nvec, x_hi.data_ptr(), x_lo.data_ptr(), ld, trans, slices, digits.data_ptr(), ldd,
           exps.data_ptr(), status.data_ptr() if status is not None else 0,
           current_stream_ptr(stream))
    else:
        fn(nvec, k, x_hi.data_ptr(), x_lo.data_ptr(), ld, trans, slices, digits.data_ptr(), ldd,
           exps.data_ptr(), status.data_ptr() if status is not None else 0,
           current_stream_ptr(stream))
    return digits[:, :, :k], exps


class Batch:
    """Many FP64x2 GEMMs C_i := A_i B_i run by one ddgemm_batched call.

    ``problems`` is a list of (a_hi, a_lo, b_hi, b_lo, c_hi, c_lo) CUDA
    tensors (row-major, unit last stride).  The constructor uploads the
    problem descriptors and allocates the workspace (PyTorch memory), so
    ``run()`` only enqueues the launches (four in either form) and can be
    captured into a CUDA graph.  The tensors must stay alive and in place
    while the batch is used, and the Batch itself (its workspace) until the
    work of its last ``run()`` has completed on the stream it was enqueued
    on."""

    def __init__(self, problems, device=None, variant=_lib.DDGEMM_VARIANT_FP64, int8_slices=0):
        """variant: DDGEMM_VARIANT_FP64 (the persistent FP64 kernel),
        DDGEMM_VARIANT_INT8_TC (the INT8 form on the tcgen05 tensor cores) or
        DDGEMM_VARIANT_INT8_TC8 (the same with eight-bit pieces)."""
        self.count = len(problems)
        self.variant = variant
        self.int8_slices = int8_slices
        arr = (_lib.ddgemm_problem * max(self.count, 1))()
        self.shapes = []
        self._keep = []
        for i, (a_hi, a_lo, b_hi, b_lo, c_hi, c_lo) in enumerate(problems):
            lda = _check_pair(a_hi, a_lo, "A")
            ldb = _check_pair(b_hi, b_lo, "B")
            ldc = _check_pair(c_hi, c_lo, "C")
            m, k = a_hi.shape
            n = b_hi.shape[1]
            if b_hi.shape[0] != k or tuple(c_hi.shape) != (m, n):
                raise ValueError(f"problem {i}: shapes do not match")
            arr[i] = _lib.ddgemm_problem(m, n, k, lda, ldb, ldc, a_hi.data_ptr(), a_lo.data_ptr(),
                                         b_hi.data_ptr(), b_lo.data_ptr(), c_hi.data_ptr(),
                                         c_lo.data_ptr())
            self.shapes.append((m, n, k))
            self._keep.append((a_hi, a_lo, b_hi, b_lo, c_hi, c_lo))
        self.host = arr
        devs = {t.device for p in problems for t in p}
        if len(devs) > 1 or (device is not None and devs and torch.device(device) not in devs):
            raise ValueError(f"problems on different devices: {sorted(map(str, devs))}")
        dev = device or (problems[0][0].device if problems else "cuda")
        raw = bytearray(ctypes.string_at(ctypes.addressof(arr), ctypes.sizeof(arr)))
        self.dev = torch.frombuffer(raw, dtype=torch.uint8).to(dev)
        nbytes = _lib.ddgemm_batched_workspace_size(
            self.count, arr, _lib.make_opts(variant=variant, int8_slices=int8_slices))
        self.workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)

    def run(self, stream=None, config=None, status=None, phase_events=None):
        """Enqueue the batch.  config: None (library default), a
        ddgemm_batch_config, or a tuple of its fields (tile, order[, orient,
        planes, row_group]); missing fields are 0.  phase_events: optional
        three recorded torch.cuda.Event objects, re-recorded before the plan,
        before the persistent kernel and after it."""
        if config is not None and not isinstance(config, _lib.ddgemm_batch_config):
            config = _lib.ddgemm_batch_config(*config)
        evs = None
        if phase_events is not None:
            if len(phase_events) != 3 or not all(e.cuda_event for e in phase_events):
                raise ValueError("phase_events: three torch.cuda.Event, each recorded once")
            evs = (ctypes.c_void_p * 3)(*[e.cuda_event for e in phase_events])
        opts = _lib.make_opts(variant=self.variant, int8_slices=self.int8_slices,
                              status_dev=status.data_ptr() if status is not None else 0,
                              phase_events=evs)
        if stream is not None and stream.device != self.workspace.device:
            raise ValueError("the stream is on another device than the batch")
        with torch.cuda.device(self.workspace.device):
            _lib.ddgemm_batched(self.count, self.host, self.dev.data_ptr(),
                                self.workspace.data_ptr(), self.workspace.numel(),
                                current_stream_ptr(stream), opts, config)
