"""Thin ctypes binding of libddgemm: the C ABI of include/ddgemm.h (and the
measurement and failure-handling aids of include/ddgemm_diag.h) under the
same names, with argument marshalling only (every step of the computation
runs in the library's CUDA kernels).  Device memory and streams come from
PyTorch; pointers and sizes go through unchanged.

There is no fallback: if the library is missing or fails to load, every
call raises."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

DDGEMM_OK = 0
DDGEMM_EINVAL = 1
DDGEMM_EWORKSPACE = 2
DDGEMM_ECUDA = 3
DDGEMM_EUNSUPPORTED = 4
DDGEMM_DEV_NONFINITE = 0x1
DDGEMM_DEV_TIMEOUT = 0x2
DDGEMM_VARIANT_FP64 = 0
DDGEMM_VARIANT_INT8 = 1
DDGEMM_VARIANT_FP64_GEMM16 = 2
DDGEMM_VARIANT_FP64_DROP456 = 3
DDGEMM_VARIANT_INT8_TC = 4
DDGEMM_VARIANT_INT8_TC8 = 5


class DdgemmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (code {code})")


class ddgemm_opts(ctypes.Structure):
    _fields_ = [("trans_a", ctypes.c_int), ("trans_b", ctypes.c_int),
                ("variant", ctypes.c_int), ("status_dev", ctypes.c_void_p),
                ("flags_dev", ctypes.c_void_p), ("phase_events", ctypes.c_void_p),
                ("int8_slices", ctypes.c_int), ("split_k", ctypes.c_int)]


class ddgemm_problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("k", ctypes.c_int),
                ("lda", ctypes.c_int), ("ldb", ctypes.c_int), ("ldc", ctypes.c_int),
                ("A_hi", ctypes.c_void_p), ("A_lo", ctypes.c_void_p),
                ("B_hi", ctypes.c_void_p), ("B_lo", ctypes.c_void_p),
                ("C_hi", ctypes.c_void_p), ("C_lo", ctypes.c_void_p)]


class ddgemm_batch_config(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("order", ctypes.c_int), ("orient", ctypes.c_int),
                ("planes", ctypes.c_int), ("row_group", ctypes.c_int)]


DDGEMM_TILE_64x64, DDGEMM_TILE_32x64, DDGEMM_TILE_64x32, DDGEMM_TILE_32x32 = 0, 1, 2, 3
DDGEMM_ORDER_GIVEN, DDGEMM_ORDER_LONGEST_K_FIRST = 0, 1
DDGEMM_ORIENT_FEWER_TILES, DDGEMM_ORIENT_GIVEN = 0, 1
DDGEMM_PLANES_INTERLEAVED, DDGEMM_PLANES_ASCENDING = 0, 1

_LIB = None

_I, _Z, _P = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
_SIGS = {
    "ddgemm_workspace_size": (_Z, [_I, _I, _I, _P]),
    "ddgemm_split_groups": (_I, [_I, _I, _I, _I, _Z, _P]),
    "ddgemm_assemble_int8": (_I, [_I, _I, _P, _P, _P, _P, _P]),
    "ddgemm_probe_wait_timeout": (_I, [ctypes.c_ulonglong, _P, _P]),
    "ddgemm": (_I, [_I, _I, _I, _P, _P, _I, _P, _P, _I, _P, _P, _I, _P, _Z, _P, _P]),
    "ddgemm_split_a": (_I, [_I, _I, _P, _P, _I, _I, _P, _I, _P, _P, _P]),
    "ddgemm_split_b": (_I, [_I, _I, _P, _P, _I, _I, _P, _I, _P, _P, _P]),
    "ddgemm_bins": (_I, [_I, _I, _I, _P, _P, _I, _P, _P, _I, _P, _P, _Z, _P, _P]),
    "ddgemm_status_string": (ctypes.c_char_p, [_I]),
    "ddgemm_probe_fp64": (ctypes.c_double, [_I, _P, _P]),
    "ddgemm_probe_int8": (ctypes.c_double, [_I, _P, _P]),
    "ddgemm_noalloc": (_I, [_I, _I, _I, _P, _P, _I, _P, _P, _I, _P, _P, _I, _P, _P]),
    "ddgemm_host_buffer_size": (_Z, [_I, _I, _I, _P]),
    "ddgemm_host": (_I, [_I, _I, _I, _P, _P, _I, _P, _P, _I, _P, _P, _I, _P, _Z, _P, _P]),
    "ddgemm_backward_workspace_size": (_Z, [_I, _I, _I, _P]),
    "ddgemm_split_int8_a": (_I, [_I, _I, _P, _P, _I, _I, _I, _P, _I, _P, _P, _P]),
    "ddgemm_batched_workspace_size": (_Z, [_I, _P, _P]),
    "ddgemm_batched": (_I, [_I, _P, _P, _P, _Z, _P, _P, _P]),
    "ddgemm_split_int8_b": (_I, [_I, _I, _P, _P, _I, _I, _I, _P, _I, _P, _P, _P]),
    "ddgemm_backward": (_I, [_I, _I, _I, _P, _P, _I, _P, _P, _I, _P, _P, _I, _P, _P, _I, _P, _P,
                             _I, _P, _Z, _P, _P]),
    "ddgemm_diag_withheld_copy": (_I, [_I, _I, _I, _P, _P, _I, _P, _P, _I, _P, _P, _I, _P, _Z, _P,
                                       _P, _I, ctypes.c_longlong, ctypes.c_ulonglong]),
    "ddgemm_diag_batched_withheld_copy": (_I, [_I, _P, _P, _P, _Z, _P, _P, _I, ctypes.c_longlong,
                                               ctypes.c_ulonglong]),
}
DDGEMM_NOALLOC_SCRATCH_BYTES = 64 << 20


def load(build_if_missing: bool = True):
    """Load libddgemm (building it first if allowed and needed)."""
    global _LIB
    if _LIB is None:
        path = _build.lib_path()
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"libddgemm is not built ({path}); run "
                                   "paper_2303_04353_gb300.build.build()")
            path = _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def lib_file() -> str:
    return _build.lib_path()


def status_string(code: int) -> str:
    return load().ddgemm_status_string(code).decode()


def _check(code: int, where: str) -> None:
    if code != DDGEMM_OK:
        raise DdgemmError(code, where)


def make_opts(trans_a=False, trans_b=False, variant=DDGEMM_VARIANT_FP64, status_dev=0,
              flags_dev=0, phase_events=None, int8_slices=0, split_k=0) -> ddgemm_opts:
    """phase_events: None or a ctypes array of three cudaEvent_t handles
    (the caller keeps it alive until the call returns)."""
    ev = ctypes.cast(phase_events, ctypes.c_void_p) if phase_events is not None else None
    return ddgemm_opts(int(trans_a), int(trans_b), int(variant), status_dev or None,
                       flags_dev or None, ev, int(int8_slices), int(split_k))


def ddgemm_workspace_size(m: int, n: int, k: int, opts: ddgemm_opts | None = None) -> int:
    return load().ddgemm_workspace_size(m, n, k, ctypes.byref(opts) if opts else None)


def ddgemm(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, c_hi, c_lo, ldc, workspace, ws_bytes,
           stream, opts: ddgemm_opts | None = None) -> None:
    """C := A B (raw pointers; see include/ddgemm.h).  Raises on error."""
    _check(load().ddgemm(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, c_hi, c_lo, ldc, workspace,
                         ws_bytes, stream, ctypes.byref(opts) if opts else None), "ddgemm")


def ddgemm_split_a(m, k, a_hi, a_lo, lda, trans_a, slices, ld_slices, exps, status_dev,
                   stream) -> None:
    _check(load().ddgemm_split_a(m, k, a_hi, a_lo, lda, int(trans_a), slices, ld_slices, exps,
                                 status_dev or None, stream), "ddgemm_split_a")


def ddgemm_split_b(k, n, b_hi, b_lo, ldb, trans_b, slices, ld_slices, exps, status_dev,
                   stream) -> None:
    _check(load().ddgemm_split_b(k, n, b_hi, b_lo, ldb, int(trans_b), slices, ld_slices, exps,
                                 status_dev or None, stream), "ddgemm_split_b")


def ddgemm_bins(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, bins, workspace, ws_bytes, stream,
                opts: ddgemm_opts | None = None) -> None:
    _check(load().ddgemm_bins(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, bins, workspace,
                              ws_bytes, stream, ctypes.byref(opts) if opts else None),
           "ddgemm_bins")


def ddgemm_probe_fp64(iters: int, sink: int, stream: int) -> float:
    """Enqueue the FP64 tensor-path throughput probe; returns its flop count."""
    flops = load().ddgemm_probe_fp64(iters, sink, stream)
    if flops < 0:
        raise DdgemmError(DDGEMM_ECUDA, "ddgemm_probe_fp64")
    return flops


def ddgemm_noalloc(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, c_hi, c_lo, ldc, stream,
                   opts: ddgemm_opts | None = None) -> None:
    """ddgemm with the library's static scratch array instead of a workspace
    (for callers that cannot allocate; see include/ddgemm.h).  Raises on error."""
    _check(load().ddgemm_noalloc(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, c_hi, c_lo, ldc,
                                 stream, ctypes.byref(opts) if opts else None), "ddgemm_noalloc")


def ddgemm_host_buffer_size(m: int, n: int, k: int, opts: ddgemm_opts | None = None) -> int:
    return load().ddgemm_host_buffer_size(m, n, k, ctypes.byref(opts) if opts else None)


def ddgemm_host(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, c_hi, c_lo, ldc, buffer, buf_bytes,
                stream, opts: ddgemm_opts | None = None) -> None:
    """ddgemm on host operands (raw host pointers, a device buffer; see
    include/ddgemm.h).  Raises on error."""
    _check(load().ddgemm_host(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, c_hi, c_lo, ldc, buffer,
                              buf_bytes, stream, ctypes.byref(opts) if opts else None),
           "ddgemm_host")


def ddgemm_backward_workspace_size(m: int, n: int, k: int, opts: ddgemm_opts | None = None) -> int:
    return load().ddgemm_backward_workspace_size(m, n, k, ctypes.byref(opts) if opts else None)


def ddgemm_backward(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, dc_hi, dc_lo, lddc, da_hi, da_lo,
                    ldda, db_hi, db_lo, lddb, workspace, ws_bytes, stream,
                    opts: ddgemm_opts | None = None) -> None:
    """dA = dC op(B)^T, dB = op(A)^T dC through the cascade.  Raises on error."""
    _check(load().ddgemm_backward(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, dc_hi, dc_lo, lddc,
                                  da_hi, da_lo, ldda, db_hi, db_lo, lddb, workspace, ws_bytes,
                                  stream, ctypes.byref(opts) if opts else None),
           "ddgemm_backward")


def ddgemm_split_int8_a(m, k, a_hi, a_lo, lda, trans_a, slices, digits, ld_digits, exps,
                        status_dev, stream) -> None:
    _check(load().ddgemm_split_int8_a(m, k, a_hi, a_lo, lda, int(trans_a), slices, digits,
                                      ld_digits, exps, status_dev or None, stream),
           "ddgemm_split_int8_a")


def ddgemm_split_int8_b(k, n, b_hi, b_lo, ldb, trans_b, slices, digits, ld_digits, exps,
                        status_dev, stream) -> None:
    _check(load().ddgemm_split_int8_b(k, n, b_hi, b_lo, ldb, int(trans_b), slices, digits,
                                      ld_digits, exps, status_dev or None, stream),
           "ddgemm_split_int8_b")


def ddgemm_assemble_int8(count, slices, diag, scale, hi, lo, stream) -> None:
    """The exact assembly step of the tensor-core INT8 form (raw pointers)."""
    _check(load().ddgemm_assemble_int8(count, slices, diag, scale, hi, lo, stream),
           "ddgemm_assemble_int8")


def ddgemm_probe_int8(iters: int, sink: int, stream: int) -> float:
    """Enqueue the integer tensor-path throughput probe; returns its op count."""
    ops = load().ddgemm_probe_int8(iters, sink, stream)
    if ops < 0:
        raise DdgemmError(DDGEMM_ECUDA, "ddgemm_probe_int8")
    return ops


def ddgemm_batched_workspace_size(count: int, probs_host, opts: ddgemm_opts | None = None) -> int:
    return load().ddgemm_batched_workspace_size(count, probs_host,
                                                ctypes.byref(opts) if opts else None)


def ddgemm_batched(count, probs_host, probs_dev, workspace, ws_bytes, stream,
                   opts: ddgemm_opts | None = None,
                   config: ddgemm_batch_config | None = None) -> None:
    """Many FP64x2 GEMMs in one pass (see include/ddgemm.h).  Raises on error."""
    _check(load().ddgemm_batched(count, probs_host, probs_dev, workspace, ws_bytes, stream,
                                 ctypes.byref(opts) if opts else None,
                                 ctypes.byref(config) if config else None), "ddgemm_batched")


def ddgemm_diag_withheld_copy(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, c_hi, c_lo, ldc,
                              workspace, ws_bytes, stream, opts: ddgemm_opts, cta: int, step: int,
                              limit_ns: int) -> None:
    """ddgemm with one copy of CTA `cta` withheld, so that its bounded waits
    run out after limit_ns (see include/ddgemm_diag.h).  Raises on error."""
    _check(load().ddgemm_diag_withheld_copy(m, n, k, a_hi, a_lo, lda, b_hi, b_lo, ldb, c_hi, c_lo,
                                            ldc, workspace, ws_bytes, stream, ctypes.byref(opts),
                                            cta, step, limit_ns), "ddgemm_diag_withheld_copy")


def ddgemm_diag_batched_withheld_copy(count, probs_host, probs_dev, workspace, ws_bytes, stream,
                                      opts: ddgemm_opts, cta: int, step: int,
                                      limit_ns: int) -> None:
    """ddgemm_batched (tcgen05 forms) with one copy withheld; see
    include/ddgemm_diag.h.  Raises on error."""
    _check(load().ddgemm_diag_batched_withheld_copy(count, probs_host, probs_dev, workspace,
                                                    ws_bytes, stream, ctypes.byref(opts), cta,
                                                    step, limit_ns),
           "ddgemm_diag_batched_withheld_copy")
