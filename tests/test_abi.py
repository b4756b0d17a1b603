"""The C ABI without a GPU: the library builds and loads, exports every
function include/*.h declares, and its host-side checks answer before any
CUDA call."""
import ctypes
import glob
import os
import re

import pytest

from paper_2303_04353_gb300 import _lib

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")
HEADER = os.path.join(INCLUDE, "ddgemm.h")
DIAG_HEADER = os.path.join(INCLUDE, "ddgemm_diag.h")
FAKE = 0x10000  # never dereferenced: every call below returns before a CUDA call


def declared_functions(path=None):
    paths = [path] if path else sorted(glob.glob(os.path.join(INCLUDE, "*.h")))
    names = set()
    for p in paths:
        text = re.sub(r"/\*.*?\*/", "", open(p).read(), flags=re.S)
        names |= set(re.findall(r"\b(ddgemm\w*)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions(HEADER)
    for want in ("ddgemm", "ddgemm_workspace_size", "ddgemm_split_a", "ddgemm_split_b",
                 "ddgemm_bins", "ddgemm_status_string", "ddgemm_batched", "ddgemm_backward"):
        assert want in names
    # the measurement and failure-handling aids live in their own header
    diag = declared_functions(DIAG_HEADER)
    assert set(diag) == {"ddgemm_probe_fp64", "ddgemm_probe_int8", "ddgemm_probe_wait_timeout",
                         "ddgemm_diag_withheld_copy", "ddgemm_diag_batched_withheld_copy"}
    assert not set(diag) & set(names)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    raw = ctypes.CDLL(_lib.lib_file())
    for name in declared_functions():
        assert hasattr(raw, name), name
    assert set(_lib._SIGS) >= set(declared_functions())
    assert lib is _lib.load()


def test_status_strings():
    assert _lib.status_string(0) == "ok"
    assert "workspace" in _lib.status_string(2)
    assert _lib.status_string(99) == "unknown status"


def test_workspace_size():
    ws = _lib.ddgemm_workspace_size
    assert ws(0, 5, 5) == 0 and ws(5, 0, 5) == 0 and ws(5, 5, 0) == 0
    assert ws(-1, 5, 5) == 0
    m, n, k = 4096, 4096, 4096
    # 4 m k + 7 k n doubles of cascaded pieces plus the block exponents
    assert ws(m, n, k) >= (4 * m * k + 7 * k * n) * 8
    assert ws(m, n, k) < (4 * m * k + 7 * k * n) * 8 * 1.01
    assert ws(3, 5, 7) % 256 == 0


def split_groups(m, n, k, sms=152, ws_bytes=None, **kw):
    opts = _lib.make_opts(**kw)
    if ws_bytes is None:
        ws_bytes = _lib.ddgemm_workspace_size(m, n, k, opts)
    return _lib.load().ddgemm_split_groups(m, n, k, sms, ws_bytes, ctypes.byref(opts))


def test_split_k_workspace_and_choice():
    """Split-k: room for partial C only for grids below 4096 tiles of 64 x
    64 (at most min(16, k-blocks, ceil(8192 / tiles)) groups), as many
    groups as give the shortest span in k-block times, none without room."""
    ws = _lib.ddgemm_workspace_size
    base = ws(512, 512, 4096, _lib.make_opts(split_k=1))
    # 64 tiles, 16 k-blocks: fifteen partial C of 512 x 512 FP64x2 entries
    assert ws(512, 512, 4096) == base + 15 * 2 * 512 * 512 * 8
    assert ws(4096, 4096, 4096) == ws(4096, 4096, 4096, _lib.make_opts(split_k=1))
    assert ws(512, 512, 4096, _lib.make_opts(split_k=2)) == base + 2 * 512 * 512 * 8
    # 2048 tiles: at most ceil(8192 / 2048) = 4 groups, 3 partials
    assert ws(8192, 1024, 4096) - ws(8192, 1024, 4096, _lib.make_opts(split_k=1)) == \
        3 * 2 * 8192 * 1024 * 8
    # 4096 tiles fill 152 SMs in 27 waves: no split
    assert split_groups(4096, 4096, 4096) == 1
    # 64 tiles on 152 SMs: 1024 CTAs of one k-block in 7 waves (span 7)
    # beat 128 CTAs of 8 k-blocks in one wave (span 8)
    assert split_groups(512, 512, 4096) == 16
    # 2048 tiles, 16 k-blocks: 27 waves of 8 blocks beat 14 waves of 16
    assert split_groups(8192, 1024, 4096) == 2
    # 256 tiles, 4 k-blocks: 7 waves of one block beat 2 waves of four
    assert split_groups(1000, 1000, 1000) == 4
    # 16 tiles, 64 k-blocks: 8 groups of 8 blocks fill one wave of 128 CTAs
    assert split_groups(256, 256, 16384) == 8
    # 256 tiles, 32 k-blocks: 27 waves of 2 blocks (span 54) beat 7 waves
    # of 8 (span 56)
    assert split_groups(1024, 1024, 8192) == 16
    # 1024 tiles, 8 k-blocks: 27 waves of 2 blocks tie 54 waves of one;
    # the tie goes to fewer groups
    assert split_groups(2048, 2048, 2048) == 4
    assert split_groups(512, 512, 256) == 1                    # one k-block
    assert split_groups(64, 64, 8192) == 16                    # at most 16
    assert split_groups(512, 512, 4096, split_k=1) == 1
    assert split_groups(512, 512, 4096, split_k=3) == 3
    assert split_groups(100, 100, 600, split_k=4) == 3         # 3 k-blocks
    assert split_groups(100, 100, 20000, split_k=40) == 16     # at most 16
    assert split_groups(512, 512, 4096, ws_bytes=base) == 1    # no room
    assert split_groups(512, 512, 4096, ws_bytes=base + 2 * 512 * 512 * 8, split_k=4) == 2
    assert split_groups(512, 512, 4096, variant=_lib.DDGEMM_VARIANT_INT8) == 1
    assert split_groups(512, 512, 4096, sms=0) == 0
    assert split_groups(512, 512, 4096, split_k=-1) == 0


def call(m, n, k, lda, ldb, ldc, ws=FAKE, ws_bytes=1 << 40, opts=None):
    lib = _lib.load()
    return lib.ddgemm(m, n, k, FAKE, FAKE, lda, FAKE, FAKE, ldb, FAKE, FAKE, ldc, ws, ws_bytes,
                      None, ctypes.byref(opts) if opts else None)


def test_host_checks():
    assert call(-1, 4, 4, 4, 4, 4) == _lib.DDGEMM_EINVAL
    assert call(4, 4, 4, 3, 4, 4) == _lib.DDGEMM_EINVAL          # lda < k
    assert call(4, 4, 4, 4, 3, 4) == _lib.DDGEMM_EINVAL          # ldb < n
    assert call(4, 4, 4, 4, 4, 3) == _lib.DDGEMM_EINVAL          # ldc < n
    assert call(4, 4, 4, 4, 4, 4, ws=0) == _lib.DDGEMM_EWORKSPACE
    assert call(4, 4, 4, 4, 4, 4, ws=FAKE + 8) == _lib.DDGEMM_EWORKSPACE  # misaligned
    assert call(4, 4, 4, 4, 4, 4, ws_bytes=16) == _lib.DDGEMM_EWORKSPACE
    assert call(0, 4, 4, 4, 4, 4) == _lib.DDGEMM_OK              # empty: nothing to do
    assert call(4, 4, 4, 4, 4, 4, opts=_lib.make_opts(variant=7)) == _lib.DDGEMM_EUNSUPPORTED
    bad = _lib.ddgemm_opts(2, 0, 0, None, None)
    assert call(4, 4, 4, 4, 4, 4, opts=bad) == _lib.DDGEMM_EINVAL
    # trans_a: A stored k x m needs lda >= m
    assert call(8, 4, 2, 2, 4, 4, opts=_lib.make_opts(trans_a=True)) == _lib.DDGEMM_EINVAL


def test_bins_and_split_host_checks():
    lib = _lib.load()
    assert lib.ddgemm_bins(4, 4, 300, FAKE, FAKE, 300, FAKE, FAKE, 4, FAKE, FAKE, 1 << 40,
                           None, None) == _lib.DDGEMM_EINVAL  # one k-block at most
    assert lib.ddgemm_split_a(4, 8, FAKE, FAKE, 7, 0, FAKE, 8, FAKE, None, None) == _lib.DDGEMM_EINVAL
    assert lib.ddgemm_split_b(8, 4, FAKE, FAKE, 4, 0, FAKE, 3, FAKE, None, None) == _lib.DDGEMM_EINVAL
    assert lib.ddgemm_split_a(0, 8, None, None, 8, 0, None, 8, None, None, None) == _lib.DDGEMM_OK


def test_ops_refuse_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_2303_04353_gb300 import ops
    a = torch.zeros(2, 2, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        ops.ddgemm(a, a, a, a)


def test_batched_host_checks():
    lib = _lib.load()
    arr = (_lib.ddgemm_problem * 2)()
    arr[0] = _lib.ddgemm_problem(4, 5, 6, 6, 5, 5, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    arr[1] = _lib.ddgemm_problem(0, 5, 6, 6, 5, 5, 0, 0, 0, 0, 0, 0)
    need = _lib.ddgemm_batched_workspace_size(2, arr)
    assert need >= (4 * 4 * 8 + 7 * 6 * 8) * 8
    # workspace too small / misaligned
    assert lib.ddgemm_batched(2, arr, FAKE, FAKE, 16, None, None, None) == _lib.DDGEMM_EWORKSPACE
    assert lib.ddgemm_batched(2, arr, FAKE, FAKE + 8, need, None, None, None) == _lib.DDGEMM_EWORKSPACE
    # a bad problem (ldc < n), trans flags, bad config, empty batch
    bad = (_lib.ddgemm_problem * 1)()
    bad[0] = _lib.ddgemm_problem(4, 5, 6, 6, 5, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    assert lib.ddgemm_batched(1, bad, FAKE, FAKE, 1 << 30, None, None, None) == _lib.DDGEMM_EINVAL
    o = _lib.make_opts(trans_a=True)
    assert lib.ddgemm_batched(2, arr, FAKE, FAKE, need, None, ctypes.byref(o), None) == \
        _lib.DDGEMM_EUNSUPPORTED
    cfg = _lib.ddgemm_batch_config(9, 0)
    assert lib.ddgemm_batched(2, arr, FAKE, FAKE, need, None, None, ctypes.byref(cfg)) == \
        _lib.DDGEMM_EINVAL
    assert lib.ddgemm_batched(0, None, None, None, 0, None, None, None) == _lib.DDGEMM_OK


def test_batched_tc_host_checks():
    """The tcgen05 batched form: its workspace (digit tiles of whole
    128 x 16 tiles), and the host checks before any CUDA call."""
    lib = _lib.load()
    arr = (_lib.ddgemm_problem * 2)()
    arr[0] = _lib.ddgemm_problem(4, 5, 6, 6, 5, 5, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    arr[1] = _lib.ddgemm_problem(0, 5, 6, 6, 5, 5, 0, 0, 0, 0, 0, 0)
    o = _lib.make_opts(variant=_lib.DDGEMM_VARIANT_INT8_TC)
    need = _lib.ddgemm_batched_workspace_size(2, arr, o)
    # 16 planes (the default) of a 128 x 16 A tile and a 16 x 16 B tile, bf16
    assert need >= 16 * (128 + 16) * 16 * 2
    assert need != _lib.ddgemm_batched_workspace_size(2, arr)
    bad_s = _lib.make_opts(variant=_lib.DDGEMM_VARIANT_INT8_TC, int8_slices=18)
    assert _lib.ddgemm_batched_workspace_size(2, arr, bad_s) == 0
    assert lib.ddgemm_batched(2, arr, FAKE, FAKE, need, None, ctypes.byref(bad_s), None) == \
        _lib.DDGEMM_EINVAL
    assert lib.ddgemm_batched(2, arr, FAKE, FAKE, 16, None, ctypes.byref(o), None) == \
        _lib.DDGEMM_EWORKSPACE
    bad = (_lib.ddgemm_problem * 1)()
    bad[0] = _lib.ddgemm_problem(4, 5, 6, 6, 5, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    assert lib.ddgemm_batched(1, bad, FAKE, FAKE, 1 << 30, None, ctypes.byref(o), None) == \
        _lib.DDGEMM_EINVAL
    int8 = _lib.make_opts(variant=_lib.DDGEMM_VARIANT_INT8)
    assert lib.ddgemm_batched(2, arr, FAKE, FAKE, need, None, ctypes.byref(int8), None) == \
        _lib.DDGEMM_EUNSUPPORTED


def host_chunk_rows(m, n, variant):
    """The row-chunk rule of ddgemm_host, restated: at least 1024 tiles of
    the form's kernel (64 x 64 FP64, 32 x 32 mma.sync INT8, 128 x 16 tcgen05)
    per chunk, at most four chunks, a multiple of 128 rows."""
    tm, tn = {_lib.DDGEMM_VARIANT_FP64: (64, 64), _lib.DDGEMM_VARIANT_INT8: (32, 32),
              _lib.DDGEMM_VARIANT_INT8_TC: (128, 16)}[variant]
    rows_min = -(-1024 // -(-n // tn)) * tm
    mc = -(-max(rows_min, -(-m // 4)) // 128) * 128
    return min(mc, m)


@pytest.mark.parametrize("m,n,k,variant,chunks", [
    (4096, 4096, 4096, _lib.DDGEMM_VARIANT_FP64, 4),
    (2100, 8192, 300, _lib.DDGEMM_VARIANT_FP64, 4),
    (4096, 4096, 4096, _lib.DDGEMM_VARIANT_INT8_TC, 4),
    (4200, 2048, 300, _lib.DDGEMM_VARIANT_INT8_TC, 4),
    (2500, 2048, 300, _lib.DDGEMM_VARIANT_INT8, 4),
    (2100, 8192, 1100, _lib.DDGEMM_VARIANT_FP64, 4),
    (1500, 4096, 300, _lib.DDGEMM_VARIANT_FP64, 2),
    (100, 70, 300, _lib.DDGEMM_VARIANT_FP64, 1),
    (100, 50, 0, _lib.DDGEMM_VARIANT_FP64, 1)])
def test_host_buffer_size(m, n, k, variant, chunks):
    """ddgemm_host's device buffer: dense hi/lo copies of A, B and C (each
    plane 256-byte aligned) and ddgemm's workspace for one row chunk; the
    shapes the GPU tests use run in the chunk counts given."""
    def r(x):
        return -(-x // 256) * 256
    o = _lib.make_opts(variant=variant)
    mc = host_chunk_rows(m, n, variant) if k else m
    assert -(-m // mc) == chunks
    ws = _lib.ddgemm_workspace_size(mc, n, k, o) if k else 0
    want = 2 * r(m * k * 8) + 2 * r(k * n * 8) + 2 * r(m * n * 8) + ws
    assert _lib.ddgemm_host_buffer_size(m, n, k, o) == want


def test_host_entry_checks():
    lib = _lib.load()

    def host(m, n, k, lda, ldb, ldc, buf=FAKE, nbytes=1 << 40, opts=None):
        return lib.ddgemm_host(m, n, k, FAKE, FAKE, lda, FAKE, FAKE, ldb, FAKE, FAKE, ldc, buf,
                               nbytes, None, ctypes.byref(opts) if opts else None)
    assert _lib.ddgemm_host_buffer_size(0, 5, 5) == 0
    assert _lib.ddgemm_host_buffer_size(5, 5, 5, _lib.make_opts(variant=9)) == 0
    assert _lib.ddgemm_host_buffer_size(-1, 5, 5) == 0
    assert host(-1, 4, 4, 4, 4, 4) == _lib.DDGEMM_EINVAL
    assert host(4, 4, 4, 3, 4, 4) == _lib.DDGEMM_EINVAL            # lda < k
    assert host(4, 4, 4, 4, 3, 4) == _lib.DDGEMM_EINVAL            # ldb < n
    assert host(4, 4, 4, 4, 4, 3) == _lib.DDGEMM_EINVAL            # ldc < n
    assert host(4, 4, 4, 4, 4, 4, buf=0) == _lib.DDGEMM_EWORKSPACE
    assert host(4, 4, 4, 4, 4, 4, buf=FAKE + 8) == _lib.DDGEMM_EWORKSPACE
    assert host(4, 4, 4, 4, 4, 4, nbytes=16) == _lib.DDGEMM_EWORKSPACE
    assert host(0, 4, 4, 4, 4, 4) == _lib.DDGEMM_OK                # empty: nothing to do
    assert host(4, 4, 4, 4, 4, 4, opts=_lib.make_opts(variant=7)) == _lib.DDGEMM_EUNSUPPORTED
    flagged = _lib.make_opts(variant=_lib.DDGEMM_VARIANT_INT8, flags_dev=FAKE)
    assert host(4, 4, 4, 4, 4, 4, opts=flagged) == _lib.DDGEMM_EUNSUPPORTED
    assert host(8, 4, 2, 2, 4, 4, opts=_lib.make_opts(trans_a=True)) == _lib.DDGEMM_EINVAL


def test_host_ops_refuse_cuda_tensors():
    torch = pytest.importorskip("torch")
    from paper_2303_04353_gb300 import ops
    a = torch.zeros(2, 2, dtype=torch.float32)
    with pytest.raises(TypeError, match="float64"):
        ops.ddgemm_host(a, a, a, a)


def test_tc8_workspace_and_pieces():
    """The eight-bit tcgen05 form: the tiled bf16 digit layout of the
    seven-bit one with k-blocks of 8192, and s in 12..15."""
    tc8 = _lib.DDGEMM_VARIANT_INT8_TC8
    s15 = _lib.ddgemm_workspace_size(300, 40, 20000, _lib.make_opts(variant=tc8))
    assert s15 == _lib.ddgemm_workspace_size(300, 40, 20000,
                                             _lib.make_opts(variant=tc8, int8_slices=15))
    # 15 planes of bf16 digits: 384 rows of A and 48 columns of B, k padded to 16
    assert s15 >= 15 * (384 + 48) * 20000 * 2
    assert _lib.ddgemm_workspace_size(300, 40, 20000, _lib.make_opts(variant=tc8,
                                                                     int8_slices=16)) == 0
    # three exponent blocks of 8192 against two of 16384 for the seven-bit form
    s7 = _lib.ddgemm_workspace_size(300, 40, 20000, _lib.make_opts(
        variant=_lib.DDGEMM_VARIANT_INT8_TC, int8_slices=15))
    assert s15 > s7
    lib = _lib.load()
    flagged = _lib.make_opts(variant=tc8, flags_dev=FAKE)
    assert call(4, 4, 4, 4, 4, 4, opts=flagged) == _lib.DDGEMM_EUNSUPPORTED
    # batched: the seven-bit form's layout with the eight-bit k-blocks, s <= 15
    arr = (_lib.ddgemm_problem * 1)()
    arr[0] = _lib.ddgemm_problem(4, 5, 20000, 20000, 5, 5, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    o = _lib.make_opts(variant=tc8)
    need8 = _lib.ddgemm_batched_workspace_size(1, arr, o)
    need7 = _lib.ddgemm_batched_workspace_size(1, arr, _lib.make_opts(
        variant=_lib.DDGEMM_VARIANT_INT8_TC, int8_slices=15))
    assert need8 >= need7 > 0
    bad = _lib.make_opts(variant=tc8, int8_slices=16)
    assert _lib.ddgemm_batched_workspace_size(1, arr, bad) == 0
    assert lib.ddgemm_batched(1, arr, FAKE, FAKE, 1 << 30, None, ctypes.byref(bad), None) == \
        _lib.DDGEMM_EINVAL
    assert lib.ddgemm_batched(1, arr, FAKE, FAKE, 16, None, ctypes.byref(o), None) == \
        _lib.DDGEMM_EWORKSPACE


def test_diag_withheld_copy_host_checks():
    """The failure-handling entry points check their arguments on the host
    (nothing is enqueued on an error): a status word is required, the wait
    limit lies in 10^3 .. 10^10 ns, the CTA and step are >= 0, and an empty
    problem has no kernel to withhold a copy from."""
    lib = _lib.load()
    with_status = _lib.make_opts(status_dev=FAKE)

    def call(m=4, n=4, k=4, opts=with_status, cta=0, step=0, limit=20_000_000):
        return lib.ddgemm_diag_withheld_copy(m, n, k, FAKE, FAKE, k, FAKE, FAKE, n, FAKE, FAKE, n,
                                             FAKE, 1 << 30, None,
                                             ctypes.byref(opts) if opts else None, cta, step,
                                             limit)
    assert call(opts=None) == _lib.DDGEMM_EINVAL
    assert call(opts=_lib.make_opts()) == _lib.DDGEMM_EINVAL      # no status word
    assert call(limit=10) == _lib.DDGEMM_EINVAL
    assert call(limit=10 ** 11) == _lib.DDGEMM_EINVAL
    assert call(cta=-1) == _lib.DDGEMM_EINVAL
    assert call(step=-1) == _lib.DDGEMM_EINVAL
    assert call(m=0) == _lib.DDGEMM_EINVAL
    assert call(opts=_lib.make_opts(status_dev=FAKE, flags_dev=FAKE)) == _lib.DDGEMM_EUNSUPPORTED
    arr = (_lib.ddgemm_problem * 1)()
    arr[0] = _lib.ddgemm_problem(4, 5, 6, 6, 5, 5, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    fp64 = _lib.make_opts(status_dev=FAKE)
    tc = _lib.make_opts(variant=_lib.DDGEMM_VARIANT_INT8_TC, status_dev=FAKE)
    batched = lib.ddgemm_diag_batched_withheld_copy
    # the FP64 batched kernel has no barrier wait to run out
    assert batched(1, arr, FAKE, FAKE, 1 << 30, None, ctypes.byref(fp64), 0, 0,
                   20_000_000) == _lib.DDGEMM_EUNSUPPORTED
    assert batched(1, arr, FAKE, FAKE, 1 << 30, None, None, 0, 0, 20_000_000) == \
        _lib.DDGEMM_EINVAL
    assert batched(1, arr, FAKE, FAKE, 1 << 30, None, ctypes.byref(tc), 0, 0, 10) == \
        _lib.DDGEMM_EINVAL
    assert batched(1, arr, FAKE, FAKE, 16, None, ctypes.byref(tc), 0, 0, 20_000_000) == \
        _lib.DDGEMM_EWORKSPACE


def test_batch_config_range_checks():
    """Out-of-range schedule fields are refused before any CUDA call, for
    both forms."""
    lib = _lib.load()
    arr = (_lib.ddgemm_problem * 1)()
    arr[0] = _lib.ddgemm_problem(4, 5, 6, 6, 5, 5, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE)
    tc = _lib.make_opts(variant=_lib.DDGEMM_VARIANT_INT8_TC)
    for bad in [(0, 2, 0, 0, 0), (0, 0, 2, 0, 0), (0, 0, 0, 2, 0), (0, 0, 0, 0, 9),
                (0, 0, 0, 0, -1), (4, 0, 0, 0, 0)]:
        cfg = _lib.ddgemm_batch_config(*bad)
        for opts in (None, ctypes.byref(tc)):
            assert lib.ddgemm_batched(1, arr, FAKE, FAKE, 1 << 30, None, opts,
                                      ctypes.byref(cfg)) == _lib.DDGEMM_EINVAL, bad
    # the workspace of the tcgen05 forms covers either tile grid
    need = _lib.ddgemm_batched_workspace_size(1, arr, tc)
    ok = _lib.ddgemm_batch_config(0, 1, 1, 1, 8)
    assert lib.ddgemm_batched(1, arr, FAKE, FAKE, need - 256, None, ctypes.byref(tc),
                              ctypes.byref(ok)) == _lib.DDGEMM_EWORKSPACE

