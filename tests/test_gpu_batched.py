"""The batched form: many problems in one pass (plan, two batched splits,
one persistent cascade kernel), captured into a CUDA graph.

The per-tile arithmetic is the single-problem kernel's and the k order is
the same, so each problem's C must be bit-identical to ddgemm() on that
problem alone, for every tile shape and schedule; ddgemm itself is checked
against the oracles in test_gpu_parity.py, and a few problems here are
checked against the double-double oracle directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dd  # noqa: E402
from workloads import batched_shapes, gemm_inputs  # noqa: E402

pytestmark = pytest.mark.gpu

MIXED = [(64, 64, 256), (100, 70, 300), (1, 1, 1), (3, 200, 17), (0, 5, 7), (6, 0, 9),
         (9, 11, 0), (130, 65, 513), (33, 97, 64), (256, 32, 1024), (17, 300, 250), (64, 1, 65)]


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04353_gb300 import _lib, autotune, ops
    return _lib, ops, autotune


def make_batch(ops, shapes, seed=0, kind="uniform", variant=0):
    probs, host = [], []
    for i, (m, n, k) in enumerate(shapes):
        a = gemm_inputs(m, n, k, kind=kind, seed=seed + i)
        t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]
        c = [torch.full((m, n), np.nan, dtype=torch.float64, device="cuda") for _ in range(2)]
        probs.append((*t, *c))
        host.append(a)
    return ops.Batch(probs, variant=variant), probs, host


def reference(ops, probs):
    out = []
    for a_hi, a_lo, b_hi, b_lo, _, _ in probs:
        # one launch per problem in the paper's k order (no split-k), which
        # the batched kernel follows bit for bit
        c_hi, c_lo = ops.ddgemm(a_hi, a_lo, b_hi, b_lo, split_k=1)
        out.append((c_hi, c_lo))
    torch.cuda.synchronize()
    return [(h.cpu().numpy(), l.cpu().numpy()) for h, l in out]


def results(probs):
    torch.cuda.synchronize()
    return [(p[4].cpu().numpy(), p[5].cpu().numpy()) for p in probs]


@pytest.mark.parametrize("tile", [0, 1, 2, 3])
@pytest.mark.parametrize("order", [0, 1])
def test_batched_bit_identical_to_ddgemm(mods, tile, order):
    _lib, ops, _ = mods
    batch, probs, _ = make_batch(ops, MIXED, seed=10, kind="wide")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    batch.run(config=(tile, order), status=status)
    got = results(probs)
    want = reference(ops, probs)
    assert int(status.item()) == 0
    for (gh, gl), (wh, wl), (m, n, k) in zip(got, want, MIXED):
        if m == 0 or n == 0:
            continue
        if k == 0:
            assert not gh.any() and not gl.any()
        assert np.array_equal(gh, wh) and np.array_equal(gl, wl), (m, n, k)


def test_batched_against_oracle(mods):
    _lib, ops, _ = mods
    shapes = [(100, 70, 300), (37, 53, 600), (5, 9, 1000)]
    batch, probs, host = make_batch(ops, shapes, seed=20)
    batch.run()
    for (ch, cl), a in zip(results(probs), host):
        oh, ol = dd.ddgemm(*a)
        absab = np.abs(a[0]) @ np.abs(a[2])
        assert np.all(np.abs((ch - oh) + (cl - ol)) <= 1e-28 * absab)


def test_batched_graph_capture_and_replay(mods):
    _lib, ops, _ = mods
    batch, probs, _ = make_batch(ops, MIXED[:8], seed=30)
    batch.run()                      # eager once (sets kernel attributes)
    eager = results(probs)
    for p in probs:
        p[4].fill_(np.nan)
        p[5].fill_(np.nan)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=stream):
        batch.run(stream=torch.cuda.current_stream())
    g.replay()
    replayed = results(probs)
    for (eh, el), (rh, rl), (m, n, k) in zip(eager, replayed, MIXED[:8]):
        if m and n:
            assert np.array_equal(eh, rh) and np.array_equal(el, rl)
    # new values in the same buffers: the graph recomputes them
    for p in probs:
        for x in p[:4]:
            x.mul_(0.5)
    g.replay()
    halved = results(probs)
    want = reference(ops, probs)
    for (hh, hl), (wh, wl), (m, n, k) in zip(halved, want, MIXED[:8]):
        if m and n:
            assert np.array_equal(hh, wh) and np.array_equal(hl, wl)


def test_batched_512_uneven_problems(mods):
    """512 problems, m, n, k each log-uniform in [64, 1024], uniform entries:
    every problem bit-identical to ddgemm, three against the oracle."""
    _lib, ops, _ = mods
    shapes = [tuple(int(v) for v in s) for s in batched_shapes(512, seed=0)]
    batch, probs, host = make_batch(ops, shapes, seed=1000)
    batch.run()
    got = results(probs)
    want = reference(ops, probs)
    for (gh, gl), (wh, wl) in zip(got, want):
        assert np.array_equal(gh, wh) and np.array_equal(gl, wl)
    for i in (0, 255, 511):
        a = host[i]
        rows = np.arange(0, shapes[i][0], max(1, shapes[i][0] // 8))
        cols = np.arange(0, shapes[i][1], max(1, shapes[i][1] // 8))
        rr, cc = np.meshgrid(rows, cols, indexing="ij")
        oh, ol = dd.ddgemm_entries(*a, rr.ravel(), cc.ravel())
        absab = np.array([np.abs(a[0][r]) @ np.abs(a[2][:, c]) for r, c in zip(rr.ravel(), cc.ravel())])
        gh, gl = got[i]
        assert np.all(np.abs((gh[rr.ravel(), cc.ravel()] - oh) + (gl[rr.ravel(), cc.ravel()] - ol))
                      <= 1e-28 * absab)


def test_autotuner_picks_and_caches(mods, tmp_path, monkeypatch):
    _lib, ops, autotune = mods
    monkeypatch.setenv("DDGEMM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    batch, probs, _ = make_batch(ops, MIXED, seed=40)
    cfg, timings = autotune.tune(batch, reps=1)
    assert cfg in autotune.CANDIDATES and len(timings) == len(autotune.CANDIDATES)
    assert all(v > 0 for v in timings.values())
    cfg2, _ = autotune.tune(batch, reps=1)           # served from the cache
    assert cfg2 == cfg and (tmp_path / "tune.json").exists()
    batch.run(config=cfg)
    want = reference(ops, probs)
    for (gh, gl), (wh, wl), (m, n, k) in zip(results(probs), want, MIXED):
        if m and n:
            assert np.array_equal(gh, wh) and np.array_equal(gl, wl)


# ---- the batched tcgen05 INT8 form -------------------------------------

TC = 4


def reference_tc(ops, probs, variant=TC):
    out = []
    for a_hi, a_lo, b_hi, b_lo, _, _ in probs:
        out.append(ops.ddgemm(a_hi, a_lo, b_hi, b_lo, variant=variant))
    torch.cuda.synchronize()
    return [(h.cpu().numpy(), l.cpu().numpy()) for h, l in out]


@pytest.mark.parametrize("kind", ["uniform", "wide"])
def test_batched_tc_bit_identical_to_ddgemm(mods, kind):
    """Every problem of a batched tcgen05 pass equals ddgemm() with the
    tcgen05 form on that problem alone, bit for bit; k = 0 gives C = 0 and
    empty problems are skipped."""
    _lib, ops, _ = mods
    batch, probs, _ = make_batch(ops, MIXED, seed=60, kind=kind, variant=TC)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    batch.run(status=status)
    got = results(probs)
    want = reference_tc(ops, probs)
    assert int(status.item()) == 0
    for (gh, gl), (wh, wl), (m, n, k) in zip(got, want, MIXED):
        if m and n:
            assert np.array_equal(gh, wh) and np.array_equal(gl, wl), (m, n, k)
        if m and n and not k:
            assert not gh.any() and not gl.any()


def test_batched_tc_512_uneven_graph_replay(mods):
    """The 512-problem workload through the tcgen05 form, captured into a
    CUDA graph and replayed: bit-identical to ddgemm per problem, and within
    1e-28 (|A||B|) of the double-double oracle on sampled entries."""
    _lib, ops, _ = mods
    shapes = [tuple(int(v) for v in s) for s in batched_shapes(512, seed=0)]
    batch, probs, host = make_batch(ops, shapes, seed=1000, variant=TC)
    batch.run()
    torch.cuda.synchronize()
    for p in probs:
        p[4].fill_(np.nan)
        p[5].fill_(np.nan)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=stream):
        batch.run(stream=torch.cuda.current_stream())
    g.replay()
    got = results(probs)
    want = reference_tc(ops, probs)
    for (gh, gl), (wh, wl) in zip(got, want):
        assert np.array_equal(gh, wh) and np.array_equal(gl, wl)
    for i in (0, 511):
        a = host[i]
        rows = np.arange(0, shapes[i][0], max(1, shapes[i][0] // 6))
        cols = np.arange(0, shapes[i][1], max(1, shapes[i][1] // 6))
        rr, cc = np.meshgrid(rows, cols, indexing="ij")
        oh, ol = dd.ddgemm_entries(*a, rr.ravel(), cc.ravel())
        absab = np.array([np.abs(a[0][r]) @ np.abs(a[2][:, c])
                          for r, c in zip(rr.ravel(), cc.ravel())])
        gh, gl = got[i]
        assert np.all(np.abs((gh[rr.ravel(), cc.ravel()] - oh) + (gl[rr.ravel(), cc.ravel()] - ol))
                      <= 1e-28 * absab)


TC8 = 5


def test_batched_tc8_bit_identical_to_ddgemm(mods):
    """The eight-bit tcgen05 form batched: every problem equals ddgemm() with
    DDGEMM_VARIANT_INT8_TC8 on that problem alone, bit for bit, including a
    problem with two k-blocks of 8192."""
    _lib, ops, _ = mods
    shapes = MIXED + [(20, 30, 8300)]
    batch, probs, _ = make_batch(ops, shapes, seed=61, kind="wide", variant=TC8)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    batch.run(status=status)
    got = results(probs)
    want = reference_tc(ops, probs, variant=TC8)
    assert int(status.item()) == 0
    for (gh, gl), (wh, wl), (m, n, k) in zip(got, want, shapes):
        if m and n:
            assert np.array_equal(gh, wh) and np.array_equal(gl, wl), (m, n, k)


@pytest.mark.parametrize("count", [1001, 2100])
def test_batched_tc_many_small_problems(mods, count):
    """Many small problems (and empty ones): the plan's ranking (its keys in
    shared memory up to 2048 problems, from global memory above) and its
    segmented prefix sums; every C equals ddgemm() with the tcgen05 form."""
    _lib, ops, _ = mods
    rng = np.random.default_rng(count)
    shapes = [(int(rng.integers(0, 40)), int(rng.integers(0, 40)), int(rng.integers(0, 300)))
              for _ in range(count)]
    batch, probs, _ = make_batch(ops, shapes, seed=7, kind="wide", variant=TC)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    batch.run(status=status)
    got = results(probs)
    want = reference_tc(ops, probs)
    assert int(status.item()) == 0
    for (gh, gl), (wh, wl), (m, n, k) in zip(got, want, shapes):
        if m and n:
            assert np.array_equal(gh, wh) and np.array_equal(gl, wl), (m, n, k)


@pytest.mark.parametrize("count,order", [(1001, 1), (2100, 1), (2100, 0)])
def test_batched_fp64_many_small_problems(mods, count, order):
    """The FP64 form's plan on many small (and empty) problems: its ranking
    (keys in shared memory up to 2048 problems, from global memory above,
    or the given order) and its segmented prefix sums; every C equals
    ddgemm() on that problem alone."""
    _lib, ops, _ = mods
    rng = np.random.default_rng(count + order)
    shapes = [(int(rng.integers(0, 40)), int(rng.integers(0, 40)), int(rng.integers(0, 600)))
              for _ in range(count)]
    batch, probs, _ = make_batch(ops, shapes, seed=11, kind="wide")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    batch.run(status=status, config=(3, order))
    got = results(probs)
    want = reference(ops, probs)
    assert int(status.item()) == 0
    for (gh, gl), (wh, wl), (m, n, k) in zip(got, want, shapes):
        if m and n:
            assert np.array_equal(gh, wh) and np.array_equal(gl, wl), (m, n, k)


@pytest.mark.parametrize("variant", [TC, 5])
def test_batched_tc_every_schedule_bit_identical(mods, variant):
    """Every schedule the autotuner may pick for the tcgen05 forms (problem
    order, tile grid over C or C^T, plane order, row group) gives each
    problem bit for bit what ddgemm() gives it alone; wide and tall shapes
    make the transposed grid win for some problems."""
    _lib, ops, autotune = mods
    shapes = MIXED + [(40, 900, 300), (700, 20, 129), (64, 64, 64), (127, 129, 200)]
    batch, probs, _ = make_batch(ops, shapes, seed=90, variant=variant)
    want = reference_tc(ops, probs, variant)
    for cfg in autotune.candidates(variant):
        for p in probs:
            p[4].fill_(np.nan)
            p[5].fill_(np.nan)
        batch.run(config=cfg)
        for (gh, gl), (wh, wl), (m, n, k) in zip(results(probs), want, shapes):
            if m and n:
                assert np.array_equal(gh, wh) and np.array_equal(gl, wl), (cfg, m, n, k)


def test_autotuner_tc_picks_a_schedule(mods, tmp_path, monkeypatch):
    _lib, ops, autotune = mods
    monkeypatch.setenv("DDGEMM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    batch, probs, _ = make_batch(ops, MIXED, seed=41, variant=TC)
    cfg, timings = autotune.tune(batch, reps=1)
    assert cfg in autotune.TC_CANDIDATES and len(timings) == len(autotune.TC_CANDIDATES)
    cfg2, _ = autotune.tune(batch, reps=1)
    assert cfg2 == cfg
    # the FP64 batch of the same shapes is tuned (and cached) on its own
    fp64, _, _ = make_batch(ops, MIXED, seed=41)
    assert autotune.tune(fp64, reps=1)[0] in autotune.CANDIDATES


@pytest.mark.parametrize("variant", [0, TC, 5])
def test_batched_phase_events(mods, variant):
    """ddgemm_batched records the three phase events (before the plan,
    before the persistent kernel, after it) in stream order, and a run with
    them gives the same bits as one without."""
    _, ops, _ = mods
    rng = np.random.default_rng(11)
    shapes = [tuple(int(v) for v in rng.integers(30, 300, 3)) for _ in range(40)]
    batch, probs, _ = make_batch(ops, shapes, seed=50, variant=variant)
    batch.run()
    want = [(h.copy(), lo.copy()) for h, lo in results(probs)]
    for p in probs:
        p[4].fill_(np.nan)
        p[5].fill_(np.nan)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for e in ev:
        e.record(stream)
    end = torch.cuda.Event(enable_timing=True)
    batch.run(phase_events=ev)
    end.record(stream)
    end.synchronize()
    split_ms, kern_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    assert split_ms > 0 and kern_ms > 0
    assert ev[2].elapsed_time(end) >= 0
    for (h, lo), (wh, wl) in zip(results(probs), want):
        assert np.array_equal(h.view(np.int64), wh.view(np.int64))
        assert np.array_equal(lo.view(np.int64), wl.view(np.int64))
