"""Benchmark of the cascading FP64x2 GEMM on GB300.

One step = one pass of the whole hot path over one problem: the split of A
(four pieces), the split of B (seven panels) and the ten FP64 products with
the fused bin assembly, through the C ABI (ddgemm).  Default workload: the
4096^3 cascade with hi log-uniform over 2^-20..2^20 (random signs) and
lo = hi 2^-53 U[-1, 1], seed 0.  The inputs (512 MiB), the cascaded panels
(1.4 GiB) and C are all larger than the 129 MB L2, so no flush is needed
between steps.

Metric: effective FP64x2 GFLOP/s = 2 m n k / time (the work of the FP64x2
product, not of the ten FP64 products), next to the fraction of the FP64
tensor-path peak that the ten products reach, and the largest error against
the double-double oracle on sampled entries.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica of the problem (the
cascade needs no exchange between GPUs): value = all ranks' work / the
slowest rank's time.  `--impl reference` times the CPU oracle (the scalar
double-double triple loop) on the host cores on a bounded sample of rows.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import gemm_inputs  # noqa: E402

METRIC = "effective FP64x2 GFLOP/s at 4096^3 & % FP64-TC peak; max err vs dd oracle"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal GB300 dense rates (TFLOP/s) for the FP64-from-bf16 ratio.
NOMINAL_FP64_TFLOPS = 1.25
NOMINAL_BF16_TFLOPS = 2250.0

# DRAM bytes per launch (read + write) of the dominant kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the current
# kernels at 4096^3; other workloads report null.
TRAFFIC_4096 = {"cascade_fp64_kernel": 9.881583e9 + 0.286808e9,
                "cascade_int8_kernel<15>": 3.096227e9 + 0.268912e9,
                "cascade_int8_tc_kernel<16>": 9.188401e9 + 0.287655e9}

VARIANT_NAMES = {1: "int8", 4: "int8 on tcgen05", 5: "int8 on tcgen05, eight-bit pieces"}

WORKLOADS = {
    "4096": dict(m=4096, n=4096, k=4096, kind="wide",
                 name="ddgemm 4096x4096x4096 FP64x2, hi log-uniform 2^-20..2^20, seed 0"),
    "rect": dict(m=8192, n=1024, k=4096, kind="wide",
                 name="ddgemm 8192x1024x4096 FP64x2, hi log-uniform 2^-20..2^20, seed 0"),
    "8192": dict(m=8192, n=8192, k=8192, kind="wide",
                 name="ddgemm 8192x8192x8192 FP64x2, hi log-uniform 2^-20..2^20, seed 0"),
    "2048": dict(m=2048, n=2048, k=2048, kind="wide",
                 name="ddgemm 2048x2048x2048 FP64x2, hi log-uniform 2^-20..2^20, seed 0"),
    "256": dict(m=256, n=256, k=256, kind="uniform",
                name="ddgemm 256x256x256 FP64x2, hi U[-1,1], seed 0"),
}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Largest value over the ranks (the slowest replica's time); the
    identity for one process.  Works on gloo (CPU tensors) and NCCL."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job rate of independent replicas: all ranks' units over the
    slowest rank's time (units per second)."""
    return world * units_per_rank / (max_ms * 1e-3)


def physical_index(local: int) -> int:
    """nvidia-smi index of this rank's GPU."""
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    if local < len(vis) and vis[local].isdigit():
        return int(vis[local])
    return local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen(
            [exe, "-i", str(self.index), f"--query-gpu={self.FIELDS}",
             "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
            stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for name, val in zip(self.NAMES, parts[3:7]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.remove(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


def fp64_peak_rule():
    """FP64 tensor-path peak = the measured bf16 peak x the nominal
    FP64/bf16 ratio.  The burst bf16 figure is used: the FP64 pipe runs at
    the maximum SM clock for the whole step (see "clocks"), so the
    power-capped sustained bf16 figure does not describe it."""
    try:
        with open(MEASURED_PEAKS) as f:
            mp = json.load(f)
        return (mp["bf16_tflops"] * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS,
                "of measured: MEASURED_PEAKS.json bf16_tflops (burst) x nominal FP64/bf16 "
                "(1.25/2250)")
    except (OSError, KeyError, ValueError):
        return (1900.0 * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS,
                "of fallback: bf16 1.9 PFLOP/s burst x nominal FP64/bf16 (1.25/2250)")


def bf16_peaks():
    """(peak, source, sustained) of the bf16 tensor path for the tcgen05
    INT8 form: MEASURED_PEAKS.json's burst figure (a conservative
    denominator; the sustained power-capped figure is reported beside it)."""
    try:
        with open(MEASURED_PEAKS) as f:
            mp = json.load(f)
        return (mp["bf16_tflops"], "of measured: MEASURED_PEAKS.json bf16_tflops (burst)",
                mp.get("bf16_tflops_sustained"))
    except (OSError, KeyError, ValueError):
        return 1900.0, "of fallback: bf16 1.9 PFLOP/s burst", 1700.0


def oracle_rows_rate(a_hi, a_lo, b_hi, b_lo, rows):
    """Time the double-double oracle on full rows of C; returns (seconds, threads)."""
    from oracle import dd
    n = b_hi.shape[1]
    rr = np.repeat(np.asarray(rows, dtype=np.int32), n)
    cc = np.tile(np.arange(n, dtype=np.int32), len(rows))
    t0 = time.perf_counter()
    dd.ddgemm_entries(a_hi, a_lo, b_hi, b_lo, rr, cc)
    return time.perf_counter() - t0, dd.num_threads()


def cpu_baseline(a_hi, a_lo, b_hi, b_lo, target_s=12.0):
    """The oracle as it stands on the host cores, on a bounded row sample."""
    m, k = a_hi.shape
    n = b_hi.shape[1]
    probe_rows = 2
    t, _ = oracle_rows_rate(a_hi, a_lo, b_hi, b_lo, list(range(probe_rows)))
    rows = int(max(1, min(m, probe_rows * target_s / max(t, 1e-6))))
    sel = np.linspace(0, m - 1, rows).astype(np.int64)
    t, threads = oracle_rows_rate(a_hi, a_lo, b_hi, b_lo, sel)
    value = 2.0 * rows * n * k / t / 1e9
    return {"value": round(value, 4), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"{rows} of {m} rows of C ({rows * n} entries, k = {k}), "
                      f"scalar double-double TwoProd/TwoSum loop, {t:.1f} s"}


# ---- the other workloads of the benchmark line ----------------------------
# Each is one compact record in the default line, timed with CUDA events on
# the launching stream after warm-up, with its own clock record and its
# largest error against the double-double oracle on sampled entries.

TC_FORMS = {1: ("int8 mma.sync, 15 x 8-bit pieces", 15),
            4: ("int8 tcgen05, 16 x 7-bit pieces", 16),
            5: ("int8 tcgen05, 15 x 8-bit pieces", 15)}


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _timed(fn, reps, warmup, stream):
    """Milliseconds per call of fn() on `stream` (CUDA events), and the
    clock record taken while the timed calls ran."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    sampler = ClockSampler(physical_index(stream.device.index or 0))
    sampler.start()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    return e0.elapsed_time(e1) / reps, clocks


def _sampled_error(a, c, rows, cols):
    """max |C - C_dd| / (|A||B|) over the sampled entries (A, B as (hi, lo)
    host arrays, C as a (hi, lo) pair of device tensors)."""
    from oracle import dd
    oh, ol = dd.ddgemm_entries(*a, rows, cols)
    ch, cl = c[0].cpu().numpy(), c[1].cpu().numpy()
    absab = np.array([np.abs(a[0][i]) @ np.abs(a[2][:, j]) for i, j in zip(rows, cols)])
    return float(np.max(np.abs((ch[rows, cols] - oh) + (cl[rows, cols] - ol)) / absab))


def _form_step(d_in, m, n, k, variant, slices, reps, warmup, stream, dev):
    """One form's whole step (split + products) timed, and its products
    kernel timed by the phase events on the same calls."""
    import torch

    from paper_2303_04353_gb300 import ops
    ws = ops.alloc_workspace(m, n, k, dev, variant, slices)
    c = (torch.empty((m, n), dtype=torch.float64, device=dev),
         torch.empty((m, n), dtype=torch.float64, device=dev))
    phase = [_events(3) for _ in range(reps)]
    for evs in phase:
        for e in evs:
            e.record(stream)            # an event must exist before the library records it
    calls = {"timed": 0}

    def step(timed=True):
        evs = None
        if timed:
            evs = phase[calls["timed"] % reps]
            calls["timed"] += 1
        ops.ddgemm(*d_in, out=c, workspace=ws, stream=stream, variant=variant,
                   int8_slices=slices, phase_events=evs)
    for _ in range(warmup):
        step(timed=False)
    ms, clocks = _timed(step, reps, 0, stream)
    kernel_ms = sum(ev[1].elapsed_time(ev[2]) for ev in phase) / reps
    del ws
    return ms, kernel_ms, clocks, c


def _roofline_of(variant, slices, flops_dd, kernel_ms, int8_peak):
    """Roofline fraction of a form's products kernel: FP64 flops against the
    FP64 peak rule, integer ops against the live mma.sync s8 probe, bf16
    digit flops against the measured bf16 burst peak."""
    if variant == 0:
        peak, src = fp64_peak_rule()
        achieved = 10 * flops_dd / (kernel_ms * 1e-3) / 1e12
        return {"bound": "fp64 pipe", "achieved": round(achieved, 4), "peak": round(peak, 4),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "peak_source": src}
    prods = slices * (slices + 1) // 2
    achieved = prods * flops_dd / (kernel_ms * 1e-3) / 1e12
    if variant == 1:
        return {"bound": "tensor (mma.sync s8)", "achieved": round(achieved, 3),
                "peak": round(int8_peak, 3), "unit": "TOPS", "frac": round(achieved / int8_peak, 4),
                "peak_source": "of measured: live mma.sync s8 probe in this run"}
    bpeak, bsrc, _ = bf16_peaks()
    return {"bound": "tensor (tcgen05 bf16)", "achieved": round(achieved, 3),
            "peak": round(bpeak, 3), "unit": "TFLOP/s", "frac": round(achieved / bpeak, 4),
            "peak_source": bsrc}


def _probe_tops(stream):
    import torch

    from paper_2303_04353_gb300 import _lib
    sink = torch.zeros(1, dtype=torch.float64, device=stream.device)
    best = 0.0
    for iters in (200, 4000, 4000):
        p0, p1 = _events(2)
        p0.record(stream)
        work = _lib.ddgemm_probe_int8(iters, sink.data_ptr(), stream.cuda_stream)
        p1.record(stream)
        torch.cuda.synchronize()
        best = max(best, work / (p0.elapsed_time(p1) * 1e-3) / 1e12)
    return best


def config_small(dev, stream):
    """256^3, uniform entries, seed 0: the latency case.  Every entry is
    checked against the full oracle."""
    from oracle import dd
    import torch
    m = n = k = 256
    a = gemm_inputs(m, n, k, kind="uniform", seed=0)
    d_in = [torch.from_numpy(x).to(dev) for x in a]
    oh, ol = dd.ddgemm(*a)
    absab = np.abs(a[0]) @ np.abs(a[2])
    out = {"workload": "ddgemm 256x256x256 FP64x2, hi U[-1,1], seed 0 (all entries checked)"}
    for name, variant, s8 in (("fp64", 0, 0), ("int8_tc", 4, 16), ("int8_tc8", 5, 15)):
        ms, kms, clocks, c = _form_step(d_in, m, n, k, variant, s8, 50, 5, stream, dev)
        ch, cl = c[0].cpu().numpy(), c[1].cpu().numpy()
        err = float(np.max(np.abs((ch - oh) + (cl - ol)) / absab))
        out[name] = {"us_per_call": round(ms * 1e3, 2), "kernel_us": round(kms * 1e3, 2),
                     "value": round(2.0 * m * n * k / (ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
                     "max_err_vs_dd_oracle": err, "launches": 3 if variant == 0 else 5,
                     "clocks": clocks}
    return out


def config_rect(dev, stream):
    """8192 x 1024 x 4096, wide entries (the rectangular case): the FP64
    form with its automatic split-k grouping."""
    import torch

    from paper_2303_04353_gb300 import ops
    m, n, k = 8192, 1024, 4096
    a = gemm_inputs(m, n, k, kind="wide", seed=0)
    d_in = [torch.from_numpy(x).to(dev) for x in a]
    rng = np.random.default_rng(11)
    rows, cols = rng.integers(0, m, 64), rng.integers(0, n, 64)
    ms, kms, clocks, c = _form_step(d_in, m, n, k, 0, 0, 3, 3, stream, dev)
    ws_bytes = ops.workspace_bytes(m, n, k)
    return {"workload": "ddgemm 8192x1024x4096 FP64x2, hi log-uniform 2^-20..2^20, seed 0",
            "ms_per_step": round(ms, 3), "value": round(2.0 * m * n * k / (ms * 1e-3) / 1e9, 4),
            "unit": "GFLOP/s", "split_k_groups": ops.split_groups(m, n, k, dev, ws_bytes),
            "roofline": _roofline_of(0, 0, 2.0 * m * n * k, kms, None),
            "max_err_vs_dd_oracle": _sampled_error(a, c, rows, cols), "steps": 3, "warmup": 3,
            "clocks": clocks}


def config_int8_large(dev, stream, int8_peak):
    """8192^3, wide entries: the three INT8 forms against one FP64-form step
    on the same inputs (equal accuracy is read off the sampled errors)."""
    import torch
    m = n = k = 8192
    a = gemm_inputs(m, n, k, kind="wide", seed=0)
    d_in = [torch.from_numpy(x).to(dev) for x in a]
    rng = np.random.default_rng(12)
    rows, cols = rng.integers(0, m, 64), rng.integers(0, n, 64)
    flops = 2.0 * m * n * k
    out = {"workload": "ddgemm 8192x8192x8192 FP64x2, hi log-uniform 2^-20..2^20, seed 0"}
    fp64_ms = None
    for name, variant, s8, reps, warm in (("fp64", 0, 0, 1, 1), ("int8", 1, 15, 3, 3),
                                          ("int8_tc", 4, 16, 5, 3), ("int8_tc8", 5, 15, 5, 3)):
        ms, kms, clocks, c = _form_step(d_in, m, n, k, variant, s8, reps, warm, stream, dev)
        rec = {"ms_per_step": round(ms, 3), "value": round(flops / (ms * 1e-3) / 1e9, 3),
               "unit": "GFLOP/s", "roofline": _roofline_of(variant, s8, flops, kms, int8_peak),
               "max_err_vs_dd_oracle": _sampled_error(a, c, rows, cols),
               "steps": reps, "warmup": warm, "clocks": clocks}
        if variant:
            rec["pieces"] = s8
            rec["products"] = s8 * (s8 + 1) // 2
            rec["speedup_vs_fp64_form"] = round(fp64_ms / ms, 3)
        else:
            fp64_ms = ms
        out[name] = rec
        del c
        torch.cuda.empty_cache()
    return out


def config_spread_sweep(dev, stream):
    """Exponent-spread sweep at 2048^3: hi = +-2^u, u ~ U[-S/2, S/2], for
    S = 0, 20, 40, 60 octaves; max error per form on 64 sampled entries."""
    import torch

    from paper_2303_04353_gb300 import ops
    m = n = k = 2048
    rng = np.random.default_rng(3)
    rows, cols = rng.integers(0, m, 64), rng.integers(0, n, 64)
    forms = (("fp64", 0, 0), ("int8", 1, 15), ("int8_tc", 4, 16), ("int8_tc8", 5, 15))
    out = {"workload": "ddgemm 2048^3, hi = +-2^u, u ~ U[-S/2, S/2], seed 0; 64 sampled entries",
           "spreads": [0, 20, 40, 60], "max_err_vs_dd_oracle": {f[0]: [] for f in forms}}
    for spread in out["spreads"]:
        a = gemm_inputs(m, n, k, kind="wide", seed=0, spread=float(spread))
        d_in = [torch.from_numpy(x).to(dev) for x in a]
        for name, variant, s8 in forms:
            c = ops.ddgemm(*d_in, stream=stream, variant=variant, int8_slices=s8)
            out["max_err_vs_dd_oracle"][name].append(_sampled_error(a, c, rows, cols))
    return out


def config_batched(dev, stream):
    """512 problems, m, n, k each log-uniform in [64, 1024], uniform entries:
    one ddgemm per problem against ddgemm_batched (autotuned tiles, eager and
    graph-replayed) for the FP64 form, and the batched tcgen05 forms
    graph-replayed.  Three problems are checked against the oracle."""
    import torch

    from paper_2303_04353_gb300 import autotune, ops
    from workloads import batched_shapes
    shapes = [tuple(int(v) for v in sh) for sh in batched_shapes(512, seed=0)]
    host, probs = [], []
    for i, (m, n, k) in enumerate(shapes):
        a = gemm_inputs(m, n, k, kind="uniform", seed=1000 + i)
        host.append(a)
        t = [torch.from_numpy(x).to(dev) for x in a]
        probs.append((*t, torch.empty((m, n), dtype=torch.float64, device=dev),
                      torch.empty((m, n), dtype=torch.float64, device=dev)))
    flops = sum(2.0 * m * n * k for m, n, k in shapes)
    checked = (0, 170, 341)

    def worst(plist):
        e = 0.0
        for i in checked:
            m, n, _ = shapes[i]
            rng = np.random.default_rng(i)
            rows, cols = rng.integers(0, m, 32), rng.integers(0, n, 32)
            e = max(e, _sampled_error(host[i], (plist[i][4], plist[i][5]), rows, cols))
        return e

    def graph_of(batch, cfg=None):
        side = torch.cuda.Stream(dev)
        g = torch.cuda.CUDAGraph()
        batch.run(stream=stream, config=cfg)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=side):
            batch.run(stream=torch.cuda.current_stream(), config=cfg)
        return g

    out = {"workload": "batched: 512 problems, m, n, k log-uniform in [64, 1024], hi U[-1,1]",
           "sum_2mnk": flops}
    ws = ops.alloc_workspace(max(sh[0] for sh in shapes), max(sh[1] for sh in shapes),
                             max(sh[2] for sh in shapes), dev)

    def per_problem():
        for a_hi, a_lo, b_hi, b_lo, c_hi, c_lo in probs:
            ops.ddgemm(a_hi, a_lo, b_hi, b_lo, out=(c_hi, c_lo), workspace=ws, stream=stream)
    per_ms, per_clocks = _timed(per_problem, 2, 1, stream)
    del ws
    batch = ops.Batch(probs)
    cfg, tune_ms = autotune.tune(batch, reps=2, use_cache=False)
    eager_ms, _ = _timed(lambda: batch.run(stream=stream, config=cfg), 3, 3, stream)
    g = graph_of(batch, cfg)
    graph_ms, graph_clocks = _timed(g.replay, 3, 3, stream)
    out["fp64"] = {"per_problem_ms": round(per_ms, 3), "per_problem_launches": 3 * len(shapes),
                   "per_problem_value": round(flops / (per_ms * 1e-3) / 1e9, 3),
                   "batched_eager_ms": round(eager_ms, 3),
                   "batched_graph_ms": round(graph_ms, 3),
                   "value": round(flops / (graph_ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
                   "autotuned": {"tile_order": list(cfg), "candidates_ms": tune_ms},
                   "max_err_vs_dd_oracle": worst(probs), "launches": 4,
                   "clocks": graph_clocks, "per_problem_clocks": per_clocks}
    bpeak, bsrc, _ = bf16_peaks()
    for name, variant, s8 in (("int8_tc", 4, 16), ("int8_tc8", 5, 15)):
        tp = [(*p[:4], torch.empty_like(p[4]), torch.empty_like(p[5])) for p in probs]
        tb = ops.Batch(tp, variant=variant)
        default_ms, _ = _timed(lambda: tb.run(stream=stream), 3, 3, stream)
        tcfg, ttimes = autotune.tune(tb, reps=2, use_cache=False)
        tg = graph_of(tb, tcfg)
        ms, clocks = _timed(tg.replay, 5, 3, stream)
        prods = s8 * (s8 + 1) // 2
        achieved = prods * flops / (ms * 1e-3) / 1e12
        # the persistent kernel alone: the library's phase events around it,
        # eager runs of the tuned schedule
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        for e in ev:
            e.record(stream)
        split_ms = kern_ms = 0.0
        reps = 5
        for _ in range(reps):
            tb.run(stream=stream, config=tcfg, phase_events=ev)
            ev[2].synchronize()
            split_ms += ev[0].elapsed_time(ev[1]) / reps
            kern_ms += ev[1].elapsed_time(ev[2]) / reps
        k_achieved = prods * flops / (kern_ms * 1e-3) / 1e12
        out[name] = {"batched_graph_ms": round(ms, 3),
                     "value": round(flops / (ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
                     "pieces": s8, "launches": 4,
                     "autotuned": {"config": list(tcfg), "fields": "tile, order, orient, "
                                   "planes, row_group", "candidates_ms": ttimes,
                                   "default_schedule_eager_ms": round(default_ms, 3)},
                     "speedup_vs_fp64_batched": round(graph_ms / ms, 3),
                     "pass_roofline": {"bound": "tensor (tcgen05 bf16)",
                                       "achieved": round(achieved, 3), "peak": round(bpeak, 3),
                                       "unit": "TFLOP/s", "frac": round(achieved / bpeak, 4),
                                       "peak_source": bsrc,
                                       "what": f"{prods} x sum 2mnk digit flops over the "
                                               "whole pass (4 launches)"},
                     "phases_ms": {"plan_and_split": round(split_ms, 3),
                                   "persistent_kernel": round(kern_ms, 3)},
                     "kernel_roofline": {"bound": "tensor (tcgen05 bf16)",
                                         "kernel": "cascade_int8_tc_kernel (BatchSource)",
                                         "achieved": round(k_achieved, 3),
                                         "peak": round(bpeak, 3), "unit": "TFLOP/s",
                                         "frac": round(k_achieved / bpeak, 4),
                                         "peak_source": bsrc,
                                         "what": f"{prods} x sum 2mnk digit flops / the "
                                                 "persistent kernel's time (phase events)"},
                     "max_err_vs_dd_oracle": worst(tp), "clocks": clocks}
        del tg, tb, tp
    return out


def config_backward(dev, stream):
    """2048^3 forward and backward (L = sum(W * C), dC = W, uniform A, B,
    W): one step = C, then dA = W B^T and dB = A^T W, each by the cascade;
    dA and dB checked on 64 sampled entries against the oracle's gradient."""
    import torch

    from paper_2303_04353_gb300 import ops
    from workloads import dd_matrix
    m = n = k = 2048
    a = gemm_inputs(m, n, k, kind="uniform", seed=0)
    w = dd_matrix(np.random.default_rng(99), (m, n))
    d_in = [torch.from_numpy(x).to(dev) for x in a]
    d_w = [torch.from_numpy(x).to(dev) for x in w]
    rng = np.random.default_rng(13)
    rows, cols = rng.integers(0, m, 64), rng.integers(0, k, 64)
    bt = (np.ascontiguousarray(a[2].T), np.ascontiguousarray(a[3].T))
    at = (np.ascontiguousarray(a[0].T), np.ascontiguousarray(a[1].T))
    out = {"workload": "ddgemm 2048^3 forward + backward, L = sum(W * C), A, B, W hi U[-1,1]"}
    for name, variant, s8 in (("fp64", 0, 0), ("int8_tc", 4, 16), ("int8_tc8", 5, 15)):
        res = {}

        def step():
            ops.ddgemm(*d_in, stream=stream, variant=variant, int8_slices=s8)
            res["g"] = ops.ddgemm_backward(*d_in, *d_w, stream=stream, variant=variant,
                                           int8_slices=s8)
        ms, clocks = _timed(step, 3, 3, stream)
        da_hi, da_lo, db_hi, db_lo = res["g"]
        err_da = _sampled_error((w[0], w[1], bt[0], bt[1]), (da_hi, da_lo), rows, cols)
        err_db = _sampled_error((at[0], at[1], w[0], w[1]), (db_hi, db_lo), rows, cols)
        out[name] = {"ms_per_step": round(ms, 3), "cascades": 3,
                     "value": round(3 * 2.0 * m * n * k / (ms * 1e-3) / 1e9, 3),
                     "unit": "GFLOP/s (3 x 2mnk per step)",
                     "max_err_dA_vs_dd_oracle": err_da, "max_err_dB_vs_dd_oracle": err_db,
                     "clocks": clocks}
    return out


def run_configs(dev, stream):
    """All the other workloads, in the order of their cost."""
    t0 = time.perf_counter()
    int8_peak = _probe_tops(stream)
    out = {"config0_256": config_small(dev, stream),
           "config1_rect": config_rect(dev, stream),
           "config2_8192": config_int8_large(dev, stream, int8_peak),
           "config2_sweep": config_spread_sweep(dev, stream),
           "config3_batched": config_batched(dev, stream),
           "config4_backward": config_backward(dev, stream)}
    out["configs_wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def run_reference(args, wl):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(wl["m"], wl["n"], wl["k"], kind=wl["kind"], seed=0)
    from oracle import dd
    dd.build()
    m, n, k = wl["m"], wl["n"], wl["k"]
    # rows per step sized for ~2-3 s of host work
    t, threads = oracle_rows_rate(a_hi, a_lo, b_hi, b_lo, [0])
    rows = int(max(1, min(m, 2.5 / max(t, 1e-6))))
    rng = np.random.default_rng(1)
    for _ in range(args.warmup):
        oracle_rows_rate(a_hi, a_lo, b_hi, b_lo, rng.integers(0, m, rows))
    times = []
    for _ in range(args.steps):
        t, threads = oracle_rows_rate(a_hi, a_lo, b_hi, b_lo, rng.integers(0, m, rows))
        times.append(t)
    step_s = sum(times) / len(times)
    value = 2.0 * rows * n * k / step_s / 1e9
    sample = f"{rows} random rows of C per step ({rows * n} entries, k = {k})"
    line = {"metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["name"], "m": m, "n": n, "k": k,
                       "sample": sample, "l2": "host run"},
            "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, wl):
    import torch

    from paper_2303_04353_gb300 import _lib, ops

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the cascade has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
    m, n, k = wl["m"], wl["n"], wl["k"]
    a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind=wl["kind"], seed=0)
    host_in = [torch.from_numpy(x).pin_memory() for x in (a_hi, a_lo, b_hi, b_lo)]
    d_in = [h.to(dev) for h in host_in]
    c_hi = torch.empty((m, n), dtype=torch.float64, device=dev)
    c_lo = torch.empty((m, n), dtype=torch.float64, device=dev)
    variant = {"int8": _lib.DDGEMM_VARIANT_INT8, "int8tc": _lib.DDGEMM_VARIANT_INT8_TC,
               "int8tc8": _lib.DDGEMM_VARIANT_INT8_TC8}.get(
        args.variant, _lib.DDGEMM_VARIANT_FP64)
    if not args.int8_slices:   # each form's default: 15 eight-bit / 16 seven-bit pieces
        args.int8_slices = 16 if variant == _lib.DDGEMM_VARIANT_INT8_TC else 15
    ws = ops.alloc_workspace(m, n, k, dev, variant, args.int8_slices)
    groups = ops.split_groups(m, n, k, dev, ws.numel(), variant)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(events=None):
        ops.ddgemm(*d_in, out=(c_hi, c_lo), workspace=ws, status=status, stream=stream,
                   phase_events=events, variant=variant, int8_slices=args.int8_slices)

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps on device-resident inputs -------------------
    phase = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    for evs in phase:
        for e in evs:
            e.record(stream)          # create the events before handing them over
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(physical_index(local))
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_start.record(stream)
    for s in range(args.steps):
        step(phase[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    split_ms = sum(ev[0].elapsed_time(ev[1]) for ev in phase) / args.steps
    casc_ms = sum(ev[1].elapsed_time(ev[2]) for ev in phase) / args.steps
    elapsed_ms = reduce_max(elapsed_ms, world, dev)
    ms_per_step = elapsed_ms / args.steps
    flops_dd = 2.0 * m * n * k
    value = replica_rate(flops_dd, world, ms_per_step) / 1e9
    st = int(status.item())
    if st:
        raise SystemExit(f"bench.py: device status {st:#x} (non-finite input or timeout)")

    # ---- accuracy on sampled entries vs the double-double oracle -----------
    from oracle import dd
    rng = np.random.default_rng(7)
    rows = rng.integers(0, m, 256)
    cols = rng.integers(0, n, 256)
    ch, cl = c_hi.cpu().numpy(), c_lo.cpu().numpy()
    oh, ol = dd.ddgemm_entries(a_hi, a_lo, b_hi, b_lo, rows, cols)
    absab = np.array([np.abs(a_hi[i]) @ np.abs(b_hi[:, j]) for i, j in zip(rows, cols)])
    err = np.abs((ch[rows, cols] - oh) + (cl[rows, cols] - ol))
    max_err = float(np.max(err / absab))

    # ---- end to end: pinned host inputs -> ddgemm_host (C ABI) -> host C ----
    # The library copies A and B in and C out on streams of its own, in row
    # chunks that overlap the cascade on `stream`; `stream` ends after the
    # last copy back.
    e2e_steps = max(1, min(args.steps, 3))
    host_out = [torch.empty((m, n), dtype=torch.float64).pin_memory() for _ in range(2)]
    hbuf = torch.empty(max(ops.host_buffer_bytes(m, n, k, variant, args.int8_slices), 1),
                       dtype=torch.uint8, device=dev)
    del ws                                   # the host path has its own workspace
    torch.cuda.empty_cache()

    def e2e_step():
        ops.ddgemm_host(*host_in, out=host_out, buffer=hbuf, status=status, stream=stream,
                        variant=variant, int8_slices=args.int8_slices)
    e2e_step()                               # warm-up (first-use costs of the copy path)
    torch.cuda.synchronize()
    # the host link's rate right now (it varies on a shared host): one plain
    # copy of A_hi in and of C_hi out, outside the timed region
    c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    c0.record(stream)
    d_in[0].copy_(host_in[0], non_blocking=True)
    c1.record(stream)
    host_out[0].copy_(c_hi, non_blocking=True)
    c2.record(stream)
    torch.cuda.synchronize()
    link = {"h2d_GBs": round(m * k * 8 / (c0.elapsed_time(c1) * 1e-3) / 1e9, 1),
            "d2h_GBs": round(m * n * 8 / (c1.elapsed_time(c2) * 1e-3) / 1e9, 1)}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_sampler = ClockSampler(physical_index(local))
    barrier()
    torch.cuda.synchronize()
    e2e_sampler.start()
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_clocks = e2e_sampler.stop()
    e2e_ms = reduce_max(e0.elapsed_time(e1) / e2e_steps, world, dev)
    h2d = sum(h.numel() * 8 for h in host_in)
    d2h = 2 * m * n * 8
    e2e_err = float(np.max(np.abs((host_out[0].numpy()[rows, cols] - oh)
                                  + (host_out[1].numpy()[rows, cols] - ol)) / absab))
    del hbuf

    # ---- the tensor-path ceilings, measured on this GPU --------------------
    sink = torch.zeros(1, dtype=torch.float64, device=dev)

    def probe(fn, iters_list):
        best = 0.0
        for iters in iters_list:
            p0 = torch.cuda.Event(enable_timing=True)
            p1 = torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            work = fn(iters, sink.data_ptr(), stream.cuda_stream)
            p1.record(stream)
            torch.cuda.synchronize()
            best = max(best, work / (p0.elapsed_time(p1) * 1e-3) / 1e12)
        return best
    probe_tflops = probe(_lib.ddgemm_probe_fp64, (200, 2000, 2000, 2000))
    probe_tops = probe(_lib.ddgemm_probe_int8, (200, 4000, 4000, 4000)) \
        if variant == _lib.DDGEMM_VARIANT_INT8 else None

    # ---- the INT8 forms on the same inputs (one line, all forms) ----------
    def time_form(form_variant):
        s8 = 16 if form_variant == _lib.DDGEMM_VARIANT_INT8_TC else 15
        ws8 = ops.alloc_workspace(m, n, k, dev, form_variant, s8)
        c8 = (torch.empty((m, n), dtype=torch.float64, device=dev),
              torch.empty((m, n), dtype=torch.float64, device=dev))

        def step8():
            ops.ddgemm(*d_in, out=c8, workspace=ws8, stream=stream, variant=form_variant,
                       int8_slices=s8)
        for _ in range(args.warmup):
            step8()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step8()
        e1.record(stream)
        torch.cuda.synchronize()
        ms8 = reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)
        h8, l8 = c8[0].cpu().numpy(), c8[1].cpu().numpy()
        err8 = np.abs((h8[rows, cols] - oh) + (l8[rows, cols] - ol))
        del ws8
        return {"pieces": s8, "piece_bits": 7 if form_variant == _lib.DDGEMM_VARIANT_INT8_TC else 8,
                "products": s8 * (s8 + 1) // 2, "ms_per_step": round(ms8, 3),
                "value": round(replica_rate(flops_dd, world, ms8) / 1e9, 4),
                "unit": "GFLOP/s",
                "max_err_vs_dd_oracle": float(np.max(err8 / absab)),
                "speedup_vs_fp64_form": round(ms_per_step / ms8, 3)}

    int8_form = int8_tc_form = int8_tc8_form = None
    if variant == _lib.DDGEMM_VARIANT_FP64 and not args.no_int8_form:
        int8_form = time_form(_lib.DDGEMM_VARIANT_INT8)
        int8_form["products_on"] = "mma.sync m16n8k32 s8 (int32 accumulation)"
        int8_tc_form = time_form(_lib.DDGEMM_VARIANT_INT8_TC)
        int8_tc8_form = time_form(_lib.DDGEMM_VARIANT_INT8_TC8)
        int8_tc8_form["products_on"] = ("tcgen05.mma kind::f16, the mma.sync form's eight-bit "
                                        "digits in bf16, FP32 in TMEM (exact per 64 entries); "
                                        "exact assembly")
        int8_tc_form["products_on"] = ("tcgen05.mma kind::f16, bf16 digits, FP32 in TMEM "
                                       "(exact per 256 entries); exact assembly")

    # ---- yardstick: a plain FP64 GEMM of the same shape (cuBLAS DGEMM via
    # torch.matmul), the unit of the paper's "10-13x DGEMM time" claim ------
    dgemm = None
    if variant == _lib.DDGEMM_VARIANT_FP64 and not args.no_int8_form:
        x, y = d_in[0], d_in[2]
        z = torch.empty((m, n), dtype=torch.float64, device=dev)
        for _ in range(2):
            torch.matmul(x, y, out=z)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            torch.matmul(x, y, out=z)
        e1.record(stream)
        torch.cuda.synchronize()
        dg_ms = e0.elapsed_time(e1) / 3
        dgemm = {"ms": round(dg_ms, 3), "tflops": round(flops_dd / (dg_ms * 1e-3) / 1e12, 4),
                 "fp64_form_over_dgemm": round(ms_per_step / dg_ms, 3),
                 "what": "cuBLAS DGEMM (torch.matmul, float64) on A_hi, B_hi: a yardstick, "
                         "not part of the path"}
        if int8_form is not None:
            dgemm["int8_form_over_dgemm"] = round(int8_form["ms_per_step"] / dg_ms, 3)
        if int8_tc_form is not None:
            dgemm["int8_tc_form_over_dgemm"] = round(int8_tc_form["ms_per_step"] / dg_ms, 3)
        if int8_tc8_form is not None:
            dgemm["int8_tc8_form_over_dgemm"] = round(int8_tc8_form["ms_per_step"] / dg_ms, 3)
        del z

    # ---- the other workloads (configs 0, 2, 3, 4 and the rectangular case) --
    configs = None
    if world == 1 and variant == _lib.DDGEMM_VARIANT_FP64 and not args.no_configs:
        torch.cuda.empty_cache()
        configs = run_configs(dev, stream)

    if rank != 0:
        return
    peak, peak_src = fp64_peak_rule()
    if variant in (_lib.DDGEMM_VARIANT_INT8_TC, _lib.DDGEMM_VARIANT_INT8_TC8):
        s8 = args.int8_slices
        prods = s8 * (s8 + 1) // 2
        achieved = prods * flops_dd / (casc_ms * 1e-3) / 1e12
        bpeak, bsrc, spk = bf16_peaks()
        kname = (f"cascade_int8_tc_kernel<{s8}>" if variant == _lib.DDGEMM_VARIANT_INT8_TC
                 else f"cascade_int8_tc_kernel<{s8}> (eight-bit pieces)")
        roofline = {"bound": "tensor", "kernel": kname,
                    "achieved": round(achieved, 3), "peak": round(bpeak, 3), "unit": "TFLOP/s",
                    "frac": round(achieved / bpeak, 4),
                    "traffic": TRAFFIC_4096.get(kname) if args.workload == "4096" else None,
                    "peak_source": bsrc,
                    "frac_vs_sustained": round(achieved / spk, 4) if spk else None,
                    "algorithmic": f"{prods} x 2mnk = {prods * flops_dd:.4g} bf16 flops "
                                   "(digit products) per launch"}
    elif variant == _lib.DDGEMM_VARIANT_INT8:
        s8 = args.int8_slices
        prods = s8 * (s8 + 1) // 2
        achieved = prods * flops_dd / (casc_ms * 1e-3) / 1e12
        roofline = {"bound": "tensor", "kernel": f"cascade_int8_kernel<{s8}>",
                    "achieved": round(achieved, 3), "peak": round(probe_tops, 3), "unit": "TOPS",
                    "frac": round(achieved / probe_tops, 4),
                    "traffic": TRAFFIC_4096.get(f"cascade_int8_kernel<{s8}>")
                    if args.workload == "4096" else None,
                    "peak_source": "of measured: live mma.sync s8 probe in this run (no INT8 "
                                   "figure in MEASURED_PEAKS.json)",
                    "algorithmic": f"{prods} x 2mnk = {prods * flops_dd:.4g} INT8 ops per launch"}
    else:
        achieved = 10.0 * flops_dd / (casc_ms * 1e-3) / 1e12
        # the FP64 MMA (mma.sync f64) runs on the FP64 pipe of sm_103a: ncu
        # shows sm__pipe_fp64_cycles_active near 97 % and the tensor pipe idle
        roofline = {"bound": "fp64 pipe", "kernel": "cascade_fp64_kernel",
                    "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                    "frac": round(achieved / peak, 4),
                    "traffic": TRAFFIC_4096["cascade_fp64_kernel"]
                    if args.workload == "4096" else None,
                    "peak_source": peak_src,
                    "probe_peak": round(probe_tflops, 4),
                    "frac_vs_probe": round(achieved / probe_tflops, 4),
                    "algorithmic": f"10 x 2mnk = {10 * flops_dd:.4g} FP64 flops per launch"}
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "m": m, "n": n, "k": k,
                   "variant": "fp64 (ten FP64 products)" if variant == _lib.DDGEMM_VARIANT_FP64
                   else f"{VARIANT_NAMES[variant]}"
                        f" ({args.int8_slices} pieces, "
                        f"{args.int8_slices * (args.int8_slices + 1) // 2} digit products)",
                   "split_k_groups": groups,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs (512 MiB) and panels larger than L2; no flush"
                         if m * k >= 1 << 22 else "small case; L2-resident"},
        **({"pct_fp64_peak": round(100.0 * 10.0 * flops_dd / (ms_per_step * 1e-3) / 1e12
                                   / probe_tflops, 2),
            "pct_fp64_peak_of": "the live FP64 MMA probe; the metric's FP64-TC path is the FP64 "
                                "pipe on sm_103a (tcgen05 has no f64 kind)"}
           if variant == _lib.DDGEMM_VARIANT_FP64 else
           {"pct_int8_tc_peak": round(100.0 * (args.int8_slices * (args.int8_slices + 1) // 2)
                                      * flops_dd / (ms_per_step * 1e-3) / 1e12 / probe_tops, 2)}
           if variant == _lib.DDGEMM_VARIANT_INT8 else
           {"pct_bf16_tc_peak": round(100.0 * (args.int8_slices * (args.int8_slices + 1) // 2)
                                      * flops_dd / (ms_per_step * 1e-3) / 1e12
                                      / bf16_peaks()[0], 2)}),
        "max_err_vs_dd_oracle": max_err,
        "phases_ms": {"split": round(split_ms, 3), "products_and_assembly": round(casc_ms, 3)},
        "roofline": roofline,
        "e2e": {"value": round(replica_rate(flops_dd, world, e2e_ms) / 1e9, 4), "unit": "GFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": round(e2e_ms, 3),
                "path": "ddgemm_host: pinned host operands, library copy streams overlapping "
                        "the cascade in row chunks",
                "max_err_vs_dd_oracle": e2e_err, "clocks": e2e_clocks,
                "link_before": link},
        # FP64 form: split A, split B, the cascade kernel, the split-k fix-up;
        # INT8 forms: exponents and digits of A and of B, the cascade kernel
        "gpu_launches": ((3 + (groups > 1)) if variant == _lib.DDGEMM_VARIANT_FP64 else 5)
        * args.steps,
        "clocks": clocks,
    }
    if int8_form is not None:
        line["int8_form"] = int8_form
    if int8_tc_form is not None:
        line["int8_tc_form"] = int8_tc_form
    if int8_tc8_form is not None:
        line["int8_tc8_form"] = int8_tc8_form
    if dgemm is not None:
        line["dgemm_yardstick"] = dgemm
    if int8_tc_form is not None and int8_tc8_form is not None:
        line["int8_tc_headline"] = (
            "int8_tc8_form (15 eight-bit pieces) is the tcgen05 form at the FP64 form's accuracy "
            "everywhere measured, ill-conditioned products included; int8_tc_form (16 seven-bit "
            "pieces) is faster and matches it on these inputs but not on ill-conditioned ones")
    if configs is not None:
        line.update(configs)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a_hi, a_lo, b_hi, b_lo)
    print(json.dumps(line), flush=True)


def run_batched_tc_only(args, shapes, probs, flops, stream):
    """The batched tcgen05 INT8 pass alone on the 512-problem workload (for
    profiling it): --steps timed calls after --warmup, no graph, no other
    form.  Study line."""
    import torch

    from paper_2303_04353_gb300 import _lib, ops

    variant = (_lib.DDGEMM_VARIANT_INT8_TC if args.variant == "int8tc"
               else _lib.DDGEMM_VARIANT_INT8_TC8)
    batch = ops.Batch(probs, variant=variant)
    status = torch.zeros(1, dtype=torch.int32, device=stream.device)
    for _ in range(args.warmup):
        batch.run(stream=stream, status=status)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batch.run(stream=stream, status=status)
    e1.record(stream)
    torch.cuda.synchronize()
    if int(status.item()):
        raise SystemExit(f"bench.py: device status {int(status.item()):#x}")
    ms = e0.elapsed_time(e1) / args.steps
    # the split and the persistent kernel apart (the library's phase events)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for e in ev:
        e.record(stream)
    split_ms = kern_ms = 0.0
    for _ in range(args.steps):
        batch.run(stream=stream, status=status, phase_events=ev)
        ev[2].synchronize()
        split_ms += ev[0].elapsed_time(ev[1]) / args.steps
        kern_ms += ev[1].elapsed_time(ev[2]) / args.steps
    tiles = sum(((m + 127) // 128) * ((n + 15) // 16) for m, n, _ in shapes if m and n)
    print(json.dumps({"study": "batched tcgen05 INT8 pass alone", "variant": args.variant,
                      "problems": len(shapes), "tiles": tiles, "ms": round(ms, 3),
                      "phases_ms": {"plan_and_split": round(split_ms, 3),
                                    "persistent_kernel": round(kern_ms, 3)},
                      "effective_gflops": round(flops / (ms * 1e-3) / 1e9, 1),
                      "launches": 4}), flush=True)


def run_batched(args):
    """Config 3: 512 independent problems, m, n, k each log-uniform in
    [64, 1024], uniform entries; one graph-captured pass of the batched form
    (autotuned tile shape and schedule) against one ddgemm call per problem.
    value = sum 2 m n k / time of the graph replay."""
    import torch

    from oracle import dd
    from paper_2303_04353_gb300 import _lib, autotune, ops
    from workloads import batched_shapes

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    shapes = [tuple(int(v) for v in sh) for sh in batched_shapes(args.batch_count, seed=0)]
    host, probs = [], []
    for i, (m, n, k) in enumerate(shapes):
        a = gemm_inputs(m, n, k, kind="uniform", seed=1000 + i)
        host.append(a)
        t = [torch.from_numpy(x).to(dev) for x in a]
        probs.append((*t, torch.empty((m, n), dtype=torch.float64, device=dev),
                      torch.empty((m, n), dtype=torch.float64, device=dev)))
    flops = sum(2.0 * m * n * k for m, n, k in shapes)
    if args.variant in ("int8tc", "int8tc8"):
        run_batched_tc_only(args, shapes, probs, flops, stream)
        return
    batch = ops.Batch(probs)
    cfg, tune_ms = autotune.tune(batch, reps=2)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # one ddgemm per problem (three launches each), shared workspace
    ws = ops.alloc_workspace(max(sh[0] for sh in shapes), max(sh[1] for sh in shapes),
                             max(sh[2] for sh in shapes), dev)

    def per_problem():
        for a_hi, a_lo, b_hi, b_lo, c_hi, c_lo in probs:
            ops.ddgemm(a_hi, a_lo, b_hi, b_lo, out=(c_hi, c_lo), workspace=ws, stream=stream)

    per_ms = timed(per_problem, args.steps)
    eager_ms = timed(lambda: batch.run(stream=stream, config=cfg), args.steps)
    side = torch.cuda.Stream(dev)
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side):
        batch.run(stream=torch.cuda.current_stream(), config=cfg)
    sampler = ClockSampler(physical_index(0))
    sampler.start()
    graph_ms = timed(graph.replay, args.steps)
    clocks = sampler.stop()
    # accuracy on sampled entries of a few problems
    worst = 0.0
    for i in range(0, len(shapes), 64):
        a = host[i]
        m, n, _ = shapes[i]
        rng = np.random.default_rng(i)
        rows, cols = rng.integers(0, m, 16), rng.integers(0, n, 16)
        oh, ol = dd.ddgemm_entries(*a, rows, cols)
        ch, cl = probs[i][4].cpu().numpy(), probs[i][5].cpu().numpy()
        absab = np.array([np.abs(a[0][r]) @ np.abs(a[2][:, c]) for r, c in zip(rows, cols)])
        worst = max(worst, float(np.max(np.abs((ch[rows, cols] - oh) + (cl[rows, cols] - ol))
                                        / absab)))
    # the same 512 problems through the batched tcgen05 INT8 forms (graph):
    # seven-bit pieces, and the mma.sync form's eight-bit ones
    def tc_pass(variant):
        tc_probs = [(*p[:4], torch.empty_like(p[4]), torch.empty_like(p[5])) for p in probs]
        tc_batch = ops.Batch(tc_probs, variant=variant)
        tc_graph = torch.cuda.CUDAGraph()
        tc_batch.run(stream=stream)
        torch.cuda.synchronize()
        with torch.cuda.graph(tc_graph, stream=side):
            tc_batch.run(stream=torch.cuda.current_stream())
        ms = timed(tc_graph.replay, args.steps)
        worst_tc = 0.0
        for i in range(0, len(shapes), 64):
            a = host[i]
            m, n, _ = shapes[i]
            rng = np.random.default_rng(i)
            rows, cols = rng.integers(0, m, 16), rng.integers(0, n, 16)
            oh, ol = dd.ddgemm_entries(*a, rows, cols)
            ch, cl = tc_probs[i][4].cpu().numpy(), tc_probs[i][5].cpu().numpy()
            absab = np.array([np.abs(a[0][r]) @ np.abs(a[2][:, c]) for r, c in zip(rows, cols)])
            worst_tc = max(worst_tc, float(np.max(np.abs((ch[rows, cols] - oh) +
                                                          (cl[rows, cols] - ol)) / absab)))
        return ms, worst_tc
    tc_ms, tc_worst = tc_pass(_lib.DDGEMM_VARIANT_INT8_TC)
    tc8_ms, tc8_worst = tc_pass(_lib.DDGEMM_VARIANT_INT8_TC8)
    value = flops / (graph_ms * 1e-3) / 1e9
    peak, peak_src = fp64_peak_rule()
    achieved = 10.0 * flops / (graph_ms * 1e-3) / 1e12
    line = {"metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(graph_ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "batched: 512 problems, m, n, k log-uniform in [64, 1024], "
                                   "hi U[-1,1], one CUDA-graph replay of ddgemm_batched",
                       "sum_2mnk": flops, "tile_order": list(cfg),
                       "l2": "inputs 1.4 GB and panels larger than L2; no flush"},
            "per_problem_launches": {"ms": round(per_ms, 3),
                                     "gflops": round(flops / (per_ms * 1e-3) / 1e9, 3),
                                     "launches": 3 * len(shapes)},
            "batched_eager": {"ms": round(eager_ms, 3),
                              "gflops": round(flops / (eager_ms * 1e-3) / 1e9, 3)},
            "autotune_ms": tune_ms, "max_err_vs_dd_oracle": worst,
            "int8_tc_batched": {"ms": round(tc_ms, 3),
                                "gflops": round(flops / (tc_ms * 1e-3) / 1e9, 3),
                                "launches": 4, "max_err_vs_dd_oracle": tc_worst,
                                "what": "the same problems, batched tcgen05 INT8 form "
                                        "(16 seven-bit pieces), one CUDA-graph replay"},
            "int8_tc8_batched": {"ms": round(tc8_ms, 3),
                                 "gflops": round(flops / (tc8_ms * 1e-3) / 1e9, 3),
                                 "launches": 4, "max_err_vs_dd_oracle": tc8_worst,
                                 "what": "the same problems, batched tcgen05 INT8 form with "
                                         "the mma.sync form's 15 eight-bit pieces"},
            "roofline": {"bound": "tensor", "kernel": "whole batched pass (4 launches)",
                         "achieved": round(achieved, 4), "peak": round(peak, 4),
                         "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "peak_source": peak_src},
            "gpu_launches": 4 * args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_ablation(args):
    """Study of eq. (Gemm16) against eq. (Gemm10): the ten folded products
    (the method), all sixteen products, and ten products with bins 4-6
    dropped, on the same GPU and inputs: max error against the
    double-double oracle on sampled entries, and time.  Study lines, not the
    benchmark line."""
    import torch

    from oracle import dd
    from paper_2303_04353_gb300 import _lib, ops

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    m = n = k = args.sweep_size
    rng = np.random.default_rng(5)
    rows, cols = rng.integers(0, m, 128), rng.integers(0, n, 128)
    for kind in ("uniform", "wide"):
        a = gemm_inputs(m, n, k, kind=kind, seed=0)
        d_in = [torch.from_numpy(x).to(dev) for x in a]
        oh, ol = dd.ddgemm_entries(*a, rows, cols)
        absab = np.array([np.abs(a[0][i]) @ np.abs(a[2][:, j]) for i, j in zip(rows, cols)])
        for name, variant in (("gemm10 (method)", _lib.DDGEMM_VARIANT_FP64),
                              ("gemm16", _lib.DDGEMM_VARIANT_FP64_GEMM16),
                              ("drop bins 4-6", _lib.DDGEMM_VARIANT_FP64_DROP456)):
            out = ops.ddgemm(*d_in, variant=variant)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = ops.ddgemm(*d_in, variant=variant, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            ch, cl = out[0].cpu().numpy(), out[1].cpu().numpy()
            err = np.abs((ch[rows, cols] - oh) + (cl[rows, cols] - ol)) / absab
            print(json.dumps({"study": "Gemm10 vs Gemm16 vs dropped bins", "size": m,
                              "entries": kind, "form": name,
                              "ms": round(e0.elapsed_time(e1), 3),
                              "max_err_rel_absAabsB": float(err.max()),
                              "median_err_rel_absAabsB": float(np.median(err))}), flush=True)


def run_illcond(args):
    """Study after the paper's ill-conditioned experiments: A = Q with
    orthonormal rows, C with entries of magnitude (t, 10t) and one 1 per
    column, B = Q^T C (workloads/illcond.py).  Max element-wise relative
    error over sampled entries against exact rationals, for the FP64x2
    triple loop (the CPU oracle) and the two CUDA forms; study lines, not
    the benchmark line."""
    from fractions import Fraction

    import torch

    from oracle import dd
    from paper_2303_04353_gb300 import _lib, ops
    from workloads.illcond import illcond_inputs

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import exact  # exact rational dot products (test helper)

    dev = torch.device("cuda", 0)
    for n in (64, 128, 256, 512):
        for t in (1e-9, 1e-14, 1e-19):
            a = illcond_inputs(n, t, seed=n)[:4]
            rng = np.random.default_rng(n)
            rows, cols = rng.integers(0, n, 256), rng.integers(0, n, 256)
            refs = [exact.exact_dot(a[0][i], a[1][i], a[2][:, j], a[3][:, j])
                    for i, j in zip(rows, cols)]

            def worst(c_hi, c_lo):
                return max(exact.err_vs_exact(c_hi[i, j], c_lo[i, j], r)
                           / abs(float(Fraction(r, 1 << (2 * exact.SHIFT))))
                           for i, j, r in zip(rows, cols, refs))
            o_hi, o_lo = dd.ddgemm_entries(*a, rows, cols)
            e_dd = max(exact.err_vs_exact(h, l, r) / abs(float(Fraction(r, 1 << (2 * exact.SHIFT))))
                       for h, l, r in zip(o_hi, o_lo, refs))
            d_in = [torch.from_numpy(x).to(dev) for x in a]
            res = {}
            for name, variant in (("cascade fp64", _lib.DDGEMM_VARIANT_FP64),
                                  ("cascade int8 s=15", _lib.DDGEMM_VARIANT_INT8),
                                  ("cascade int8 tcgen05 s=16", _lib.DDGEMM_VARIANT_INT8_TC),
                                  ("cascade int8 tcgen05 eight-bit s=15",
                                   _lib.DDGEMM_VARIANT_INT8_TC8)):
                c = ops.ddgemm(*d_in, variant=variant)
                torch.cuda.synchronize()
                res[name] = worst(c[0].cpu().numpy(), c[1].cpu().numpy())
            print(json.dumps({"study": "ill-conditioned products", "n": n, "t": t,
                              "max_rel_err_fp64x2_triple_loop": e_dd,
                              **{f"max_rel_err_{k}": v for k, v in res.items()},
                              "ratio_fp64x2_over_cascade_fp64": e_dd / max(res["cascade fp64"],
                                                                            1e-300)}),
                  flush=True)


def run_splitk(args):
    """Split-k study: effective GFLOP/s of the FP64 form with no split,
    the automatic choice and forced group counts, on shapes whose grids of
    64 x 64 tiles fill the 152 SMs in few waves.  Study lines, not the
    benchmark line."""
    import torch

    from paper_2303_04353_gb300 import ops

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    shapes = [(8192, 1024, 4096), (3000, 3000, 3000), (2048, 2048, 2048), (1024, 1024, 8192),
              (1000, 1000, 1000), (512, 512, 4096), (256, 256, 16384)]
    for m, n, k in shapes:
        d_in = [torch.from_numpy(x).to(dev) for x in gemm_inputs(m, n, k, kind="uniform", seed=1)]
        out = (torch.empty((m, n), dtype=torch.float64, device=dev),
               torch.empty((m, n), dtype=torch.float64, device=dev))
        for split_k in (1, 0, 2, 4, 8, 16):
            ws = ops.alloc_workspace(m, n, k, dev, split_k=split_k)
            for _ in range(3):
                ops.ddgemm(*d_in, out=out, workspace=ws, split_k=split_k)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = 5
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                ops.ddgemm(*d_in, out=out, workspace=ws, split_k=split_k)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            print(json.dumps({"study": "split-k", "m": m, "n": n, "k": k,
                              "split_k": split_k if split_k else "auto",
                              "groups": ops.split_groups(m, n, k, dev, ws.numel(),
                                                         split_k=split_k),
                              "ms": round(ms, 3),
                              "effective_gflops": round(2.0 * m * n * k / (ms * 1e-3) / 1e9, 2)}),
                  flush=True)
            del ws


def run_sweep(args):
    """Config-2 study: error and throughput of the FP64 form and the INT8
    form as the exponent spread of the entries grows (hi = +-2^u,
    u ~ U[-S/2, S/2]), at 2048^3.  One JSON line per (spread, form); these
    are study lines, not the benchmark line."""
    import torch

    from oracle import dd
    from paper_2303_04353_gb300 import _lib, ops

    dev = torch.device("cuda", 0)
    m = n = k = args.sweep_size
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(3)
    rows, cols = rng.integers(0, m, 128), rng.integers(0, n, 128)
    forms = [("fp64", _lib.DDGEMM_VARIANT_FP64, 0)] + [
        (f"int8 s={s8}", _lib.DDGEMM_VARIANT_INT8, s8) for s8 in (13, 14, 15)] + [
        (f"int8 tcgen05 s={s8}", _lib.DDGEMM_VARIANT_INT8_TC, s8) for s8 in (14, 15, 16)] + [
        (f"int8 tcgen05 eight-bit s={s8}", _lib.DDGEMM_VARIANT_INT8_TC8, s8) for s8 in (14, 15)]
    for spread in range(0, 61, 10):
        a_hi, a_lo, b_hi, b_lo = gemm_inputs(m, n, k, kind="wide", seed=0, spread=float(spread))
        d_in = [torch.from_numpy(x).to(dev) for x in (a_hi, a_lo, b_hi, b_lo)]
        oh, ol = dd.ddgemm_entries(a_hi, a_lo, b_hi, b_lo, rows, cols)
        absab = np.array([np.abs(a_hi[i]) @ np.abs(b_hi[:, j]) for i, j in zip(rows, cols)])
        for name, variant, s8 in forms:
            ws = ops.alloc_workspace(m, n, k, dev, variant, s8)
            out = (torch.empty((m, n), dtype=torch.float64, device=dev),
                   torch.empty((m, n), dtype=torch.float64, device=dev))
            for _ in range(3):
                ops.ddgemm(*d_in, out=out, workspace=ws, variant=variant, int8_slices=s8)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = 1 if variant == _lib.DDGEMM_VARIANT_FP64 else 5
            e0.record(stream)
            for _ in range(reps):
                ops.ddgemm(*d_in, out=out, workspace=ws, variant=variant, int8_slices=s8)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            ch, cl = out[0].cpu().numpy(), out[1].cpu().numpy()
            err = np.abs((ch[rows, cols] - oh) + (cl[rows, cols] - ol)) / absab
            print(json.dumps({"study": "exponent-spread sweep", "size": m, "spread_octaves": spread,
                              "form": name, "ms": round(ms, 3),
                              "effective_gflops": round(2.0 * m * n * k / (ms * 1e-3) / 1e9, 2),
                              "max_err_rel_absAabsB": float(err.max()),
                              "median_err_rel_absAabsB": float(np.median(err))}), flush=True)


def make_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched"], default="4096")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the records of the other workloads in the default line")
    ap.add_argument("--no-int8-form", action="store_true",
                    help="skip the INT8 form's entry in the FP64 line")
    ap.add_argument("--variant", choices=("fp64", "int8", "int8tc", "int8tc8"), default="fp64",
                    help="fp64: the ten FP64 products (default); int8: the INT8 form on "
                         "mma.sync s8; int8tc: the INT8 form on the tcgen05 tensor cores; "
                         "int8tc8: the same with the mma.sync form's eight-bit pieces")
    ap.add_argument("--int8-slices", type=int, default=0,
                    help="pieces of the INT8 forms; 0: 15 eight-bit (mma.sync) or 16 "
                         "seven-bit (tcgen05)")
    ap.add_argument("--sweep", action="store_true",
                    help="exponent-spread study of both forms instead of the benchmark line")
    ap.add_argument("--sweep-size", type=int, default=2048)
    ap.add_argument("--batch-count", type=int, default=512,
                    help="problems of the batched workload (512; fewer for a small profile)")
    ap.add_argument("--illcond", action="store_true",
                    help="ill-conditioned accuracy study instead of the benchmark line")
    ap.add_argument("--ablation", action="store_true",
                    help="Gemm10 / Gemm16 / dropped-bins accuracy study instead of the line")
    ap.add_argument("--splitk", action="store_true",
                    help="split-k study on grids of few waves instead of the line")
    return ap


def main():
    args = make_parser().parse_args()
    if args.splitk:
        run_splitk(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.ablation:
        run_ablation(args)
        return
    if args.illcond:
        run_illcond(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.warmup < 3:
        raise SystemExit("bench.py: at least 3 warm-up steps")
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
