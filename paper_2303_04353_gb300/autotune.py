"""Autotuner for the batched cascade: picks the persistent kernel's schedule
by timing every candidate on the actual batch with CUDA events, and caches
the choice in a JSON file keyed by the batch's form and shape list.

FP64 form: C tile 64x64, 32x64, 64x32 or 32x32 x the order in which CTAs
take tiles (given, longest k first).  Small problems waste less of a
32-wide tile; large ones keep more warps per CTA busy with 64-wide tiles;
longest-k-first shortens the tail of the persistent schedule.

tcgen05 forms (128 x 16 tiles): the problem order (given, longest k first),
each problem's tile grid (over C, or over C^T when that needs fewer tiles),
the order of a k-step's MMAs over the digit planes (interleaved narrow and
wide, or ascending: the slice schedule) and the row tiles per group of a
problem's tile order (1 or 4).

Results do not depend on the choice: every configuration computes each
problem bit-identically."""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import _lib
from .build import OUT_DIR

CANDIDATES = [(t, o) for t in (_lib.DDGEMM_TILE_64x64, _lib.DDGEMM_TILE_32x64,
                               _lib.DDGEMM_TILE_64x32, _lib.DDGEMM_TILE_32x32)
              for o in (_lib.DDGEMM_ORDER_GIVEN, _lib.DDGEMM_ORDER_LONGEST_K_FIRST)]
# (tile (unused), order, orient, planes, row_group)
TC_CANDIDATES = [(0, o, r, p, g)
                 for o in (_lib.DDGEMM_ORDER_GIVEN, _lib.DDGEMM_ORDER_LONGEST_K_FIRST)
                 for r in (_lib.DDGEMM_ORIENT_FEWER_TILES, _lib.DDGEMM_ORIENT_GIVEN)
                 for p in (_lib.DDGEMM_PLANES_INTERLEAVED, _lib.DDGEMM_PLANES_ASCENDING)
                 for g in (1, 4)]
TC_VARIANTS = (_lib.DDGEMM_VARIANT_INT8_TC, _lib.DDGEMM_VARIANT_INT8_TC8)


def cache_path() -> str:
    return os.environ.get("DDGEMM_AUTOTUNE_CACHE", os.path.join(OUT_DIR, "autotune.json"))


def signature(shapes, variant: int = _lib.DDGEMM_VARIANT_FP64, slices: int = 0) -> str:
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    h = hashlib.sha1(json.dumps([dev, variant, slices, sorted(map(list, shapes))]).encode())
    return h.hexdigest()[:20]


def candidates(variant: int = _lib.DDGEMM_VARIANT_FP64):
    """The configurations the tuner times for a batch of this form."""
    return TC_CANDIDATES if variant in TC_VARIANTS else CANDIDATES


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(db: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_config(batch, config, reps: int = 2, stream=None) -> float:
    """Milliseconds per run of the batch with this config (after one warm-up)."""
    stream = stream or torch.cuda.current_stream()
    batch.run(stream=stream, config=config)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        batch.run(stream=stream, config=config)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(batch, reps: int = 2, use_cache: bool = True):
    """Best configuration for this batch's form and shapes; returns (config
    tuple, timings in ms by candidate)."""
    variant = getattr(batch, "variant", _lib.DDGEMM_VARIANT_FP64)
    key = signature(batch.shapes, variant, getattr(batch, "int8_slices", 0))
    db = _load() if use_cache else {}
    if key in db:
        return tuple(db[key]["config"]), db[key].get("ms", {})
    timings = {",".join(map(str, c)): time_config(batch, c, reps) for c in candidates(variant)}
    best = min(timings, key=timings.get)
    cfg = tuple(int(x) for x in best.split(","))
    if use_cache:
        db[key] = {"config": list(cfg), "ms": timings, "problems": batch.count,
                   "variant": variant}
        _save(db)
    return cfg, timings
