"""Autotuner for the batched cascade: picks the persistent kernel's C tile
shape and the order in which its CTAs take tiles, by timing every
candidate on the actual batch with CUDA events, and caches the choice in a
JSON file keyed by the batch's shape list.

Candidates: tiles 64x64, 32x64, 64x32, 32x32 x orders {given, longest k
first}.  Small problems waste less of a 32-wide tile; large ones keep more
warps per CTA busy with 64-wide tiles; longest-k-first shortens the tail
of the persistent schedule.  Results do not depend on the choice (every
configuration computes each problem bit-identically)."""
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


def cache_path() -> str:
    return os.environ.get("DDGEMM_AUTOTUNE_CACHE", os.path.join(OUT_DIR, "autotune.json"))


def signature(shapes) -> str:
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    h = hashlib.sha1(json.dumps([dev, sorted(map(list, shapes))]).encode()).hexdigest()
    return h[:20]


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
    """Best (tile, order) for this batch; returns (config tuple, timings)."""
    key = signature(batch.shapes)
    db = _load() if use_cache else {}
    if key in db:
        return tuple(db[key]["config"]), db[key].get("ms", {})
    timings = {f"{t},{o}": time_config(batch, (t, o), reps) for t, o in CANDIDATES}
    best = min(timings, key=timings.get)
    cfg = tuple(int(x) for x in best.split(","))
    if use_cache:
        db[key] = {"config": list(cfg), "ms": timings, "problems": batch.count}
        _save(db)
    return cfg, timings
