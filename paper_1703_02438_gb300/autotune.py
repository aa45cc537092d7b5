"""Autotuner for batched compression: picks the number of concurrent lanes and the grid share
(each variable's kernels sized for 1/grid_share of the GPU) by timing the actual batch.

The best setting is cached per (GPU name, batch signature) in _lib/autotune.json next to the
built library, so later runs of a batch with the same shape reuse it without timing again.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import numarck as N

CANDIDATES = ((1, 1), (2, 2), (4, 2), (4, 4), (8, 4), (8, 8), (16, 8), (16, 16), (32, 16))
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")


def signature(batch: N.Batch) -> str:
    """Shape of a batch: count, dtype mix and size buckets (log2 of element counts)."""
    sizes = sorted(int(math.log2(max(1, p.numel()))) for p, _ in batch.pairs)
    f64 = sum(p.dtype == torch.float64 for p, _ in batch.pairs)
    return f"n{batch.count}-f64{f64}-" + ",".join(str(s) for s in sizes)


def _load():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _time(batch: N.Batch, reps: int) -> float:
    batch.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        batch.run()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune(batch: N.Batch, reps: int = 2, candidates=CANDIDATES, use_cache: bool = True):
    """Sets batch.lanes / batch.grid_share to the fastest candidate; returns
    (lanes, grid_share, {candidate: ms})."""
    key = torch.cuda.get_device_name() + "|" + signature(batch)
    cache = _load() if use_cache else {}
    if key in cache:
        lanes, share = cache[key]["best"]
        batch.set_lanes(lanes, share)
        return lanes, share, cache[key]["ms"]
    timings = {}
    for lanes, share in candidates:
        batch.set_lanes(lanes, share)
        timings[f"{lanes}x{share}"] = _time(batch, reps)
    best = min(timings, key=timings.get)
    lanes, share = (int(v) for v in best.split("x"))
    batch.set_lanes(lanes, share)
    cache[key] = {"best": [lanes, share], "ms": timings}
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return lanes, share, timings
