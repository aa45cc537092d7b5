"""Autotuner for batched compression: times the actual batch (compression and decompression)
under every candidate configuration and keeps the fastest.

Two families of configurations give byte-identical results:
  * lanes (numarck_compress_batch): `lanes` variables in flight on forked streams, each
    variable's kernels sized for 1/grid_share of the GPU;
  * fused (numarck_compress_batch_fused): one launch per phase over a work list of variables;
    the shape knobs are the CTA size of the ratio/histogram pass (512 or 1024 threads), the
    warps per CTA of the incompressible copy (4 or 8), how many warps share a 4096-element tile
    in the decode (2^decode_seg_log2), and how many work lists (groups) run on how many streams
    (each launch sized for 1/streams of the GPU).

The best setting is cached per (GPU name, batch signature) in _lib/autotune.json next to the
built library, so later runs of a batch with the same shape reuse it without timing again.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import numarck as N

LANE_CANDIDATES = ((1, 1), (2, 2), (4, 2), (4, 4), (8, 4), (8, 8), (16, 8), (16, 16), (32, 16))
FUSED_CANDIDATES = tuple((k1, xw, sl, g, st) for k1 in (512, 1024) for xw, sl in ((8, 0), (4, 1))
                         for g, st in ((1, 1), (4, 2), (8, 2), (8, 4), (16, 4)))
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


def _time(batch: N.Batch, prevs, outs, reps: int) -> float:
    """Mean ms of one compression of the batch plus one decompression of its blobs."""
    def once():
        batch.run()
        batch.decompress(prevs, outs=outs)
    once()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        once()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _apply(batch: N.Batch, key: str):
    kind, rest = key.split(":")
    vals = [int(v) for v in rest.split("x")]
    if kind == "lanes":
        batch.set_lanes(*vals)
    else:
        batch.set_fused(tuple(vals))


def tune(batch: N.Batch, reps: int = 2, lane_candidates=LANE_CANDIDATES,
         fused_candidates=FUSED_CANDIDATES, use_cache: bool = True):
    """Sets the batch to the fastest candidate; returns (best key, {key: ms}). Keys are
    "lanes:<lanes>x<grid_share>" and
    "fused:<k1_threads>x<exact_warps>x<decode_seg_log2>x<groups>x<streams>"."""
    key = torch.cuda.get_device_name() + "|" + signature(batch)
    cache = _load() if use_cache else {}
    if key in cache:
        _apply(batch, cache[key]["best"])
        return cache[key]["best"], cache[key]["ms"]
    prevs = [p for p, _ in batch.pairs]
    outs = [torch.empty_like(p) for p in prevs]
    timings = {}
    for lanes, share in lane_candidates:
        k = f"lanes:{lanes}x{share}"
        _apply(batch, k)
        timings[k] = _time(batch, prevs, outs, reps)
    for cand in fused_candidates:
        k = "fused:" + "x".join(str(v) for v in cand)
        _apply(batch, k)
        timings[k] = _time(batch, prevs, outs, reps)
    best = min(timings, key=timings.get)
    _apply(batch, best)
    cache[key] = {"best": best, "ms": timings}
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return best, timings
