#!/usr/bin/env python3
"""NUMARCK compress + decompress throughput on GB300.

Workload (default, the configuration the headline metric is quoted on): a FLASH-like 3-D float64
density field of 1024^3 cells (8 GiB per timestep), 4 consecutive timesteps compressed pairwise
in a closed loop (prev = previous reconstruction), for every E in {1e-3, 1e-4} and B in {8, 10}.
One step = those 12 (pair, E, B) compressions and their 12 decompressions. Inputs are 8 GiB
arrays, far larger than the 129 MB L2, so no L2 flush is needed between iterations.

Each (E, B) chain runs through the public API as a user of a chain of timesteps would: timestep
1 compressed against timestep 0 (numarck_compress), timesteps 2 and 3 by the chained step
(numarck_decompress_compress: the previous blob decompressed and the new timestep compressed
against that reconstruction, with the decompression and the first compression pass fused in one
kernel), and the last blob decompressed (numarck_decompress). Every compression and
decompression of the step is done in full; --no-fuse runs them as 12 separate pairs instead.

value = input bytes (n * 8 per pair, once for compression and once for decompression counted as
one pass of the variable) / (compress time + decompress time), i.e. n*L / (t_c + t_d) summed
over the step, in GB/s of the uncompressed variable, on the device with CUDA events.

--impl reference times the CPU oracle (plain numpy, one host core) on a bounded sample of the
same workload; it is the reference arm of this comparison (the paper has no GPU code).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
import zlib
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

COMBOS = [(1e-3, 8), (1e-3, 10), (1e-4, 8), (1e-4, 10)]
METRIC = "compress+decompress input GB/s (and % of HBM peak) on 1 GB300, bit-exact vs oracle"
WORKLOAD = ("FLASH-like 3-D float64 field 1024^3 (8 GiB/step), 4 timesteps, 3 closed-loop pairs "
            "x E{1e-3,1e-4} x B{8,10}")


def workload_label(side: int, f32: bool) -> str:
    """The workload string of a run (the headline workload is side 1024, float64)."""
    L = 4 if f32 else 8
    gib = side ** 3 * L / 2 ** 30
    size = f"{gib:.0f} GiB" if gib >= 1 else f"{side ** 3 * L / 2 ** 20:.0f} MiB"
    return (f"FLASH-like 3-D {'float32 (cast)' if f32 else 'float64'} field {side}^3 "
            f"({size}/step), 4 timesteps, 3 closed-loop pairs x E{{1e-3,1e-4}} x B{{8,10}}")
KERNEL_FILES = {"k3_assign": ["k_assign.cu", "common.cuh"],
                "k3_exact": ["k_assign.cu", "common.cuh"],
                "k1_hist": ["k_hist.cu", "k1.cuh", "common.cuh"],
                "k4_decode": ["k_decode.cu", "k4.cuh", "common.cuh"],
                "k41_step": ["k_step.cu", "k1.cuh", "k4.cuh", "common.cuh"]}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="numarck", choices=["numarck", "reference"])
    ap.add_argument("--side", type=int, default=1024, help="grid side (1024 = the full workload)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1 << 24,
                    help="elements of the oracle's bounded sample")
    ap.add_argument("--f32", action="store_true",
                    help="the same series as float32 (4 bytes per element)")
    ap.add_argument("--no-fuse", action="store_true",
                    help="every pair as a separate compression and decompression (no chained "
                         "step that fuses a decompression with the next histogram pass)")
    ap.add_argument("--auto-b", action="store_true",
                    help="choose B per pair from the histogram (Eqs. 5-6) instead of B = 8, 10")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--workload", default="flash",
                    choices=["flash", "batched", "served", "zindex", "climate"],
                    help="flash: the headline 1024^3 series; batched: 256 mixed variables, "
                         "per-variable launches vs one graph-captured batch; climate: 120 "
                         "CMIP-like float32 months chained, plain launches vs one CUDA graph")
    ap.add_argument("--batch-count", type=int, default=256)
    return ap.parse_args()


# ----------------------------------------------------------------------------------------
def _rank_world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def _init_dist(world):
    import torch
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return dist if world > 1 else None


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index),
                                       f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(rows),
                "reasons": sorted(reasons)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _kernel_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_FILES[kernel]:
        with open(os.path.join(ROOT, "paper_1703_02438_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str, side: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        e = tr[kernel]
        if e.get("source_sha") != _kernel_hash(kernel):
            return None
        return float(e["bytes_per_launch_full"]) * (side ** 3) / float(e["n_full"])
    except (OSError, KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------------------
def cpu_oracle_sample(pair, sample: int):
    """The oracle as it stands, on `sample` contiguous elements of pair (x1 -> x2) at E=1e-3,
    B=8: compress + decompress; returns (GB/s of input, seconds, description)."""
    from oracle import numarck_oracle as O
    p, x = pair
    n = min(sample, p.numel())
    lo = (p.numel() - n) // 2
    ps = p[lo: lo + n].cpu().numpy().copy()
    xs = x[lo: lo + n].cpu().numpy().copy()
    t0 = time.perf_counter()
    blob = O.compress(ps, xs, 1e-3, 8).to_bytes()
    t1 = time.perf_counter()
    O.decompress(blob, ps)
    t2 = time.perf_counter()
    gbs = n * ps.itemsize / (t2 - t0) / 1e9
    return gbs, t2 - t0, (f"{n} contiguous float64 elements (middle of timestep pair 1->2), "
                          f"E=1e-3 B=8, compress {t1 - t0:.2f}s + decompress {t2 - t1:.2f}s")


def cpu_parallel_pair(pair, gpu_blob=None):
    """The all-cores CPU baseline (oracle/numarck_cpu.c, POSIX threads on every host core this
    process may use) on the whole pair at E=1e-3, B=8: compress + decompress; returns a dict for
    the bench line. With gpu_blob (the library's blob of the same pair), also whether the two
    blobs are byte-identical."""
    from oracle import cpu_parallel as C
    C.build()
    p = pair[0].cpu().numpy()
    x = pair[1].cpu().numpy()
    cores = C.threads_available()
    t0 = time.perf_counter()
    blob = C.compress(p, x, 1e-3, 8, threads=cores)
    t1 = time.perf_counter()
    C.decompress(blob, p, threads=cores)
    t2 = time.perf_counter()
    out = {"value": p.size * p.itemsize / (t2 - t0) / 1e9, "unit": "GB/s", "cores": cores,
           "kind": "parallel C (POSIX threads; chunked ratio/bin pass, per-thread histograms, "
                   "tiles in parallel)",
           "sample": f"the whole timestep pair 1->2 ({p.size} float64 elements), E=1e-3 B=8, "
                     f"compress {t1 - t0:.2f}s + decompress {t2 - t1:.2f}s",
           "seconds": round(t2 - t0, 2)}
    if gpu_blob is not None:
        out["blob_equals_gpu"] = blob == gpu_blob
    return out


def run_reference(args):
    rank, world = _rank_world()
    if rank != 0:
        return
    import numpy as np
    import torch
    from paper_1703_02438_gb300 import synth
    side = 256       # bounded sample of the same workload: a 256^3 sub-volume recipe
    series = synth.flash_series(side=side, steps=3, device="cpu")
    p, x = series[1], series[2]
    times = []
    for i in range(args.warmup + args.steps):
        gbs, sec, desc = cpu_oracle_sample((p, x), args.cpu_sample)
        if i >= args.warmup:
            times.append(sec)
    n = min(args.cpu_sample, p.numel())
    value = n * 8 / statistics.mean(times) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------
def run_batched(args):
    """256 variables (sizes log-uniform in [1e4, 2e8], float32/float64, per-variable E and B):
    per-variable launches on one stream vs the autotuned lane batch and the autotuned fused
    batch (one launch per phase over all variables), each captured in a CUDA graph."""
    import torch
    from paper_1703_02438_gb300 import autotune
    from paper_1703_02438_gb300 import build as nbuild
    from paper_1703_02438_gb300 import numarck as N
    from paper_1703_02438_gb300 import synth
    nbuild.build()
    dev = torch.device("cuda", 0)
    specs = synth.batch_specs(count=args.batch_count)
    pairs = []
    for i, (n, dtype, E, B, scale) in enumerate(specs):
        pairs.append(synth.plain_pair(n, dtype=dtype, seed=synth.seed_for(3, 1000 + i),
                                      scale=scale, device=dev))
    torch.cuda.synchronize()
    nbytes = sum(p.numel() * p.element_size() for p, _ in pairs)
    batch = N.Batch(pairs, [(E, B) for _, _, E, B, _ in specs])
    prevs = [p for p, _ in pairs]
    outs = [torch.empty_like(p) for p in prevs]
    ws = N.Workspace(dev)
    stream = torch.cuda.current_stream()

    def plain_compress():
        for (p, x), (_, _, E, B, _), blob in zip(pairs, specs, batch.blobs):
            N.compress(p, x, E, B, blob=blob, workspace=ws)

    def plain_decompress():
        for p, blob, o in zip(prevs, batch.blobs, outs):
            N.decompress(blob, p, out=o)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    reps = max(1, args.steps)
    for _ in range(args.warmup):
        plain_compress()
        plain_decompress()
    t_pc = timed(plain_compress, reps)
    t_pd = timed(plain_decompress, reps)
    best, tune_ms = autotune.tune(batch, reps=1, use_cache=False)

    def graphed(key):
        """Compression and decompression graphs of the batch in configuration `key`."""
        kind, rest = key.split(":")
        vals = [int(v) for v in rest.split("x")]
        if kind == "lanes":
            batch.set_lanes(*vals)
        else:
            batch.set_fused(tuple(vals))
        batch.run()
        batch.decompress(prevs, outs=outs)
        torch.cuda.synchronize()
        gc, gd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            with torch.cuda.graph(gc, stream=cs):
                batch.run()
            with torch.cuda.graph(gd, stream=cs):
                batch.decompress(prevs, outs=outs)
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            gc.replay()
            gd.replay()
        t_c, t_d = timed(gc.replay, reps), timed(gd.replay, reps)
        return {"config": key, "compress_ms": t_c, "decompress_ms": t_d,
                "value": nbytes / ((t_c + t_d) / 1e3) / 1e9,
                "compress_gbs": nbytes / (t_c / 1e3) / 1e9,
                "decompress_gbs": nbytes / (t_d / 1e3) / 1e9}

    best_of = {kind: min((k for k in tune_ms if k.startswith(kind)), key=tune_ms.get)
               for kind in ("lanes", "fused")}
    res = {kind: graphed(k) for kind, k in best_of.items()}
    # the fused batch's output equals the single calls (checked by the tests); here a spot check
    # that the timed configuration produced complete blobs
    for b in batch.blobs[:4]:
        N.blob_size(N.header_bytes(b))
    top = max(res.values(), key=lambda r: r["value"])
    sizes = [n for n, *_ in specs]
    line = {"metric": "batched compress+decompress input GB/s (graph-captured batch vs "
                      "per-variable launches)",
            "value": top["value"], "unit": "GB/s", "n_gpus": 1,
            "steps": reps, "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"{len(specs)} variables, n log-uniform [1e4, 2e8] "
                                   f"(total {sum(sizes)} elements, {nbytes / 1e9:.1f} GB), "
                                   "float32/float64 50/50, E in {1e-2,1e-3,1e-4}, B in {6,8,10}",
                       "best": top["config"]},
            "fused": res["fused"], "lanes": res["lanes"],
            "per_variable": {"compress_ms": t_pc, "decompress_ms": t_pd,
                             "value": nbytes / ((t_pc + t_pd) / 1e3) / 1e9,
                             "compress_gbs": nbytes / (t_pc / 1e3) / 1e9,
                             "decompress_gbs": nbytes / (t_pd / 1e3) / 1e9},
            "speedup_vs_per_variable": (t_pc + t_pd) / (top["compress_ms"] + top["decompress_ms"]),
            "fused_vs_lanes": res["lanes"]["value"] and res["fused"]["value"] / res["lanes"]["value"],
            "autotune_ms": tune_ms}
    print(json.dumps(line), flush=True)


def run_climate(args):
    """CMIP-like 2-D float32 fields (3600 x 1800, 6.48 M points, 25.9 MB per month), 120 monthly
    fields chained at E = 1e-3, B = 8: month 1 compressed against month 0, months 2..119 by the
    chained step, the last blob decompressed (119 compressions + 119 decompressions). All months
    are resident (3.1 GB, > L2): each step's new month comes from HBM, while its prev (the
    reconstruction just made) is usually still in L2, as in any chain of fields this size.
    A field this small takes microseconds per kernel, so the chain is timed as plain launches on
    one stream and as one CUDA graph holding every launch of the chain."""
    import torch
    from paper_1703_02438_gb300 import build as nbuild
    from paper_1703_02438_gb300 import numarck as N
    from paper_1703_02438_gb300 import synth
    nbuild.build()
    dev = torch.device("cuda", 0)
    months = [f for _, f in synth.climate_series(steps=120, device=dev)]
    n = months[0].numel()
    E, B = 1e-3, 8
    params = N.make_params(torch.float32, B, E)
    bound = N.compress_bound(n, params)
    blobs = [torch.empty(bound, dtype=torch.uint8, device=dev) for _ in range(2)]
    recs = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = N.Workspace(dev)
    ws.get(N.workspace_bytes(n, params))
    stream = torch.cuda.current_stream()

    def chain():
        N.compress(months[0], months[1], E, B, blob=blobs[0], workspace=ws)
        prev = months[0]
        for t in range(2, len(months)):
            out = recs[t % 2]
            N.decompress_compress(blobs[t % 2], prev, months[t], E, B, out=out,
                                  next_blob=blobs[(t + 1) % 2], workspace=ws, status=status)
            prev = out
        N.decompress(blobs[len(months) % 2], prev, out=recs[len(months) % 2], status=status)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    for _ in range(args.warmup):
        chain()
    reps = max(1, args.steps)
    clocks = Clocks(0)
    t_plain = timed(chain, reps)
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    cs.wait_stream(stream)
    with torch.cuda.stream(cs):
        with torch.cuda.graph(g, stream=cs):
            chain()
    torch.cuda.synchronize()
    t_graph = timed(g.replay, reps)
    clk = clocks.stop()
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {int(status.item())}")
    pairs = len(months) - 1
    nbytes = pairs * n * 4
    hdr = N.parse_header(N.header_bytes(blobs[len(months) % 2]))
    line = {"metric": "chained compress+decompress input GB/s, CMIP-like float32 fields",
            "value": nbytes / (t_graph / 1e3) / 1e9, "unit": "GB/s", "n_gpus": 1,
            "steps": reps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "CMIP-like 3600 x 1800 float32 monthly fields, 120 months "
                                   "(119 chained pairs), 3% ocean mask = 0, E = 1e-3, B = 8",
                       "n": n, "pairs_per_step": pairs,
                       "l2": "3.1 GB of months resident: each new month read from HBM"},
            "graph": {"ms_per_chain": t_graph, "us_per_pair": 1e3 * t_graph / pairs,
                      "gbs": nbytes / (t_graph / 1e3) / 1e9},
            "plain_launches": {"ms_per_chain": t_plain, "us_per_pair": 1e3 * t_plain / pairs,
                               "gbs": nbytes / (t_plain / 1e3) / 1e9},
            "gpu_launches_per_chain": 6 + (pairs - 1) * 6 + 1,
            "alpha_last": hdr["n_inc"] / n, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_zindex(args):
    """Lossless index compression (§IV.C) on the FLASH-like pair (timesteps 1 -> 2) at each
    (E, B): deflate throughput (raw index bytes / time) and ratio, full inflate, and a partial
    decompression of 1% of the points (inflate its sub-blocks + range decode) against the whole
    decompression."""
    import torch
    from paper_1703_02438_gb300 import build as nbuild
    from paper_1703_02438_gb300 import numarck as N
    from paper_1703_02438_gb300 import synth
    nbuild.build()
    dev = torch.device("cuda", 0)
    side = args.side
    n = side ** 3
    xs = synth.flash_series(side=side, steps=3, device=dev, seed=synth.seed_for(1, 0))
    p, x = xs[1], xs[2]
    del xs
    stream = torch.cuda.current_stream()

    def timed(fn, reps=5, warm=2):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    rows = []
    rng = np.random.default_rng(7)
    for E, B in ((1e-3, 8), (1e-4, 10)):
        blob = N.compress(p, x, E, B)
        hb = N.header_bytes(blob)
        h = N.parse_header(hb)
        raw = sum(((min(n, (q + 1) * h["epb"]) - q * h["epb"]) * B + 7) // 8
                  for q in range(h["nblocks"]))
        zbuf = torch.empty(N.lib().numarck_zindex_bound(hb), dtype=torch.uint8, device=dev)
        zws = torch.empty(N.lib().numarck_zindex_workspace_bytes(hb), dtype=torch.uint8, device=dev)
        t_def = timed(lambda: N.deflate_index(blob, hb, zindex=zbuf, workspace=zws))
        zh = N.zindex_header(zbuf)
        zb = zh["total_bytes"]
        copy = blob.clone()
        t_inf = timed(lambda: N.inflate_index(zbuf, zb, hb, copy))
        out = torch.empty_like(p)
        t_full = timed(lambda: N.decompress(blob, p, header=hb, out=out))
        cnt = n // 100
        start = int(rng.integers(0, n - cnt))
        seg = torch.empty(cnt, dtype=torch.float64, device=dev)

        def partial():
            N.inflate_index(zbuf, zb, hb, copy, start=start, count=cnt)
            N.decompress_range(copy, p[start: start + cnt], start, cnt, header=hb, out=seg)
        t_part = timed(partial)
        # the host's zlib (level 6, every index block as one stream) on the same blocks
        index_host = blob[h["off_index"]: h["off_exact"]].cpu().numpy().tobytes()
        blocks = [index_host[q * h["block_stride"]:
                             q * h["block_stride"] + ((min(n, (q + 1) * h["epb"]) - q * h["epb"])
                                                      * B + 7) // 8]
                  for q in range(h["nblocks"])]
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max(1, len(os.sched_getaffinity(0)))) as ex:
            zl = sum(ex.map(lambda b: len(zlib.compress(b, 6)), blocks))
        t_zl = time.perf_counter() - t0
        del index_host, blocks
        rows.append({"E": E, "B": B, "index_bytes": raw, "zindex_bytes": zb,
                     "host_zlib6_bytes": zl, "host_zlib6_ratio": raw / zl,
                     "host_zlib6_seconds": round(t_zl, 2),
                     "index_ratio": raw / zb, "deflate_ms": t_def,
                     "deflate_gbs": raw / (t_def / 1e3) / 1e9, "inflate_all_ms": t_inf,
                     "inflate_gbs": raw / (t_inf / 1e3) / 1e9,
                     "decompress_all_ms": t_full, "partial_1pct_ms": t_part,
                     "blob_bytes": N.blob_size(hb),
                     "blob_ratio_raw": n * 8 / N.blob_size(hb),
                     "blob_ratio_deflated": n * 8 / (N.blob_size(hb)
                                                     - (h["off_exact"] - h["off_index"]) + zb)})
    line = {"metric": "lossless index compression (zlib streams): deflate/inflate GB/s, ratio, "
                      "partial decode", "value": rows[0]["deflate_gbs"], "unit": "GB/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"FLASH-like float64 {side}^3 pair, E/B in (1e-3, 8), (1e-4, 10)"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_served(args):
    """The served form: 32 series (sizes log-uniform in [1 MB, 2 GB] of float32/float64 data,
    50/50), Poisson arrivals at --serve-rate requests/s for --serve-seconds; 80% compressions of
    the next timestep, 20% decompressions of the latest one (half whole, half a 1-10% range at
    a random start). Reports latency percentiles from the server's own timestamps (completion -
    submission, the request being submitted at its arrival time) and the aggregate input GB/s."""
    import torch
    from paper_1703_02438_gb300 import build as nbuild
    from paper_1703_02438_gb300 import numarck as N
    from paper_1703_02438_gb300 import synth
    nbuild.build()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(synth.seed_for(4))
    n_series, steps = 32, 3
    series = []
    for s_ in range(n_series):
        size = int(np.exp(rng.uniform(np.log(1 << 20), np.log(2 << 30))))
        dtype = torch.float64 if rng.random() < 0.5 else torch.float32
        L = 8 if dtype == torch.float64 else 4
        n = max(1, size // L)
        g = torch.Generator(device=dev)
        g.manual_seed(synth.seed_for(4, s_))
        x = torch.empty(n, dtype=torch.float64, device=dev).log_normal_(0.0, 1.0, generator=g)
        ts = []
        for t in range(steps):
            if t:
                r = torch.randn(n, generator=g, device=dev, dtype=torch.float64).mul_(1e-3)
                x = x * (1.0 + r)
            h = torch.empty(n, dtype=dtype, pin_memory=True)
            h.copy_(x.to(dtype))
            ts.append(h)
        params = N.make_params(dtype, (6, 8, 10)[s_ % 3], (1e-3, 1e-4)[s_ % 2])
        out_blob = torch.empty(N.compress_bound(n, params), dtype=torch.uint8, pin_memory=True)
        out_dec = torch.empty(n, dtype=dtype, pin_memory=True)
        series.append(dict(n=n, L=L, ts=ts, params=params, blob=out_blob, dec=out_dec))
        del x
    torch.cuda.synchronize()
    arena = torch.empty(64 << 30, dtype=torch.uint8, device=dev)
    srv = N.Server(arena, slots=8, max_series=n_series)
    for s_, sr in enumerate(series):                  # reference timesteps (not timed)
        srv.submit(N.REQ_COMPRESS, s_, sr["n"], sr["params"], host_in=sr["ts"][0],
                   host_out=sr["blob"])
    got = 0
    while got < n_series:
        got += len(srv.poll(wait_ms=100))
    next_t = [1] * n_series
    compressed = [False] * n_series          # a decompression needs a compressed timestep
    arrivals = np.cumsum(rng.exponential(1.0 / args.serve_rate,
                                         int(args.serve_rate * args.serve_seconds * 1.2) + 10))
    arrivals = arrivals[arrivals < args.serve_seconds]
    kinds = rng.random(arrivals.size)
    picks = rng.integers(0, n_series, arrivals.size)
    info, done = {}, []
    t0 = time.perf_counter()
    for a_t, k, s_ in zip(arrivals, kinds, picks):
        while True:
            now = time.perf_counter() - t0
            if now >= a_t:
                break
            done += srv.poll(wait_ms=0)
            time.sleep(min(0.0005, a_t - now))
        sr = series[s_]
        if k < 0.8 or not compressed[s_]:
            compressed[s_] = True
            t = next_t[s_]
            next_t[s_] = t % (steps - 1) + 1
            rid = srv.submit(N.REQ_COMPRESS, int(s_), sr["n"], sr["params"], host_in=sr["ts"][t],
                             host_out=sr["blob"])
            info[rid] = ("compress", sr["n"] * sr["L"])
        else:
            if k < 0.9:
                start, count = 0, sr["n"]
            else:
                count = max(1, int(sr["n"] * rng.uniform(0.01, 0.10)))
                start = int(rng.integers(0, sr["n"] - count + 1))
            rid = srv.submit(N.REQ_DECOMPRESS, int(s_), sr["n"], sr["params"],
                             host_out=sr["dec"][:count], start=start, count=count)
            info[rid] = ("decompress", count * sr["L"])
    while len(done) < len(info):
        done += srv.poll(wait_ms=100)
    st = srv.stats()
    srv.close()
    ok = [c for c in done if c["status"] == 0]
    lat = {"compress": [], "decompress": []}
    for c in ok:
        lat[info[c["id"]][0]].append((c["t_end"] - c["t_submit"]) * 1e3)
    span = max(c["t_end"] for c in done) - min(c["t_submit"] for c in done)
    moved = sum(info[c["id"]][1] for c in ok)
    offered = sum(v[1] for v in info.values()) / args.serve_seconds / 1e9
    allv = lat["compress"] + lat["decompress"]
    pct = lambda v, q: float(np.percentile(v, q)) if v else None
    # where the time goes: waiting for a slot (and for the series' earlier requests, and for
    # arena space) against running on a slot; and the latency of large against small requests
    wait = [(c["t_start"] - c["t_submit"]) * 1e3 for c in ok]
    run_ = [(c["t_end"] - c["t_start"]) * 1e3 for c in ok]
    big = [(c["t_end"] - c["t_submit"]) * 1e3 for c in ok if info[c["id"]][1] >= (1 << 30)]
    small = [(c["t_end"] - c["t_submit"]) * 1e3 for c in ok if info[c["id"]][1] < (64 << 20)]
    worst = sorted(ok, key=lambda c: c["t_end"] - c["t_submit"])[-max(1, len(ok) // 100):]
    t_first = min(c["t_submit"] for c in ok) if ok else 0.0
    late = [(c["t_end"] - c["t_submit"]) * 1e3 for c in ok if c["t_submit"] >= t_first + 5.0]
    line = {"metric": "served compress/decompress requests: latency p50/p99 and aggregate input GB/s",
            "value": moved / span / 1e9, "unit": "GB/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"{n_series} series, sizes log-uniform [1 MB, 2 GB], float32/"
                                   f"float64 50/50, Poisson {args.serve_rate:g} req/s for "
                                   f"{args.serve_seconds:g} s, 80% compress / 20% decompress "
                                   "(half whole, half 1-10% range)",
                       "slots": 8, "arena_gb": 64},
            "requests": len(info), "completed_ok": len(ok),
            "failed": len(done) - len(ok),
            "failed_status": {str(k): v for k, v in
                              sorted(__import__("collections").Counter(
                                  c["status"] for c in done if c["status"]).items())},
            "offered_gbs": offered,
            "p50_ms": pct(allv, 50), "p99_ms": pct(allv, 99),
            "compress_p50_ms": pct(lat["compress"], 50), "compress_p99_ms": pct(lat["compress"], 99),
            "decompress_p50_ms": pct(lat["decompress"], 50),
            "decompress_p99_ms": pct(lat["decompress"], 99),
            "breakdown": {
                "wait_p50_ms": pct(wait, 50), "wait_p99_ms": pct(wait, 99),
                "run_p50_ms": pct(run_, 50), "run_p99_ms": pct(run_, 99),
                "ge_1GB_requests": len(big), "ge_1GB_p50_ms": pct(big, 50),
                "ge_1GB_p99_ms": pct(big, 99),
                "lt_64MB_requests": len(small), "lt_64MB_p50_ms": pct(small, 50),
                "lt_64MB_p99_ms": pct(small, 99),
                "after_5s_requests": len(late), "after_5s_p50_ms": pct(late, 50),
                "after_5s_p99_ms": pct(late, 99),
                "slowest_1pct": {"count": len(worst),
                                 "mean_submit_s": float(np.mean([c["t_submit"] - t_first
                                                                 for c in worst])),
                                 "mean_wait_ms": float(np.mean([(c["t_start"] - c["t_submit"]) * 1e3
                                                                for c in worst])),
                                 "mean_run_ms": float(np.mean([(c["t_end"] - c["t_start"]) * 1e3
                                                               for c in worst])),
                                 "mean_input_mb": float(np.mean([info[c["id"]][1]
                                                                 for c in worst])) / 1e6}},
            "server": {k: st[k] for k in ("deferred_memory", "arena_peak", "max_inflight")}}
    print(json.dumps(line), flush=True)


def _host_mem_available():
    """MemAvailable of this host in bytes (None where /proc/meminfo is missing)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def run_e2e(args, xs, n, bound, dist, dev, ws, recon_out=True):
    """End-to-end metric through the public API: host timesteps in, blobs (and reconstructions)
    out, each (E, B) chain as in the device-resident run (compress, two chained steps,
    decompress), with the host<->device copies overlapped with the kernels and with each other.

    Inputs are double-buffered on the device, so the next step's four timesteps are copied in
    while this step computes; the copies out run on their own streams as soon as each result is
    ready. The timed region starts before the first timed step's inputs are copied in."""
    import torch
    from paper_1703_02438_gb300 import numarck as N
    nC = len(COMBOS)
    tdt = xs[0].dtype
    L = xs[0].element_size()
    host_x = [xs[t].cpu().pin_memory() for t in range(4)]
    host_blob = torch.empty(bound, dtype=torch.uint8).pin_memory()
    host_rec = torch.empty(n if recon_out else 1, dtype=tdt).pin_memory()
    host_status = torch.zeros(1, dtype=torch.int32).pin_memory()
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    xin = [[torch.empty(n, dtype=tdt, device=dev) for _ in range(4)] for _ in range(2)]
    NB, NR = 3, 3
    blobs = [torch.empty(bound, dtype=torch.uint8, device=dev) for _ in range(NB)]
    recs = [torch.empty(n, dtype=tdt, device=dev) for _ in range(NR)]
    hdrs = [torch.empty(N.HEADER_BYTES, dtype=torch.uint8).pin_memory() for _ in range(NB)]
    comp = torch.cuda.current_stream()
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    parts = 4                                         # each large copy is split over 4 streams
    h2d_s = [torch.cuda.Stream() for _ in range(parts)]
    d2h_s = [torch.cuda.Stream() for _ in range(parts)]
    tally = {"h2d": 0, "d2h": 0}

    def split_copy(dst, src, lead, streams):
        """dst.copy_(src) as `parts` chunks on `streams`, ordered after stream `lead`; `lead`
        then waits for all chunks."""
        m = src.numel()
        step_ = (m + parts - 1) // parts
        for i, st in enumerate(streams):
            st.wait_stream(lead)
            lo, hi = i * step_, min(m, (i + 1) * step_)
            if lo < hi:
                with torch.cuda.stream(st):
                    dst[lo:hi].copy_(src[lo:hi], non_blocking=True)
        for st in streams:
            lead.wait_stream(st)

    def record(stream):
        ev = torch.cuda.Event()
        ev.record(stream)
        return ev

    state = {"set_free": [None, None], "blob_free": [None] * NB, "rec_free": [None] * NR,
             "bi": 0, "ri": 0, "loaded": {}}

    def load(k):
        """Queue the copy-in of step k's four timesteps into input set k % 2."""
        st = k % 2
        if state["set_free"][st] is not None:
            h2d.wait_event(state["set_free"][st])
        evs = []
        for t in range(4):
            split_copy(xin[st][t], host_x[t], h2d, h2d_s)
            evs.append(record(h2d))
            tally["h2d"] += n * L
        state["loaded"][k] = evs

    pending = []   # (event after the producing call, blob index or None, recon index or None)

    def flush(keep):
        """Queue the copies out of every pending result but the last `keep`."""
        while len(pending) > keep:
            ev, bi, ri = pending.pop(0)
            d2h.wait_event(ev)
            if bi is not None:
                ev.synchronize()                      # the blob's header is in pinned memory
                size = N.blob_size(bytes(hdrs[bi].numpy().tobytes()))
                split_copy(host_blob[:size], blobs[bi][:size], d2h, d2h_s)
                tally["d2h"] += size
                state["blob_free"][bi] = record(d2h)
            if ri is not None:
                if recon_out:
                    split_copy(host_rec, recs[ri], d2h, d2h_s)
                    tally["d2h"] += n * L
                    state["rec_free"][ri] = record(d2h)
                else:
                    with torch.cuda.stream(d2h):
                        host_status.copy_(status, non_blocking=True)
                    tally["d2h"] += 4

    def new_blob():
        bi = state["bi"]
        state["bi"] = (bi + 1) % NB
        if state["blob_free"][bi] is not None:
            comp.wait_event(state["blob_free"][bi])
        return bi

    def new_rec():
        ri = state["ri"]
        state["ri"] = (ri + 1) % NR
        if state["rec_free"][ri] is not None:
            comp.wait_event(state["rec_free"][ri])
        return ri

    def produced(bi, ri):
        if bi is not None:
            hdrs[bi].copy_(blobs[bi][:N.HEADER_BYTES], non_blocking=True)
        pending.append((record(comp), bi, ri))
        flush(1)

    def compute(k):
        st = k % 2
        X = xin[st]
        ld = state["loaded"].pop(k)
        for c, (E, B) in enumerate(COMBOS):
            if c == 0:
                comp.wait_event(ld[0])
                comp.wait_event(ld[1])
            b0 = new_blob()
            N.compress(X[0], X[1], E, B, blob=blobs[b0], workspace=ws, stream=comp)
            produced(b0, None)
            if c == 0:
                comp.wait_event(ld[2])
            ra, b1 = new_rec(), new_blob()
            N.decompress_compress(blobs[b0], X[0], X[2], E, B, out=recs[ra], next_blob=blobs[b1],
                                  workspace=ws, status=status, stream=comp)
            produced(b1, ra)
            if c == 0:
                comp.wait_event(ld[3])
            rb, b2 = new_rec(), new_blob()
            N.decompress_compress(blobs[b1], recs[ra], X[3], E, B, out=recs[rb],
                                  next_blob=blobs[b2], workspace=ws, status=status, stream=comp)
            produced(b2, rb)
            rc = new_rec()
            N.decompress(blobs[b2], recs[rb], out=recs[rc], status=status, stream=comp)
            produced(None, rc)
        state["set_free"][st] = record(comp)

    def run(steps):
        load(0)
        if steps > 1:
            load(1)
        for k in range(steps):
            compute(k)
            if k + 2 < steps:
                load(k + 2)
        flush(0)

    run(1)                                            # warm-up (pins pages, loads code)
    torch.cuda.synchronize()
    tally["h2d"] = tally["d2h"] = 0
    _barrier(dist)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(comp)
    h2d.wait_stream(comp)                             # nothing of the timed steps before `a`
    d2h.wait_stream(comp)
    run(args.e2e_steps)
    comp.wait_stream(h2d)
    comp.wait_stream(d2h)
    b.record(comp)
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {int(status.item())} in the end-to-end run")
    e2e_ms = _max_over_ranks(dist, a.elapsed_time(b))
    n_pairs = 3 * nC
    val = _sum_over_ranks(dist, args.e2e_steps * n_pairs * n * L) / (e2e_ms / 1e3) / 1e9

    # the host link's own copy rates (one timestep each way, then both ways at once), for the
    # bound that the copies above put on E
    def issue(dst, src, streams):
        m = src.numel()
        st_ = (m + parts - 1) // parts
        for i, st in enumerate(streams):
            st.wait_stream(comp)
            with torch.cuda.stream(st):
                dst[i * st_:(i + 1) * st_].copy_(src[i * st_:(i + 1) * st_], non_blocking=True)

    def link_rate(pairs_):
        def once():
            for dst, src, streams in pairs_:
                issue(dst, src, streams)
            for _, _, streams in pairs_:
                for st in streams:
                    comp.wait_stream(st)
        once()
        torch.cuda.synchronize()
        a.record(comp)
        for _ in range(3):
            once()
        b.record(comp)
        torch.cuda.synchronize()
        nbytes = 3 * sum(src.numel() * src.element_size() for _, src, _ in pairs_)
        return nbytes / (a.elapsed_time(b) / 1e3) / 1e9

    link = {"d2h_gbs": link_rate([(host_x[0], xin[0][0], d2h_s)]),
            "h2d_gbs": link_rate([(xin[0][1], host_x[1], h2d_s)]),
            "both_ways_gbs": link_rate([(host_x[0], xin[0][0], d2h_s), (xin[0][1], host_x[1], h2d_s)])}
    hb_, db_ = tally["h2d"] / args.e2e_steps, tally["d2h"] / args.e2e_steps
    # E if the step took exactly as long as its copies: each direction at its own rate, and
    # both together at the measured two-way rate
    t_copy = max(hb_ / link["h2d_gbs"], db_ / link["d2h_gbs"],
                 (hb_ + db_) / link["both_ways_gbs"]) / 1e9
    link["bound_gbs"] = n_pairs * n * L / t_copy / 1e9
    out = {"value": val, "unit": "GB/s",
           "h2d_bytes_per_step": tally["h2d"] // args.e2e_steps,
           "d2h_bytes_per_step": tally["d2h"] // args.e2e_steps,
           "steps": args.e2e_steps,
           "link": {k: round(v, 1) for k, v in link.items()},
           "note": ("each timestep copied in once per step (inputs double-buffered: the next "
                    "step's are copied in while this one computes); every pair's blob and "
                    + ("reconstruction" if recon_out else "decode status word")
                    + " copied out as soon as it is ready; copies split over 4 streams each way "
                      "and overlapped with the kernels; chains as in the device-resident run")}
    del host_x, host_blob, host_rec, xin, recs, blobs
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "climate":
        return run_climate(args)
    if args.workload == "zindex":
        return run_zindex(args)
    if args.workload == "batched":
        return run_batched(args)
    rank, world = _rank_world()
    import numpy as np
    import torch
    from paper_1703_02438_gb300 import build as nbuild
    from paper_1703_02438_gb300 import numarck as N
    from paper_1703_02438_gb300 import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = _init_dist(world)
    if rank == 0:
        nbuild.build()
    _barrier(dist)
    nbuild.build()
    N.lib()
    dev = torch.device("cuda", local)
    side = args.side
    n = side ** 3
    xs = synth.flash_series(side=side, steps=4, device=dev, seed=synth.seed_for(1, rank))
    tdt = torch.float32 if args.f32 else torch.float64
    L = 4 if args.f32 else 8
    if args.f32:
        xs = [x.float() for x in xs]
    torch.cuda.synchronize()
    combos = [(E, 0 if args.auto_b else B) for E, B in COMBOS]
    params = {(E, B): N.make_params(tdt, B, E) for E, B in combos}
    bound = max(N.compress_bound(n, p) for p in params.values())
    blob = torch.empty(bound, dtype=torch.uint8, device=dev)
    recon = [torch.empty(n, dtype=tdt, device=dev) for _ in range(2)]
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = N.Workspace(dev)
    ws.get(max(N.workspace_bytes(n, p) for p in params.values()))
    stream = torch.cuda.current_stream()

    n_pairs = len(COMBOS) * 3
    blobs = [blob, torch.empty(bound, dtype=torch.uint8, device=dev)]
    # (kind, events): "c" a compression (K1, K2, K3a+K3f, K3b, K3c), "s" a chained step (K41,
    # then the same four), "d" a decompression (K4)
    ev_pool = []

    def new_events(kind, k):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        for e in evs:          # torch creates the CUDA event on first record
            e.record(stream)
        ev_pool.append((kind, evs))
        return evs

    def step(trace: bool):
        for E, B in combos:
            if args.no_fuse:
                prev = xs[0]
                for t in range(1, 4):
                    if trace:
                        N.trace_events(new_events("c", 6))
                    N.compress(prev, xs[t], E, B, blob=blobs[0], workspace=ws)
                    if trace:
                        N.trace_events(new_events("d", 2))
                    out = recon[t % 2]
                    N.decompress(blobs[0], prev, out=out, status=status)
                    prev = out
            else:
                # timestep 1 compressed alone; timesteps 2 and 3 by the chained step, which also
                # decompresses the blob before (Eq. 4: prev = that reconstruction); the last blob
                # decompressed alone
                if trace:
                    N.trace_events(new_events("c", 6))
                N.compress(xs[0], xs[1], E, B, blob=blobs[0], workspace=ws)
                prev = xs[0]
                for t in range(2, 4):
                    out = recon[t % 2]
                    if trace:
                        N.trace_events(new_events("s", 6))
                    N.decompress_compress(blobs[t % 2], prev, xs[t], E, B, out=out,
                                          next_blob=blobs[(t + 1) % 2], workspace=ws,
                                          status=status)
                    prev = out
                if trace:
                    N.trace_events(new_events("d", 2))
                N.decompress(blobs[0], prev, out=recon[0], status=status)
        if trace:
            N.trace_events(None)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {int(status.item())} after warm-up")

    clocks = Clocks(local)
    _barrier(dist)
    torch.cuda.synchronize()
    ev_pool.clear()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step(True)
    t_end.record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    clk = clocks.stop()
    ms_total = t_start.elapsed_time(t_end)
    ms_total = _max_over_ranks(dist, ms_total)
    ms_step = ms_total / args.steps
    bytes_rank = args.steps * n_pairs * n * L
    value = _sum_over_ranks(dist, bytes_rank) / (ms_total / 1e3) / 1e9

    # per-kernel times from the trace events
    kt, kn = {}, {}
    tail = (("k2_topk", 1, 2), ("k3_assign", 2, 3), ("k3_scan", 3, 4), ("k3_exact", 4, 5))

    def add(name, ms):
        kt[name] = kt.get(name, 0.0) + ms
        kn[name] = kn.get(name, 0) + 1

    for kind, evs in ev_pool:
        if kind == "d":
            add("k4_decode", evs[0].elapsed_time(evs[1]))
        else:
            add("k1_hist" if kind == "c" else "k41_step", evs[0].elapsed_time(evs[1]))
            for name, a, b in tail:
                add(name, evs[a].elapsed_time(evs[b]))
    avg = {k: kt[k] / kn[k] for k in kt}
    # algorithmic bytes per launch (HBM roofline); n_inc / B from the last blob of the step
    hdr = N.parse_header(N.header_bytes(blobs[0]))
    alpha = hdr["n_inc"] / n
    Bl = hdr["B"]
    # K1 reads p, x and writes a 2-byte code per point; K3a reads the codes and writes the
    # packed indices and 1 bit per point of incompressible flags; K3c reads the flags, gathers
    # the incompressible values of cur and writes them; K4 reads p (compressible points), the
    # packed indices and the incompressible values and writes R; K41 does K4's traffic plus
    # K1's without reading p (its p is the R it has just made)
    alg = {"k1_hist": 2 * L * n + 2 * n,
           "k3_assign": 2 * n + n * Bl / 8 + n / 8,
           "k3_exact": n / 8 + 2 * alpha * n * L,
           "k4_decode": (1 - alpha) * n * L + n * Bl / 8 + alpha * n * L + n * L}
    alg["k41_step"] = alg["k4_decode"] + L * n + 2 * n
    alg = {k: v for k, v in alg.items() if k in avg}
    dominant = max(alg, key=lambda k: avg[k])
    peak, peak_kind = _peaks()
    achieved = alg[dominant] / (avg[dominant] / 1e3) / 1e9
    kernel_ms = {k: round(v, 4) for k, v in avg.items()}
    kernel_gbs = {k: round(alg[k] / (avg[k] / 1e3) / 1e9, 1) for k in alg}
    launches = {k: kn[k] // args.steps for k in kn}              # per step
    step_alg = sum(alg[k] * launches[k] for k in alg)            # whole step, all kernels
    # the compressions and decompressions run alone (every one without chaining)
    t_comp = sum(avg[k] for k in ("k1_hist", "k2_topk", "k3_assign", "k3_scan", "k3_exact"))
    comp_alg = alg["k1_hist"] + alg["k3_assign"] + alg["k3_exact"]
    one_pass = 2 * L * n + n * Bl / 8 + alpha * n * L      # read p, x once; write the blob once

    # end to end through the public API with host buffers, pipelined: each timestep is copied
    # host->device once per step (pinned; the next step's inputs while this one computes);
    # every pair's blob (the used bytes, sized from its header) and reconstruction are copied
    # device->host on their own streams as soon as they are ready
    e2e = e2e_blob = None
    if not args.no_e2e and args.e2e_steps > 0:
        # host memory per rank: the 4 timesteps, a blob and a reconstruction pinned, plus one
        # pageable timestep while pinning; every rank of the node holds its own
        local_ranks = int(os.environ.get("LOCAL_WORLD_SIZE", "1"))
        need = local_ranks * (6 * n * L + bound)
        avail = _host_mem_available()
        if avail is not None and need > 0.8 * avail:
            why = (f"skipped: the end-to-end run pins {need / 1e9:.0f} GB of host memory on this "
                   f"node ({local_ranks} ranks) and {avail / 1e9:.0f} GB are available")
            e2e = {"value": None, "unit": "GB/s", "note": why}
            e2e_blob = {"value": None, "unit": "GB/s", "note": why}
        else:
            e2e = run_e2e(args, xs, n, bound, dist, dev, ws)
            # the same without the reconstruction leaving the device (it is the next prev of the
            # closed loop, Eq. 4): the blobs and the decode status are the step's results
            e2e_blob = run_e2e(args, xs, n, bound, dist, dev, ws, recon_out=False)

    # quality of every pair of the step, from one more run of each chain (outside the timed
    # region): CR (Eq. 2, raw blob), ME (Eq. 3), the largest relative error, and the points
    # whose reconstruction fails |R - x| <= E|x| evaluated in T (none may: markers are exact
    # and every indexed point passed that check when it was compressed)
    quality = []
    for E, B in combos:
        row = {"E": E, "B": B, "CR": [], "ME": [], "max_rel_err": [], "alpha": [],
               "bound_violations": 0}
        N.compress(xs[0], xs[1], E, B, blob=blobs[0], workspace=ws)
        prev = xs[0]
        for t in range(1, 4):
            if t < 3:
                rec, _ = N.decompress_compress(blobs[(t - 1) % 2], prev, xs[t + 1], E, B,
                                               out=recon[t % 2], next_blob=blobs[t % 2],
                                               workspace=ws, status=status)
            else:
                rec = N.decompress(blobs[(t - 1) % 2], prev, out=recon[t % 2], status=status)
            h = N.parse_header(N.header_bytes(blobs[(t - 1) % 2]))
            x = xs[t]
            xd, rd = x.double(), rec.double()
            nz = xd != 0
            rel = torch.where(nz, (xd - rd).abs_().div_(xd.abs()), torch.zeros((), dtype=torch.float64,
                                                                            device=dev))
            row["CR"].append(n * L / h["total_bytes"])
            row["ME"].append(float(rel.sum().item()) / max(1, int(nz.sum().item())))
            row["max_rel_err"].append(float(rel.max().item()))
            row["alpha"].append(h["n_inc"] / n)
            row["bound_violations"] += int(((rec - x).abs_() > x.abs().mul_(E)).sum().item())
            del xd, rd, nz, rel
            prev = rec
        quality.append(row)
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {int(status.item())} in the quality run")

    cpu = None
    if rank == 0 and not args.no_cpu:
        gbs, sec, desc = cpu_oracle_sample((xs[1], xs[2]), args.cpu_sample)
        cpu = {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc,
               "seconds": round(sec, 2)}
        if not args.f32 and (_host_mem_available() or 0) > 8 * n * 8:
            ref = N.compress(xs[1], xs[2], 1e-3, 8)
            torch.cuda.synchronize()
            ref_bytes = ref[:N.blob_size(N.header_bytes(ref))].cpu().numpy().tobytes()
            del ref
            cpu["all_cores"] = cpu_parallel_pair((xs[1], xs[2]), ref_bytes)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.f32 else "f64",
            "data": "synthetic",
            "config": {"workload": workload_label(side, args.f32),
                       "n": n, "pairs_per_step": n_pairs,
                       "chained": not args.no_fuse, "seed": synth.seed_for(1, rank),
                       "l2": (f"inputs {n * L / 2 ** 30:.2f} GiB per array > 129 MB L2: no flush"
                              if n * L > 129e6 else "inputs fit in L2: warm-cache figure"),
                       "parallelism": f"replicas x{world} (independent series per GPU)"},
            "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": _traffic(dominant, side),
                         "algorithmic_bytes_per_launch": alg[dominant],
                         # the same fractions of the peak for the whole step and for a
                         # compression alone (also given below, outside this object)
                         "step_frac": step_alg / (ms_step / 1e3) / 1e9 / peak,
                         "compress_path_frac": comp_alg / (t_comp / 1e3) / 1e9 / peak,
                         "compress_one_pass_frac": one_pass / (t_comp / 1e3) / 1e9 / peak},
            "kernels_ms": kernel_ms, "kernels_gbs": kernel_gbs, "launches_per_step": launches,
            "step_hbm_frac": step_alg / (ms_step / 1e3) / 1e9 / peak,
            "compress_gbs": n * L / (t_comp / 1e3) / 1e9,
            "compress_path_hbm_frac": comp_alg / (t_comp / 1e3) / 1e9 / peak,
            "compress_one_pass_frac": one_pass / (t_comp / 1e3) / 1e9 / peak,
            "decompress_gbs": n * L / (avg["k4_decode"] / 1e3) / 1e9,
            "alpha_last": alpha, "B_last": Bl, "auto_b": bool(args.auto_b),
            "quality": {"per_chain": quality,
                        "max_rel_err_over_E": max(max(r["max_rel_err"]) / r["E"] for r in quality),
                        "bound_violations": sum(r["bound_violations"] for r in quality)},
            "clocks": clk, "e2e": e2e, "e2e_blobs_only": e2e_blob, "cpu_baseline": cpu,
            "gpu_launches": args.steps * len(COMBOS) * ((21 if args.no_fuse else 19)
                                                        + (3 if args.auto_b else 0)),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
