"""Parity at the full size of the headline workload (FLASH-like 1024^3 float64, 8 GiB per array),
in the launch configuration bench.py times.

The oracle's whole compress() cannot run at this size in test time, so its per-step functions run
on contiguous chunks of the host copies, in threads (numpy releases the GIL in its array loops):
  * the histogram, the top-k selection and the centre table come from the oracle's counts over
    all 2^30 points (counts of chunks add up), and the GPU's centre table must match byte for
    byte;
  * every point's index: the oracle's change ratio, bin id and indexing with the error-bound check
    (§III.C), chunk by chunk with that selection, must equal the GPU's packed index of the point,
    for all 2^30 points;
  * the incompressible table must hold the oracle's incompressible points' values bit for bit, in
    element order, and the sub-block offset table must be the prefix counts of the oracle's
    markers;
  * the reconstruction: every compressible point reconstructs within E (in T, as the check
    defines it), every incompressible one bit for bit, and a range decode equals the slice of the
    full decode.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

from oracle import numarck_oracle as O
from paper_1703_02438_gb300 import numarck as N
from paper_1703_02438_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SIDE = 1024
CHUNK = 1 << 22
THREADS = max(1, min(32, len(os.sched_getaffinity(0))))


@pytest.fixture(scope="module")
def series():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1703_02438_gb300 import build
    build.build()
    xs = synth.flash_series(side=SIDE, steps=2, device=DEV, seed=synth.seed_for(1, 0))
    return xs[0], xs[1]


@pytest.fixture(scope="module")
def host(series):
    """Host copies of the pair, for the oracle."""
    return series[0].cpu().numpy(), series[1].cpu().numpy()


def _chunks(n):
    return range(0, n, CHUNK)


def _oracle_selection(p_h, x_h, E, B):
    """Oracle histogram over all points (counts per chunk, added up), then its top-k and
    centres."""
    T = np.float64
    E_T, w, inv_w, cap = O.grid_constants(T, E)
    a = O.grid_anchor(np.zeros(0), np.zeros(0, bool), E_T, O.ANCHOR_ZERO)

    def count(lo):
        ratio, ok = O.change_ratio(p_h[lo: lo + CHUNK], x_h[lo: lo + CHUNK], cap)
        return O.histogram(O.bin_ids(ratio, ok, a, inv_w), ok)

    counts = {}
    with ThreadPoolExecutor(THREADS) as ex:
        for bins, cnt in ex.map(count, _chunks(p_h.size)):
            for k, v in zip(bins.tolist(), cnt.tolist()):
                counts[k] = counts.get(k, 0) + v
    bins = np.array(sorted(counts), dtype=np.int64)
    cnts = np.array([counts[k] for k in bins.tolist()], dtype=np.int64)
    sel = O.top_k(bins, cnts, (1 << B) - 1)
    return sel, O.centres_of(sel, a, w, T), (E_T, inv_w, cap, a)


def _oracle_indices(p_h, x_h, sel, centres, consts, M):
    """The oracle's index of every point (chunks in threads), as int16 (B <= 15)."""
    E_T, inv_w, cap, a = consts
    out = np.empty(p_h.size, dtype=np.int16)

    def index(lo):
        p, x = p_h[lo: lo + CHUNK], x_h[lo: lo + CHUNK]
        ratio, ok = O.change_ratio(p, x, cap)
        b = O.bin_ids(ratio, ok, a, inv_w)
        out[lo: lo + CHUNK] = O.assign_indices(p, x, ok, b, sel, centres, E_T, M)

    with ThreadPoolExecutor(THREADS) as ex:
        list(ex.map(index, _chunks(p_h.size)))
    return out


def _gpu_indices_at(blob_u8: np.ndarray, h: dict, j: np.ndarray) -> np.ndarray:
    """Read the B-bit indices of elements j from the packed index section (test-side reader:
    block q at idx_off[q], index i of a block at bits [iB, iB+B), least significant bit first)."""
    B, epb = h["B"], h["epb"]
    idx_off = np.frombuffer(blob_u8.tobytes()[h["off_idx_off"]: h["off_idx_off"] + 8 * (h["nblocks"] + 1)],
                            dtype=np.int64)
    q = j // epb
    bit = (j - q * epb) * B
    byte = h["off_index"] + idx_off[q] + bit // 8
    v = (blob_u8[byte].astype(np.int64) | (blob_u8[byte + 1].astype(np.int64) << 8)
         | (blob_u8[byte + 2].astype(np.int64) << 16))
    return (v >> (bit % 8)) & ((1 << B) - 1)


@pytest.mark.parametrize("E,B", [(1e-4, 10), (1e-3, 8)])
def test_fullsize_flash_pair(series, host, E, B):
    p_dev, x_dev = series
    p_h, x_h = host
    n = p_dev.numel()
    M = (1 << B) - 1
    blob = N.compress(p_dev, x_dev, E, B)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    rec = N.decompress(blob, p_dev, status=status)
    torch.cuda.synchronize()
    hb = N.header_bytes(blob)
    size = N.blob_size(hb)
    h = N.parse_header(hb)
    assert int(status.item()) == 0 and h["n"] == n

    # 1. histogram / top-k / centres over all points, by the oracle
    sel, centres, consts = _oracle_selection(p_h, x_h, E, B)
    E_T = consts[0]
    assert h["n_sel"] == sel.size
    want_c = np.zeros(1 << B, dtype=np.float64)
    want_c[: sel.size] = centres
    got_c = blob[h["off_centres"]: h["off_centres"] + 8 * (1 << B)].cpu().numpy().view(np.float64)
    assert np.array_equal(got_c.view(np.uint64), want_c.view(np.uint64))

    blob_u8 = blob[:size + 16].cpu().numpy()   # +16: the reader may touch 2 bytes past the end

    # 2. every point's index: the GPU's packed indices, unpacked on the device by a test-side
    # reader (block q at idx_off[q], index i of a block at bits [iB, iB+B), least significant
    # bit first), against the oracle's indexing of every point
    jj = torch.arange(n, device=DEV, dtype=torch.int64)
    idx_off = torch.from_numpy(np.frombuffer(
        blob_u8.tobytes()[h["off_idx_off"]: h["off_idx_off"] + 8 * (h["nblocks"] + 1)],
        dtype=np.int64).copy()).to(DEV)
    q = jj // h["epb"]
    bit = (jj - q * h["epb"]) * B
    byte = h["off_index"] + idx_off[q] + bit // 8
    del q, jj
    bu = blob[: size + 16].to(torch.int32)
    v = bu[byte] | (bu[byte + 1] << 8) | (bu[byte + 2] << 16)
    del byte, bu
    idx_all = ((v >> (bit % 8)) & M).to(torch.int16)
    del v, bit
    got_idx = idx_all.cpu().numpy()
    want_idx = _oracle_indices(p_h, x_h, sel, centres, consts, M)
    bad = np.flatnonzero(got_idx != want_idx)
    assert bad.size == 0, f"{bad.size} indices differ, first at {bad[:5].tolist()}"
    # the spot reader agrees with the device unpacking (a check of the test's own reader)
    j = np.random.default_rng(1).integers(0, n, 4096)
    assert np.array_equal(_gpu_indices_at(blob_u8, h, j), want_idx[j].astype(np.int64))
    del got_idx

    # 3. incompressible values and offsets against the oracle's markers
    marker_h = want_idx == M
    n_inc = int(marker_h.sum())
    assert n_inc == h["n_inc"]
    exact = blob_u8[h["off_exact"]: h["off_exact"] + 8 * n_inc].view(np.uint64)
    assert np.array_equal(exact, x_h.view(np.uint64)[marker_h])
    csum = np.concatenate([[0], np.cumsum(marker_h, dtype=np.int64)])
    starts = np.concatenate([np.arange(qq * h["epb"], min(n, (qq + 1) * h["epb"]), h["sub"])
                             for qq in range(h["nblocks"])])
    sub_off = blob_u8[h["off_sub_off"]: h["off_sub_off"] + 8 * h["nsub"]].view(np.int64)
    assert np.array_equal(sub_off, csum[starts])
    inc_off = blob_u8[h["off_inc_off"]: h["off_inc_off"] + 8 * (h["nblocks"] + 1)].view(np.int64)
    assert np.array_equal(inc_off, csum[np.minimum(np.arange(h["nblocks"] + 1) * h["epb"], n)])
    del csum, starts

    # 4. the reconstruction over every point
    marker = idx_all == M
    del idx_all
    comp = ~marker
    err = (rec - x_dev).abs()
    tol = x_dev.abs() * E_T
    assert bool((err[comp] <= tol[comp]).all())
    del err, tol, comp
    rec_b, x_b = rec.view(torch.int64), x_dev.view(torch.int64)
    assert bool((rec_b[marker] == x_b[marker]).all())
    del marker
    # a range decode equals the slice
    s, c = n // 3 + 12345, 50_000_000
    seg = N.decompress_range(blob, p_dev[s: s + c], s, c, status=status)
    torch.cuda.synchronize()
    assert torch.equal(seg.view(torch.int64), rec[s: s + c].view(torch.int64))
    assert int(status.item()) == 0


@pytest.mark.parametrize("E,B", [(1e-4, 10), (1e-3, 8)])
def test_fullsize_chained_step_equals_separate_calls(series, E, B):
    """At the full size and in the launch configuration of the timed run, the chained step
    (decompression fused with the next compression's first pass) gives byte for byte the
    reconstruction and the next blob of the separate calls, whose parity with the oracle the
    test above establishes. The next timestep is the pair's cur scaled by a smooth factor, so
    its ratios against the reconstruction spread over many bins."""
    p_dev, x_dev = series
    n = p_dev.numel()
    idx = torch.arange(n, device=DEV, dtype=torch.float64)
    y_dev = x_dev * (1.0 + 3e-3 * torch.sin(idx * 1e-5))
    del idx
    b1 = N.compress(p_dev, x_dev, E, B)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    rec_sep = N.decompress(b1, p_dev, status=status)
    sep = N.compress(rec_sep, y_dev, E, B)
    torch.cuda.synchronize()
    sep_bytes = sep[:N.blob_size(N.header_bytes(sep))]
    rec, nxt = N.decompress_compress(b1, p_dev, y_dev, E, B, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(rec.view(torch.int64), rec_sep.view(torch.int64))
    got = nxt[:N.blob_size(N.header_bytes(nxt))]
    assert got.numel() == sep_bytes.numel() and torch.equal(got, sep_bytes)
