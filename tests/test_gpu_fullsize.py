"""Parity at the full size of the headline workload (FLASH-like 1024^3 float64, 8 GiB per array),
in the launch configuration bench.py times.

The oracle cannot run whole at this size in test time, so the check is split:
  * the histogram, the top-k selection and the centre table are computed by the oracle over all
    2^30 points (its per-step functions on contiguous chunks; counts of chunks add up) and the
    GPU's centre table must match byte for byte;
  * indices: 2^20 sampled points (plus every sub-block and block boundary region) are indexed by
    the oracle one by one and must equal the GPU's packed indices at those positions;
  * properties over every point: each compressible point reconstructs within E (in T, as the
    check defines it), each incompressible point is stored bit for bit at the position given by
    the sub-block offset table, the offset tables are prefix counts of the GPU's own indices, and
    a range decode equals the slice of the full decode.
"""
import numpy as np
import pytest
import torch

from oracle import numarck_oracle as O
from paper_1703_02438_gb300 import numarck as N
from paper_1703_02438_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SIDE = 1024
CHUNK = 1 << 24


@pytest.fixture(scope="module")
def series():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1703_02438_gb300 import build
    build.build()
    xs = synth.flash_series(side=SIDE, steps=2, device=DEV, seed=synth.seed_for(1, 0))
    return xs[0], xs[1]


def _oracle_selection(p_dev, x_dev, E, B):
    """Oracle histogram over all points (chunked counting), then its top-k and centres."""
    T = np.float64
    E_T, w, inv_w, cap = O.grid_constants(T, E)
    a = T(-E_T)
    n = p_dev.numel()
    counts = {}
    for lo in range(0, n, CHUNK):
        p = p_dev[lo: lo + CHUNK].cpu().numpy()
        x = x_dev[lo: lo + CHUNK].cpu().numpy()
        ratio, ok = O.change_ratio(p, x, cap)
        b = O.bin_ids(ratio, ok, a, inv_w)[ok]
        if b.size:
            bmin = int(b.min())
            c = np.bincount(b - bmin)
            nz = np.nonzero(c)[0]
            for k, v in zip((nz + bmin).tolist(), c[nz].tolist()):
                counts[k] = counts.get(k, 0) + v
    bins = np.array(sorted(counts), dtype=np.int64)
    cnts = np.array([counts[k] for k in bins.tolist()], dtype=np.int64)
    sel = O.top_k(bins, cnts, (1 << B) - 1)
    return sel, O.centres_of(sel, a, w, T), (E_T, inv_w, cap, a)


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
def test_fullsize_flash_pair(series, E, B):
    p_dev, x_dev = series
    n = p_dev.numel()
    blob = N.compress(p_dev, x_dev, E, B)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    rec = N.decompress(blob, p_dev, status=status)
    torch.cuda.synchronize()
    hb = N.header_bytes(blob)
    size = N.blob_size(hb)
    h = N.parse_header(hb)
    assert int(status.item()) == 0 and h["n"] == n

    # 1. histogram / top-k / centres over all points, by the oracle
    sel, centres, (E_T, inv_w, cap, a) = _oracle_selection(p_dev, x_dev, E, B)
    assert h["n_sel"] == sel.size
    want_c = np.zeros(1 << B, dtype=np.float64)
    want_c[: sel.size] = centres
    got_c = blob[h["off_centres"]: h["off_centres"] + 8 * (1 << B)].cpu().numpy().view(np.float64)
    assert np.array_equal(got_c.view(np.uint64), want_c.view(np.uint64))

    blob_u8 = blob[:size + 16].cpu().numpy()   # +16: the reader may touch 2 bytes past the end

    # 2. sampled indices, computed by the oracle one by one
    rng = np.random.default_rng(1)
    sub = h["sub"]
    edges = np.concatenate([(np.arange(0, n, h["epb"])[:, None] + np.arange(-3, 3)[None, :]).ravel(),
                            (np.arange(0, n, sub * 977)[:, None] + np.arange(-2, 2)[None, :]).ravel()])
    j = np.unique(np.clip(np.concatenate([rng.integers(0, n, 1 << 20), edges, [0, n - 1]]), 0, n - 1))
    jt = torch.from_numpy(j).to(DEV)
    ps = p_dev[jt].cpu().numpy()
    xsm = x_dev[jt].cpu().numpy()
    ratio, ok = O.change_ratio(ps, xsm, cap)
    b = O.bin_ids(ratio, ok, a, inv_w)
    want_idx = O.assign_indices(ps, xsm, ok, b, sel, centres, E_T, (1 << B) - 1)
    got_idx = _gpu_indices_at(blob_u8, h, j)
    assert np.array_equal(got_idx, want_idx)

    # 3. properties over every point
    M = (1 << B) - 1
    # per-element indices on the device: unpack with the same reader logic in torch
    jj = torch.arange(n, device=DEV, dtype=torch.int64)
    idx_off = torch.from_numpy(np.frombuffer(
        blob_u8.tobytes()[h["off_idx_off"]: h["off_idx_off"] + 8 * (h["nblocks"] + 1)],
        dtype=np.int64).copy()).to(DEV)
    q = jj // h["epb"]
    bit = (jj - q * h["epb"]) * B
    byte = h["off_index"] + idx_off[q] + bit // 8
    del q
    bu = blob[: size + 16].to(torch.int64)
    v = bu[byte] | (bu[byte + 1] << 8) | (bu[byte + 2] << 16)
    del byte
    idx_all = (v >> (bit % 8)) & M
    del v, bit, bu, jj
    marker = idx_all == M
    n_inc = int(marker.sum().item())
    assert n_inc == h["n_inc"]
    # compressible points: |R - x| <= E_T |x| in float64, the check of the method
    comp = ~marker
    err = (rec - x_dev).abs()
    tol = x_dev.abs() * E_T
    assert bool((err[comp] <= tol[comp]).all())
    del err, tol
    # incompressible points: bit copies, stored in element order
    rec_b, x_b = rec.view(torch.int64), x_dev.view(torch.int64)
    assert bool((rec_b[marker] == x_b[marker]).all())
    exact = blob[h["off_exact"]: h["off_exact"] + 8 * n_inc].view(torch.int64)
    assert torch.equal(exact, x_b[marker])
    # sub-block offsets = prefix counts of the GPU's own indices
    sub_off = blob[h["off_sub_off"]: h["off_sub_off"] + 8 * h["nsub"]].view(torch.int64)
    csum = torch.cumsum(marker.to(torch.int64), 0)
    starts = []
    for qq in range(h["nblocks"]):
        lo, hi = qq * h["epb"], min(n, (qq + 1) * h["epb"])
        starts.append(torch.arange(lo, hi, sub, device=DEV))
    starts = torch.cat(starts)
    before = torch.where(starts > 0, csum[(starts - 1).clamp(min=0)], torch.zeros_like(starts))
    assert torch.equal(sub_off, before)
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
