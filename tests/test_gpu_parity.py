"""GPU parity: the CUDA path against the CPU oracle, through the C ABI.

Floating point decides only integers and bit copies here (bin ids, indices, packed bits,
incompressible values), and the reconstruction is one T multiply, so the bar is bit-exact:
the whole blob (header, centre table, offset tables, index blocks, incompressible table) must be
byte-identical to the oracle's, and decompression bit-identical. Inputs are the seeded synthetic
workloads (scaled and full size) plus adversarial cases.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import numarck_oracle as O
from paper_1703_02438_gb300 import numarck as N
from paper_1703_02438_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1703_02438_gb300 import build
    build.build()
    N.lib()


def _u(a: np.ndarray) -> np.ndarray:
    return a.view(np.uint64 if a.dtype == np.float64 else np.uint32)


def _first_diff(a: bytes, b: bytes) -> str:
    n = min(len(a), len(b))
    i = next((k for k in range(n) if a[k] != b[k]), n)
    return f"len {len(a)} vs {len(b)}, first difference at byte {i}"


def gpu_compress(prev, cur, E, B, anchor=0, block_bytes=0):
    blob = N.compress(prev, cur, E, B, anchor=anchor, block_bytes=block_bytes)
    torch.cuda.synchronize()
    hb = N.header_bytes(blob)
    size = N.blob_size(hb)
    return blob, hb, blob[:size].cpu().numpy().tobytes()


def check_pair(p_np, x_np, E, B, anchor=0, block_bytes=0, ranges=(), p_dev=None, x_dev=None):
    """Compress on the GPU and with the oracle; compare blob bytes, decompression and ranges."""
    want = O.compress(p_np, x_np, E, B, anchor=anchor,
                      block_bytes=block_bytes or O.DEFAULT_BLOCK_BYTES).to_bytes()
    p_dev = torch.from_numpy(p_np).to(DEV) if p_dev is None else p_dev
    x_dev = torch.from_numpy(x_np).to(DEV) if x_dev is None else x_dev
    blob, hb, got = gpu_compress(p_dev, x_dev, E, B, anchor, block_bytes)
    if got != want:
        hg, hw = O.parse_header(got), O.parse_header(want)
        diff = {k: (hg[k], hw[k]) for k in hw if hg.get(k) != hw[k]}
        raise AssertionError(f"blob mismatch: {_first_diff(got, want)}; header diff {diff}")
    ref = O.decompress(want, p_np)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    rec = N.decompress(blob, p_dev, header=hb, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(_u(rec.cpu().numpy()), _u(ref)), "decompression mismatch"
    for s, c in ranges:
        seg = N.decompress_range(blob, p_dev[s: s + c], s, c, header=hb, status=status)
        torch.cuda.synchronize()
        assert np.array_equal(_u(seg.cpu().numpy()), _u(ref[s: s + c])), (s, c)
    assert int(status.item()) == 0
    return O.parse_header(want), rec


# ---------------------------------------------------------------------------------------
# the plain 1-D pair at full size (2^20 float64), both anchors
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("anchor", [N.ANCHOR_ZERO, N.ANCHOR_MIN])
def test_plain_pair_full_size(anchor):
    p, x = synth.plain_pair(1 << 20)
    rng = np.random.default_rng(0)
    ranges = [(0, 1 << 20), (12345, 777), (4095, 2), (1 << 19, 1 << 18)]
    ranges += [(int(s), int(rng.integers(1, 50000))) for s in rng.integers(0, 1 << 19, 6)]
    h, _ = check_pair(p.numpy(), x.numpy(), 1e-3, 8, anchor=anchor, ranges=ranges)
    assert h["n_sel"] == 255 and 0.05 < h["n_inc"] / h["n"] < 0.08


@pytest.mark.parametrize("B", [6, 10])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_plain_pair_dtypes_and_widths(B, dtype):
    p, x = synth.plain_pair(300_001, dtype=dtype, seed=synth.seed_for(0, B))
    check_pair(p.numpy(), x.numpy(), 1e-3, B, ranges=[(0, 300_001), (299_000, 1001)])


# ---------------------------------------------------------------------------------------
# FLASH-like 3-D series (scaled), closed loop: prev = previous reconstruction
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("E,B", [(1e-3, 8), (1e-4, 10), (1e-4, 8), (1e-3, 10)])
def test_flash_series_closed_loop(E, B):
    steps = synth.flash_series(side=96, steps=4, device=DEV)
    prev = steps[0]
    for t in range(1, 4):
        cur = steps[t]
        h, rec = check_pair(prev.cpu().numpy(), cur.cpu().numpy(), E, B,
                            ranges=[(1000, 50_000)], p_dev=prev, x_dev=cur)
        assert 0.001 < h["n_inc"] / h["n"] < 0.2     # shocks: 5% of cells, U(-0.5, 2)
        prev = rec


# ---------------------------------------------------------------------------------------
# CMIP-like 2-D float32 fields: full 3600 x 1800 grid, three monthly pairs
# ---------------------------------------------------------------------------------------
def test_climate_full_grid():
    months = dict(synth.climate_series(steps=4, device=DEV))
    for t in range(1, 4):
        p, x = months[t - 1], months[t]
        h, _ = check_pair(p.cpu().numpy(), x.cpu().numpy(), 1e-3, 8,
                          ranges=[(0, 64), (3_000_000, 100_000)], p_dev=p, x_dev=x)
        assert h["n_inc"] / h["n"] >= 0.03          # the ocean mask alone is 3%


# ---------------------------------------------------------------------------------------
# adversarial inputs
# ---------------------------------------------------------------------------------------
def _edge_case_arrays(T, n=50_000, seed=5):
    rng = np.random.default_rng(seed)
    E = 2.0 ** -10
    w = 2 * E
    p = rng.lognormal(size=n).astype(T)
    # ratios exactly on bin edges, on centres, and a few ulps either side
    m = rng.integers(-300, 300, n)
    base = (-E + m * w)
    jitter = rng.choice([0.0, 1.0, -1.0, 0.5, -0.5], n) * np.finfo(T).eps
    r = (base + jitter).astype(T)
    x = (p * (T(1) + r)).astype(T)
    k = n // 20
    sel = rng.permutation(n)
    # special values
    p[sel[0:k]] = 0
    x[sel[k:2 * k]] = 0
    p[sel[2 * k:2 * k + 50]] = np.inf
    x[sel[2 * k + 50:2 * k + 100]] = -np.inf
    x[sel[2 * k + 100:2 * k + 150]] = np.nan
    p[sel[2 * k + 150:2 * k + 200]] = -p[sel[2 * k + 150:2 * k + 200]]
    tiny = np.finfo(T).smallest_subnormal
    p[sel[2 * k + 200:2 * k + 250]] = tiny * 3
    x[sel[2 * k + 250:2 * k + 300]] = tiny * 5
    p[sel[2 * k + 300:2 * k + 350]] = -0.0
    # ratios near the cap 2^21 * w and beyond
    cap = T(w) * T(2 ** 21)
    for i, f in enumerate((1.0, 1.0 - 1e-6, 1.0 + 1e-6, 0.5, 2.0)):
        j = sel[2 * k + 350 + 10 * i: 2 * k + 360 + 10 * i]
        p[j] = 1
        x[j] = T(1) + T(cap * f)
    return p, x, E


@pytest.mark.parametrize("T", [np.float32, np.float64])
@pytest.mark.parametrize("anchor", [N.ANCHOR_ZERO, N.ANCHOR_MIN])
def test_adversarial_edges_and_specials(T, anchor):
    p, x, E = _edge_case_arrays(T)
    nanpay = np.array([0x7FF8DEADBEEF0001 if T == np.float64 else 0x7FC0BEEF],
                      dtype=np.uint64 if T == np.float64 else np.uint32).view(T)[0]
    x[7] = nanpay
    check_pair(p, x, E, 9, anchor=anchor, ranges=[(0, 50_000), (3, 4000)])


@pytest.mark.parametrize("T", [np.float32, np.float64])
@pytest.mark.parametrize("anchor", [N.ANCHOR_ZERO, N.ANCHOR_MIN])
def test_zero_prev_against_every_kind_of_cur(T, anchor):
    """p = +0 and -0 against x = +-0, +-1, +-inf, NaN, subnormal and huge values, spread among
    ordinary points (one zero every 97 points): (x - p) / p is +-inf or NaN, never binnable,
    whichever x; the kernels decide these points without dividing."""
    rng = np.random.default_rng(41)
    n = 20_000
    p = rng.lognormal(size=n).astype(T)
    x = (p * (T(1) + rng.normal(0, 1e-3, n))).astype(T)
    fi = np.finfo(T)
    xs = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, fi.smallest_subnormal,
                   -fi.smallest_subnormal, fi.max, -fi.max, 3.5], dtype=T)
    idx = np.arange(0, n, 97)
    p[idx] = np.where(np.arange(idx.size) % 2 == 0, T(0.0), T(-0.0))
    x[idx] = xs[np.arange(idx.size) % xs.size]
    h, _ = check_pair(p, x, 1e-3, 8, anchor=anchor, ranges=[(0, n), (95, 300)])
    assert h["n_inc"] >= idx.size


@pytest.mark.parametrize("B", [1, 2, 3, 5, 7, 8, 11, 13, 16])
def test_all_widths_small_blocks(B):
    """Index widths whose blocks do not hold a multiple of 32 indices; many blocks and
    sub-blocks, partial last sub-block in every block."""
    p, x = synth.plain_pair(123_457, seed=synth.seed_for(0, 100 + B))
    bb = 3001                                   # epb = 24008 // B
    rng = np.random.default_rng(B)
    ranges = [(int(s), int(rng.integers(1, 9000))) for s in rng.integers(0, 110_000, 8)]
    check_pair(p.numpy(), x.numpy(), 1e-3, B, block_bytes=bb, ranges=ranges)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 4095, 4096, 4097, 8191, 65537])
def test_sizes(n):
    p, x = synth.plain_pair(max(n, 1), seed=synth.seed_for(0, 7))
    p, x = p[:n].numpy().copy(), x[:n].numpy().copy()
    check_pair(p, x, 1e-3, 8, ranges=[(0, n), (n // 2, n - n // 2)])


def test_many_ties_in_counts():
    """Every bin holds the same count: the selection is decided by the tie-break alone."""
    n = 64 * 1000
    E = 2.0 ** -8
    m = np.repeat(np.arange(-500, 500), 64)
    rng = np.random.default_rng(9)
    rng.shuffle(m)
    p = np.ones(n)
    x = 1 + m * (2 * E)
    for B in (4, 8, 10):
        h, _ = check_pair(p, x, E, B)
        assert h["n_sel"] == min(1000, (1 << B) - 1)


def test_all_non_finite_and_constant():
    n = 10_000
    p = np.full(n, np.nan)
    check_pair(p, p.copy(), 1e-3, 8)
    q = np.full(n, 3.5)
    h, rec = check_pair(q, q.copy(), 1e-3, 8)
    assert h["n_inc"] == 0 and h["n_sel"] == 1


def test_misaligned_views_take_the_scalar_path():
    p, x = synth.plain_pair(100_003, seed=synth.seed_for(0, 11))
    pd, xd = p.to(DEV), x.to(DEV)
    # one-element offsets: 8-byte aligned but not 16-byte aligned
    check_pair(p[1:].numpy().copy(), x[1:].numpy().copy(), 1e-3, 8, p_dev=pd[1:], x_dev=xd[1:])
    p32, x32 = p.float(), x.float()
    check_pair(p32[3:].numpy().copy(), x32[3:].numpy().copy(), 1e-3, 8,
               p_dev=p32.to(DEV)[3:], x_dev=x32.to(DEV)[3:])


def test_worked_example_golden(golden_dir):
    import json
    import os
    g = json.load(open(os.path.join(golden_dir, "worked_example.json")))
    p = np.array(g["prev"], dtype=np.float64)
    x = np.array(g["cur"], dtype=np.float64)
    for anchor in (N.ANCHOR_ZERO, N.ANCHOR_MIN):
        for bb in (16, g["block_bytes_small"]):
            _, rec = check_pair(p, x, g["E"], g["B"], anchor=anchor, block_bytes=bb)
            assert rec.cpu().numpy().tolist() == g["recon"]


def test_repeatable_and_workspace_reuse():
    """Same inputs -> same bytes, across workspace reuse with other sizes and dtypes in between
    (the workspace is left ready for the next call)."""
    p, x = synth.plain_pair(200_000, seed=synth.seed_for(0, 13))
    pd, xd = p.to(DEV), x.to(DEV)
    _, _, first = gpu_compress(pd, xd, 1e-3, 8)
    q, y = synth.plain_pair(77_777, dtype=torch.float32, seed=synth.seed_for(0, 14))
    gpu_compress(q.to(DEV), y.to(DEV), 1e-4, 10, anchor=N.ANCHOR_MIN)
    _, _, second = gpu_compress(pd, xd, 1e-3, 8)
    assert first == second


@pytest.mark.parametrize("T", [np.float32, np.float64])
def test_min_anchor_negative_zero_minimum(T):
    """Reading R2 on the MIN grid: an unchanged point with a negative prev has ratio -0, so the
    smallest binnable ratio can be -0; the grid origin (and the header's `a`) is +0."""
    cases = [([2.0, -1.0], [2.0, -1.0]), ([-1.0, 2.0], [-1.0, 2.0]), ([-3.0], [-3.0]),
             ([1.0, -1.0, 1.0], [1.5, -1.0, 1.5])]
    rng = np.random.default_rng(61)
    n = 100_003
    p = rng.lognormal(size=n) * rng.choice([-1.0, 1.0], n)
    x = p * (1.0 + rng.uniform(0.0, 0.02, n))      # every ratio >= 0 ...
    keep = rng.random(n) < 0.3
    x[keep] = p[keep]                              # ... and 30% unchanged: +0 or -0
    cases.append((p, x))
    for prev, cur in cases:
        h, _ = check_pair(np.array(prev, dtype=T), np.array(cur, dtype=T), 1e-3, 8,
                          anchor=N.ANCHOR_MIN)
        assert h["a"] == 0.0 and not np.signbit(h["a"])


# byte offset of the window-error flag in the workspace's 256-byte control block (the
# library's internal layout: 4 + 4 + 8 + 4 + 4 + 6 * 4 bytes of counters, then the anchor
# as a double at 48, then this flag)
_CTRL_WIN_ERR = 56


def test_workspace_ready_after_device_reported_error():
    """A compression whose kernels report an error (here a histogram-window error, planted in
    the workspace's control block) marks its blob and still leaves the workspace ready: the
    next compression on the same workspace equals the oracle's."""
    ws = N.Workspace(DEV)
    rng = np.random.default_rng(62)
    n = 200_000
    pa = rng.lognormal(size=n)
    xa = pa * (1.0 + 0.3 + rng.uniform(-0.01, 0.01, n))   # ratios around 0.3: bins ~150
    pb, xb = synth.plain_pair(n, seed=synth.seed_for(0, 63))
    pb, xb = pb.numpy(), xb.numpy()
    pad, xad = torch.from_numpy(pa).to(DEV), torch.from_numpy(xa).to(DEV)
    pbd, xbd = torch.from_numpy(pb).to(DEV), torch.from_numpy(xb).to(DEV)
    N.compress(pbd, xbd, 1e-3, 8, workspace=ws)            # initialises the workspace
    torch.cuda.synchronize()
    for anchor in (N.ANCHOR_ZERO, N.ANCHOR_MIN):
        ws.buf[_CTRL_WIN_ERR:_CTRL_WIN_ERR + 4].view(torch.int32).fill_(1)
        bad = N.compress(pad, xad, 1e-3, 8, anchor=anchor, workspace=ws)
        torch.cuda.synchronize()
        assert N.parse_header(N.header_bytes(bad))["status"] == N.ERR_CORRUPT
        want = O.compress(pb, xb, 1e-3, 8).to_bytes()
        blob = N.compress(pbd, xbd, 1e-3, 8, workspace=ws)
        torch.cuda.synchronize()
        got = blob[:len(want)].cpu().numpy().tobytes()
        assert got == want, _first_diff(got, want)


def _fraction_pair(n, frac, T, seed):
    """A pair whose incompressible fraction is close to `frac` at E = 1e-4, B = 4: the bulk
    moves by a ratio inside two bins, the chosen fraction by ratios spread over thousands."""
    rng = np.random.default_rng(seed)
    p = rng.lognormal(0.0, 1.0, n)
    r = np.where(rng.random(n) < 0.5, 1e-5, 3.1e-4)
    far = rng.random(n) < frac
    r[far] = rng.uniform(0.3, 0.9, int(far.sum()))
    return p.astype(T), (p * (1.0 + r)).astype(T)


@pytest.mark.parametrize("T,frac,n", [(np.float64, 0.7, 5_000_017), (np.float64, 0.8, 5_000_017),
                                      (np.float64, 1.0, (1 << 24) + 12_345),
                                      (np.float32, 0.4, 5_000_017), (np.float32, 0.6, 5_000_017),
                                      (np.float32, 0.95, (1 << 24) + 12_345)])
def test_high_incompressible_fractions(T, frac, n):
    """Incompressible fractions on both sides of the point where the incompressible table can
    reach the scratch area in the blob tail (75% for float64, 50% for float32), at sizes of
    thousands of sub-blocks (several waves of the copy kernel)."""
    p, x = _fraction_pair(n, frac, T, seed=int(frac * 100) + (T == np.float32))
    h, _ = check_pair(p, x, 1e-4, 4, ranges=[(n // 3, 70_000), (n - 5000, 5000)])
    L = np.dtype(T).itemsize
    assert abs(h["n_inc"] / n - frac) < 0.05
    assert (h["n_inc"] * L > n * (L - 2)) == (frac > (L - 2) / L)


_BOUNDARY_BINS = (0, 1, -1, 5, -7, 100, -250, 1000, 5000, -9000, 16000, 16382, 16383, 16384,
                  -16383, -16384, 20000, -30000)


def _check_boundary_pair(T, E, per_bin=3000, seed=17):
    """Points a few ulps either side of the error bound |p m - x| = E |x| (§III.C) of their
    own bin, for bins near the zero change and far from it (beyond +-16383 bins as well)."""
    rng = np.random.default_rng(seed)
    Et = T(E)
    w = T(Et + Et)
    a = T(-Et)
    ps, xs = [], []
    for b in _BOUNDARY_BINS:
        m = T(T(1) + T(a + T(T(b) + T(0.5)) * w))
        p = rng.lognormal(size=per_bin).astype(T)
        R = (p * m).astype(T)
        sign = rng.choice([-1.0, 1.0], per_bin)
        x = (R.astype(np.float64) / (1.0 + sign * float(Et))).astype(T)
        x = (x + rng.integers(-3, 4, per_bin).astype(T) * np.spacing(x)).astype(T)
        ps.append(p)
        xs.append(x)
    order = rng.permutation(per_bin * len(_BOUNDARY_BINS))
    return np.concatenate(ps)[order], np.concatenate(xs)[order]


@pytest.mark.parametrize("T", [np.float32, np.float64])
@pytest.mark.parametrize("E", [1e-3, 3.3e-5])
@pytest.mark.parametrize("anchor", [N.ANCHOR_ZERO, N.ANCHOR_MIN])
def test_check_boundary_near_and_far_bins(T, E, anchor):
    p, x = _check_boundary_pair(T, E)
    h, _ = check_pair(p, x, E, 8, anchor=anchor)
    assert 0 < h["n_inc"] < h["n"]


# ---------------------------------------------------------------------------------------
# automatic index length (B = 0, §IV.B.2)
# ---------------------------------------------------------------------------------------
def _many_bins_pair(n=1 << 21, seed=31):
    """Ratios spread over about 470000 bins of width 2^-19: more than 65535 non-empty bins."""
    rng = np.random.default_rng(seed)
    p = rng.lognormal(size=n)
    return p, p * (1.0 + rng.uniform(-0.45, 0.45, n))


@pytest.mark.parametrize("case", ["plain", "plain_min", "climate", "flash", "many_bins"])
def test_auto_B_matches_oracle(case):
    anchor = N.ANCHOR_MIN if case == "plain_min" else N.ANCHOR_ZERO
    if case.startswith("plain"):
        p, x = synth.plain_pair(1 << 20, seed=synth.seed_for(0, 41))
        p, x, E = p.numpy(), x.numpy(), 1e-3
    elif case == "climate":
        (_, a), (_, b) = list(synth.climate_series(360, 720, steps=2))
        p, x, E = a.numpy(), b.numpy(), 1e-3
    elif case == "flash":
        xs = synth.flash_series(side=64, steps=2)
        p, x, E = xs[0].numpy(), xs[1].numpy(), 1e-4
    else:
        p, x = _many_bins_pair()
        E = 2.0 ** -20
    h, _ = check_pair(p, x, E, 0, anchor=anchor, ranges=[(1000, 5000)])
    bins, counts = O.histogram(*_oracle_bins(p, x, E, anchor))
    assert h["B"] == O.choose_B(counts, p.size, p.dtype.itemsize)


def _oracle_bins(p, x, E, anchor):
    T = p.dtype.type
    E_T, w, inv_w, cap = O.grid_constants(T, E)
    ratio, binnable = O.change_ratio(p, x, cap)
    a = O.grid_anchor(ratio, binnable, E_T, anchor)
    return O.bin_ids(ratio, binnable, a, inv_w), binnable


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_auto_B_refused_while_capturing():
    p, x = synth.plain_pair(4096, seed=synth.seed_for(0, 42))
    pd, xd = p.to(DEV), x.to(DEV)
    params = N.make_params(torch.float64, 0, 1e-3)
    blob = torch.empty(N.compress_bound(4096, params), dtype=torch.uint8, device=DEV)
    ws = torch.zeros(N.workspace_bytes(4096, params), dtype=torch.uint8, device=DEV)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    rc = None
    with torch.cuda.graph(graph, stream=s):
        rc = N.lib().numarck_compress(pd.data_ptr(), xd.data_ptr(), 4096, ctypes.byref(params),
                                      blob.data_ptr(), blob.numel(), ws.data_ptr(), ws.numel(),
                                      s.cuda_stream)
    assert rc == N.ERR_INVALID_ARG


def test_corrupted_offset_tables_are_reported():
    """A blob whose offset tables disagree with its index table is refused through the status
    word, by the decoder and by the chained step (whose next blob then carries the error)."""
    p, x = synth.plain_pair(200_000, seed=synth.seed_for(0, 95))
    y, _ = synth.plain_pair(200_000, seed=synth.seed_for(0, 96))
    pd, xd, yd = p.to(DEV), x.to(DEV), y.to(DEV)
    blob = N.compress(pd, xd, 1e-3, 8)
    torch.cuda.synchronize()
    h = N.parse_header(N.header_bytes(blob))
    assert h["nsub"] > 8
    for field, idx, how in (("off_sub_off", 5, lambda v: v + 3),
                            ("off_sub_off", 7, lambda v: -10 ** 9),
                            ("off_sub_off", 2, lambda v: h["n_inc"] + 1),
                            ("off_idx_off", 0, lambda v: v + 16)):
        bad = blob.clone()
        at = h[field] + 8 * idx
        word = bad[at: at + 8].view(torch.int64)
        word.copy_(torch.tensor([how(int(word.item()))], dtype=torch.int64, device=DEV))
        status = torch.zeros(1, dtype=torch.int32, device=DEV)
        N.decompress(bad, pd, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == N.ERR_CORRUPT, (field, idx)
        status.zero_()
        _, nxt = N.decompress_compress(bad, pd, yd, 1e-3, 8, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == N.ERR_CORRUPT, (field, idx)
        assert N.parse_header(N.header_bytes(nxt))["status"] == N.ERR_CORRUPT
    # the intact blob still decodes
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    N.decompress(blob, pd, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
