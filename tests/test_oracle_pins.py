"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: hand-computed values,
closed forms, brute force on tiny inputs, the DP optimum of §V.D, the worked numbers of
Fig. 2, exact rational arithmetic, or invariants. A plausible slip in the oracle (a dropped
term, a wrong sign or index, a swapped operand, a wrong tie-break or bit order) fails at least
one of them.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import numarck_oracle as O


# ---------------------------------------------------------------------------------------
# helpers written for the tests (independent of the oracle's code)
# ---------------------------------------------------------------------------------------
def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def _dp_max_coverage(values, width, k):
    """§V.D, Fig. 15 prose: OPT(i, j) = max(OPT(i+1, j), OPT(i+c(i), j-1) + c(i)) over the
    sorted values, c(i) = #values in [v_i, v_i + width]; OPT(N+1, *) = OPT(*, 0) = 0."""
    v = sorted(values)
    N = len(v)
    c = [sum(1 for x in v[i:] if x <= v[i] + width) for i in range(N)]
    OPT = [[0] * (k + 1) for _ in range(N + 2)]
    for i in range(N - 1, -1, -1):
        for j in range(1, k + 1):
            OPT[i][j] = max(OPT[i + 1][j], OPT[i + c[i]][j - 1] + c[i])
    return OPT[0][k]


def _bits_lsb_first(indices, B):
    """Reference bit writer with Python integers: index i occupies bits [iB, iB+B)."""
    acc = 0
    for i, v in enumerate(indices):
        acc |= int(v) << (i * B)
    nbytes = (len(indices) * B + 7) // 8
    return acc.to_bytes(nbytes, "little") if nbytes else b""


# ---------------------------------------------------------------------------------------
# Step 0: grid constants
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("T", [np.float32, np.float64])
def test_grid_constants_dyadic(T):
    E_T, w, inv_w, cap = O.grid_constants(T, 2.0 ** -10)
    assert E_T == T(2.0 ** -10) and w == T(2.0 ** -9) and inv_w == T(512) and cap == T(4096)
    assert all(type(v) is T for v in (E_T, w, inv_w, cap))


def test_grid_constants_fp32_rounds_E_first():
    # E = 1e-3 is rounded to float32 before doubling (all arithmetic in T)
    E_T, w, inv_w, _ = O.grid_constants(np.float32, 1e-3)
    assert E_T == np.float32(1e-3) and w == np.float32(2) * np.float32(1e-3)
    assert inv_w == np.float32(np.float32(1) / w)


# ---------------------------------------------------------------------------------------
# Step 1: change ratio (Eq. 1)
# ---------------------------------------------------------------------------------------
def test_change_ratio_closed_forms():
    cap = np.float64(4096)
    prev = np.array([1.0, 2.0, -4.0, 1.0, 0.0, 0.0, np.inf, 1.0, np.nan, 1.0, 1.0, 4.0])
    cur = np.array([1.0 + 3 * 2 ** -9, 3.0, -3.0, 0.0, 5.0, 0.0, 1.0, np.inf, 1.0,
                    1.0 + 4096.0, 1.0 + 4096.0 + 2 ** -40, -4.0])
    r, ok = O.change_ratio(prev, cur, cap)
    assert r[0] == 3 * 2 ** -9                 # (x - p) / p, exact
    assert r[1] == 0.5 and r[2] == -0.25       # sign follows Eq. 1 (p negative)
    assert r[3] == -1.0 and ok[3]              # cur = 0 is binnable (ratio -1)
    assert not ok[4] and not ok[5]             # prev = 0: inf and NaN
    assert not ok[6] and not ok[7] and not ok[8]
    assert ok[9] and r[9] == 4096.0            # |ratio| == cap is binnable
    assert not ok[10]                          # just above the cap is not
    assert r[11] == -2.0 and ok[11]


def test_change_ratio_is_T_precision():
    # float32: (x - p) / p rounded twice in float32, not computed in double
    p = np.array([3.0], dtype=np.float32)
    x = np.array([np.float32(3.0) + np.float32(2 ** -20)], dtype=np.float32)
    r, _ = O.change_ratio(p, x, np.float32(1e9))
    assert r.dtype == np.float32
    d32 = np.float32(x[0] - p[0])
    assert r[0] == np.float32(d32 / np.float32(3.0))


# ---------------------------------------------------------------------------------------
# Step 3: bin ids and edges (readings R2, R3)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("T", [np.float32, np.float64])
def test_bin_ids_dyadic_centres_and_edges(T):
    E_T, w, inv_w, cap = O.grid_constants(T, 2.0 ** -10)
    m = np.arange(-40, 41)
    ratio = (m * 2.0 ** -9).astype(T)             # on the centres of the ZERO grid
    b = O.bin_ids(ratio, np.ones(m.size, bool), T(-E_T), inv_w)
    assert np.array_equal(b, m)
    # edges: a + b*w belongs to bin b (half-open bins [edge, edge + w))
    edges = (-(2.0 ** -10) + m * 2.0 ** -9).astype(T)
    b = O.bin_ids(edges, np.ones(m.size, bool), T(-E_T), inv_w)
    assert np.array_equal(b, m)
    # 2^-20 below an edge: every step stays exact in float32 and float64 -> previous bin
    below = (edges.astype(np.float64) - 2.0 ** -20).astype(T)
    b = O.bin_ids(below, np.ones(m.size, bool), T(-E_T), inv_w)
    assert np.array_equal(b, m - 1)


def test_bin_ids_monotone_in_ratio():
    rng = np.random.default_rng(5)
    for T in (np.float32, np.float64):
        E_T, w, inv_w, cap = O.grid_constants(T, 1e-3)
        r = np.sort(rng.uniform(-0.6, 0.6, 20000).astype(T))
        b = O.bin_ids(r, np.ones(r.size, bool), T(-E_T), inv_w)
        assert np.all(np.diff(b) >= 0)
        # every ratio lies within one ulp-scale slack of its bin [a + b w, a + (b+1) w)
        lo = -E_T + b.astype(np.float64) * float(w)
        assert np.all(r.astype(np.float64) >= lo - 1e-5) and np.all(r < lo + float(w) + 1e-5)


def test_min_anchor_puts_minimum_in_bin_zero():
    rng = np.random.default_rng(7)
    p = rng.lognormal(size=500)
    x = p * (1 + rng.normal(0, 0.01, 500))
    T = np.float64
    E_T, w, inv_w, cap = O.grid_constants(T, 1e-3)
    r, ok = O.change_ratio(p, x, cap)
    a = O.grid_anchor(r, ok, E_T, O.ANCHOR_MIN)
    assert a == r.min()
    b = O.bin_ids(r, ok, a, inv_w)
    assert b.min() == 0 and b[np.argmin(r)] == 0
    assert O.grid_anchor(r, np.zeros_like(ok), E_T, O.ANCHOR_MIN) == 0.0
    assert O.grid_anchor(r, ok, E_T, O.ANCHOR_ZERO) == -E_T


def test_min_anchor_zero_minimum_is_positive_zero():
    """Reading R2: a zero minimum ratio is taken as +0. An unchanged point with a negative prev
    has ratio (x - p) / p = +0 / (-1) = -0, so the raw minimum can be -0; the grid origin, and
    the header's `a` field written from it, must still be +0 (sign bit clear)."""
    for T in (np.float32, np.float64):
        for prev, cur in (([-1.0], [-1.0]),                     # only a -0 ratio
                          ([2.0, -1.0], [2.0, -1.0]),           # +0 then -0
                          ([-1.0, 2.0], [-1.0, 2.0]),           # -0 then +0
                          ([1.0, -1.0, 1.0], [1.5, -1.0, 1.5])):
            p = np.array(prev, dtype=T)
            x = np.array(cur, dtype=T)
            E_T, w, inv_w, cap = O.grid_constants(T, 1e-3)
            r, ok = O.change_ratio(p, x, cap)
            a = O.grid_anchor(r, ok, E_T, O.ANCHOR_MIN)
            assert a == 0 and not np.signbit(a), (T, prev, cur)
            blob = O.compress(p, x, 1e-3, 8, anchor=O.ANCHOR_MIN)
            h = O.parse_header(blob.to_bytes())
            assert h["a"] == 0.0 and not np.signbit(h["a"])
            # the unchanged points sit in bin 0, whose centre is +E (0 + 0.5 * 2E)
            assert blob.centres[0] == T(0.5) * w


# ---------------------------------------------------------------------------------------
# Step 3b: histogram, hand counted
# ---------------------------------------------------------------------------------------
def test_histogram_hand_counted():
    b = np.array([3, -1, 3, 0, 7, 3, -1, 0, 0, 0, 99, 5])
    ok = np.array([1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 0, 1], bool)   # b=99 is not binnable
    bins, counts = O.histogram(b, ok)
    assert bins.tolist() == [-1, 0, 3, 5, 7]
    assert counts.tolist() == [2, 4, 3, 1, 1]
    assert counts.sum() == ok.sum()


# ---------------------------------------------------------------------------------------
# Step 4: top-k selection vs brute force and the DP optimum (§IV.B.1, §V.D)
# ---------------------------------------------------------------------------------------
def _brute_top_k(bins, counts, k):
    """Among all subsets of min(k, #bins) bins: maximum coverage, then the lexicographically
    smallest ascending tuple (equivalent to ties going to smaller bins)."""
    m = min(k, len(bins))
    best = None
    for sub in itertools.combinations(range(len(bins)), m):
        cov = sum(counts[i] for i in sub)
        key = (-cov, tuple(sorted(bins[i] for i in sub)))
        if best is None or key < best:
            best = key
    return list(best[1]) if best else []


def test_top_k_matches_brute_force():
    rng = np.random.default_rng(11)
    for trial in range(300):
        nb = int(rng.integers(1, 9))
        bins = np.sort(rng.choice(np.arange(-20, 20), nb, replace=False))
        counts = rng.integers(1, 5, nb)          # small counts: many ties
        k = int(rng.integers(1, 5))
        got = O.top_k(bins, counts, k).tolist()
        assert got == _brute_top_k(bins.tolist(), counts.tolist(), k), (bins, counts, k)
        # tie-break independent statement: coverage equals the sum of the k largest counts
        cov = sum(int(counts[bins.tolist().index(x)]) for x in got)
        assert cov == int(np.sort(counts)[::-1][:k].sum())


def test_top_k_fewer_bins_than_k_selects_all():
    bins = np.array([-3, 2, 9])
    counts = np.array([1, 5, 2])
    assert O.top_k(bins, counts, 255).tolist() == [-3, 2, 9]
    assert O.top_k(np.zeros(0, np.int64), np.zeros(0, np.int64), 3).tolist() == []


def test_top_k_coverage_bounded_by_dp_optimum():
    rng = np.random.default_rng(13)
    E = 2.0 ** -6
    for trial in range(60):
        n = int(rng.integers(3, 14))
        r = np.round(rng.normal(0, 0.05, n) * 2 ** 12) / 2 ** 12     # dyadic ratios
        p = np.ones(n)
        x = p + r
        T = np.float64
        E_T, w, inv_w, cap = O.grid_constants(T, E)
        ratio, ok = O.change_ratio(p, x, cap)
        b = O.bin_ids(ratio, ok, T(-E_T), inv_w)
        bins, counts = O.histogram(b, ok)
        k = int(rng.integers(1, 4))
        sel = O.top_k(bins, counts, k)
        cov = int(sum(counts[np.searchsorted(bins, s)] for s in sel))
        assert cov <= _dp_max_coverage(ratio.tolist(), 2 * E, k)


def test_dp_optimum_reached_on_grid_aligned_clusters():
    # clusters sit inside single grid bins, >= 2 bins apart, so no interval of width 2E
    # covers two of them and grid-aligned top-k is optimal
    E = 2.0 ** -6
    w = 2 * E
    rng = np.random.default_rng(17)
    centres = np.array([-6, -2, 1, 4, 9]) * w
    sizes = [3, 6, 1, 4, 2]
    ratio = np.concatenate([c + rng.uniform(-0.3, 0.3, s) * w for c, s in zip(centres, sizes)])
    T = np.float64
    E_T, _, inv_w, _ = O.grid_constants(T, E)
    b = O.bin_ids(ratio, np.ones(ratio.size, bool), T(-E_T), inv_w)
    bins, counts = O.histogram(b, np.ones(ratio.size, bool))
    for k in (1, 2, 3):
        sel = O.top_k(bins, counts, k)
        cov = int(sum(counts[np.searchsorted(bins, s)] for s in sel))
        assert cov == _dp_max_coverage(ratio.tolist(), w, k)


# ---------------------------------------------------------------------------------------
# Step 4b: centres (reading R6)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("T", [np.float32, np.float64])
def test_centres_closed_form(T):
    E_T, w, inv_w, cap = O.grid_constants(T, 2.0 ** -10)
    sel = np.array([-7, -1, 0, 1, 12])
    c = O.centres_of(sel, T(-E_T), w, T)
    assert c.dtype == T
    assert np.array_equal(c, (sel * 2.0 ** -9).astype(T))        # ZERO grid: c = 2E*b
    assert c[2] == 0.0 and not np.signbit(c[2])
    a = T(-0.3125)
    c = O.centres_of(sel, a, w, T)
    assert np.array_equal(c, (-0.3125 + (sel + 0.5) * 2.0 ** -9).astype(T))


# ---------------------------------------------------------------------------------------
# Step 5: indexing with the error check, Eq. 4 reconstruction
# ---------------------------------------------------------------------------------------
def test_worked_example(golden_dir):
    g = _load(golden_dir, "worked_example.json")
    p = np.array(g["prev"], dtype=np.float64)
    x = np.array(g["cur"], dtype=np.float64)
    for anchor, sel_key in ((O.ANCHOR_ZERO, "selected_zero"), (O.ANCHOR_MIN, "selected_min")):
        T = np.float64
        E_T, w, inv_w, cap = O.grid_constants(T, g["E"])
        ratio, ok = O.change_ratio(p, x, cap)
        a = O.grid_anchor(ratio, ok, E_T, anchor)
        b = O.bin_ids(ratio, ok, a, inv_w)
        if anchor == O.ANCHOR_ZERO:
            assert [int(v) if o else None for v, o in zip(b, ok)] == g["bins_zero"]
            bins, counts = O.histogram(b, ok)
            assert {str(int(k)): int(c) for k, c in zip(bins, counts)} == g["hist_zero"]
        else:
            assert a == g["a_min"]
        bins, counts = O.histogram(b, ok)
        assert O.top_k(bins, counts, 3).tolist() == g[sel_key]
        blob = O.compress(p, x, g["E"], g["B"], anchor=anchor, block_bytes=16)
        assert blob.centres.tolist() == g["centres"]
        assert blob.indices.tolist() == g["indices"]
        assert blob.exact.tolist() == g["exact"]
        assert b"".join(blob.index_blocks).hex() == g["packed_one_block_hex"]
        assert O.decompress(blob.to_bytes(), p).tolist() == g["recon"]
        small = O.compress(p, x, g["E"], g["B"], anchor=anchor, block_bytes=g["block_bytes_small"])
        assert [d.hex() for d in small.index_blocks] == g["packed_blocks_small_hex"]
        assert small.inc_off.tolist() == g["inc_off_small"]
        assert O.decompress(small.to_bytes(), p).tolist() == g["recon"]


def test_value_space_check_rejects_decreasing_edge_point():
    # bin -3 of the E = 1/16 ZERO grid covers ratios [-7/16, -5/16); centre -3/8.
    p = np.array([1.0, 1.0, 1.0])
    x = np.array([1 - 7 / 16, 1 - 3 / 8, 1 - 3 / 8])
    blob = O.compress(p, x, 1 / 16, 1)             # k = 1: only bin -3 is selected
    assert blob.centres[0] == -0.375
    # ratio -7/16: |0.625 - 0.5625| = 1/16 > (1/16) * 0.5625 -> incompressible
    assert blob.indices.tolist() == [1, 0, 0]


def test_unchanged_points_reconstruct_exactly_zero_anchor():
    rng = np.random.default_rng(19)
    for T in (np.float32, np.float64):
        p = rng.lognormal(size=3000).astype(T) * T(-1) ** rng.integers(0, 2, 3000).astype(T)
        x = p.copy()
        blob = O.compress(p, x, 1e-3, 4)
        assert np.all(blob.indices == 0) and blob.header["n_sel"] == 1
        assert blob.centres[0] == 0
        R = O.decompress(blob.to_bytes(), p)
        assert np.array_equal(R.view(np.uint8), x.view(np.uint8))


def test_error_bound_holds_exactly_for_compressible_points():
    """Every compressible point: |R - x| <= E_T * |x| up to the two roundings of the T check,
    verified in exact rational arithmetic."""
    rng = np.random.default_rng(23)
    for T, eps in ((np.float32, 2.0 ** -24), (np.float64, 2.0 ** -53)):
        n = 4000
        p = rng.lognormal(size=n).astype(T)
        x = (p * (1 + rng.normal(0, 0.02, n))).astype(T)
        E = 1e-3
        blob = O.compress(p, x, E, 6)
        R = O.decompress(blob.to_bytes(), p)
        E_T = Fraction(float(T(E)))
        bound = E_T * (1 + Fraction(4) * Fraction(eps))
        comp = np.nonzero(blob.indices != 63)[0]
        assert comp.size > n // 2
        for j in comp[:: max(1, comp.size // 800)]:
            xr, Rr = Fraction(float(x[j])), Fraction(float(R[j]))
            assert abs(Rr - xr) <= bound * abs(xr)


def test_special_inputs_become_markers_and_roundtrip_bits():
    T = np.float64
    p = np.array([0.0, -0.0, np.inf, np.nan, 1.0, 1.0, 1e-310, 2.0])
    nanpay = np.frombuffer(np.uint64(0x7FF8DEADBEEF0001).tobytes(), dtype=np.float64)[0]
    x = np.array([1.0, 0.0, 1.0, 1.0, nanpay, -np.inf, 1.0, 2.0])
    blob = O.compress(p, x, 1e-3, 3)
    M = 7
    assert blob.indices[:7].tolist() == [M] * 7 and blob.indices[7] == 0
    R = O.decompress(blob.to_bytes(), p)
    assert np.array_equal(R.view(np.uint64), x.view(np.uint64))     # incl. the NaN payload


def test_all_non_finite_and_empty_inputs():
    p = np.full(10, np.nan)
    blob = O.compress(p, p.copy(), 1e-3, 8)
    assert blob.header["n_sel"] == 0 and np.all(blob.centres == 0)
    assert blob.header["n_inc"] == 10
    e = O.compress(np.zeros(0), np.zeros(0), 1e-3, 8)
    assert e.header["nblocks"] == 0 and e.header["n_inc"] == 0 and e.header["nsub"] == 0
    assert e.idx_off.tolist() == [0] and e.inc_off.tolist() == [0]
    assert O.decompress(e.to_bytes(), np.zeros(0)).size == 0


def test_B1_single_bin():
    rng = np.random.default_rng(29)
    p = rng.lognormal(size=100)
    x = p * (1 + rng.normal(0, 1e-4, 100))
    blob = O.compress(p, x, 1e-3, 1)
    assert blob.header["n_sel"] == 1 and set(blob.indices.tolist()) <= {0, 1}


# ---------------------------------------------------------------------------------------
# Step 6: bit packing and block layout (§IV.C, Fig. 2, Eq. 6)
# ---------------------------------------------------------------------------------------
def test_pack_hand_example():
    # B = 3, [1,2,3,4,5]: stream bits 100 010 110 001 101 -> 0xD1, 0x58
    assert O.pack_block(np.array([1, 2, 3, 4, 5]), 3) == bytes([0xD1, 0x58])
    assert O.pack_block(np.array([0x12, 0xFF, 0x00]), 8) == bytes([0x12, 0xFF, 0x00])
    assert O.pack_block(np.array([0x1234, 0xBEEF]), 16) == bytes([0x34, 0x12, 0xEF, 0xBE])


@pytest.mark.parametrize("B", [1, 2, 3, 5, 7, 8, 10, 13, 16])
def test_pack_matches_integer_bit_writer_and_roundtrips(B):
    rng = np.random.default_rng(B)
    for n in (1, 7, 8, 33, 257):
        v = rng.integers(0, 1 << B, n)
        data = O.pack_block(v, B)
        assert data == _bits_lsb_first(v.tolist(), B)
        assert len(data) == -(-(n * B) // 8)
        assert np.array_equal(O.unpack_block(data, n, B), v)


def test_fig2_block_layout(golden_dir):
    g = _load(golden_dir, "fig2_header.json")
    lay = O.layout(g["n"], np.float32, g["B"], g["block_bytes"])
    assert O.elements_per_block(g["block_bytes"], g["B"]) == g["elements_per_block"]
    assert lay["epb"] == g["elements_per_block"] and lay["nblocks"] == g["nblocks"]
    assert (lay["off_idx_off"] - lay["off_centres"]) >= g["bin_centers"] * 4
    assert sum(lay["counts"]) == g["n"]
    alpha = O.incompressible_ratio(g["n"], g["n"] - g["n_incompressible"])
    assert abs(alpha - 0.0245) < 1e-4                  # 2.45% for the UU example


def test_blob_size_matches_eq6_plus_layout_overhead():
    rng = np.random.default_rng(31)
    for T, B, bb in ((np.float64, 8, 1 << 20), (np.float32, 10, 4096), (np.float64, 13, 1000)):
        n = 50000
        p = rng.lognormal(size=n).astype(T)
        x = (p * (1 + rng.normal(0, 0.01, n))).astype(T)
        blob = O.compress(p, x, 1e-3, B, block_bytes=bb)
        h = blob.header
        L = np.dtype(T).itemsize
        alpha = h["n_inc"] / n
        eq6 = O.estimated_file_size(n, B, alpha, L)
        # Eq. 6 counts n*B/8 index bytes; each block is rounded up to whole bytes and then
        # to 16, the centre table and offset tables/sections are 256-aligned, plus header.
        index_exact = sum(-(-(c * B) // 8) for c in O.layout(n, T, B, bb)["counts"])
        assert abs(index_exact - n * B / 8) < h["nblocks"]
        assert len(blob.to_bytes()) == h["total_bytes"]
        assert h["total_bytes"] == h["off_exact"] + h["n_inc"] * L
        overhead = h["total_bytes"] - eq6
        assert 0 <= overhead <= (256 * 6 + 16 * (h["nblocks"] + 1) + 8 * (2 * h["nblocks"] + 2)
                                 + 8 * h["nsub"] + 16 * h["nblocks"] + 1)


def test_offsets_tables_are_prefix_counts():
    rng = np.random.default_rng(37)
    n = 30000
    p = rng.lognormal(size=n)
    x = p * (1 + np.where(rng.random(n) < 0.2, rng.uniform(-0.5, 0.5, n), rng.normal(0, 1e-3, n)))
    blob = O.compress(p, x, 1e-3, 4, block_bytes=1500)       # epb = 3000, 10 blocks
    M = 15
    mk = blob.indices == M
    epb = blob.header["epb"]
    for q in range(blob.header["nblocks"] + 1):
        assert blob.inc_off[q] == mk[: min(n, q * epb)].sum()
    starts = [s for q in range(blob.header["nblocks"])
              for s in range(q * epb, min(n, (q + 1) * epb), O.SUB_BLOCK)]
    assert blob.sub_off.tolist() == [int(mk[:s].sum()) for s in starts]
    assert blob.exact.size == mk.sum() and np.array_equal(blob.exact, x[mk])


# ---------------------------------------------------------------------------------------
# Decompression and partial decompression
# ---------------------------------------------------------------------------------------
def test_decompress_closed_form():
    rng = np.random.default_rng(41)
    for T in (np.float32, np.float64):
        n = 20000
        p = rng.lognormal(size=n).astype(T)
        x = (p * (1 + rng.normal(0, 0.003, n))).astype(T)
        blob = O.compress(p, x, 1e-3, 5)
        R = O.decompress(blob.to_bytes(), p)
        M = 31
        c = blob.centres
        comp = blob.indices != M
        expect = p[comp] * (T(1) + c[blob.indices[comp]])
        assert np.array_equal(R[comp], expect.astype(T))
        assert np.array_equal(R[~comp].view(np.uint8), x[~comp].view(np.uint8))


def test_decompress_range_equals_slice():
    rng = np.random.default_rng(43)
    n = 25000
    p = rng.lognormal(size=n).astype(np.float32)
    x = (p * (1 + np.where(rng.random(n) < 0.1, rng.uniform(-0.5, 0.5, n),
                           rng.normal(0, 2e-3, n)))).astype(np.float32)
    data = O.compress(p, x, 1e-3, 7, block_bytes=700).to_bytes()   # epb = 800
    full = O.decompress(data, p)
    cases = [(0, n), (0, 0), (n, 0), (799, 2), (800, 800), (123, 5000), (n - 1, 1)]
    cases += [(int(s), int(rng.integers(0, n - s + 1))) for s in rng.integers(0, n, 20)]
    for s, c in cases:
        seg = O.decompress_range(data, p[s: s + c], s, c)
        assert np.array_equal(seg.view(np.uint32), full[s: s + c].view(np.uint32)), (s, c)


# ---------------------------------------------------------------------------------------
# Metrics (Eq. 2, 3, 5, 6) against the paper's worked numbers
# ---------------------------------------------------------------------------------------
def test_metrics_against_paper_examples():
    # §V.B CMIP example: 32-bit data, B = 12, index table zlib ratio 2.2, 2% incompressible
    per_point_bits = 12 / 2.2 + 0.02 * 32
    cr = O.compression_ratio(32, per_point_bits)
    assert int(cr * 10) / 10 == 5.2                 # the paper prints 5.25... as 5.2
    # Eq. 6 by hand: B = 2, L = 8, n = 16, alpha = 1/4 -> 4*8 + 16*2/8 + 16*(1/4)*8 = 68
    assert O.estimated_file_size(16, 2, 0.25, 8) == 68
    # Eq. 3 by hand: errors 0, 0.1, 0.2 over n = 4 points (one point is 0 -> skipped)
    cur = np.array([1.0, 2.0, 5.0, 0.0])
    rec = np.array([1.0, 2.2, 4.0, 0.0])
    assert abs(O.mean_error_rate(cur, rec) - 0.3 / 4) < 1e-15
    # Eq. 5: alpha = (n - compressible) / n
    assert O.incompressible_ratio(200, 150) == 0.25


# ---------------------------------------------------------------------------------------
# Automatic index length (§IV.B.2, Eqs. 5 and 6), reading R10
# ---------------------------------------------------------------------------------------
def test_file_size_hand_example():
    """Six bins holding 600, 200, 100, 50, 30, 20 of n = 1000 float64 points. By hand, in bytes:
    B=1: 2*8 + 1000/8 + 400*8 = 3341; B=2: 32 + 250 + 100*8 = 1082; B=3: 64 + 375 + 0 = 439;
    B=4: 128 + 500 = 628; B=5: 256 + 625 = 881. The smallest is B = 3."""
    counts = np.array([30, 600, 20, 100, 200, 50])
    bits = O.file_size_bits(counts, 1000, 8, B_max=5)
    assert bits == [8 * 3341, 8 * 1082, 8 * 439, 8 * 628, 8 * 881]
    assert O.choose_B(counts, 1000, 8) == 3


def test_choose_B_single_bin_and_uniform_bins():
    # every point in one bin: the 1-bit table already covers it, B = 1
    assert O.choose_B(np.array([10 ** 6]), 10 ** 6, 8) == 1
    # 15 equal bins of 10^4 float32 points: B = 4 covers them all (64 + 75000 bytes);
    # B = 3 leaves 8 bins out (32 + 56250 + 80000 * 4), B = 5 doubles the table (128 + 93750)
    assert O.choose_B(np.full(15, 10 ** 4), 150_000, 4) == 4


def test_choose_B_tie_goes_to_smaller_B():
    """n = 96 float32 points: one bin of 80, bins of 3 and 2, eleven bins of 1. In bits,
    B=1: 64 + 96 + 32 * 16 = 672 and B=2: 128 + 192 + 32 * 11 = 672 tie; B=3 is 768."""
    counts = np.array([80, 3, 2] + [1] * 11)
    bits = O.file_size_bits(counts, 96, 4, B_max=3)
    assert bits == [672, 672, 768]
    assert O.choose_B(counts, 96, 4) == 1


def test_auto_B_blob_equals_the_chosen_B():
    rng = np.random.default_rng(21)
    p = rng.lognormal(size=20_000)
    x = p * (1 + rng.normal(0, 3e-3, p.size))
    auto = O.compress(p, x, 1e-3, 0)
    B = O.parse_header(auto.to_bytes())["B"]
    assert 1 <= B <= 16
    assert auto.to_bytes() == O.compress(p, x, 1e-3, B).to_bytes()
