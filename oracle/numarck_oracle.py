"""NUMARCK oracle: a plain, slow, obviously correct CPU restatement of the compression hot path.

TEST INFRASTRUCTURE ONLY. This module exists to check the CUDA library. Only the test suite
(tests/), ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and its
``--impl reference`` arm) may import it. The library and its Python binding never import it,
and it imports nothing from them: it shares no code, tables or constants generators with the
GPU path. Its only inputs are arrays (seeded synthetic data from the separate generator
module, or hand-written fixtures).

Source: Z. Yuan et al., "Parallel Implementation of Lossy Data Compression for Temporal Data
Sets", arXiv 1703.02438. Section, equation and figure numbers below are the paper's.

Arithmetic. Every floating-point step is done in the element type T (numpy float32 or
float64). numpy evaluates each elementwise operation on its own and rounds it once,
round-to-nearest-even, so no multiply-add is fused and the order of operations is exactly
the order written here. Library primitives used as steps: np.unique / np.bincount (counting),
np.lexsort / np.sort (ordering), np.packbits (bit order), np.searchsorted (lookup).

Readings of the paper where it is silent, ambiguous or garbled (each is used below):
  R1  a ratio that is not finite (prev = 0, non-finite inputs) is not binnable: the point
      is incompressible. A ratio with |ratio| > cap = 2^21 * 2E is not binnable either
      (it keeps every bin id inside a 2^22-bin window).
  R2  grid anchor: ZERO (a = -E, default: bin 0 is centred on ratio 0) or MIN (a = the
      minimum binnable ratio, 0 when there is none; a zero minimum is +0, never -0).
  R3  bin id = floor((ratio - a) * (1 / (2E))), all in T.
  R4  the histogram counts every binnable point.
  R5  k = 2^B - 1 bins; ties in count go to the smaller bin id; selected bins are numbered
      0..|S|-1 in ascending bin order; with fewer than k non-empty bins all are selected.
  R6  centre = a + ((T)bin + 0.5) * 2E in T; decompression multiplies by m = 1 + centre.
  R7  Eq. 4 is garbled in the paper (it multiplies by the ratio itself); the reconstruction
      is R = prev * (1 + centre), the inverse of Eq. 1. A point in a selected bin is
      compressible only if |prev * m - cur| <= E * |cur| holds in T (the element-wise
      relative error bound of §VI, measured as in Eq. 3); otherwise it is incompressible.
  R8  index blocks hold epb = floor(8 * block_bytes / B) indices, least significant bit
      first; block byte images are padded with zero bytes to a multiple of 16.
  R9  offset tables are int64 with nblocks + 1 entries; a sub-block table (one int64 per
      4096 elements) is added for decoders.
  R10 automatic index length (§IV.B.2): B ranges over 1..16; alpha(B) of Eq. 5 counts as
      compressible every point of the top 2^B - 1 bins (the histogram's estimate, before
      the error check); the smallest file_size(B) of Eq. 6 wins, ties to the smaller B.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------------------
# Format constants of the blob (these restate the documented format; they are not shared
# with the library's sources).
# ---------------------------------------------------------------------------------------
MAGIC = 0x314B4D4E          # "NMK1"
VERSION = 1
HEADER_BYTES = 256
SECTION_ALIGN = 256
SUB_BLOCK = 4096
WINDOW_LOG2 = 21
ANCHOR_ZERO = 0
ANCHOR_MIN = 1
DEFAULT_BLOCK_BYTES = 1 << 20

_HEADER_FMT = "<IIiid ii qqqqqqqq d qqqqqqqq"   # 168 bytes, then 88 reserved zero bytes
_HEADER_FIELDS = ("magic", "version", "dtype", "B", "E", "anchor", "status", "n",
                  "block_bytes", "epb", "nblocks", "sub", "nsub", "n_sel", "n_inc", "a",
                  "block_stride", "off_centres", "off_idx_off", "off_inc_off", "off_sub_off",
                  "off_index", "off_exact", "total_bytes")


def _dtype_code(T) -> int:
    return {np.float32: 0, np.float64: 1}[T]


def _round_up(x: int, m: int) -> int:
    return (x + m - 1) // m * m


# ---------------------------------------------------------------------------------------
# Step 0: derived constants (§IV.B.1: bins of width 2E).
# ---------------------------------------------------------------------------------------
def grid_constants(T, E: float):
    """E_T = (T)E, bin width w = 2E, its reciprocal and the ratio cap (reading R1)."""
    E_T = T(E)
    w = T(E_T + E_T)
    inv_w = T(T(1) / w)
    cap = T(w * T(2 ** WINDOW_LOG2))      # a power-of-two scaling: exact
    return E_T, w, inv_w, cap


# ---------------------------------------------------------------------------------------
# Step 1: change ratios, Eq. 1 (§III.A, §IV.A).
# ---------------------------------------------------------------------------------------
def change_ratio(prev: np.ndarray, cur: np.ndarray, cap):
    """ratio_j = (cur_j - prev_j) / prev_j in T; binnable iff finite and |ratio| <= cap."""
    with np.errstate(all="ignore"):
        d = cur - prev
        ratio = d / prev
    binnable = np.isfinite(ratio) & (np.abs(ratio) <= cap)
    return ratio, binnable


# ---------------------------------------------------------------------------------------
# Step 2: grid anchor (reading R2; §IV.A computes the global min/max of the ratios).
# ---------------------------------------------------------------------------------------
def grid_anchor(ratio: np.ndarray, binnable: np.ndarray, E_T, anchor: int):
    T = type(E_T)
    if anchor == ANCHOR_ZERO:
        return T(-E_T)
    if anchor == ANCHOR_MIN:
        if not binnable.any():
            return T(0)
        a = T(ratio[binnable].min())
        # An unchanged point with a negative prev has ratio +0 / (-p) = -0; reading R2 takes a
        # zero minimum as +0 whichever signed zero the minimum search meets first.
        return T(0) if a == 0 else a
    raise ValueError("anchor must be 0 (ZERO) or 1 (MIN)")


# ---------------------------------------------------------------------------------------
# Step 3: bin ids (reading R3) and the histogram (§IV.B.1, reading R4).
# ---------------------------------------------------------------------------------------
def bin_ids(ratio: np.ndarray, binnable: np.ndarray, a, inv_w) -> np.ndarray:
    """floor((ratio - a) * inv_w) for binnable points; 0 (unused) for the others."""
    with np.errstate(all="ignore"):
        t = ratio - a
        u = t * inv_w
    b = np.zeros(ratio.shape, dtype=np.int64)
    b[binnable] = np.floor(u[binnable]).astype(np.int64)
    return b


def histogram(b: np.ndarray, binnable: np.ndarray):
    """Distinct bins of the binnable points (ascending) and how many points fall in each."""
    bins, counts = np.unique(b[binnable], return_counts=True)
    return bins.astype(np.int64), counts.astype(np.int64)


# ---------------------------------------------------------------------------------------
# Step 4: top-k selection (§IV.B.1, reading R5).
# ---------------------------------------------------------------------------------------
def top_k(bins: np.ndarray, counts: np.ndarray, k: int) -> np.ndarray:
    """The min(k, #bins) bins with the largest counts (ties: smaller bin first),
    returned in ascending bin order; position in the result = the bin's index r."""
    order = np.lexsort((bins, -counts))      # last key is primary: count descending
    return np.sort(bins[order[:k]])


def file_size_bits(counts: np.ndarray, n: int, L: int, B_max: int = 16) -> list:
    """8 * file_size(B) of Eq. 6 for B = 1..B_max (§IV.B.2): the compressible points are those
    in the top k = 2^B - 1 bins of the histogram (reading R10), alpha(B) of Eq. 5 is
    (n - compressible) / n, file_size(B) = 2^B * L + n * B / 8 + n * alpha(B) * L. Exact
    integers (bits), so that sizes compare without rounding."""
    desc = np.sort(np.asarray(counts, dtype=np.int64))[::-1]
    prefix = np.concatenate([[0], np.cumsum(desc, dtype=np.int64)])
    out = []
    for B in range(1, B_max + 1):
        compressible = int(prefix[min((1 << B) - 1, desc.size)])
        out.append(8 * (1 << B) * L + n * B + 8 * L * (n - compressible))
    return out


def choose_B(counts: np.ndarray, n: int, L: int, B_max: int = 16) -> int:
    """The B of smallest file_size(B) (§IV.B.2); ties go to the smaller B."""
    bits = file_size_bits(counts, n, L, B_max)
    return 1 + int(np.argmin(bits))          # argmin returns the first (smallest B) minimum


def centres_of(selected: np.ndarray, a, w, T) -> np.ndarray:
    """centre_r = a + (((T)bin_r + 0.5) * w), in T (reading R6)."""
    bf = selected.astype(T)
    return (a + ((bf + T(0.5)) * w)).astype(T)


# ---------------------------------------------------------------------------------------
# Step 5: indexing with the error-bound check (§III.C, reading R7).
# ---------------------------------------------------------------------------------------
def assign_indices(prev, cur, binnable, b, selected, centres, E_T, M: int) -> np.ndarray:
    T = type(E_T)
    n = prev.shape[0]
    idx = np.full(n, M, dtype=np.int64)
    if selected.size == 0 or n == 0:
        return idx
    pos = np.searchsorted(selected, b)
    pos_c = np.minimum(pos, selected.size - 1)
    in_sel = binnable & (selected[pos_c] == b)
    m = (T(1) + centres).astype(T)
    with np.errstate(all="ignore"):
        R = prev * m[pos_c]
        e = R - cur
        tol = E_T * np.abs(cur)
        ok = np.abs(e) <= tol
    take = in_sel & ok
    idx[take] = pos_c[take]
    return idx


# ---------------------------------------------------------------------------------------
# Step 6: block layout and bit packing (§IV.C, reading R8).
# ---------------------------------------------------------------------------------------
def elements_per_block(block_bytes: int, B: int) -> int:
    """Indices that fit in one byte-aligned block (§IV.C; Fig. 2 shows 645277 = 2^23 // 13)."""
    return (8 * block_bytes) // B


def pack_block(indices: np.ndarray, B: int) -> bytes:
    """B least significant bits of each index, index i at bits [i*B, i*B+B), LSB first;
    bit t of the stream is bit (t mod 8) of byte t // 8; the last byte is zero-padded."""
    if indices.size == 0:
        return b""
    bits = ((indices[:, None] >> np.arange(B, dtype=np.int64)[None, :]) & 1).astype(np.uint8)
    return np.packbits(bits.reshape(-1), bitorder="little").tobytes()


def unpack_block(data: bytes, count: int, B: int) -> np.ndarray:
    """Inverse of pack_block for `count` indices."""
    if count == 0:
        return np.zeros(0, dtype=np.int64)
    bits = np.unpackbits(np.frombuffer(data, dtype=np.uint8), bitorder="little")
    bits = bits[: count * B].reshape(count, B).astype(np.int64)
    return (bits << np.arange(B, dtype=np.int64)[None, :]).sum(axis=1)


# ---------------------------------------------------------------------------------------
# The blob (§IV.D, Fig. 2 arrays + the documented header).
# ---------------------------------------------------------------------------------------
@dataclass
class Blob:
    header: dict
    centres: np.ndarray            # T[2^B]
    idx_off: np.ndarray            # int64[nblocks+1]
    inc_off: np.ndarray            # int64[nblocks+1]
    sub_off: np.ndarray            # int64[nsub]
    index_blocks: list = field(default_factory=list)   # bytes per block, unpadded
    exact: np.ndarray = None       # T[n_inc]
    indices: np.ndarray = None     # int64[n] (kept for tests; not part of the bytes)

    def to_bytes(self) -> bytes:
        h = self.header
        out = bytearray(h["total_bytes"])
        out[0:HEADER_BYTES] = pack_header(h)
        out[h["off_centres"]: h["off_centres"] + self.centres.nbytes] = self.centres.tobytes()
        out[h["off_idx_off"]: h["off_idx_off"] + self.idx_off.nbytes] = self.idx_off.tobytes()
        out[h["off_inc_off"]: h["off_inc_off"] + self.inc_off.nbytes] = self.inc_off.tobytes()
        out[h["off_sub_off"]: h["off_sub_off"] + self.sub_off.nbytes] = self.sub_off.tobytes()
        for q, data in enumerate(self.index_blocks):
            start = h["off_index"] + int(self.idx_off[q])
            out[start: start + len(data)] = data
        out[h["off_exact"]: h["off_exact"] + self.exact.nbytes] = self.exact.tobytes()
        return bytes(out)


def pack_header(h: dict) -> bytes:
    raw = struct.pack(_HEADER_FMT, *[h[f] for f in _HEADER_FIELDS])
    return raw + bytes(HEADER_BYTES - len(raw))


def parse_header(data: bytes) -> dict:
    size = struct.calcsize(_HEADER_FMT)
    return dict(zip(_HEADER_FIELDS, struct.unpack(_HEADER_FMT, bytes(data[:size]))))


def layout(n: int, T, B: int, block_bytes: int) -> dict:
    """Section offsets of a blob (everything but n_inc / total_bytes)."""
    L = np.dtype(T).itemsize
    epb = elements_per_block(block_bytes, B)
    nblocks = -(-n // epb) if n > 0 else 0
    counts = [min(epb, n - q * epb) for q in range(nblocks)]
    nsub = sum(-(-c // SUB_BLOCK) for c in counts)
    block_stride = _round_up(-(-(epb * B) // 8), 16)
    index_bytes = 0
    if nblocks:
        index_bytes = (nblocks - 1) * block_stride + _round_up(-(-(counts[-1] * B) // 8), 16)
    off_centres = HEADER_BYTES
    off_idx_off = _round_up(off_centres + (1 << B) * L, SECTION_ALIGN)
    off_inc_off = _round_up(off_idx_off + (nblocks + 1) * 8, SECTION_ALIGN)
    off_sub_off = _round_up(off_inc_off + (nblocks + 1) * 8, SECTION_ALIGN)
    off_index = _round_up(off_sub_off + nsub * 8, SECTION_ALIGN)
    off_exact = _round_up(off_index + index_bytes, SECTION_ALIGN)
    return dict(epb=epb, nblocks=nblocks, counts=counts, nsub=nsub, block_stride=block_stride,
                index_bytes=index_bytes, off_centres=off_centres, off_idx_off=off_idx_off,
                off_inc_off=off_inc_off, off_sub_off=off_sub_off, off_index=off_index,
                off_exact=off_exact)


# ---------------------------------------------------------------------------------------
# Compression: steps 1-6 in the paper's order (§III.A-C, §IV.A-C).
# ---------------------------------------------------------------------------------------
def compress(prev: np.ndarray, cur: np.ndarray, E: float, B: int, anchor: int = ANCHOR_ZERO,
             block_bytes: int = DEFAULT_BLOCK_BYTES) -> Blob:
    prev = np.ascontiguousarray(prev)
    cur = np.ascontiguousarray(cur)
    assert prev.dtype == cur.dtype and prev.dtype in (np.float32, np.float64)
    assert prev.ndim == 1 and prev.shape == cur.shape
    assert 0 <= B <= 16                                              # 0: choose B (§IV.B.2)
    T = prev.dtype.type
    L = prev.dtype.itemsize
    n = prev.shape[0]

    E_T, w, inv_w, cap = grid_constants(T, E)
    ratio, binnable = change_ratio(prev, cur, cap)                   # Eq. 1
    a = grid_anchor(ratio, binnable, E_T, anchor)                    # R2
    b = bin_ids(ratio, binnable, a, inv_w)                           # R3
    bins, counts = histogram(b, binnable)                            # §IV.B.1
    if B == 0:
        B = choose_B(counts, n, L)                                   # §IV.B.2, Eqs. 5-6
    k = (1 << B) - 1
    M = (1 << B) - 1
    selected = top_k(bins, counts, k)                                # §IV.B.1
    c_sel = centres_of(selected, a, w, T)                            # R6
    idx = assign_indices(prev, cur, binnable, b, selected, c_sel, E_T, M)   # §III.C

    lay = layout(n, T, B, block_bytes)
    epb, nblocks = lay["epb"], lay["nblocks"]
    centres = np.zeros(1 << B, dtype=T)
    centres[: selected.size] = c_sel

    is_marker = idx == M
    exact = cur[is_marker].copy()                                    # §III.C, bit copies
    # markers_before[j] = number of incompressible points with index < j
    markers_before = np.concatenate([[0], np.cumsum(is_marker, dtype=np.int64)])
    blocks, idx_off, inc_off, sub_off = [], [], [], []
    for q in range(nblocks):
        lo, hi = q * epb, min(n, (q + 1) * epb)
        idx_off.append(q * lay["block_stride"])
        inc_off.append(int(markers_before[lo]))
        for s in range(lo, hi, SUB_BLOCK):
            sub_off.append(int(markers_before[s]))
        blocks.append(pack_block(idx[lo:hi], B))
    idx_off.append(lay["index_bytes"])
    n_inc = int(markers_before[n])
    inc_off.append(n_inc)

    header = dict(magic=MAGIC, version=VERSION, dtype=_dtype_code(T), B=B, E=float(E),
                  anchor=anchor, status=0, n=n, block_bytes=block_bytes, epb=epb,
                  nblocks=nblocks, sub=SUB_BLOCK, nsub=lay["nsub"], n_sel=int(selected.size),
                  n_inc=n_inc, a=float(a), block_stride=lay["block_stride"],
                  off_centres=lay["off_centres"], off_idx_off=lay["off_idx_off"],
                  off_inc_off=lay["off_inc_off"], off_sub_off=lay["off_sub_off"],
                  off_index=lay["off_index"], off_exact=lay["off_exact"],
                  total_bytes=lay["off_exact"] + n_inc * L)
    return Blob(header=header, centres=centres,
                idx_off=np.array(idx_off, dtype=np.int64),
                inc_off=np.array(inc_off, dtype=np.int64),
                sub_off=np.array(sub_off, dtype=np.int64),
                index_blocks=blocks, exact=exact, indices=idx)


def compress_bound(n: int, T, B: int, block_bytes: int = DEFAULT_BLOCK_BYTES) -> int:
    """Largest blob for n elements: all points incompressible (B = 0, chosen at run time: the
    largest over B = 1..16)."""
    Bs = [B] if B else range(1, 17)
    return max(layout(n, T, b, block_bytes)["off_exact"] for b in Bs) + n * np.dtype(T).itemsize


# ---------------------------------------------------------------------------------------
# Decompression, Eq. 4 (§III.E, reading R7), and partial decompression (§IV.C, §V.C).
# ---------------------------------------------------------------------------------------
def _sections(data: bytes):
    h = parse_header(data)
    if h["magic"] != MAGIC or h["version"] != VERSION:
        raise ValueError("not a NUMARCK v1 blob")
    T = np.float64 if h["dtype"] == 1 else np.float32
    L = np.dtype(T).itemsize
    B, nblocks = h["B"], h["nblocks"]
    centres = np.frombuffer(data, dtype=T, count=1 << B, offset=h["off_centres"])
    inc_off = np.frombuffer(data, dtype=np.int64, count=nblocks + 1, offset=h["off_inc_off"])
    idx_off = np.frombuffer(data, dtype=np.int64, count=nblocks + 1, offset=h["off_idx_off"])
    exact = np.frombuffer(data, dtype=T, count=h["n_inc"], offset=h["off_exact"])
    return h, T, L, centres, idx_off, inc_off, exact


def _block_indices(data: bytes, h: dict, idx_off, q: int) -> np.ndarray:
    epb, n, B = h["epb"], h["n"], h["B"]
    count = min(epb, n - q * epb)
    start = h["off_index"] + int(idx_off[q])
    nbytes = -(-(count * B) // 8)
    return unpack_block(data[start: start + nbytes], count, B)


def decompress(data: bytes, prev: np.ndarray) -> np.ndarray:
    """R_j = exact value (next in order) if idx_j = M, else prev_j * (1 + centre[idx_j])."""
    h, T, L, centres, idx_off, inc_off, exact = _sections(data)
    n, B = h["n"], h["B"]
    M = (1 << B) - 1
    assert prev.dtype == T and prev.shape == (n,)
    idx = np.concatenate([_block_indices(data, h, idx_off, q) for q in range(h["nblocks"])]) \
        if h["nblocks"] else np.zeros(0, dtype=np.int64)
    m = (T(1) + centres).astype(T)
    out = np.empty(n, dtype=T)
    marker = idx == M
    with np.errstate(all="ignore"):
        out[~marker] = prev[~marker] * m[idx[~marker]]
    out[marker] = exact
    return out


def decompress_range(data: bytes, prev_seg: np.ndarray, start: int, count: int) -> np.ndarray:
    """Decode only the blocks covering [start, start+count): the exact-value cursor starts at
    the block's incompressible offset plus the markers that precede `start` in that block."""
    h, T, L, centres, idx_off, inc_off, exact = _sections(data)
    n, B, epb = h["n"], h["B"], h["epb"]
    M = (1 << B) - 1
    assert 0 <= start <= start + count <= n and prev_seg.shape == (count,)
    out = np.empty(count, dtype=T)
    if count == 0:
        return out
    q0, q1 = start // epb, (start + count - 1) // epb
    idx = np.concatenate([_block_indices(data, h, idx_off, q) for q in range(q0, q1 + 1)])
    lo = start - q0 * epb
    before = int((idx[:lo] == M).sum())
    seg = idx[lo: lo + count]
    marker = seg == M
    cursor = int(inc_off[q0]) + before
    m = (T(1) + centres).astype(T)
    with np.errstate(all="ignore"):
        out[~marker] = prev_seg[~marker] * m[seg[~marker]]
    out[marker] = exact[cursor: cursor + int(marker.sum())]
    return out


# ---------------------------------------------------------------------------------------
# Metrics (Eq. 2, 3, 5, 6) — computed from outputs, used by tests and the bench report.
# ---------------------------------------------------------------------------------------
def compression_ratio(original_bytes: int, compressed_bytes: int) -> float:
    """Eq. 2."""
    return original_bytes / compressed_bytes


def mean_error_rate(cur: np.ndarray, recon: np.ndarray) -> float:
    """Eq. 3, over the points with cur != 0 (the ratio is undefined at 0)."""
    nz = cur != 0
    if not nz.any():
        return 0.0
    c = cur[nz].astype(np.float64)
    r = recon[nz].astype(np.float64)
    return float(np.abs((c - r) / c).sum() / cur.size)


def incompressible_ratio(n: int, n_compressible: int) -> float:
    """Eq. 5: alpha = (n - compressible points) / n."""
    return (n - n_compressible) / n if n else 0.0


def estimated_file_size(n: int, B: int, alpha: float, L: int) -> float:
    """Eq. 6: 2^B * L + n * B / 8 + n * alpha * L bytes."""
    return (1 << B) * L + n * B / 8 + n * alpha * L
