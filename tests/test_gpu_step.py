"""GPU parity of the chained step numarck_decompress_compress: decompressing one blob and
compressing the next timestep against that reconstruction (fused into one kernel on the
zero-centred grid) must give exactly what the oracle gives for the two operations one after the
other — the reconstruction bit for bit and the next blob byte for byte — and what the separate
GPU calls give. Errors that the decompression finds on the device reach the next blob's header.
"""
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


def _used(blob):
    torch.cuda.synchronize()
    hb = N.header_bytes(blob)
    return blob[:N.blob_size(hb)].cpu().numpy().tobytes()


def run_chain(series, E, B, anchor=N.ANCHOR_ZERO, block_bytes=0, header=False):
    """Chain over `series` (device tensors) with the fused step; checks every reconstruction
    and every blob against the oracle. Returns the GPU blobs."""
    kw = dict(anchor=anchor, block_bytes=block_bytes or O.DEFAULT_BLOCK_BYTES)
    prev_np = series[0].cpu().numpy()
    want = O.compress(prev_np, series[1].cpu().numpy(), E, B, **kw).to_bytes()
    blob = N.compress(series[0], series[1], E, B, anchor=anchor, block_bytes=block_bytes)
    assert _used(blob) == want, "first blob"
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    prev = series[0]
    blobs = [want]
    for t in range(2, len(series)):
        hb = N.header_bytes(blob) if header else None
        rec, nxt = N.decompress_compress(blob, prev, series[t], E, B, anchor=anchor,
                                         block_bytes=block_bytes, status=status, header=hb)
        got = _used(nxt)
        assert int(status.item()) == 0
        ref = O.decompress(want, prev_np)
        assert np.array_equal(_u(rec.cpu().numpy()), _u(ref)), f"reconstruction {t - 1}"
        want = O.compress(ref, series[t].cpu().numpy(), E, B, **kw).to_bytes()
        assert got == want, f"blob {t}: {len(got)} vs {len(want)} bytes"
        blobs.append(got)
        prev_np, prev, blob = ref, rec, nxt
    last = N.decompress(blob, prev, status=status)
    torch.cuda.synchronize()
    assert np.array_equal(_u(last.cpu().numpy()), _u(O.decompress(want, prev_np)))
    return blobs


@pytest.mark.parametrize("E,B", [(1e-3, 8), (1e-4, 10), (1e-4, 8), (1e-3, 0)])
def test_flash_chain_matches_oracle(E, B):
    run_chain(synth.flash_series(side=96, steps=5, device=DEV), E, B)


@pytest.mark.parametrize("B", [6, 9, 13])
def test_flash_chain_float32_and_odd_block_lengths(B):
    """float32, and index blocks whose length is not a multiple of the 4096-point tile (B = 9,
    13: odd block lengths, so tiles start off the 16-byte boundary)."""
    s = [x.float() for x in synth.flash_series(side=64, steps=4, device=DEV,
                                                seed=synth.seed_for(1, 40 + B))]
    run_chain(s, 1e-3, B)
    run_chain(synth.flash_series(side=64, steps=4, device=DEV, seed=synth.seed_for(1, 50 + B)),
              1e-4, B, block_bytes=3001, header=True)


def test_min_anchor_chain_runs_unfused_with_the_same_results():
    run_chain(synth.flash_series(side=64, steps=4, device=DEV, seed=synth.seed_for(1, 60)),
              1e-3, 8, anchor=N.ANCHOR_MIN)


@pytest.mark.parametrize("n", [1, 2, 31, 4095, 4097, 65537, 300_001])
def test_sizes_and_spread_ratios(n):
    """The plain pair (zeros, ratios spread over thousands of bins: bins outside the shared
    window, undecided points) followed by an unrelated third array."""
    p, x = synth.plain_pair(n, seed=synth.seed_for(0, 70))
    y, _ = synth.plain_pair(n, seed=synth.seed_for(0, 71), zero_frac=0.02)
    run_chain([p.to(DEV), x.to(DEV), y.to(DEV)], 1e-3, 8)


def test_misaligned_views():
    p, x = synth.plain_pair(100_003, seed=synth.seed_for(0, 72))
    y, _ = synth.plain_pair(100_003, seed=synth.seed_for(0, 73))
    s = [t.to(DEV)[1:] for t in (p, x, y)]            # 8-byte but not 16-byte aligned
    run_chain(s, 1e-3, 8)


def test_fused_equals_separate_calls_and_workspace_is_left_ready():
    s = synth.flash_series(side=80, steps=3, device=DEV, seed=synth.seed_for(1, 80))
    b1 = N.compress(s[0], s[1], 1e-3, 10)
    rec_sep = N.decompress(b1, s[0])
    sep = _used(N.compress(rec_sep, s[2], 1e-3, 10))
    rec, nxt = N.decompress_compress(b1, s[0], s[2], 1e-3, 10)
    assert _used(nxt) == sep
    assert torch.equal(rec.view(torch.int64), rec_sep.view(torch.int64))
    # the workspace is left as a plain compression expects it
    assert _used(N.compress(rec_sep, s[2], 1e-3, 10)) == sep


def test_device_error_reaches_the_next_blob():
    s = synth.flash_series(side=48, steps=3, device=DEV, seed=synth.seed_for(1, 90))
    b1 = N.compress(s[0], s[1], 1e-3, 8)
    torch.cuda.synchronize()
    bad = b1.clone()
    off = N.HEADER_FIELDS.index("status")
    import struct
    fmt = N._HEADER_FMT
    fields = list(struct.unpack(fmt, N.header_bytes(b1)[:struct.calcsize(fmt)]))
    fields[off] = N.ERR_CORRUPT
    hdr = struct.pack(fmt, *fields)
    bad[:len(hdr)] = torch.frombuffer(bytearray(hdr), dtype=torch.uint8).to(DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    for anchor in (N.ANCHOR_ZERO, N.ANCHOR_MIN):
        status.zero_()
        _, nxt = N.decompress_compress(bad, s[0], s[2], 1e-3, 8, anchor=anchor, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == N.ERR_CORRUPT
        assert N.parse_header(N.header_bytes(nxt))["status"] == N.ERR_CORRUPT
        with pytest.raises(N.NumarckError):
            N.blob_size(N.header_bytes(nxt))
    # a float32 blob offered as the start of a float64 step: refused on the device
    b32 = N.compress(s[0].float(), s[1].float(), 1e-3, 8)
    status.zero_()
    _, nxt = N.decompress_compress(b32, s[0], s[2], 1e-3, 8, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == N.ERR_INVALID_ARG
    assert N.parse_header(N.header_bytes(nxt))["status"] == N.ERR_INVALID_ARG
    # and a good step afterwards still matches the separate calls (no state left behind)
    rec_sep = N.decompress(b1, s[0])
    sep = _used(N.compress(rec_sep, s[2], 1e-3, 8))
    _, nxt = N.decompress_compress(b1, s[0], s[2], 1e-3, 8)
    assert _used(nxt) == sep


@pytest.mark.parametrize("E,B", [(1e-3, 8), (1e-4, 10)])
def test_chain_helper_matches_oracle(E, B):
    """numarck.Chain (push one timestep at a time) gives the oracle's chain: every blob byte for
    byte, and the reconstruction of the latest timestep bit for bit."""
    s = synth.flash_series(side=64, steps=5, device=DEV, seed=synth.seed_for(1, 120 + B))
    ch = N.Chain(s[0].numel(), torch.float64, E, B, device=DEV)
    assert ch.push(s[0]) is None
    prev_np = s[0].cpu().numpy()
    for t in range(1, 5):
        blob = ch.push(s[t])
        want = O.compress(prev_np, s[t].cpu().numpy(), E, B).to_bytes()
        assert _used(blob) == want, f"blob {t}"
        prev_np = O.decompress(want, prev_np)
        if t == 2:          # an on-demand reconstruction between pushes does not disturb the chain
            assert np.array_equal(_u(ch.reconstruction().cpu().numpy()), _u(prev_np))
    rec = ch.reconstruction()
    torch.cuda.synchronize()
    assert ch.check() == 0
    assert np.array_equal(_u(rec.cpu().numpy()), _u(prev_np))


def test_empty_step():
    """n = 0: nothing to decompress; the next blob is the empty compression's."""
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    b = N.compress(e, e, 1e-3, 8)
    rec, nxt = N.decompress_compress(b, e, e, 1e-3, 8)
    assert rec.numel() == 0
    assert _used(nxt) == O.compress(np.empty(0), np.empty(0), 1e-3, 8).to_bytes()
