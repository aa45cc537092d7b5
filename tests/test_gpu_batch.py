"""Batched compression (many variables of mixed dtype, size, E and B in one call) must give, byte
for byte, the blobs of the single-variable entry point, for every lane count and grid share, and
also when the batch is captured into a CUDA graph and replayed on new data."""
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


def _variables(seed_base=0):
    sizes = [1, 100, 4095, 4096, 4097, 10_000, 65_537, 300_000, 1_000_003, 2_500_000]
    pairs, specs = [], []
    Es, Bs = (1e-2, 1e-3, 1e-4), (6, 8, 10)
    for i in range(24):
        n = sizes[i % len(sizes)]
        dtype = torch.float64 if i % 2 == 0 else torch.float32
        p, x = synth.plain_pair(n, dtype=dtype, seed=synth.seed_for(3, seed_base + i),
                                scale=0.5 + 3.5 * ((i * 37) % 11) / 10)
        pairs.append((p.to(DEV), x.to(DEV)))
        anchor = N.ANCHOR_MIN if i % 7 == 3 else N.ANCHOR_ZERO
        block_bytes = 3001 if i % 5 == 4 else 0
        specs.append((Es[i % 3], Bs[(i // 3) % 3], anchor, block_bytes))
    return pairs, specs


def _used(blob):
    return blob[: N.blob_size(N.header_bytes(blob))].cpu()


def _single(pairs, specs):
    out = []
    for (p, x), spec in zip(pairs, specs):
        anchor = spec[2] if len(spec) > 2 else 0
        bb = spec[3] if len(spec) > 3 else 0
        out.append(_used(N.compress(p, x, spec[0], spec[1], anchor=anchor, block_bytes=bb)))
    return out


@pytest.mark.parametrize("lanes,share", [(1, 1), (3, 2), (8, 4), (64, 16)])
def test_batch_equals_single_calls(lanes, share):
    pairs, specs = _variables()
    want = _single(pairs, specs)
    batch = N.Batch(pairs, specs, lanes=lanes, grid_share=share)
    blobs = batch.run()
    torch.cuda.synchronize()
    for i, (b, w) in enumerate(zip(blobs, want)):
        assert torch.equal(_used(b), w), i
    # decompression of the whole batch
    prevs = [p for p, _ in pairs]
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    outs = N.decompress_batch(blobs, prevs, lanes=lanes, grid_share=share, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    for (p, _), b, o in zip(pairs, blobs, outs):
        ref = N.decompress(b, p)
        torch.cuda.synchronize()
        assert torch.equal(o.view(torch.uint8), ref.view(torch.uint8))


def test_batch_small_items_match_oracle():
    pairs, specs = _variables(seed_base=100)
    batch = N.Batch(pairs[:6], specs[:6], lanes=4, grid_share=4)
    blobs = batch.run()
    torch.cuda.synchronize()
    for (p, x), spec, b in zip(pairs[:6], specs[:6], blobs):
        anchor = spec[2] if len(spec) > 2 else 0
        bb = spec[3] if len(spec) > 3 else O.DEFAULT_BLOCK_BYTES
        want = O.compress(p.cpu().numpy(), x.cpu().numpy(), spec[0], spec[1], anchor=anchor,
                          block_bytes=bb or O.DEFAULT_BLOCK_BYTES).to_bytes()
        assert _used(b).numpy().tobytes() == want


def test_batch_graph_capture_and_replay_on_new_data():
    pairs, specs = _variables(seed_base=200)
    batch = N.Batch(pairs, specs, lanes=8, grid_share=4)
    batch.run()                       # first call: lane streams, kernel set-up, workspace
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.run()
    torch.cuda.synchronize()
    for round_ in range(2):
        new_pairs, _ = _variables(seed_base=300 + 50 * round_)
        for (p, x), (np_, nx) in zip(batch.pairs, new_pairs):
            p.copy_(np_)
            x.copy_(nx)
        g.replay()
        torch.cuda.synchronize()
        want = _single(batch.pairs, specs)
        for i, (b, w) in enumerate(zip(batch.blobs, want)):
            assert torch.equal(_used(b), w), (round_, i)


# ---------------------------------------------------------------------------------------
# the fused batch: one launch per phase over all variables (numarck_*_batch_fused)
# ---------------------------------------------------------------------------------------
TUNINGS = [(1024, 8, 0, 1, 1), (512, 4, 1, 4, 2), (1024, 4, 2, 8, 4), (512, 8, 3, 3, 3)]


def _with_empty(pairs, specs):
    """The mixed list plus a variable of no elements (its blob is a header and tables only)."""
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    return pairs[:5] + [(e, e.clone())] + pairs[5:], specs[:5] + [(1e-3, 8)] + specs[5:]


@pytest.mark.parametrize("tuning", TUNINGS)
def test_fused_batch_equals_single_calls(tuning):
    pairs, specs = _with_empty(*_variables(seed_base=400))
    want = _single(pairs, specs)
    batch = N.Batch(pairs, specs, mode="fused", tuning=tuning)
    for _ in range(2):                   # the second run reuses the workspace the first left
        blobs = batch.run()
        torch.cuda.synchronize()
        for i, (b, w) in enumerate(zip(blobs, want)):
            assert torch.equal(_used(b), w), i
    prevs = [p for p, _ in pairs]
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    outs = batch.decompress(prevs, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    for (p, _), b, o in zip(pairs, blobs, outs):
        ref = N.decompress(b, p) if p.numel() else torch.empty_like(p)
        torch.cuda.synchronize()
        assert torch.equal(o.view(torch.uint8), ref.view(torch.uint8))


def test_fused_batch_matches_oracle():
    pairs, specs = _variables(seed_base=500)
    sel = [0, 1, 3, 4, 7, 9, 13, 17]         # both dtypes, MIN grid, odd block size, 2.5M points
    pairs, specs = [pairs[i] for i in sel], [specs[i] for i in sel]
    batch = N.Batch(pairs, specs, mode="fused")
    blobs = batch.run()
    torch.cuda.synchronize()
    for (p, x), spec, b in zip(pairs, specs, blobs):
        want = O.compress(p.cpu().numpy(), x.cpu().numpy(), spec[0], spec[1], anchor=spec[2],
                          block_bytes=spec[3] or O.DEFAULT_BLOCK_BYTES).to_bytes()
        assert _used(b).numpy().tobytes() == want
    outs = batch.decompress([p for p, _ in pairs])
    torch.cuda.synchronize()
    for (p, _), b, o in zip(pairs, blobs, outs):
        ref = O.decompress(_used(b).numpy().tobytes(), p.cpu().numpy())
        assert o.cpu().numpy().tobytes() == ref.tobytes()


def test_fused_batch_graph_capture_and_replay_on_new_data():
    pairs, specs = _variables(seed_base=600)
    batch = N.Batch(pairs, specs, mode="fused", tuning=(512, 4, 1, 4, 2))
    prevs = [p for p, _ in pairs]
    outs = [torch.empty_like(p) for p in prevs]
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    batch.run()                       # first call: kernel set-up, workspace
    batch.decompress(prevs, outs=outs, status=status)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.run()
            batch.decompress(prevs, outs=outs, status=status)
    torch.cuda.synchronize()
    for round_ in range(2):
        new_pairs, _ = _variables(seed_base=700 + 50 * round_)
        for (p, x), (np_, nx) in zip(batch.pairs, new_pairs):
            p.copy_(np_)
            x.copy_(nx)
        g.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        want = _single(batch.pairs, specs)
        for i, (b, w) in enumerate(zip(batch.blobs, want)):
            assert torch.equal(_used(b), w), (round_, i)
        for (p, _), b, o in zip(batch.pairs, batch.blobs, outs):
            ref = N.decompress(b, p)
            torch.cuda.synchronize()
            assert torch.equal(o.view(torch.uint8), ref.view(torch.uint8)), round_


def test_fused_decode_reports_a_bad_blob_and_decodes_the_rest():
    pairs, specs = _variables(seed_base=800)
    pairs, specs = pairs[:8], specs[:8]
    batch = N.Batch(pairs, specs, mode="fused")
    blobs = batch.run()
    torch.cuda.synchronize()
    bad = [b.clone() for b in blobs]
    bad[3][0:4] = 0                          # magic destroyed
    prevs = [p for p, _ in pairs]
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    outs = N.decompress_batch_fused(bad, prevs, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == N.ERR_CORRUPT
    for i, ((p, _), b, o) in enumerate(zip(pairs, blobs, outs)):
        if i == 3:
            continue
        ref = N.decompress(b, p)
        torch.cuda.synchronize()
        assert torch.equal(o.view(torch.uint8), ref.view(torch.uint8)), i


def test_lane_batch_after_another_lane_count():
    """A lane batch whose workspace served another lane count (slices elsewhere) still equals
    the single calls."""
    pairs, specs = _variables(seed_base=900)
    want = _single(pairs, specs)
    batch = N.Batch(pairs, specs, lanes=2, grid_share=2)
    for lanes, share in ((2, 2), (8, 4), (3, 2), (16, 8)):
        batch.set_lanes(lanes, share)
        blobs = batch.run()
        torch.cuda.synchronize()
        for i, (b, w) in enumerate(zip(blobs, want)):
            assert torch.equal(_used(b), w), (lanes, i)
