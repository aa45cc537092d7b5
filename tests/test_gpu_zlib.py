"""Lossless index compression (§IV.C) on the GPU: every index block's stream is a zlib stream
that the host's zlib inflates to exactly the block's bytes (the oracle's), the GPU inflater
restores the blob's index section bit for bit, a partial decompression inflates only its
sub-blocks, and malformed data is reported, not decoded."""
import zlib

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


def _case(kind):
    if kind == "plain":
        p, x = synth.plain_pair(300_001, seed=synth.seed_for(0, 51))
        return p.numpy(), x.numpy(), 1e-3, 8, 0
    if kind == "flash":
        xs = synth.flash_series(side=64, steps=2)
        return xs[0].numpy(), xs[1].numpy(), 1e-4, 10, 0
    if kind == "climate":
        (_, a), (_, b) = list(synth.climate_series(360, 720, steps=2))
        return a.numpy(), b.numpy(), 1e-3, 6, 0
    B = int(kind[1:])                      # small blocks, partial last tiles, every B
    p, x = synth.plain_pair(123_457, seed=synth.seed_for(0, 60 + B))
    return p.numpy(), x.numpy(), 1e-3, B, 3001


@pytest.mark.parametrize("kind", ["plain", "flash", "climate", "B1", "B3", "B13", "B16"])
def test_streams_inflate_to_the_index_blocks(kind):
    p, x, E, B, bb = _case(kind)
    want = O.compress(p, x, E, B, block_bytes=bb or O.DEFAULT_BLOCK_BYTES).to_bytes()
    h = O.parse_header(want)
    blob = N.compress(torch.from_numpy(p).to(DEV), torch.from_numpy(x).to(DEV), E, B,
                      block_bytes=bb)
    hb = N.header_bytes(blob)
    z = N.deflate_index(blob, hb)
    zh = N.zindex_header(z)
    zoff, sub_zoff = N.zindex_offsets(z, zh)
    zimg = bytes(z[:zh["total_bytes"]].cpu().numpy().tobytes())
    assert zh["nblocks"] == h["nblocks"] and zh["nsub"] == h["nsub"] and zh["B"] == B
    epb, n = h["epb"], h["n"]
    raw = 0
    for q in range(h["nblocks"]):
        cnt = min(n, (q + 1) * epb) - q * epb
        lo = h["off_index"] + q * h["block_stride"]
        block = want[lo: lo + (cnt * B + 7) // 8]
        assert zlib.decompress(zimg[zoff[q]: zoff[q + 1]]) == block, q
        raw += len(block)
    # a sub-block that fixed Huffman codes would expand is stored: the container stays within
    # a few bytes per sub-block of the raw index; the plain pair's indices compress
    assert zh["total_bytes"] <= zh["off_data"] + raw + 5 * h["nsub"] + 8 * h["nblocks"]
    if kind == "plain":
        assert zh["total_bytes"] < raw

    # the GPU inflater restores the whole index section bit for bit
    size = N.blob_size(hb)
    copy = blob[:size].clone()
    copy[h["off_index"]: h["off_exact"]] = 0
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    N.inflate_index(z, zh["total_bytes"], hb, copy, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert bytes(copy.cpu().numpy().tobytes()) == want


def test_partial_decode_inflates_only_its_sub_blocks():
    p, x, E, B, _ = _case("plain")
    want = O.compress(p, x, E, B).to_bytes()
    h = O.parse_header(want)
    pd = torch.from_numpy(p).to(DEV)
    blob = N.compress(pd, torch.from_numpy(x).to(DEV), E, B)
    hb = N.header_bytes(blob)
    z = N.deflate_index(blob, hb)
    zh = N.zindex_header(z)
    size = N.blob_size(hb)
    copy = blob[:size].clone()
    copy[h["off_index"]: h["off_exact"]] = 0xAB          # nothing outside the range is restored
    start, count = 150_000, 7000
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    N.inflate_index(z, zh["total_bytes"], hb, copy, start=start, count=count, status=status)
    seg = N.decompress_range(copy, pd[start: start + count], start, count, header=hb,
                             status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = O.decompress_range(want, p[start: start + count], start, count)
    assert np.array_equal(seg.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    img = copy.cpu().numpy()
    t0, t1 = start // 4096, (start + count - 1) // 4096
    assert (img[h["off_index"]: h["off_index"] + t0 * 512 * B] == 0xAB).all()
    assert (img[h["off_index"] + (t1 + 1) * 512 * B: h["off_exact"]] == 0xAB).all()


def test_malformed_stream_is_reported():
    p, x, E, B, _ = _case("plain")
    blob = N.compress(torch.from_numpy(p).to(DEV), torch.from_numpy(x).to(DEV), E, B)
    hb = N.header_bytes(blob)
    z = N.deflate_index(blob, hb)
    zh = N.zindex_header(z)
    zoff, sub_zoff = N.zindex_offsets(z, zh)
    bad = z.clone()
    bad[int(sub_zoff[3])] ^= 0x06                        # the block type bits of sub-block 3
    copy = blob.clone()
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    N.inflate_index(bad, zh["total_bytes"], hb, copy, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == N.ERR_CORRUPT


def test_bulk_inflate_restores_a_large_index():
    """More than 16384 sub-blocks (the one-thread-per-sub-block inflater): deflate then inflate
    gives back the blob byte for byte; a sample of the streams also goes through the host's
    zlib."""
    n = (1 << 26) + 12_345
    p, x = synth.plain_pair(n, seed=synth.seed_for(0, 77), device=DEV)
    blob = N.compress(p, x, 1e-3, 8)
    hb = N.header_bytes(blob)
    h = N.parse_header(hb)
    assert h["nsub"] >= 16384
    z = N.deflate_index(blob, hb)
    zh = N.zindex_header(z)
    size = N.blob_size(hb)
    copy = blob[:size].clone()
    copy[h["off_index"]: h["off_exact"]] = 0
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    N.inflate_index(z, zh["total_bytes"], hb, copy, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(copy, blob[:size])
    zoff, _ = N.zindex_offsets(z, zh)
    for q in (0, h["nblocks"] // 2, h["nblocks"] - 1):
        cnt = min(n, (q + 1) * h["epb"]) - q * h["epb"]
        lo = h["off_index"] + q * h["block_stride"]
        stream = bytes(z[int(zoff[q]): int(zoff[q + 1])].cpu().numpy().tobytes())
        assert zlib.decompress(stream) == bytes(blob[lo: lo + cnt].cpu().numpy().tobytes())


@pytest.mark.parametrize("kind", ["plain", "flash", "climate"])
def test_ratio_against_host_zlib(kind, record_property):
    """The container against the host's zlib (level 6) on the same index blocks: the per-sub-block
    dynamic Huffman codes keep it within a small factor of zlib's size, although every
    sub-block restarts its code and its matches (for partial decoding)."""
    p, x, E, B, bb = _case(kind)
    blob = N.compress(torch.from_numpy(p).to(DEV), torch.from_numpy(x).to(DEV), E, B,
                      block_bytes=bb)
    hb = N.header_bytes(blob)
    h = N.parse_header(hb)
    z = N.deflate_index(blob, hb)
    zh = N.zindex_header(z)
    img = blob.cpu().numpy().tobytes()
    raw = zl = 0
    for q in range(h["nblocks"]):
        cnt = min(h["n"], (q + 1) * h["epb"]) - q * h["epb"]
        lo = h["off_index"] + q * h["block_stride"]
        block = img[lo: lo + (cnt * B + 7) // 8]
        raw += len(block)
        zl += len(zlib.compress(block, 6))
    ours = zh["total_bytes"] - zh["off_data"]
    record_property("index_bytes", raw)
    record_property("container_bytes", ours)
    record_property("host_zlib6_bytes", zl)
    print(f"{kind}: index {raw} bytes, container {ours} ({raw / ours:.2f}x), "
          f"host zlib -6 {zl} ({raw / zl:.2f}x)")
    assert ours < raw and ours <= 2 * zl + 64 * h["nsub"]
