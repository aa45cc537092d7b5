"""The all-cores CPU baseline (oracle/numarck_cpu.c: C, POSIX threads) against the numpy oracle,
on the CPU: byte-identical blobs and bit-identical decompression for every input family the GPU
parity tests use, at any thread count. Two CPU implementations written separately from the same
readings of the paper agree, which also checks the oracle."""
import numpy as np
import pytest

from oracle import cpu_parallel as C
from oracle import numarck_oracle as O
from paper_1703_02438_gb300 import synth


def _u(a):
    return a.view(np.uint64 if a.dtype == np.float64 else np.uint32)


def check(p, x, E, B, anchor=0, block_bytes=O.DEFAULT_BLOCK_BYTES, threads=(1, 5, 8)):
    want = O.compress(p, x, E, B, anchor=anchor, block_bytes=block_bytes).to_bytes()
    rec = O.decompress(want, p)
    for t in threads:
        got = C.compress(p, x, E, B, anchor=anchor, block_bytes=block_bytes, threads=t)
        assert got == want, (t, len(got), len(want))
        assert np.array_equal(_u(C.decompress(got, p, threads=t)), _u(rec))
    return O.parse_header(want)


@pytest.mark.parametrize("anchor", [0, 1])
@pytest.mark.parametrize("B", [0, 6, 8, 10])
def test_plain_pair(anchor, B):
    p, x = synth.plain_pair(300_001, seed=synth.seed_for(0, 200 + B))
    check(p.numpy(), x.numpy(), 1e-3, B, anchor=anchor)


@pytest.mark.parametrize("B", [1, 2, 3, 5, 7, 9, 11, 13, 16])
def test_all_widths_small_blocks(B):
    p, x = synth.plain_pair(50_003, seed=synth.seed_for(0, 300 + B))
    check(p.numpy(), x.numpy(), 1e-3, B, block_bytes=3001)


def test_float32_and_flash_like():
    p, x = synth.plain_pair(200_000, dtype=__import__("torch").float32, seed=synth.seed_for(0, 17))
    check(p.numpy(), x.numpy(), 1e-4, 10)
    s = synth.flash_series(side=48, steps=2)
    check(s[0].numpy(), s[1].numpy(), 1e-3, 8)
    check(s[0].numpy().astype(np.float32), s[1].numpy().astype(np.float32), 1e-3, 8, anchor=1)


@pytest.mark.parametrize("T", [np.float32, np.float64])
def test_specials_edges_and_signed_zero(T):
    rng = np.random.default_rng(23)
    n = 40_000
    E = 2.0 ** -10
    w = 2 * E
    p = rng.lognormal(size=n).astype(T)
    r = ((-E + rng.integers(-300, 300, n) * w) *
         (1 + rng.choice([0.0, 1.0, -1.0], n) * np.finfo(T).eps)).astype(T)
    x = (p * (T(1) + r)).astype(T)
    sel = rng.permutation(n)
    p[sel[:400]] = 0
    x[sel[400:800]] = np.nan
    p[sel[800:850]] = np.inf
    p[sel[850:900]] = -0.0
    x[sel[900:950]] = np.finfo(T).smallest_subnormal * 3
    p[sel[950:2000]] = -p[sel[950:2000]]
    x[sel[950:1500]] = p[sel[950:1500]]                    # unchanged with negative prev: -0
    for anchor in (0, 1):
        check(p, x, E, 9, anchor=anchor)


@pytest.mark.parametrize("n", [0, 1, 31, 4095, 4096, 4097, 65537])
def test_sizes(n):
    p, x = synth.plain_pair(max(n, 1), seed=synth.seed_for(0, 31))
    check(p[:n].numpy().copy(), x[:n].numpy().copy(), 1e-3, 8)


def test_many_ties():
    n = 64 * 1000
    m = np.repeat(np.arange(-500, 500), 64)
    np.random.default_rng(9).shuffle(m)
    p = np.ones(n)
    x = 1 + m * (2 * 2.0 ** -8)
    for B in (4, 8, 10):
        check(p, x, 2.0 ** -8, B)
