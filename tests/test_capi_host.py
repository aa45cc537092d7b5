"""Host-side checks of the C ABI (no GPU): the library loads and exports every function that
include/numarck.h declares; sizing and validation paths agree with the documented format
(restated by the oracle's layout) and reject bad arguments before touching any device memory."""
import ctypes
import os
import re
import struct

import numpy as np
import pytest

from oracle import numarck_oracle as O
from paper_1703_02438_gb300 import build as B_
from paper_1703_02438_gb300 import numarck as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B_.build()
    return N.lib()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "numarck.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(numarck_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "numarck_compress" in names and "numarck_decompress_range" in names
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    assert "sm_103a" in N.version()
    for code in range(8):
        assert N.status_string(code)
    assert N.status_string(99) == "unknown status"


@pytest.mark.parametrize("dtype,T", [(N.F32, np.float32), (N.F64, np.float64)])
@pytest.mark.parametrize("B", [1, 6, 8, 10, 13, 16])
@pytest.mark.parametrize("n", [0, 1, 4095, 4096, 4097, 1 << 20, 3758400])
def test_compress_bound_matches_format(lib, dtype, T, B, n):
    for bb in (0, 2, 16, 1000, 1 << 20):
        p = N.Params(dtype, B, 1e-3, 0, 0, bb)
        want = O.compress_bound(n, T, B, bb or O.DEFAULT_BLOCK_BYTES)
        assert N.compress_bound(n, p) == want
        assert N.workspace_bytes(n, p) > (1 << 22) * 8


def test_invalid_params_rejected(lib):
    bad = [N.Params(2, 8, 1e-3, 0, 0, 0), N.Params(0, -1, 1e-3, 0, 0, 0),
           N.Params(0, 17, 1e-3, 0, 0, 0), N.Params(0, 8, 0.0, 0, 0, 0),
           N.Params(0, 8, 1.0, 0, 0, 0), N.Params(0, 8, float("nan"), 0, 0, 0),
           N.Params(0, 8, 2.0 ** -61, 0, 0, 0), N.Params(0, 8, 1e-3, 2, 0, 0),
           N.Params(0, 8, 1e-3, 0, 1, 0), N.Params(0, 8, 1e-3, 0, 0, 1),
           N.Params(0, 8, 1e-3, 0, 0, (1 << 30) + 1)]
    for p in bad:
        assert N.compress_bound(10, p) == 0
        assert N.workspace_bytes(10, p) == 0
    good = N.Params(0, 8, 1e-3, 0, 0, 0)
    assert N.compress_bound(-1, good) == 0 and N.compress_bound((1 << 40) + 1, good) == 0


def test_automatic_B_is_sized_for_every_layout(lib):
    """B = 0 (chosen from the histogram, §IV.B.2) needs room for any B = 1..16: the blob bound
    and the workspace are the largest over B (a smaller B can have more sub-blocks: every
    index block ends in a partial tile)."""
    for dtype, T in ((N.F64, np.float64), (N.F32, np.float32)):
        for n in (0, 1, 4097, 3_000_001, 1 << 30):
            auto = N.Params(dtype, 0, 1e-3, 0, 0, 0)
            each = [N.Params(dtype, B, 1e-3, 0, 0, 0) for B in range(1, 17)]
            assert N.compress_bound(n, auto) == O.compress_bound(n, T, 0)
            assert N.compress_bound(n, auto) == max(N.compress_bound(n, p) for p in each)
            assert N.workspace_bytes(n, auto) == max(N.workspace_bytes(n, p) for p in each)
    # at 2^30 elements B = 6 has more sub-blocks than B = 16
    big = 1 << 30
    assert (N.workspace_bytes(big, N.Params(N.F64, 6, 1e-3, 0, 0, 0))
            > N.workspace_bytes(big, N.Params(N.F64, 16, 1e-3, 0, 0, 0)))


def test_batch_rejects_automatic_B(lib):
    item = N.BatchItem(None, None, 1000, N.Params(N.F64, 0, 1e-3, 0, 0, 0), None, 0)
    arr = (N.BatchItem * 1)(item)
    assert lib.numarck_batch_workspace_bytes(arr, 1, 1) == 0


def test_compress_argument_errors_before_device(lib):
    """Every case returns before any CUDA call (fake device addresses are never touched)."""
    p = N.Params(N.F64, 8, 1e-3, 0, 0, 0)
    n = 1000
    bound, wsb = N.compress_bound(n, p), N.workspace_bytes(n, p)
    A = 1 << 20   # a 256-aligned fake address
    C = lambda prev, cur, n, blob, cap, ws, wsz, pp=p: lib.numarck_compress(
        ctypes.c_void_p(prev), ctypes.c_void_p(cur), n, ctypes.byref(pp), ctypes.c_void_p(blob),
        cap, ctypes.c_void_p(ws), wsz, None)
    assert C(A, A, n, 0, bound, A, wsb) == N.ERR_INVALID_ARG          # null blob
    assert C(A, A, n, A, bound, 0, wsb) == N.ERR_INVALID_ARG          # null workspace
    assert C(0, A, n, A, bound, A, wsb) == N.ERR_INVALID_ARG          # null prev
    assert C(A, A, -5, A, bound, A, wsb) == N.ERR_INVALID_ARG         # negative n
    assert C(A + 4, A, n, A, bound, A, wsb) == N.ERR_INVALID_ARG      # prev not 8-aligned
    assert C(A, A, n, A + 16, bound, A, wsb) == N.ERR_INVALID_ARG     # blob not 256-aligned
    assert C(A, A, n, A, bound - 1, A, wsb) == N.ERR_CAPACITY
    assert C(A, A, n, A, bound, A, wsb - 1) == N.ERR_CAPACITY
    bad = N.Params(N.F64, 8, 1e-3, 5, 0, 0)
    assert C(A, A, n, A, bound, A, wsb, bad) == N.ERR_INVALID_ARG


def _oracle_header(n=5000, T=np.float64, B=8, bb=1 << 20):
    rng = np.random.default_rng(3)
    p = rng.lognormal(size=n).astype(T)
    x = (p * (1 + rng.normal(0, 0.01, n))).astype(T)
    return O.compress(p, x, 1e-3, B, block_bytes=bb).to_bytes()


def test_blob_size_and_header_validation(lib):
    for T, B, bb in ((np.float64, 8, 1 << 20), (np.float32, 13, 100), (np.float64, 3, 17)):
        data = _oracle_header(T=T, B=B, bb=bb)
        hb = data[:256]
        assert N.blob_size(hb) == len(data)
        hdr = N.parse_header(hb)
        assert hdr["total_bytes"] == len(data)
    data = bytearray(_oracle_header())
    for off, val in ((0, 0xDEAD), (4, 2), (12, 40), (48, 7)):       # magic, version, B, epb
        bad = bytearray(data[:256])
        bad[off:off + 4] = struct.pack("<I", val)
        with pytest.raises(N.NumarckError) as e:
            N.blob_size(bytes(bad))
        assert e.value.code == N.ERR_CORRUPT
    st = bytearray(data[:256])
    st[28:32] = struct.pack("<i", N.ERR_TIMEOUT)                       # device status word
    with pytest.raises(N.NumarckError) as e:
        N.blob_size(bytes(st))
    assert e.value.code == N.ERR_TIMEOUT


def test_decompress_argument_errors_before_device(lib):
    data = _oracle_header(n=5000)
    hb = ctypes.c_char_p(data[:256])
    A = 1 << 20
    D = lambda start, count: lib.numarck_decompress_range(
        ctypes.c_void_p(A), hb, ctypes.c_void_p(A), start, count, ctypes.c_void_p(A), None, None)
    assert D(-1, 10) == N.ERR_RANGE
    assert D(0, 5001) == N.ERR_RANGE
    assert D(4990, 11) == N.ERR_RANGE
    assert D(5000, 0) == N.OK                 # empty segment: nothing to launch
    full = lambda n: lib.numarck_decompress(ctypes.c_void_p(A), hb, ctypes.c_void_p(A),
                                            ctypes.c_void_p(A), n, None, None)
    assert full(4999) == N.ERR_INVALID_ARG    # n must match the header
    assert lib.numarck_decompress(ctypes.c_void_p(A + 8), hb, ctypes.c_void_p(A),
                                  ctypes.c_void_p(A), 5000, None, None) == N.ERR_INVALID_ARG


def test_chained_step_argument_errors_before_device(lib):
    """numarck_decompress_compress validates both halves, the blob header against the
    parameters and the aliasing of its buffers on the host, before any CUDA call."""
    n = 5000
    data = _oracle_header(n=n)
    hb = ctypes.c_char_p(data[:256])
    p = N.Params(N.F64, 8, 1e-3, 0, 0, 0)
    bound, wsb = N.compress_bound(n, p), N.workspace_bytes(n, p)
    blob, prev, out, cur, nblob, ws = (k << 30 for k in range(1, 7))   # disjoint fake buffers
    C = lambda blob=blob, prev=prev, out=out, cur=cur, nblob=nblob, ws=ws, n=n, pp=p, hb=hb: \
        lib.numarck_decompress_compress(
            ctypes.c_void_p(blob), hb, ctypes.c_void_p(prev), ctypes.c_void_p(out), n, None,
            ctypes.c_void_p(cur), ctypes.byref(pp), ctypes.c_void_p(nblob), bound,
            ctypes.c_void_p(ws), wsb, None)
    assert C(n=-1) == N.ERR_INVALID_ARG
    assert C(blob=blob + 16) == N.ERR_INVALID_ARG                    # blob not 256-aligned
    assert C(out=0) == N.ERR_INVALID_ARG
    assert C(nblob=blob) == N.ERR_INVALID_ARG                        # next blob = this blob
    assert C(out=nblob + 256) == N.ERR_INVALID_ARG                   # out inside the next blob
    assert C(out=ws) == N.ERR_INVALID_ARG                            # out inside the workspace
    assert C(out=cur + 8) == N.ERR_INVALID_ARG                       # out overlaps next_cur
    assert C(out=prev) == N.ERR_INVALID_ARG                          # out is prev
    assert C(n=n - 1) == N.ERR_INVALID_ARG                           # n differs from the header
    p32 = N.Params(N.F32, 8, 1e-3, 0, 0, 0)
    assert C(pp=p32) == N.ERR_INVALID_ARG                            # float64 blob, float32 step
    bad = bytearray(data[:256])
    bad[0:4] = struct.pack("<I", 0xDEAD)
    assert C(hb=ctypes.c_char_p(bytes(bad))) == N.ERR_CORRUPT


def test_selftest_wait_argument_errors(lib):
    A = 1 << 20
    W = lambda flag, limit, status: lib.numarck_selftest_wait(
        ctypes.c_void_p(flag), limit, ctypes.c_void_p(status), None)
    assert W(0, 10 ** 7, A) == N.ERR_INVALID_ARG                     # null flag
    assert W(A, 10 ** 7, 0) == N.ERR_INVALID_ARG                     # null status
    assert W(A + 4, 10 ** 7, A) == N.ERR_INVALID_ARG                 # flag not 8-byte aligned
    assert W(A, 999_999, A) == N.ERR_INVALID_ARG                     # limit below 1 ms
    assert W(A, 10 ** 10 + 1, A) == N.ERR_INVALID_ARG                # limit above 10 s


def test_batch_validation_before_device(lib):
    """Batch calls validate every item on the host before queueing anything."""
    A = 1 << 20
    good = N.Params(N.F64, 8, 1e-3, 0, 0, 0)
    bad = N.Params(N.F64, 0, 1e-3, 0, 0, 0)
    n = 5000
    bound = N.compress_bound(n, good)
    items = (N.BatchItem * 3)(N.BatchItem(A, A, n, good, A, bound),
                              N.BatchItem(A, A, 2 * n, good, A, N.compress_bound(2 * n, good)),
                              N.BatchItem(A, A, n, bad, A, bound))
    assert lib.numarck_batch_workspace_bytes(items, 3, 2) == 0          # invalid item 2
    assert lib.numarck_batch_workspace_bytes(items, 2, 2) >= 2 * N.workspace_bytes(n, good)
    assert lib.numarck_batch_workspace_bytes(items, 2, 1) == N.workspace_bytes(2 * n, good)
    assert lib.numarck_batch_workspace_bytes(items, 2, 0) == 0
    assert lib.numarck_compress_batch(items, 3, 2, 1, ctypes.c_void_p(A), 1 << 40, None) \
        == N.ERR_INVALID_ARG
    assert lib.numarck_compress_batch(items, 2, 2, 0, ctypes.c_void_p(A), 1 << 40, None) \
        == N.ERR_INVALID_ARG                                              # grid_share < 1
    need = lib.numarck_batch_workspace_bytes(items, 2, 2)
    assert lib.numarck_compress_batch(items, 2, 2, 1, ctypes.c_void_p(A), need - 1, None) \
        == N.ERR_CAPACITY
    short = (N.BatchItem * 1)(N.BatchItem(A, A, n, good, A, bound - 1))
    assert lib.numarck_compress_batch(short, 1, 1, 1, ctypes.c_void_p(A), 1 << 40, None) \
        == N.ERR_CAPACITY
    assert lib.numarck_compress_batch(items, 0, 1, 1, None, 0, None) == N.OK


def test_fused_batch_validation_before_device(lib):
    """The fused batch calls validate the tuning, every item and the workspace on the host
    before queueing anything."""
    A = 1 << 20
    good = N.Params(N.F64, 8, 1e-3, 0, 0, 0)
    f32 = N.Params(N.F32, 10, 1e-4, 1, 0, 3001)
    n = 5000
    items = (N.BatchItem * 3)(N.BatchItem(A, A, n, good, A, N.compress_bound(n, good)),
                              N.BatchItem(A, A, 3 * n, f32, A, N.compress_bound(3 * n, f32)),
                              N.BatchItem(A, A, n, N.Params(N.F64, 0, 1e-3, 0, 0, 0), A,
                                          N.compress_bound(n, good)))
    need = lib.numarck_fused_workspace_bytes(items, 2)
    assert need >= N.workspace_bytes(n, good) + N.workspace_bytes(3 * n, f32)
    assert lib.numarck_fused_workspace_bytes(items, 3) == 0              # automatic B
    assert lib.numarck_fused_workspace_bytes(items, 0) == 0
    ws = ctypes.c_void_p(A)
    for t in ((1000, 8, 0, 1, 1, 0), (1024, 6, 0, 1, 1, 0), (1024, 8, 4, 1, 1, 0),
              (1024, 8, -1, 1, 1, 0), (0, 0, 0, 0, 0, 1), (1024, 8, 0, 65, 1, 0),
              (1024, 8, 0, 4, 9, 0), (1024, 8, 0, -1, 1, 0)):
        tu = N.FusedTuning(*t)
        assert lib.numarck_compress_batch_fused(items, 2, ctypes.byref(tu), ws, need, None) \
            == N.ERR_INVALID_ARG, t
        assert lib.numarck_decompress_batch_fused(None, 0, ctypes.byref(tu), ws, 1 << 20, None,
                                                  None) in (N.OK, N.ERR_INVALID_ARG)
    assert lib.numarck_compress_batch_fused(items, 3, None, ws, 1 << 40, None) == N.ERR_INVALID_ARG
    assert lib.numarck_compress_batch_fused(items, 2, None, ws, need - 1, None) == N.ERR_CAPACITY
    assert lib.numarck_compress_batch_fused(items, 2, None, ctypes.c_void_p(A + 16), need, None) \
        == N.ERR_INVALID_ARG                                              # 256-byte alignment
    short = (N.BatchItem * 1)(N.BatchItem(A, A, n, good, A, N.compress_bound(n, good) - 1))
    assert lib.numarck_compress_batch_fused(short, 1, None, ws, 1 << 40, None) == N.ERR_CAPACITY
    assert lib.numarck_compress_batch_fused(items, 0, None, None, 0, None) == N.OK
    # decode: workspace size and alignment, item pointers
    dn = lib.numarck_fused_decode_workspace_bytes(4)
    assert dn >= 4 * 32 + 5 * 8 and lib.numarck_fused_decode_workspace_bytes(0) == 0
    ditems = (N.BatchDecodeItem * 2)(N.BatchDecodeItem(A, A, A, 100), N.BatchDecodeItem(A + 8, A, A, 100))
    assert lib.numarck_decompress_batch_fused(ditems, 2, None, ws, 1 << 20, None, None) \
        == N.ERR_INVALID_ARG                                              # blob not 256-aligned
    assert lib.numarck_decompress_batch_fused(ditems, 1, None, ws, 8, None, None) \
        == N.ERR_CAPACITY
