"""The allocation-free compression entry point, for callers that cannot allocate device memory
(a simulation whose memory pool already owns the GPU, code that must avoid the implicit device
synchronisation of cudaMalloc, plugins whose host forbids raw CUDA allocations).

numarck_compress_noalloc is called through the C ABI and its blob must equal, byte for byte, the
blob of numarck_compress with a caller-supplied workspace, on two calls in a row with different
inputs (the shared scratch array keeps the previous call's contents, so the second call checks
that nothing leaks from the first). This file is collected last on purpose.
"""
import ctypes

import pytest
import torch

from paper_1703_02438_gb300 import numarck as N
from paper_1703_02438_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(prev, cur, params, blob):
    L = N.lib()
    L.numarck_compress_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.POINTER(N.Params), ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]
    L.numarck_compress_noalloc.restype = ctypes.c_int
    return L.numarck_compress_noalloc(
        ctypes.c_void_p(prev.data_ptr()), ctypes.c_void_p(cur.data_ptr()), prev.numel(),
        ctypes.byref(params), ctypes.c_void_p(blob.data_ptr()), blob.numel(),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _used(blob):
    hb = N.header_bytes(blob)
    return blob[: N.blob_size(hb)].cpu()


def test_noalloc_matches_workspace_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1703_02438_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    cases = [
        (synth.plain_pair(1 << 20, seed=synth.seed_for(0, 21)), 1e-3, 8, N.ANCHOR_ZERO),
        (synth.plain_pair(300_007, dtype=torch.float32, seed=synth.seed_for(0, 22)), 1e-4, 10,
         N.ANCHOR_MIN),
    ]
    for (p, x), E, B, anchor in cases:
        p, x = p.to(dev), x.to(dev)
        params = N.make_params(p.dtype, B, E, anchor)
        bound = N.compress_bound(p.numel(), params)
        blob = torch.empty(bound, dtype=torch.uint8, device=dev)
        assert _noalloc(p, x, params, blob) == N.OK
        torch.cuda.synchronize()
        want = N.compress(p, x, E, B, anchor=anchor)
        torch.cuda.synchronize()
        got, ref = _used(blob), _used(want)
        assert torch.equal(got, ref)
        rec = N.decompress(blob, p)
        ref_rec = N.decompress(want, p)
        torch.cuda.synchronize()
        assert torch.equal(rec.view(torch.uint8), ref_rec.view(torch.uint8))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    params = N.make_params(torch.float64, 8, 1e-3, N.ANCHOR_ZERO, block_bytes=2)
    n = 10_000_000          # 2-byte blocks: one sub-block per element -> 80 MB of scan state
    assert N.workspace_bytes(n, params) > 48 * 1024 * 1024
    A = torch.empty(1, device="cuda:0")
    L = N.lib()
    L.numarck_compress_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.POINTER(N.Params), ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]
    rc = L.numarck_compress_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()),
                                    n, ctypes.byref(params), ctypes.c_void_p(A.data_ptr()), 1, None)
    assert rc == N.ERR_CAPACITY
