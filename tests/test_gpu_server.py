"""The served form on the GPU: a closed-loop series through the server equals the oracle bit for
bit (blobs, full and partial decompression), and results do not depend on what else runs:
the same requests alone and mixed give byte-identical outputs."""
import time

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


def _pinned(a: np.ndarray) -> torch.Tensor:
    t = torch.empty(a.size, dtype=torch.from_numpy(a[:1]).dtype, pin_memory=True)
    t.copy_(torch.from_numpy(a))
    return t


def _drain(srv, want, timeout=120.0):
    out, t0 = [], time.time()
    while len(out) < want and time.time() - t0 < timeout:
        out += srv.poll(wait_ms=100)
    assert len(out) == want
    return {c["id"]: c for c in out}


def _series(n, dtype, seed, steps=3):
    rng = np.random.default_rng(seed)
    x = [rng.lognormal(size=n)]
    for _ in range(steps - 1):
        r = np.where(rng.random(n) < 0.9, rng.normal(0, 1e-3, n), rng.uniform(-0.3, 0.3, n))
        x.append(x[-1] * (1 + r))
    return [v.astype(dtype) for v in x]


def test_closed_loop_series_matches_oracle():
    n, E, B = 300_001, 1e-3, 9
    xs = _series(n, np.float64, 5)
    arena = torch.empty(1 << 30, dtype=torch.uint8, device=DEV)
    srv = N.Server(arena, slots=2, max_series=1)
    params = N.make_params(torch.float64, B, E)
    bound = N.compress_bound(n, params)
    prev = xs[0]
    for t, x in enumerate(xs):
        out = torch.empty(bound, dtype=torch.uint8, pin_memory=True)
        rid = srv.submit(N.REQ_COMPRESS, 0, n, params, host_in=_pinned(x), host_out=out)
        c = _drain(srv, 1)[rid]
        assert c["status"] == 0
        if t == 0:
            assert c["reference"] == 1 and c["out_bytes"] == 0
            continue
        want = O.compress(prev, x, E, B).to_bytes()
        assert bytes(out[: c["out_bytes"]].numpy().tobytes()) == want
        rec = O.decompress(want, prev)
        full = torch.empty(n, dtype=torch.float64, pin_memory=True)
        part = torch.empty(20_000, dtype=torch.float64, pin_memory=True)
        a = srv.submit(N.REQ_DECOMPRESS, 0, n, params, host_out=full)
        b = srv.submit(N.REQ_DECOMPRESS, 0, n, params, host_out=part, start=123_457, count=20_000)
        done = _drain(srv, 2)
        assert done[a]["status"] == 0 and done[b]["status"] == 0
        assert np.array_equal(full.numpy().view(np.uint64), rec.view(np.uint64))
        assert np.array_equal(part.numpy().view(np.uint64), rec[123_457:143_457].view(np.uint64))
        prev = rec                                   # the server's next prev
    srv.close()


def _workload(seed=11):
    rng = np.random.default_rng(seed)
    series = []
    for s in range(6):
        n = int(rng.integers(5_000, 400_000))
        T = np.float64 if s % 2 else np.float32
        series.append((n, T, _series(n, T, 100 + s, steps=4)))
    reqs = []
    for t in range(4):
        for s, (n, T, xs) in enumerate(series):
            reqs.append(("c", s, t))
            if t >= 1 and (s + t) % 2 == 0:
                reqs.append(("d", s, t))
    return series, reqs


def _run(series, reqs, slots, mixed):
    arena = torch.empty(2 << 30, dtype=torch.uint8, device=DEV)
    srv = N.Server(arena, slots=slots, max_series=len(series))
    outs, ids = {}, []
    for i, (kind, s, t) in enumerate(reqs):
        n, T, xs = series[s]
        params = N.make_params(torch.float64 if T == np.float64 else torch.float32,
                               6 + s, 1e-3 if s < 3 else 1e-4)
        if kind == "c":
            out = torch.empty(N.compress_bound(n, params), dtype=torch.uint8, pin_memory=True)
            rid = srv.submit(N.REQ_COMPRESS, s, n, params, host_in=_pinned(xs[t]), host_out=out)
        else:
            cnt = n // 3
            out = torch.empty(cnt, dtype=torch.from_numpy(xs[0][:1]).dtype, pin_memory=True)
            rid = srv.submit(N.REQ_DECOMPRESS, s, n, params, host_out=out, start=n // 5, count=cnt)
        outs[i] = (rid, out)
        if not mixed:
            _drain(srv, 1)                               # one at a time
    done = _drain(srv, len(reqs)) if mixed else None
    srv.close()
    res = {}
    for i, (rid, out) in outs.items():
        nbytes = out.numel() * out.element_size()
        res[i] = bytes(out.numpy().tobytes()[:nbytes]) if reqs[i][0] == "d" else out
    return res, done


def test_alone_equals_mixed():
    series, reqs = _workload()
    alone, _ = _run(series, reqs, slots=1, mixed=False)
    mixed, done = _run(series, reqs, slots=8, mixed=True)
    assert all(c["status"] == 0 for c in done.values())
    for i, (kind, s, t) in enumerate(reqs):
        if kind == "c":
            a, m = alone[i], mixed[i]
            hb = bytes(a[:N.HEADER_BYTES].numpy().tobytes())
            if t == 0:
                continue
            size = N.blob_size(hb)
            assert bytes(a[:size].numpy().tobytes()) == bytes(m[:size].numpy().tobytes()), i
        else:
            assert alone[i] == mixed[i], i
