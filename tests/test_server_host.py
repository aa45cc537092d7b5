"""The served form's scheduling on the host (dry run: no CUDA call is made, every request stage
takes a fixed time): per-series order, the slot limit, admission by free arena space, requests
that can never fit, no starvation of large requests, and argument errors."""
import time

import pytest
import torch

from paper_1703_02438_gb300 import numarck as N

MB = 1 << 20


@pytest.fixture(scope="module")
def lib():
    from paper_1703_02438_gb300 import build
    build.build()
    return N.lib()


def _params(B=8):
    return N.make_params(torch.float64, B, 1e-3)


def _drain(srv, want, timeout=20.0):
    out, t0 = [], time.time()
    while len(out) < want and time.time() - t0 < timeout:
        out += srv.poll(wait_ms=50)
    assert len(out) == want, f"{len(out)} of {want} completions"
    return out


def test_series_order_and_slot_limit(lib):
    srv = N.Server(None, slots=3, max_series=8, dry_run_us=2000)
    dummy = torch.empty(1)
    ids = {}
    for t in range(4):                        # 4 timesteps of 5 series, interleaved
        for s in range(5):
            ids[srv.submit(N.REQ_COMPRESS, s, 1000, _params(), host_in=dummy,
                           host_out=torch.empty(16))] = (s, t)
    done = _drain(srv, 20)
    st = srv.stats()
    srv.close()
    assert all(c["status"] == 0 for c in done)
    assert st["max_inflight"] == 3
    for s in range(5):
        mine = sorted((c for c in done if c["series"] == s), key=lambda c: c["t_start"])
        assert [ids[c["id"]][1] for c in mine] == [0, 1, 2, 3]           # submission order
        assert [c["reference"] for c in mine] == [1, 0, 0, 0]
        for a, b in zip(mine, mine[1:]):                                   # one at a time
            assert b["t_start"] >= a["t_end"]


def test_admission_by_free_arena_space(lib):
    n = 1000
    ws = N.workspace_bytes(n, _params())
    res = 2 * n * 8 + N.compress_bound(n, _params(16))
    # room for the resident buffers of 4 series plus the transient buffers of one compression
    arena = 4 * (res + 4096) + (ws + n * 8) + ws // 2
    srv = N.Server(None, slots=4, max_series=4, dry_run_us=3000, arena_bytes=arena)
    dummy = torch.empty(1)
    for s in range(4):
        srv.submit(N.REQ_COMPRESS, s, n, _params(), host_in=dummy, host_out=torch.empty(16))
    _drain(srv, 4)                                                         # references
    for s in range(4):
        srv.submit(N.REQ_COMPRESS, s, n, _params(), host_in=dummy, host_out=torch.empty(16))
    done = _drain(srv, 4)
    st = srv.stats()
    srv.close()
    assert all(c["status"] == 0 for c in done)
    assert st["deferred_memory"] > 0 and st["arena_peak"] <= arena
    spans = sorted((c["t_start"], c["t_end"]) for c in done)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):                       # never two at once
        assert b0 >= a1


def test_request_that_can_never_fit(lib):
    srv = N.Server(None, slots=2, max_series=2, dry_run_us=100, arena_bytes=8 * MB)
    rid = srv.submit(N.REQ_COMPRESS, 0, 1 << 20, _params(), host_in=torch.empty(1),
                     host_out=torch.empty(16))
    (c,) = _drain(srv, 1)
    srv.close()
    assert c["id"] == rid and c["status"] == N.ERR_CAPACITY


def _g(b):
    return (max(b, 1) + 255) // 256 * 256          # the arena's 256-byte granules


def test_large_request_is_not_starved(lib):
    """A large compression that does not fit beside running small requests of other series is
    not overtaken by younger small requests (which would keep it waiting as long as they keep
    coming)."""
    small, big = 1000, 200_000
    res = lambda n: 2 * _g(n * 8) + _g(N.compress_bound(n, _params(16)))
    big_t = _g(N.workspace_bytes(big, _params())) + _g(big * 8)
    arena = 4 * res(small) + res(big) + big_t      # the big transient fits only when alone
    srv = N.Server(None, slots=4, max_series=5, dry_run_us=3000, arena_bytes=arena)
    dummy = torch.empty(1)
    for s in range(4):                             # series 0..3 small, series 4 large
        srv.submit(N.REQ_COMPRESS, s, small, _params(), host_in=dummy, host_out=torch.empty(16))
        srv.submit(N.REQ_COMPRESS, s, small, _params(), host_in=dummy, host_out=torch.empty(16))
    srv.submit(N.REQ_COMPRESS, 4, big, _params(), host_in=dummy, host_out=torch.empty(16))
    _drain(srv, 9)
    older = []
    for s in range(4):                             # staggered: some are always running
        older.append(srv.submit(N.REQ_DECOMPRESS, s, small, _params(), host_out=torch.empty(small)))
        time.sleep(0.0008)
    big_id = srv.submit(N.REQ_COMPRESS, 4, big, _params(), host_in=dummy, host_out=torch.empty(16))
    younger = [srv.submit(N.REQ_DECOMPRESS, i % 4, small, _params(), host_out=torch.empty(small))
               for i in range(40)]
    done = {c["id"]: c for c in _drain(srv, 45)}
    st = srv.stats()
    srv.close()
    assert all(c["status"] == 0 for c in done.values())
    assert st["deferred_memory"] > 0
    assert all(done[i]["t_start"] >= done[big_id]["t_start"] for i in younger)


def test_argument_errors(lib):
    srv = N.Server(None, slots=1, max_series=2, dry_run_us=100)
    with pytest.raises(N.NumarckError):
        srv.submit(N.REQ_COMPRESS, 2, 10, _params(), host_in=torch.empty(1))     # series range
    with pytest.raises(N.NumarckError):
        srv.submit(N.REQ_COMPRESS, 0, 10, _params(0), host_in=torch.empty(1))    # B = 0
    with pytest.raises(N.NumarckError):
        srv.submit(7, 0, 10, _params())                                           # kind
    a = srv.submit(N.REQ_DECOMPRESS, 0, 10, _params(), host_out=torch.empty(10))
    srv.submit(N.REQ_COMPRESS, 1, 10, _params(), host_in=torch.empty(1), host_out=torch.empty(4))
    b = srv.submit(N.REQ_COMPRESS, 1, 11, _params(), host_in=torch.empty(1), host_out=torch.empty(4))
    done = {c["id"]: c for c in _drain(srv, 3)}
    srv.close()
    assert done[a]["status"] == N.ERR_INVALID_ARG           # nothing compressed yet
    assert done[b]["status"] == N.ERR_INVALID_ARG           # n differs from the series'
