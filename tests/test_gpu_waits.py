"""Failure detection on the GPU without a fault: the library's bounded device wait (used by the
incompressible-offset scan's look-back) run on a flag that nothing sets must give up after its
limit, report NUMARCK_ERR_TIMEOUT through the status word, and leave the context usable."""
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


def test_wait_on_a_flag_nothing_sets_times_out_and_the_context_stays_usable():
    flag = torch.zeros(1, dtype=torch.int64, device=DEV)
    status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    limit = 50_000_000                                   # 50 ms
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    N.selftest_wait(flag, limit, status)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(status.item()) == N.ERR_TIMEOUT
    assert 0.05 <= dt < 5.0
    # a flag that is set is seen at once
    flag.fill_(1)
    status.fill_(-1)
    N.selftest_wait(flag, limit, status)
    torch.cuda.synchronize()
    assert int(status.item()) == N.OK
    # the context still works: a compression after the timeout matches the oracle
    p, x = synth.plain_pair(50_000, seed=synth.seed_for(0, 90))
    blob = N.compress(p.to(DEV), x.to(DEV), 1e-3, 8)
    torch.cuda.synchronize()
    got = blob[:N.blob_size(N.header_bytes(blob))].cpu().numpy().tobytes()
    assert got == O.compress(p.numpy(), x.numpy(), 1e-3, 8).to_bytes()
