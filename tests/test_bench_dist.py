"""The multi-rank plumbing of bench.py on CPU: two gloo ranks (world size 2) run the same
barrier / max-over-ranks / sum-over-ranks helpers that the GPU bench uses under torchrun, and
the whole-job value is the units of all ranks over the slowest rank's time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w = bench._rank_world()
    assert (r, w) == (rank, world)
    d = bench._init_dist(w)
    assert d is not None and dist.get_backend() == "gloo"
    bench._barrier(d)
    ms = 100.0 + 50.0 * rank               # rank 1 is the slowest
    slowest = bench._max_over_ranks(d, ms)
    units = bench._sum_over_ranks(d, 1000.0 * (rank + 1))
    out[rank] = (slowest, units, units / (slowest / 1e3))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_max_and_sum():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    slowest, units, value = out[0]
    assert slowest == 150.0 and units == 3000.0
    assert value == pytest.approx(3000.0 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench._init_dist(1) is None
    assert bench._max_over_ranks(None, 7.0) == 7.0 and bench._sum_over_ranks(None, 3.0) == 3.0
