"""Host logic of the multi-process benchmark path (replicas only: one
independent solve per rank, no data-path collective), on CPU with gloo and
world size 2: the timing barrier takes the max over ranks and the job-level
seconds per solve divide the slowest step by the number of replicas."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank)   # rank 1 is the slow one
    out[rank] = (ms, bench.job_seconds_per_solve(ms, world), bench._dist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, per_solve, d = out[r]
        assert ms == 150.0
        assert per_solve == pytest.approx(0.075)
        assert d == (2, r, 0)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_seconds_per_solve(1500.0, 1) == 1.5
