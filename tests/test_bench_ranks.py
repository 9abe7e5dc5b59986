"""The benchmark's multi-GPU arithmetic (replicas, one process per GPU) on
CPU ranks over gloo: the job's time is the slowest rank's, units add up over
ranks, so value = all ranks' steps / the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dev = torch.device("cpu")
    t = bench.slowest(1000.0 + 250.0 * rank, dev)     # rank 1 is slower
    k = bench.job_total(4.0, dev)                     # 4 steps on each rank
    q.put((rank, t, k, k / (t / 1000.0)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slowest_rank_and_job_total(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = 1000.0 + 250.0 * (world - 1)
    for rank, t, k, rate in res:
        assert t == slowest and k == 4.0 * world
        assert abs(rate - 4.0 * world / (slowest / 1000.0)) < 1e-12


def test_single_process_is_identity():
    import torch
    import bench
    assert bench.slowest(12.5, torch.device("cpu")) == 12.5
    assert bench.job_total(3.0, torch.device("cpu")) == 3.0
