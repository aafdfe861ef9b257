"""The multi-GPU mode is replicas (one field per rank, no data-path collective); its
host logic runs here on CPU with two gloo ranks: each rank has its own field seed,
the step time is the slowest rank's, and the throughput counts every rank's bytes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2603_26968_b300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                      # rank 1 is the slowest
        slowest = replicas.max_over_ranks(ms, dist)
        out[rank] = (replicas.rank_seed(1, rank), slowest, replicas.whole_job_gbs(1 << 29, world, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_as_replicas():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    seeds = {res[r][0] for r in range(world)}
    assert len(seeds) == world                       # every rank compresses its own field
    assert all(res[r][1] == 15.0 for r in range(world))   # the slowest rank's step time
    expect = world * (1 << 29) / 15e-3 / 1e9
    assert all(abs(res[r][2] - expect) < 1e-9 for r in range(world))


def test_single_process_needs_no_collective():
    from paper_2603_26968_b300 import replicas
    assert replicas.max_over_ranks(12.5) == 12.5
    assert abs(replicas.whole_job_gbs(1 << 29, 1, 12.5) - (1 << 29) / 12.5e-3 / 1e9) < 1e-12
    with pytest.raises(ValueError):
        replicas.whole_job_gbs(1, 1, 0.0)
