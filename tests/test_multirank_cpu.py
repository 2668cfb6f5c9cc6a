"""The sharded (multi-GPU) bench path's host logic on CPU: two gloo ranks.
SNPs are independent, so ranks own disjoint SNP blocks and exchange nothing but
the timing max; the job rate is all ranks' SNPs over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    starts = bench.shard_block_starts(rank, world, nb=8, bs=4096)
    gathered = [None] * world
    dist.all_gather_object(gathered, starts)
    slowest = bench.max_over_ranks(1.0 + rank, dist)  # rank 1 is slower
    out[rank] = (gathered, slowest, bench.job_rate(world, 8 * 4096, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_disjoint_and_time_by_slowest():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    g0, slow0, rate0 = out[0]
    g1, slow1, rate1 = out[1]
    assert g0 == g1
    cols = [set(range(c, c + 4096)) for starts in g0 for c in starts]
    union = set().union(*cols)
    assert len(union) == sum(len(c) for c in cols) == world * 8 * 4096  # disjoint, complete
    assert min(union) == 0 and max(union) == world * 8 * 4096 - 1
    assert slow0 == slow1 == 2.0
    assert rate0 == rate1 == pytest.approx(world * 8 * 4096 / 2.0)
