"""The sharded (multi-GPU) path's host logic on CPU: two gloo ranks.
SNPs are independent, so ranks own disjoint SNP blocks and exchange nothing but
the timing max; the job rate is all ranks' SNPs over the slowest rank's time;
the per-rank results are gathered on the host into SNP column order."""
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


def _fake_block(c0, ncols, p=4):
    """Stand-in results of the SNP columns c0 .. c0+ncols-1 (values encode the column)."""
    import numpy as np
    cols = np.arange(c0, c0 + ncols, dtype=np.float64)
    return (np.vstack([cols + 0.25 * j for j in range(p)]), np.vstack([-cols] * p), (cols % 3).astype(np.int32))


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
    # results of this rank's blocks, listed last block first: the gather restores column order
    from paper_1302_4332_b300.shard import gather_columns
    parts = [(c0, _fake_block(c0, 4096)) for c0 in reversed(starts)]
    full = gather_columns(dist, parts)
    out[rank] = (gathered, slowest, bench.job_rate(world, 8 * 4096, slowest),
                 None if full is None else tuple(a.tolist() for a in full))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_disjoint_and_time_by_slowest():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    g0, slow0, rate0, full0 = out[0]
    g1, slow1, rate1, full1 = out[1]
    assert g0 == g1
    cols = [set(range(c, c + 4096)) for starts in g0 for c in starts]
    union = set().union(*cols)
    assert len(union) == sum(len(c) for c in cols) == world * 8 * 4096  # disjoint, complete
    assert min(union) == 0 and max(union) == world * 8 * 4096 - 1
    assert slow0 == slow1 == 2.0
    assert rate0 == rate1 == pytest.approx(world * 8 * 4096 / 2.0)
    # the gather: rank 0 holds every column in order, the other rank nothing
    import numpy as np
    assert full1 is None
    b, se, st = (np.asarray(a) for a in full0)
    ref = _fake_block(0, world * 8 * 4096)
    assert np.array_equal(b, ref[0]) and np.array_equal(se, ref[1]) and np.array_equal(st, ref[2])


def test_assemble_columns_rejects_gaps_and_overlaps():
    import numpy as np
    from paper_1302_4332_b300.shard import assemble_columns
    a = [(0, _fake_block(0, 5)), (5, _fake_block(5, 3))]
    b, se, st = assemble_columns([a[1:], a[:1]])
    assert np.array_equal(b, _fake_block(0, 8)[0]) and np.array_equal(st, _fake_block(0, 8)[2])
    with pytest.raises(ValueError):
        assemble_columns([[(0, _fake_block(0, 5))], [(6, _fake_block(6, 3))]])
    with pytest.raises(ValueError):
        assemble_columns([[(0, _fake_block(0, 5))], [(4, _fake_block(4, 3))]])
