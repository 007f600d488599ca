"""Multi-rank host logic on CPU (gloo, world size 2): the bench's sharding of the
batched workload and its reduction of times over ranks.

Independent Hamiltonians need no exchange, so the only multi-rank pieces are
the partition of the systems (longest-processing-time rule on N^3) and the
maximum of the per-rank times. Both run here as two gloo processes.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import synthetic
    from paper_1503_07037_gb300.shard import cube_weights, lpt_partition

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = synthetic.cluster_sizes()
        w = cube_weights(sizes)
        share = lpt_partition(w, world)[rank]
        shares = [None] * world
        dist.all_gather_object(shares, share)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(sizes)))              # every system exactly once
        loads = [sum(w[i] for i in s) for s in shares]
        bound = max(max(w), sum(w) / world)
        assert max(loads) <= (4.0 / 3.0 - 1.0 / (3 * world)) * bound * 1.0000001
        # bench's timing reduction: the slowest rank's time
        t = 1.5 * (rank + 1)
        assert bench.reduce_max(dist, t, "cpu") == 1.5 * world
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_lpt_partition_single_process():
    from paper_1503_07037_gb300.shard import lpt_partition
    assert lpt_partition([5, 1, 4, 2, 3], 1) == [[0, 1, 2, 3, 4]]
    parts = lpt_partition([5, 1, 4, 2, 3], 2)
    assert sorted(parts[0] + parts[1]) == [0, 1, 2, 3, 4]
    assert {sum([5, 1, 4, 2, 3][i] for i in p) for p in parts} == {7, 8}
    assert lpt_partition([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        lpt_partition([1.0], 0)


def test_two_gloo_ranks_share_the_batch_and_reduce_times():
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)
