"""The multi-rank plumbing of bench.py on CPU (gloo, two ranks): the batch's independent
systems are sharded over the ranks with no data-path collective, and the job time is the
slowest rank's."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sizes = [7, 3, 9, 1, 4, 4, 8, 2]
    mine = bench.shard_systems(sizes, world)[rank]
    slowest = bench.max_over_ranks(1.5 + rank, "cpu")
    dist.barrier()
    q.put((rank, mine, slowest))
    dist.destroy_process_group()


def test_shard_and_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    shards = [o[1] for o in out]
    assert sorted(shards[0] + shards[1]) == list(range(8))      # every system exactly once
    assert not set(shards[0]) & set(shards[1])
    assert all(o[2] == 2.5 for o in out)                          # both ranks see the slowest time


def test_shard_systems_balance():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1908_10169_gb300 import workloads as W
    sizes = [w.A.nnz for w in W.cd_batch(count=64, seed0=100)]
    for world in (1, 2, 4, 8):
        parts = bench.shard_systems(sizes, world)
        assert sorted(i for p in parts for i in p) == list(range(64))
        loads = [sum(sizes[i] for i in p) for p in parts]
        # largest first onto the least loaded rank: within the largest system of the average
        assert max(loads) - min(loads) <= max(sizes)
        assert max(loads) <= sum(sizes) / world + max(sizes)
    assert bench.shard_systems([5, 5, 5], 2) == [[0, 2], [1]]       # ties: lower rank, in order
