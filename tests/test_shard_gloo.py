"""Multi-rank host logic on CPU: ensemble members split over ranks by particle
count, and the timing protocol (max elapsed, summed work) over a world of 2
gloo ranks.  No GPU and no CUDA library are involved."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1612_03369_gb300 import shard
from paper_1612_03369_gb300 import workloads as W


def test_partition_covers_and_balances():
    rng = np.random.default_rng(7)
    for world in (1, 2, 3, 4, 8):
        for n in (0, 1, 5, 64):
            w = rng.integers(0, 10**6, size=n)
            parts = shard.partition_by_weight(w, world)
            assert len(parts) == world
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            for p in parts:
                assert p == sorted(p)
            if n:
                loads = [int(sum(w[i] for i in p)) for p in parts]
                lower = max(int(w.sum()) / world, int(w.max()))
                # longest-processing-time rule: within 4/3 of any split
                assert max(loads) <= (4.0 / 3.0) * lower + 1e-9


def test_partition_small_cases_exact():
    assert shard.partition_by_weight([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    assert shard.partition_by_weight([1, 9, 3], 2) == [[1], [0, 2]]
    assert shard.partition_by_weight([3, 3], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        shard.partition_by_weight([1], 0)
    with pytest.raises(ValueError):
        shard.partition_by_weight([-1], 2)


def test_reduce_timing_single_process():
    assert shard.reduce_timing([1.5, 2.0], [3.0]) == ([1.5, 2.0], [3.0])


def _ensemble_counts():
    # particle counts of the 64-member ensemble without building meshes
    return [int(W.member_per_cell(s, W.c5_member_seed(p)).sum()) for p, s in enumerate(W.c5_sides())]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        r, ws, lr = shard.rank_env()
        assert (r, ws, lr) == (rank, world, rank)
        counts = _ensemble_counts()
        mine = shard.partition_by_weight(counts, world)[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t, u = shard.reduce_timing([10.0 + rank, 1.0 * (world - rank)], [float(sum(counts[i] for i in mine))])
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, gathered, t, u, sum(counts)))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, repr(e), None, None, None))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, gathered, t, u, total = q.get(timeout=120)
        res[rank] = (gathered, t, u, total)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        gathered, t, u, total = res[rank]
        assert not isinstance(gathered, str), gathered
        # both ranks computed the same split; it is disjoint and covers every member
        assert gathered == res[0][0]
        flat = sorted(i for g in gathered for i in g)
        assert flat == list(range(64))
        # max of elapsed times, sum of work
        assert t == [11.0, 2.0]
        assert u == [float(total)]
