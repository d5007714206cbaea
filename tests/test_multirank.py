"""The N > 1 host logic on the CPU: two gloo ranks split the batched form's
graphs, agree on the job's time (max over ranks) and work (sum), and run
independent replicas of the single-graph workload with distinct seeds."""
import os
import socket

import pytest

from paper_1904_08553_gb300 import shard


def test_partition_covers_every_graph_once_and_balances():
    cost = [5, 1, 9, 3, 3, 7, 2, 2, 8, 4, 6, 1]
    for world in (1, 2, 3, 5, 16):
        shares = shard.partition_graphs(cost, world)
        assert len(shares) == world
        flat = sorted(g for s in shares for g in s)
        assert flat == list(range(len(cost)))
        loads = [sum(cost[g] for g in s) for s in shares]
        assert max(loads) - min(loads) <= max(cost)
    assert shard.partition_graphs([], 2) == [[], []]
    with pytest.raises(ValueError):
        shard.partition_graphs([1], 0)


def test_reductions_without_a_process_group_are_identity():
    assert shard.max_over_ranks(3.5) == 3.5
    assert shard.sum_over_ranks(2.0) == 2.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1904_08553_gb300 import synth

        cost = [100, 3, 50, 50, 7, 90, 1, 60]
        mine = shard.partition_graphs(cost, world)[rank]
        t = float(10 * (rank + 1))
        work = float(sum(cost[g] for g in mine))
        out.put((rank, mine, shard.max_over_ranks(t), shard.sum_over_ranks(work), synth.seed_for(1, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, w0, seed0), (r1, s1, m1, w1, seed1) = res
    assert (r0, r1) == (0, 1)
    assert sorted(s0 + s1) == list(range(8)) and not set(s0) & set(s1)
    assert m0 == m1 == 20.0
    assert w0 == w1 == float(100 + 3 + 50 + 50 + 7 + 90 + 1 + 60)
    assert seed0 != seed1
