"""The multi-rank host logic on CPU: two gloo ranks deal scans, check the
deal is a partition, and reduce timings and counts the way bench.py does."""
import os
import socket

import pytest

from paper_2308_07173_gb300 import sharding


def test_deal_is_a_partition():
    for n in (1, 2, 7, 64):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in sharding.scans_for_rank(n, world, r))
            assert got == list(range(n))
    with pytest.raises(ValueError):
        sharding.scans_for_rank(4, 2, 2)


def test_reductions_without_a_process_group_are_identity():
    assert sharding.reduce_max(3.5) == 3.5
    assert sharding.reduce_sum(7) == 7.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = sharding.scans_for_rank(10, world, rank)
    worst = sharding.reduce_max(1.0 + rank)       # per-rank elapsed time
    total = sharding.reduce_sum(len(mine))        # queries answered by all ranks
    out.put((rank, mine, worst, total))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == [0, 2, 4, 6, 8] and res[1][1] == [1, 3, 5, 7, 9]
    assert all(r[2] == 2.0 for r in res)      # max over ranks
    assert all(r[3] == 10.0 for r in res)     # every scan answered once
