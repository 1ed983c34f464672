"""The sharded path with the product kernels: two ranks (gloo for the
host-side reductions; both on the one visible GPU, each with its own copy of
the map, and no kernel of one rank waits on the other) each answer their
round-robin share of the scans.  Every scan's idx, d2 and cov equal the
single-process answer bit for bit, and the reductions bench.py uses (max
over ranks of the elapsed time, sum of the queries) come out right."""
import os
import socket

import numpy as np
import pytest

from paper_2308_07173_gb300 import sharding

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_SCANS, K, EPS = 6, 20, 1e-3


def _world():
    from paper_2308_07173_gb300 import workloads as W

    tr = W.oval_1500()
    m = tr.sample_map(300_000, seed=41)
    g = W.rng_for(42)
    scans = [tr.raycast(*tr.random_pose(g), g)[: 20_000 + 3_000 * i] for i in range(N_SCANS)]
    return m, scans


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    from paper_2308_07173_gb300 import pc

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        m, scans = _world()
        t = pc.Target(torch.from_numpy(m).cuda())
        mine = sharding.scans_for_rank(len(scans), world, rank)
        res = {}
        for i in mine:
            idx, d2, cov = t.knn_cov(torch.from_numpy(scans[i]).cuda(), K, EPS)
            torch.cuda.synchronize()
            res[i] = (idx.cpu().numpy(), d2.cpu().numpy(), cov.cpu().numpy())
        ok = t.sync_status() == pc.PC_OK
        t.close()
        worst = sharding.reduce_max(1.0 + rank)
        total = sharding.reduce_sum(sum(len(scans[i]) for i in mine))
        out.put((rank, ok, res, worst, total))
    finally:
        dist.destroy_process_group()


def test_two_ranks_answer_their_scans_like_one_process(gpu_lib):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    m, scans = _world()
    t = gpu_lib.Target(torch.from_numpy(m).cuda())
    try:
        seen = set()
        for rank, ok, res, worst, total in got:
            assert ok
            assert worst == 2.0
            assert total == sum(len(s) for s in scans)
            assert sorted(res) == sharding.scans_for_rank(len(scans), 2, rank)
            for i, (gi, gd, gc) in res.items():
                idx, d2, cov = t.knn_cov(torch.from_numpy(scans[i]).cuda(), K, EPS)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(gi, idx.cpu().numpy())
                np.testing.assert_array_equal(gd.view(np.uint32), d2.cpu().numpy().view(np.uint32))
                np.testing.assert_array_equal(gc.view(np.uint32), cov.cpu().numpy().view(np.uint32))
                seen.add(i)
        assert seen == set(range(len(scans)))
    finally:
        t.close()
