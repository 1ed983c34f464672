"""Served form: continuous batching gives every scan the same neighbours,
distances and covariances it gets alone, and so does the per-scan baseline;
the caller-scratch batched entry matches too."""
import numpy as np
import pytest

from paper_2308_07173_gb300 import serve
from paper_2308_07173_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def small_world(gpu_lib):
    tr = W.oval_1500()
    m = tr.sample_map(400_000, seed=31)
    t = gpu_lib.Target(torch.from_numpy(m).cuda())
    arr = W.arrival_stream(duration=0.25, vehicles=2, sensors=3, lo=3000, hi=30000, pool=6, seed=32)
    yield t, arr
    t.close()


def _alone(t, pts, k, eps):
    i, d, c = t.knn_cov(torch.from_numpy(pts).cuda(), k, eps)
    torch.cuda.synchronize()
    return i.cpu(), d.cpu(), c.cpu()


def _same(a, b):
    return (torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))
            and torch.equal(a[2].view(torch.int32), b[2].view(torch.int32)))


@pytest.mark.parametrize("in_place", [False, True])
@pytest.mark.parametrize("speed", [1.0, 1e6])
def test_served_results_equal_alone(small_world, gpu_lib, speed, in_place):
    t, arr = small_world
    k, eps = 20, 1e-3
    reqs = serve.requests_from_arrivals(arr)
    assert len(reqs) > 10
    serve.prepare(reqs)
    srv = serve.Server(t, k, eps, hbm_budget=256 << 20, max_step_scans=4, slots=2, keep_results=True,
                       in_place=in_place)
    if in_place:
        assert srv.device_bytes() == 2 * 512 * -(-srv.scratch_bytes // 512)  # scan tables only
    rep = srv.serve(reqs, speed=speed)
    assert rep["scans"] == len(reqs) and rep["p99_ms"] >= rep["p50_ms"] > 0
    if speed > 1:
        assert rep["mean_scans_per_step"] > 1.0  # requests really were batched
    for r in reqs:
        assert r.t_done >= r.t_admit >= r.t_sched
        assert _same(r.out_host, _alone(t, r.points, k, eps))
    assert t.sync_status() == gpu_lib.PC_OK


def test_per_scan_baseline_equal_alone(small_world, gpu_lib):
    t, arr = small_world
    k, eps = 20, 1e-3
    reqs = serve.requests_from_arrivals(arr[:8])
    serve.prepare(reqs)
    rep = serve.serve_per_scan(t, k, eps, reqs, speed=1e6, keep_results=True)
    assert rep["scans"] == 8
    for r in reqs:
        assert _same(r.out_host, _alone(t, r.points, k, eps))


def test_batch_scratch_entry_checks_scratch(small_world, gpu_lib):
    t, arr = small_world
    pts = torch.from_numpy(arr[0].points).cuda()
    n, k = pts.shape[0], 12
    idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((n, k), dtype=torch.float32, device="cuda")
    descs = [gpu_lib.pc_scan(pts.data_ptr(), n, idx.data_ptr(), d2.data_ptr(), None)]
    need = gpu_lib.pc_batch_scratch_bytes(1)
    scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    assert gpu_lib.pc_batch_run_scratch(t.handle, descs, k, -1.0, scratch.data_ptr(), need - 1, 0) \
        == gpu_lib.PC_ERR_INVALID_ARG
    assert gpu_lib.pc_batch_run_scratch(t.handle, descs, k, -1.0, scratch.data_ptr() + 8, need, 0) \
        == gpu_lib.PC_ERR_INVALID_ARG
    assert gpu_lib.pc_batch_run_scratch(t.handle, descs, k, -1.0, scratch.data_ptr(), need, 0) == gpu_lib.PC_OK
    ri, rd = t.knn(pts, k)
    torch.cuda.synchronize()
    assert torch.equal(ri, idx) and torch.equal(rd.view(torch.int32), d2.view(torch.int32))


def test_tiny_budget_serves_one_scan_at_a_time(small_world, gpu_lib):
    t, arr = small_world
    k, eps = 16, -1.0
    reqs = serve.requests_from_arrivals(arr[:10])
    serve.prepare(reqs)
    srv = serve.Server(t, k, eps, hbm_budget=1, max_step_scans=8, slots=2, keep_results=True)
    assert srv.capacity == 1
    rep = srv.serve(reqs, speed=1e6)
    assert rep["scans"] == 10 and rep["steps"] == 10  # every scan exceeds the capacity: one per step
    for r in reqs:
        assert _same(r.out_host, _alone(t, r.points, k, eps))


def test_budget_that_forces_waits(small_world, gpu_lib):
    """A budget that gives each of two slots room for about two scans:
    requests that arrive together wait for a slot or for room in a step,
    no step exceeds the capacity the budget allows, the server holds no more
    device memory than the budget, and every result is still the one the scan
    gets alone."""
    t, arr = small_world
    k, eps = 20, 1e-3
    reqs = serve.requests_from_arrivals(arr)
    serve.prepare(reqs)
    biggest = max(r.n for r in reqs)
    point_bytes = 12 + 8 * k + 24
    budget = 2 * (int(2.2 * biggest) * point_bytes + (1 << 16))
    srv = serve.Server(t, k, eps, hbm_budget=budget, max_step_scans=4, slots=2, keep_results=True)
    assert biggest <= srv.capacity < 3 * biggest
    assert srv.device_bytes() <= budget
    rep = srv.serve(reqs, speed=1e6)
    assert rep["scans"] == len(reqs)
    assert rep["admission_waits"] > 0
    assert rep["peak_step_points"] <= srv.capacity
    for r in reqs:
        assert _same(r.out_host, _alone(t, r.points, k, eps))
    assert t.sync_status() == gpu_lib.PC_OK


@pytest.mark.parametrize("k,cov", [(20, True), (12, False), (32, True), (40, True)])
def test_batch_entries_write_page_locked_outputs_in_place(small_world, gpu_lib, k, cov):
    """Batched entries with outputs (and scans) in page-locked host memory
    run the staged kernel; every scan's rows equal the device entry's."""
    t, arr = small_world
    scans = [a.points for a in arr[:5]]
    qs = [torch.from_numpy(np.ascontiguousarray(p)).pin_memory() for p in scans]
    outs = [(torch.full((len(p), k), -7, dtype=torch.int32).pin_memory(),
             torch.full((len(p), k), -7.0).pin_memory(),
             torch.full((len(p), 6), -7.0).pin_memory() if cov else None) for p in scans]
    descs = [gpu_lib.pc_scan(q.data_ptr(), q.shape[0], o[0].data_ptr(), o[1].data_ptr(),
                             o[2].data_ptr() if cov else None) for q, o in zip(qs, outs)]
    need = gpu_lib.pc_batch_scratch_bytes(len(descs))
    scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    eps = 1e-3 if cov else -1.0
    assert gpu_lib.pc_batch_run_scratch(t.handle, descs, k, eps, scratch.data_ptr(), need, 0) == gpu_lib.PC_OK
    torch.cuda.synchronize()
    for p, o in zip(scans, outs):
        if cov:
            ref = _alone(t, p, k, eps)
            assert _same(o, ref)
        else:
            ri, rd = t.knn(torch.from_numpy(p).cuda(), k)
            torch.cuda.synchronize()
            assert torch.equal(o[0], ri.cpu()) and torch.equal(o[1].view(torch.int32), rd.cpu().view(torch.int32))
    # the planned form (direct launch and graph replay) takes the same tables
    b = gpu_lib.Batch(t, [(q, o[0], o[1], o[2]) for q, o in zip(qs, outs)], k, eps)
    try:
        for stream in (None, torch.cuda.Stream()):
            for o in outs:
                o[0].fill_(-7)
                o[1].fill_(-7.0)
            b.run(stream)
            torch.cuda.synchronize()
            for p, o in zip(scans, outs):
                ri, rd = t.knn(torch.from_numpy(p).cuda(), k)
                torch.cuda.synchronize()
                assert torch.equal(o[0], ri.cpu()) and torch.equal(o[1].view(torch.int32), rd.cpu().view(torch.int32))
    finally:
        b.close()
    assert t.sync_status() == gpu_lib.PC_OK


def test_batch_entry_refuses_pageable_host_memory(small_world, gpu_lib):
    t, arr = small_world
    p = np.ascontiguousarray(arr[0].points)
    q = torch.from_numpy(p)  # pageable
    idx = torch.empty((len(p), 8), dtype=torch.int32)
    d2 = torch.empty((len(p), 8))
    descs = [gpu_lib.pc_scan(q.data_ptr(), len(p), idx.data_ptr(), d2.data_ptr(), None)]
    need = gpu_lib.pc_batch_scratch_bytes(1)
    scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    assert gpu_lib.pc_batch_run_scratch(t.handle, descs, 8, -1.0, scratch.data_ptr(), need, 0) \
        == gpu_lib.PC_ERR_BAD_POINTER
