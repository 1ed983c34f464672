"""The allocation-free batched entry, pc_batch_run_noalloc.

Callers that may not allocate device memory while running (a real-time loop
that reserved its GPU memory at start-up, where a cudaMalloc or cudaFree
could stall the whole device, or an application that serves all device
buffers from its own pool) use this entry: its scratch lives in a fixed
device array inside the library instead of memory from cudaMalloc.

Through the C ABI this checks that two calls in a row give exactly the
neighbours and covariances of the regular entry pc_knn_cov on each scan
(bit for bit), that the calls change neither the device's free memory nor
torch's reserved memory, that an empty scan and a scan without covariance
output are handled, and that the call refuses an over-long scan list, a
target with appended points, k above the map size and a stream that is
being captured (leaving the capture intact).  It sits in its own file that
pytest collects last, and needs nothing from the other test files.
"""
import time

import numpy as np
import pytest

from paper_2308_07173_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FILL = -7


def test_noalloc_batch_matches_regular_entry_twice(gpu_lib):
    pc = gpu_lib
    tr = W.oval_1500()
    m = tr.sample_map(300_000, seed=21)
    g = W.rng_for(22)
    scans = []
    for size in (1, 31, 4000, 0, 777, 20_000, 900):
        full = tr.raycast(*tr.random_pose(g), g)
        scans.append(full[np.sort(g.choice(len(full), size, replace=False))])
    no_cov = 6  # this scan asks for neighbours only
    k, eps = 20, 1e-3
    t = pc.Target(torch.from_numpy(m).cuda())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        qs = [torch.from_numpy(s).cuda() for s in scans]
        ref = [t.knn_cov(q, k, eps, stream=stream) for q in qs]
        outs = [(torch.empty((len(q), k), dtype=torch.int32, device="cuda"),
                 torch.empty((len(q), k), dtype=torch.float32, device="cuda"),
                 torch.empty((len(q), 6), dtype=torch.float32, device="cuda")) for q in qs]
    descs = [pc.pc_scan(q.data_ptr(), q.shape[0], o[0].data_ptr(), o[1].data_ptr(),
                        0 if i == no_cov else o[2].data_ptr())
             for i, (q, o) in enumerate(zip(qs, outs))]
    sh = int(stream.cuda_stream)
    dev = torch.cuda.current_device()
    for call in range(2):
        with torch.cuda.stream(stream):
            for o in outs:
                o[0].fill_(FILL)
                o[1].fill_(float(FILL))
                o[2].fill_(float(FILL))
        stream.synchronize()
        free0, reserved0 = torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_reserved(dev)
        rc = pc.pc_batch_run_noalloc(t.handle, descs, k, eps, sh)
        assert rc == pc.PC_OK, pc.pc_status_string(rc)
        stream.synchronize()
        if call == 1:  # the first call per device may look up the array's address
            assert torch.cuda.mem_get_info(dev)[0] == free0, "device memory was allocated"
            assert torch.cuda.memory_reserved(dev) == reserved0
        assert t.sync_status(stream) == pc.PC_OK
        for i, ((ri, rd, rc_), (oi, od, oc)) in enumerate(zip(ref, outs)):
            assert torch.equal(oi, ri), f"call {call} scan {i}: neighbour indices differ"
            assert torch.equal(od.view(torch.int32), rd.view(torch.int32)), f"call {call} scan {i}: d2 differs"
            if i == no_cov:
                assert bool((oc == FILL).all()), "a scan without covariance output was written"
            else:
                assert torch.equal(oc.view(torch.int32), rc_.view(torch.int32)), \
                    f"call {call} scan {i}: covariance differs"

    # host time of one call queued behind ~50 ms of other work on the stream
    # (the table copy from pageable memory may wait for it)
    with torch.cuda.stream(stream):
        torch.cuda._sleep(100_000_000)
    t0 = time.perf_counter()
    assert pc.pc_batch_run_noalloc(t.handle, descs, k, eps, sh) == pc.PC_OK
    host_ms = (time.perf_counter() - t0) * 1e3
    stream.synchronize()
    print(f"pc_batch_run_noalloc host time behind a busy stream: {host_ms:.3f} ms")

    # refusals, none of which enqueues anything
    too_many = descs * (pc.PC_NOALLOC_MAX_SCANS // len(descs) + 1)
    assert pc.pc_batch_run_noalloc(t.handle, too_many, k, eps, sh) == pc.PC_ERR_INVALID_ARG
    small = pc.Target(torch.from_numpy(m[:10].copy()).cuda())
    assert pc.pc_batch_run_noalloc(small.handle, descs, k, eps, sh) == pc.PC_ERR_K_GT_M
    small.close()
    grown = pc.Target(torch.from_numpy(m[:100_000].copy()).cuda())
    grown.append(torch.from_numpy(m[100_000:101_000].copy()).cuda())
    assert pc.pc_batch_run_noalloc(grown.handle, descs, k, eps, sh) == pc.PC_ERR_INVALID_ARG
    grown.close()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        marker = torch.zeros(1, device="cuda")
        graph.capture_begin()
        marker += 1
        rc = pc.pc_batch_run_noalloc(t.handle, descs, k, eps, int(side.cuda_stream))
        graph.capture_end()
    assert rc == pc.PC_ERR_INVALID_ARG
    graph.replay()  # the capture survived the refusal
    torch.cuda.synchronize()
    assert marker.item() == 1.0
    t.close()


def test_noalloc_batch_writes_page_locked_outputs(gpu_lib):
    """Outputs in page-locked host memory: the staged kernel writes them in
    place, equal bit for bit to the regular entry, an empty scan untouched."""
    pc = gpu_lib
    tr = W.oval_1500()
    m = tr.sample_map(200_000, seed=23)
    g = W.rng_for(24)
    scans = [tr.raycast(*tr.random_pose(g), g)[:n] for n in (5000, 0, 1234, 31)]
    k, eps = 16, 1e-3
    t = pc.Target(torch.from_numpy(m).cuda())
    try:
        qs = [torch.from_numpy(np.ascontiguousarray(s)).cuda() for s in scans]
        ref = [t.knn_cov(q, k, eps) for q in qs]
        outs = [(torch.full((len(s), k), FILL, dtype=torch.int32).pin_memory(),
                 torch.full((len(s), k), float(FILL)).pin_memory(),
                 torch.full((len(s), 6), float(FILL)).pin_memory()) for s in scans]
        descs = [pc.pc_scan(q.data_ptr(), q.shape[0], o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr())
                 for q, o in zip(qs, outs)]
        assert pc.pc_batch_run_noalloc(t.handle, descs, k, eps, 0) == pc.PC_OK
        torch.cuda.synchronize()
        for (ri, rd, rc), o in zip(ref, outs):
            assert torch.equal(o[0], ri.cpu())
            assert torch.equal(o[1].view(torch.int32), rd.cpu().view(torch.int32))
            assert torch.equal(o[2].view(torch.int32), rc.cpu().view(torch.int32))
        assert t.sync_status() == pc.PC_OK
    finally:
        t.close()
