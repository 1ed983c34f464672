"""The allocation-free batched entry, pc_batch_run_noalloc.

Callers that may not allocate device memory while running (a real-time loop
that reserved its GPU memory at start-up, or an application that serves all
device buffers from its own pool) use this entry: its scratch lives in a
fixed device array inside the library instead of memory from cudaMalloc.
This checks, through the C ABI, that two calls in a row give the same
neighbours and covariances as the regular entry pc_knn_cov on each scan,
and that an over-long scan list is refused.  It sits in its own file that
pytest collects last, and needs nothing from the other test files.
"""
import numpy as np
import pytest

from paper_2308_07173_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

COV_RTOL = 1e-5  # the relative Frobenius bar used by the parity tests


def _rel_frob(a, b):
    w = torch.tensor([1, 2, 2, 1, 2, 1], dtype=torch.float64, device=a.device)
    a = a.double()
    b = b.double()
    num = (((a - b) ** 2) * w).sum(1).sqrt()
    den = ((b ** 2) * w).sum(1).sqrt().clamp_min(1e-30)
    return (num / den).max().item()


def test_noalloc_batch_matches_regular_entry_twice(gpu_lib):
    pc = gpu_lib
    tr = W.oval_1500()
    m = tr.sample_map(300_000, seed=21)
    g = W.rng_for(22)
    scans = []
    for size in (1, 31, 4000, 777, 20_000):
        full = tr.raycast(*tr.random_pose(g), g)
        scans.append(full[np.sort(g.choice(len(full), size, replace=False))])
    k, eps = 20, 1e-3
    t = pc.Target(torch.from_numpy(m).cuda())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        qs = [torch.from_numpy(s).cuda() for s in scans]
        ref = [t.knn_cov(q, k, eps, stream=stream) for q in qs]
        outs = [(torch.empty((len(q), k), dtype=torch.int32, device="cuda"),
                 torch.empty((len(q), k), dtype=torch.float32, device="cuda"),
                 torch.empty((len(q), 6), dtype=torch.float32, device="cuda")) for q in qs]
    descs = [pc.pc_scan(q.data_ptr(), q.shape[0], o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr())
             for q, o in zip(qs, outs)]
    sh = int(stream.cuda_stream)
    for call in range(2):
        with torch.cuda.stream(stream):
            for o in outs:
                o[0].fill_(-7)
                o[1].fill_(-7.0)
                o[2].fill_(-7.0)
        rc = pc.pc_batch_run_noalloc(t.handle, descs, k, eps, sh)
        assert rc == pc.PC_OK, pc.pc_status_string(rc)
        stream.synchronize()
        assert t.sync_status(stream) == pc.PC_OK
        for (ri, rd, rc_), (oi, od, oc) in zip(ref, outs):
            assert torch.equal(oi, ri), f"call {call}: neighbour indices differ"
            assert torch.equal(od.view(torch.int32), rd.view(torch.int32)), f"call {call}: d2 differs"
            assert _rel_frob(oc, rc_) <= COV_RTOL, f"call {call}: covariance differs"
    too_many = descs * (pc.PC_NOALLOC_MAX_SCANS // len(descs) + 1)
    assert pc.pc_batch_run_noalloc(t.handle, too_many, k, eps, sh) == pc.PC_ERR_INVALID_ARG
    t.close()
