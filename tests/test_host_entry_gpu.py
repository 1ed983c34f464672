"""pc_knn_cov_host with page-locked buffers: the search writes idx, d2 and
cov in place in host memory (each warp's block of rows staged in shared
memory, then written as whole lines), and reads a page-locked q in place.
Every case must equal the device entry bit for bit: ragged tiles, every
output vector width (k % 4, k % 2, odd k), both survivor-list sizes, the
warp path (k > 32 and far queries), non-finite queries, a window, and the
copy path taken by pageable or mixed buffers and by a target with appended
points."""
import numpy as np
import pytest

import oracle
from paper_2308_07173_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def pinned_out(n, k):
    return (torch.empty((n, k), dtype=torch.int32).pin_memory(),
            torch.empty((n, k), dtype=torch.float32).pin_memory(),
            torch.empty((n, 6), dtype=torch.float32).pin_memory())


def device_ref(t, q, k, eps):
    idx, d2, cov = t.knn_cov(torch.from_numpy(np.ascontiguousarray(q)).cuda(), k, eps)
    st = t.sync_status()
    return idx.cpu().numpy(), d2.cpu().numpy(), cov.cpu().numpy(), st


def assert_same(got, ref):
    gi, gd, gc = (np.asarray(x.numpy() if hasattr(x, "numpy") else x) for x in got)
    np.testing.assert_array_equal(gi, ref[0])
    np.testing.assert_array_equal(gd.view(np.uint32), ref[1].view(np.uint32))
    np.testing.assert_array_equal(gc.view(np.uint32), ref[2].view(np.uint32))


@pytest.fixture(scope="module")
def box(gpu_lib):
    p = W.uniform_box(8192, seed=1)
    t = gpu_lib.Target(torch.from_numpy(p).cuda())
    yield p, t
    t.close()


@pytest.mark.parametrize("n", [1, 33, 1000, 4099])
@pytest.mark.parametrize("k", [1, 7, 10, 20, 24, 25, 32, 40])
def test_pinned_buffers_equal_device_entry(box, n, k):
    p, t = box
    q = np.ascontiguousarray(p[(np.arange(n) * 7919) % len(p)] + np.float32(0.013))
    ref = device_ref(t, q, k, 1e-3)
    out = pinned_out(n, k)
    for o in out:
        o.fill_(-7)
    t.knn_cov_host(torch.from_numpy(q).pin_memory(), k, 1e-3, out=out)
    assert_same(out, ref)


def test_pinned_outputs_with_pageable_queries(box):
    p, t = box
    q = np.ascontiguousarray(p[::5][:1500] * np.float32(1.01))
    ref = device_ref(t, q, 20, 1e-3)
    out = pinned_out(len(q), 20)
    t.knn_cov_host(torch.from_numpy(q), 20, 1e-3, out=out)
    assert_same(out, ref)


def test_mixed_pageable_and_pinned_outputs_take_the_copy_path(box):
    p, t = box
    q = np.ascontiguousarray(p[3::9][:700])
    ref = device_ref(t, q, 12, 1e-3)
    out = (torch.empty((len(q), 12), dtype=torch.int32).pin_memory(), torch.empty((len(q), 12)),
           torch.empty((len(q), 6)).pin_memory())
    t.knn_cov_host(torch.from_numpy(q), 12, 1e-3, out=out)
    assert_same(out, ref)


def test_pinned_path_far_queries_on_the_warp_path(box):
    p, t = box
    q = np.array([[1e4, 0, 0], [-3e3, 5e3, 2], [20, 20, 1e5], [20, 20, 2]] * 9, np.float32)
    ref = device_ref(t, q, 9, 1e-3)
    out = pinned_out(len(q), 9)
    t.knn_cov_host(torch.from_numpy(q).pin_memory(), 9, 1e-3, out=out)
    assert_same(out, ref)
    ri, rd = oracle.knn_brute(q, p, 9)
    np.testing.assert_array_equal(out[0].numpy(), ri)


def test_pinned_path_nonfinite_rows(box, gpu_lib):
    p, t = box
    q = np.ascontiguousarray(p[:64].copy())
    q[5] = [np.nan, 0, 0]
    q[40] = [0, np.inf, 0]
    ref = device_ref(t, q, 8, 1e-3)
    assert ref[3] == gpu_lib.PC_ERR_NONFINITE
    out = pinned_out(len(q), 8)
    with pytest.raises(gpu_lib.PcError) as e:
        t.knn_cov_host(torch.from_numpy(q).pin_memory(), 8, 1e-3, out=out)
    assert e.value.code == gpu_lib.PC_ERR_NONFINITE
    assert_same(out, ref)
    assert (out[0].numpy()[[5, 40]] == -1).all() and np.isnan(out[2].numpy()[[5, 40]]).all()


def test_pinned_path_under_a_window(gpu_lib):
    p = W.uniform_box(20000, seed=3)
    t = gpu_lib.Target(torch.from_numpy(p).cuda())
    try:
        t.set_window((5.0, 5.0, -1.0), (30.0, 25.0, 5.0))
        q = np.ascontiguousarray(p[::13] + np.float32(0.02))
        ref = device_ref(t, q, 16, 1e-3)
        out = pinned_out(len(q), 16)
        t.knn_cov_host(torch.from_numpy(q).pin_memory(), 16, 1e-3, out=out)
        assert_same(out, ref)
    finally:
        t.close()


def test_appended_target_takes_the_copy_path(gpu_lib):
    p = W.uniform_box(12000, seed=4)
    t = gpu_lib.Target(torch.from_numpy(p[:10000]).cuda())
    try:
        t.append(torch.from_numpy(p[10000:]).cuda())
        q = np.ascontiguousarray(p[::17] + np.float32(0.01))
        ref = device_ref(t, q, 20, 1e-3)
        out = pinned_out(len(q), 20)
        t.knn_cov_host(torch.from_numpy(q).pin_memory(), 20, 1e-3, out=out)
        assert_same(out, ref)
    finally:
        t.close()


def test_scan_vs_map_pinned_equals_device(gpu_lib):
    q, m = W.scan_vs_map()
    t = gpu_lib.Target(torch.from_numpy(m).cuda())
    try:
        ref = device_ref(t, q, 20, 1e-3)
        out = pinned_out(len(q), 20)
        for _ in range(2):
            t.knn_cov_host(torch.from_numpy(q).pin_memory(), 20, 1e-3, out=out)
            assert_same(out, ref)
    finally:
        t.close()
