"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

idx and d2 must match bit for bit (d2 in the pinned fmaf order, ties to the
lower index); covariances within the relative Frobenius bar of
tests/helpers.py against the binary64 oracle.  Sizes span many warp tiles
and ragged tails; edge cases cover empty and tiny inputs, k = M, exact
ties, duplicates, far queries (exact exhaustive scan), non-finite input and
the search-limit status.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2308_07173_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def run_knn_cov(pc, target, q, k, eps):
    idx, d2, cov = target.knn_cov(dev(q), k, eps)
    st = target.sync_status()
    return host(idx), host(d2), host(cov), st


# ---------------------------------------------------------------- C1
@pytest.fixture(scope="module")
def c1(gpu_lib):
    p = W.uniform_box(8192, seed=1)
    t = gpu_lib.Target(dev(p))
    yield p, t
    t.close()


@pytest.fixture(scope="module")
def c1_oracle():
    p = W.uniform_box(8192, seed=1)
    idx, d2 = oracle.knn_brute(p, p, 10)
    return idx, d2


def test_c1_self_knn_bit_exact(c1, c1_oracle, gpu_lib):
    p, t = c1
    idx, d2, cov, st = run_knn_cov(gpu_lib, t, p, 10, 1e-3)
    assert st == gpu_lib.PC_OK
    np.testing.assert_array_equal(idx, c1_oracle[0])
    np.testing.assert_array_equal(d2.view(np.uint32), c1_oracle[1].view(np.uint32))
    # every query finds itself first (query set == target set)
    assert (idx[:, 0] == np.arange(len(p))).all()


def test_c1_cov_regularised_and_raw(c1, c1_oracle, gpu_lib):
    p, t = c1
    ref_idx = c1_oracle[0]
    _, _, cov_reg, _ = run_knn_cov(gpu_lib, t, p, 10, 1e-3)
    raw = host(t.cov(dev(ref_idx), -1.0))
    raw64 = oracle.cov(p, ref_idx, -1.0)
    reg64 = oracle.cov(p, ref_idx, 1e-3)
    H.check_raw_cov(raw, raw64)
    H.check_regularised_cov(cov_reg, reg64, raw64, raw, 1e-3, label="C1")


def test_fused_equals_separate_calls(c1, gpu_lib):
    p, t = c1
    q = dev(p[::3])
    i1, d1, c1_ = t.knn_cov(q, 10, 1e-3)
    i2, d2_ = t.knn(q, 10)
    c2 = t.cov(i2, 1e-3)
    c3 = t.cov(i1, -1.0)
    i4, d4, c4 = t.knn_cov(q, 10, -1.0)
    torch.cuda.synchronize()
    assert torch.equal(i1, i2) and torch.equal(d1.view(torch.int32), d2_.view(torch.int32))
    assert torch.equal(c1_.view(torch.int32), c2.view(torch.int32))
    assert torch.equal(c3.view(torch.int32), c4.view(torch.int32))
    assert torch.equal(i1, i4)


@pytest.mark.parametrize("n", [1, 31, 33, 1000])
@pytest.mark.parametrize("k", [1, 7, 24, 25, 32, 33, 64])
def test_ragged_sizes_and_k(c1, gpu_lib, n, k):
    p, t = c1
    g = np.random.default_rng(n * 100 + k)
    q = (g.random((n, 3)) * [44, 44, 6] - [2, 2, 1]).astype(np.float32)
    idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, k, -1.0)
    assert st == gpu_lib.PC_OK
    ri, rd = oracle.knn_brute(q, p, k)
    np.testing.assert_array_equal(idx, ri)
    np.testing.assert_array_equal(d2.view(np.uint32), rd.view(np.uint32))
    H.check_raw_cov(cov, oracle.cov(p, ri, -1.0))


def test_stats_count_every_query(c1, gpu_lib):
    p, t = c1
    t.stats(reset=True)
    t.knn_cov(dev(p[:1000]), 10, 1e-3)
    t.knn(dev(p[:77]), 40)
    st = t.stats(reset=True)
    assert st["queries"] == 1077
    assert 77 <= st["warp_search"] <= 1077  # k > 32 always takes the warp search
    assert t.stats()["queries"] == 0


def test_empty_query_is_noop(c1, gpu_lib):
    _, t = c1
    q = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    idx, d2, cov = t.knn_cov(q, 5, 1e-3)
    assert idx.shape == (0, 5)
    assert t.sync_status() == gpu_lib.PC_OK


@pytest.mark.parametrize("tune", [(1, 1, 0.5, 0), (7, 3, 3.0, 1), (32, 8, 1.0, 0), (16, 8, 20.0, 1),
                                  (32, 2, 0.2, 0), (32, 4, 0.9, 1)])
def test_launch_shape_never_changes_results(c1, gpu_lib, tune):
    p, t = c1
    q = dev(p[::5])
    ref = [x.clone() for x in t.knn_cov(q, 12, 1e-3)]
    t.set_tune(*tune)
    try:
        out = t.knn_cov(q, 12, 1e-3)
    finally:
        t.set_tune()
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))


@pytest.mark.parametrize("cell", [0.3, 1.0, 2.5, 9.0])
def test_cell_size_never_changes_results(c1, gpu_lib, cell):
    p, t = c1
    q = dev(p[::7])
    ref = [x.clone() for x in t.knn_cov(q, 16, 1e-3)]
    t2 = gpu_lib.Target(dev(p), cell_size=cell)
    out = t2.knn_cov(q, 16, 1e-3)
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    t2.close()


# ---------------------------------------------------------------- edge cases
def test_lattice_exact_ties(gpu_lib):
    g = np.stack(np.meshgrid(np.arange(12), np.arange(10), np.arange(5), indexing="ij"), -1)
    p = (g.reshape(-1, 3) * 0.5).astype(np.float32)
    p = p[np.random.default_rng(1).permutation(len(p))]
    q = np.concatenate([p[::5], p[::9] + np.float32(0.25), p[::13] + np.float32([0.25, 0, 0])])
    t = gpu_lib.Target(dev(p), cell_size=0.5)  # cell faces through lattice points
    for k in (6, 19, 27, 64):
        idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, k, -1.0)
        ri, rd = oracle.knn_brute(q, p, k)
        np.testing.assert_array_equal(idx, ri)
        np.testing.assert_array_equal(d2, rd)
    t.close()


@pytest.mark.parametrize("cell", [1.0, 0.8, 2.0])
def test_points_and_queries_on_sub_cell_boundaries(gpu_lib, cell):
    """The row walks skip the eighths of their end cells beyond a query's
    chord.  A lattice of spacing cell / 8 puts points exactly on those
    boundaries (and on the cell faces), queries sit on lattice points,
    midpoints and chord-length offsets, and the answers must still equal
    brute force bit for bit, ties to the lower index."""
    s = cell / 8.0
    g = np.stack(np.meshgrid(np.arange(40), np.arange(9), np.arange(3), indexing="ij"), -1)
    p = (g.reshape(-1, 3) * s).astype(np.float32)
    p = p[np.random.default_rng(7).permutation(len(p))]
    rng = np.random.default_rng(8)
    q = np.concatenate([p[::7], p[::11] + np.float32([s / 2, 0, 0]), p[::13] + np.float32([s / 2, s / 2, 0]),
                        p[::17] + rng.integers(-3, 4, (len(p[::17]), 3)).astype(np.float32) * np.float32(s / 4)])
    t = gpu_lib.Target(dev(p), cell_size=cell)
    for k in (5, 20, 32):
        idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, k, -1.0)
        assert st == gpu_lib.PC_OK
        ri, rd = oracle.knn_brute(q, p, k)
        np.testing.assert_array_equal(idx, ri)
        np.testing.assert_array_equal(d2.view(np.uint32), rd.view(np.uint32))
    t.close()


def test_duplicates_tie_break_by_index(gpu_lib):
    base = np.random.default_rng(3).random((50, 3)).astype(np.float32)
    p = base[np.random.default_rng(4).integers(0, 50, 3000)]
    t = gpu_lib.Target(dev(p))
    idx, d2, cov, st = run_knn_cov(gpu_lib, t, base, 40, 1e-3)
    ri, rd = oracle.knn_brute(base, p, 40)
    np.testing.assert_array_equal(idx, ri)
    np.testing.assert_array_equal(d2, rd)
    # an all-duplicate neighbourhood has C = 0 and C' = diag(1, 1, eps)
    one = np.repeat(base[:1], 5, 0)
    t1 = gpu_lib.Target(dev(one))
    _, _, c, _ = run_knn_cov(gpu_lib, t1, base[:1], 5, 0.25)
    np.testing.assert_array_equal(c[0], np.float32([1, 0, 0, 1, 0, 0.25]))
    t.close()
    t1.close()


def test_k_equals_m_and_single_point_target(gpu_lib):
    p = np.random.default_rng(5).random((23, 3)).astype(np.float32)
    t = gpu_lib.Target(dev(p))
    q = np.random.default_rng(6).random((40, 3)).astype(np.float32) * 3
    idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, 23, -1.0)
    ri, rd = oracle.knn_brute(q, p, 23)
    np.testing.assert_array_equal(idx, ri)
    np.testing.assert_array_equal(d2, rd)
    t.close()
    t1 = gpu_lib.Target(dev(p[:1]))
    idx, d2, _, _ = run_knn_cov(gpu_lib, t1, q, 1, -1.0)
    assert (idx == 0).all()
    t1.close()


def test_k_greater_than_m_is_rejected(gpu_lib):
    p = np.zeros((4, 3), np.float32)
    t = gpu_lib.Target(dev(p))
    with pytest.raises(gpu_lib.PcError) as e:
        t.knn(dev(p), 5)
    assert e.value.code == gpu_lib.PC_ERR_K_GT_M
    with pytest.raises(gpu_lib.PcError) as e:
        t.knn(dev(p), 65)
    assert e.value.code == gpu_lib.PC_ERR_INVALID_ARG
    t.close()


def test_far_queries_take_the_exact_exhaustive_scan(c1, gpu_lib):
    p, t = c1
    q = np.array([[1e4, 0, 0], [-3e3, 5e3, 2], [20, 20, 1e5], [20, 20, 2]], np.float32)
    idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, 9, 1e-3)
    assert st == gpu_lib.PC_OK
    ri, rd = oracle.knn_brute(q, p, 9)
    np.testing.assert_array_equal(idx, ri)
    np.testing.assert_array_equal(d2, rd)


def test_search_limit_sets_status_without_trapping(gpu_lib):
    p = W.uniform_box(2000, seed=9)
    t = gpu_lib.Target(dev(p), max_box_cells=8, exhaustive=False)
    q = np.array([[20, 20, 2], [5e3, 0, 0]], np.float32)
    idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, 5, 1e-3)
    assert st == gpu_lib.PC_ERR_SEARCH_LIMIT
    assert (idx[1] == -1).all() and np.isinf(d2[1]).all() and np.isnan(cov[1]).all()
    assert t.sync_status() == gpu_lib.PC_OK  # read-and-clear
    t.close()


def test_nonfinite_query_marks_row(c1, gpu_lib):
    p, t = c1
    q = np.array([[1, 2, 3], [np.nan, 0, 0], [0, np.inf, 0], [4, 5, 1]], np.float32)
    idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, 4, 1e-3)
    assert st == gpu_lib.PC_ERR_NONFINITE
    assert (idx[1:3] == -1).all() and np.isinf(d2[1:3]).all() and np.isnan(cov[1:3]).all()
    ri, rd = oracle.knn_brute(q[[0, 3]], p, 4)
    np.testing.assert_array_equal(idx[[0, 3]], ri)


def test_nonfinite_target_is_rejected(gpu_lib):
    p = W.uniform_box(100, seed=2)
    p[17, 1] = np.nan
    with pytest.raises(gpu_lib.PcError) as e:
        gpu_lib.Target(dev(p))
    assert e.value.code == gpu_lib.PC_ERR_NONFINITE


def test_host_pointer_where_device_required(c1, gpu_lib):
    _, t = c1
    q = np.zeros((4, 3), np.float32)
    idx = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    d2 = torch.empty((4, 3), dtype=torch.float32, device="cuda")
    rc = gpu_lib.pc_knn(t.handle, q.ctypes.data, 4, 3, idx.data_ptr(), d2.data_ptr(), 0)
    assert rc == gpu_lib.PC_ERR_BAD_POINTER


def test_cov_rejects_out_of_range_index(c1, gpu_lib):
    p, t = c1
    bad = torch.tensor([[0, 1, 2], [0, len(p), 1], [-5, 0, 0]], dtype=torch.int32, device="cuda")
    c = host(t.cov(bad, -1.0))
    assert t.sync_status() == gpu_lib.PC_ERR_BAD_INDEX
    assert np.isfinite(c[0]).all() and np.isnan(c[1:]).all()


def test_destroyed_handle(gpu_lib):
    t = gpu_lib.Target(dev(W.uniform_box(64, seed=3)))
    h = t.handle
    t.close()
    assert gpu_lib.pc_sync_status(h, 0) == gpu_lib.PC_ERR_DESTROYED


def test_host_buffer_entry_matches_device_entry(c1, gpu_lib):
    p, t = c1
    q = p[::11].copy()
    ih, dh, ch = t.knn_cov_host(q, 10, 1e-3)
    idv, ddv, cdv = t.knn_cov(dev(q), 10, 1e-3)
    np.testing.assert_array_equal(ih, host(idv))
    np.testing.assert_array_equal(dh.view(np.uint32), host(ddv).view(np.uint32))
    np.testing.assert_array_equal(ch.view(np.uint32), host(cdv).view(np.uint32))


# ---------------------------------------------------------------- C2 full size
@pytest.fixture(scope="module")
def c2(gpu_lib):
    from paper_2308_07173_gb300 import autotune

    q, m = W.scan_vs_map()
    # the configuration the benchmark runs: the cached tuned one if any
    tuned = autotune.lookup(autotune.default_cache(), 20, len(m), len(q))
    t = autotune.apply(dev(m), tuned) if tuned else gpu_lib.Target(dev(m))
    tree = oracle.KDTree(m)
    yield q, m, t, tree
    t.close()


def test_c2_full_size_parity_every_row(c2, gpu_lib):
    """The headline workload (131k-point scan, 2M-point map, k = 20) in the
    launch configuration the benchmark times: every row against the oracle's
    k-d tree -- idx and d2 bit-exact, raw and regularised covariances within
    the per-band bar."""
    q, m, t, tree = c2
    k, eps = 20, 1e-3
    idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, k, eps)
    assert st == gpu_lib.PC_OK
    ri, rd = tree.knn(q, k)
    np.testing.assert_array_equal(idx, ri)
    np.testing.assert_array_equal(d2.view(np.uint32), rd.view(np.uint32))
    raw64 = oracle.cov(m, ri, -1.0)
    reg64 = oracle.cov(m, ri, eps)
    raw = host(t.cov(dev(ri), -1.0))
    H.check_raw_cov(raw, raw64)
    bands = H.check_regularised_cov(cov, reg64, raw64, raw, eps, label="C2")
    assert bands["well"]["rows"] + bands["mid"]["rows"] + bands["degenerate"]["rows"] == len(q)


def test_c2_batch_equals_single_scans(c2, gpu_lib):
    q, m, t, tree = c2
    scans = W.scan_batch(6, lo=2000, hi=40000, seed=44)
    k, eps = 20, 1e-3
    bufs = []
    for s in scans:
        n = len(s)
        bufs.append((dev(s), torch.empty((n, k), dtype=torch.int32, device="cuda"),
                     torch.empty((n, k), dtype=torch.float32, device="cuda"),
                     torch.empty((n, 6), dtype=torch.float32, device="cuda")))
    b = gpu_lib.Batch(t, bufs, k, eps)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.run(stream)
        b.run(stream)  # graph replay
    stream.synchronize()
    for (qd, bi, bd, bc), s in zip(bufs, scans):
        i1, d1, c1_ = t.knn_cov(qd, k, eps)
        torch.cuda.synchronize()
        assert torch.equal(bi, i1)
        assert torch.equal(bd.view(torch.int32), d1.view(torch.int32))
        assert torch.equal(bc.view(torch.int32), c1_.view(torch.int32))
    ri, rd = tree.knn(scans[0][:500], k)
    np.testing.assert_array_equal(host(bufs[0][1])[:500], ri)
    assert t.sync_status() == gpu_lib.PC_OK
    b.close()


# ---------------------------------------------------------------- uneven occupancy
@pytest.fixture(scope="module")
def pit_world(gpu_lib):
    tr = W.oval_4000_pit()
    m = tr.sample_map(400_000, seed=61, noise=0.01)
    g = W.rng_for(62)
    q = tr.raycast(*tr.random_pose(g), g)[::16].copy()
    t = gpu_lib.Target(dev(m))
    tree = oracle.KDTree(m)
    yield q, m, t, tree
    t.close()


@pytest.mark.parametrize("k", [10, 20, 32])
def test_uneven_occupancy_map_parity(pit_world, gpu_lib, k):
    q, m, t, tree = pit_world
    idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, k, 1e-3)
    assert st == gpu_lib.PC_OK
    ri, rd = tree.knn(q, k)
    np.testing.assert_array_equal(idx, ri)
    np.testing.assert_array_equal(d2.view(np.uint32), rd.view(np.uint32))
    raw = host(t.cov(dev(ri), -1.0))
    H.check_raw_cov(raw, oracle.cov(m, ri, -1.0))
    H.check_regularised_cov(cov, oracle.cov(m, ri, 1e-3), oracle.cov(m, ri, -1.0), raw, 1e-3, label=f"pit k={k}")


def test_retries_and_fallbacks_stay_exact(gpu_lib):
    # a dense clump (too many points inside the smallest trial radius), a
    # sparse surface, and queries well off the surface (too few inside the
    # largest): the lane path must narrow, widen or hand over, never err
    rng = np.random.default_rng(71)
    plane = np.c_[rng.uniform(0, 30, (20000, 2)), np.zeros(20000)]
    clump = rng.normal([15, 15, 0], 0.002, (3000, 3))
    p = np.concatenate([plane, clump]).astype(np.float32)
    q = np.concatenate([
        np.c_[rng.uniform(1, 29, (300, 2)), rng.normal(0, 0.01, 300)],     # on the plane
        rng.normal([15, 15, 0], 0.003, (200, 3)),                          # inside the clump
        np.c_[rng.uniform(1, 29, (200, 2)), rng.uniform(0.5, 3.0, 200)],   # above the plane
    ]).astype(np.float32)
    t = gpu_lib.Target(dev(p))
    for k in (8, 20, 32):
        t.stats(reset=True)
        idx, d2, cov, st = run_knn_cov(gpu_lib, t, q, k, -1.0)
        assert st == gpu_lib.PC_OK
        ri, rd = oracle.knn_brute(q, p, k)
        np.testing.assert_array_equal(idx, ri)
        np.testing.assert_array_equal(d2.view(np.uint32), rd.view(np.uint32))
        H.check_raw_cov(cov, oracle.cov(p, ri, -1.0))
        assert t.stats()["queries"] == len(q)
    t.close()
