"""Windowed searches (pc_set_window, the sliding-window submap) against the
oracle's search over the same submap.

idx and d2 must match bit for bit (indices into the whole map, ties to the
lower index); covariances within the relative bar of tests/helpers.py.
Cases: a box around a scan pose on the track map (lane and warp paths), a
window edge cutting through the queries, the infinite window (identical to
no window), a window with fewer than k points, one that misses the map,
clearing, the batched form and GICP pairing restricted to the window.
"""
import numpy as np
import pytest

import oracle
from paper_2308_07173_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

INF = float("inf")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def scene(gpu_lib):
    tr = W.oval_1500()
    mp = tr.sample_map(300_000, 2)
    g = W.rng_for(3)
    scan = tr.raycast(*tr.random_pose(g), g)
    q = scan[np.sort(g.choice(len(scan), 20_000, replace=False))]
    c = np.median(scan, axis=0)
    t = gpu_lib.Target(dev(mp))
    yield {"map": mp, "q": q, "c": c, "t": t}
    t.close()


def run(t, q, k, eps=1e-3):
    idx, d2, cov = t.knn_cov(dev(q), k, eps)
    st = t.sync_status()
    return host(idx), host(d2), host(cov), st


@pytest.mark.parametrize("k", [10, 20, 32, 40])
def test_box_around_pose(scene, gpu_lib, k):
    s = scene
    lo = [s["c"][0] - 40.0, s["c"][1] - 40.0, -INF]
    hi = [s["c"][0] + 40.0, s["c"][1] + 40.0, INF]
    s["t"].set_window(lo, hi)
    try:
        idx, d2, cov, st = run(s["t"], s["q"], k)
    finally:
        s["t"].set_window()
    assert st == gpu_lib.PC_OK
    wi, wd = oracle.knn_window(s["q"], s["map"], k, lo, hi)
    np.testing.assert_array_equal(idx, wi)
    np.testing.assert_array_equal(d2.view(np.uint32), wd.view(np.uint32))
    raw_gpu = host(s["t"].cov(dev(idx), -1.0))
    H.check_regularised_cov(cov, oracle.cov(s["map"], wi, 1e-3), oracle.cov(s["map"], wi, -1.0), raw_gpu, 1e-3)


def test_edge_through_the_queries(scene, gpu_lib):
    s = scene
    # the window's x edge at the median query: half the queries sit outside
    xm = float(np.median(s["q"][:, 0]))
    lo, hi = [-INF, -INF, -INF], [xm, INF, INF]
    s["t"].set_window(lo, hi)
    idx, d2, cov, st = run(s["t"], s["q"], 20)
    s["t"].set_window()
    assert st == gpu_lib.PC_OK
    wi, wd = oracle.knn_window(s["q"], s["map"], 20, lo, hi)
    np.testing.assert_array_equal(idx, wi)
    np.testing.assert_array_equal(d2.view(np.uint32), wd.view(np.uint32))
    assert (s["map"][idx.ravel(), 0] <= np.float32(xm)).all()


def test_infinite_window_and_clear_are_identical(scene, gpu_lib):
    s = scene
    a = run(s["t"], s["q"], 20)
    s["t"].set_window([-INF] * 3, [INF] * 3)
    b = run(s["t"], s["q"], 20)
    s["t"].set_window()
    c = run(s["t"], s["q"], 20)
    for x, y in ((a, b), (a, c)):
        for u, v in zip(x[:3], y[:3]):
            assert u.tobytes() == v.tobytes()


def test_short_and_missing_windows(scene, gpu_lib):
    s = scene
    q = s["q"][:300]
    # a window with 5 map points, k = 10 (lane queries fall back to the warp
    # search, whose exhaustive scan finds too few)
    p = s["map"]
    box_lo = p[0] - 0.05
    box_hi = p[0] + 0.05
    n_in = int(oracle.window_mask(p, box_lo, box_hi).sum())
    assert n_in < 10
    for lo, hi in ((box_lo, box_hi), ([1e5, 1e5, 1e5], [1e5 + 1, 1e5 + 1, 1e5 + 1])):
        s["t"].set_window(lo, hi)
        idx, d2, cov, st = run(s["t"], q, 10)
        s["t"].set_window()
        assert st == gpu_lib.PC_ERR_K_GT_M
        assert (idx == -1).all() and np.isinf(d2).all() and np.isnan(cov).all()


def test_window_with_exactly_k_points(gpu_lib):
    g = np.random.default_rng(3)
    mp = (g.random((20_000, 3)) * [40, 40, 3]).astype(np.float32)
    lo, hi = [10.0, 10.0, 0.0], [11.5, 11.0, 3.0]
    n_in = int(oracle.window_mask(mp, lo, hi).sum())
    q = np.vstack([mp[:200], [[10.5, 10.5, 1.0], [30, 30, 1]]]).astype(np.float32)
    t = gpu_lib.Target(dev(mp))
    t.set_window(lo, hi)
    idx, d2, cov, st = run(t, q, n_in)
    assert st == gpu_lib.PC_OK
    wi, wd = oracle.knn_window(q, mp, n_in, lo, hi)
    np.testing.assert_array_equal(idx, wi)
    t.close()


def test_batched_form_keeps_the_window(scene, gpu_lib):
    s = scene
    lo = [s["c"][0] - 30.0, s["c"][1] - 30.0, -INF]
    hi = [s["c"][0] + 30.0, s["c"][1] + 30.0, INF]
    s["t"].set_window(lo, hi)
    parts = [s["q"][:9000], s["q"][9000:]]
    outs = []
    for x in parts:
        outs.append((dev(x), torch.empty((len(x), 20), dtype=torch.int32, device="cuda"),
                     torch.empty((len(x), 20), dtype=torch.float32, device="cuda"),
                     torch.empty((len(x), 6), dtype=torch.float32, device="cuda")))
    b = gpu_lib.Batch(s["t"], outs, 20, 1e-3)
    s["t"].set_window()
    b.run()  # the plan keeps the window set when it was planned
    st = s["t"].sync_status()
    assert st == gpu_lib.PC_OK
    for x, o in zip(parts, outs):
        wi, wd = oracle.knn_window(x, s["map"], 20, lo, hi)
        np.testing.assert_array_equal(host(o[1]), wi)
    b.close()


def test_gicp_pairs_only_inside_the_window(scene, gpu_lib):
    s = scene
    rng = np.random.default_rng(4)
    iso = np.array([1, 0, 0, 1, 0, 1], np.float32)
    mcov = (iso[None] * rng.uniform(0.5, 2, (len(s["map"]), 1))).astype(np.float32)
    scov = (iso[None] * rng.uniform(0.5, 2, (len(s["q"]), 1))).astype(np.float32)
    pose = np.concatenate([np.eye(3).ravel(), [0.05, -0.02, 0.01]]).astype(np.float32)
    lo = [s["c"][0] - 25.0, s["c"][1] - 25.0, -INF]
    hi = [s["c"][0] + 25.0, s["c"][1] + 25.0, INF]
    sel = np.nonzero(oracle.window_mask(s["map"], lo, hi))[0]
    tree = oracle.KDTree(s["map"][sel])
    want = oracle.gicp_linearize(tree, mcov[sel], s["q"], scov, pose, 1.0)
    wcorr = np.where(want["corr"] >= 0, sel[np.maximum(want["corr"], 0)], -1)
    s["t"].set_window(lo, hi)
    c = torch.empty(len(s["q"]), dtype=torch.int32, device="cuda")
    out, _ = s["t"].gicp_linearize(dev(mcov), dev(s["q"]), dev(scov), dev(pose), 1.0, corr=c)
    st = s["t"].sync_status()
    s["t"].set_window()
    assert st == gpu_lib.PC_OK
    np.testing.assert_array_equal(host(c), wcorr)
    v = host(out)
    Hm = np.zeros((6, 6))
    Hm[np.triu_indices(6)] = v[:21]
    got = {"H": Hm + np.triu(Hm, 1).T, "b": v[21:27], "error": float(v[27]), "pairs": int(v[28])}
    H.check_gicp(got, want, 64 * H.U32)
    assert 0 < want["pairs"] < len(s["q"])


def test_window_arguments(scene, gpu_lib):
    pc = gpu_lib
    t = scene["t"]
    assert pc.pc_set_window(t.handle, [0, 0, 1], [1, 1, 0]) == pc.PC_ERR_INVALID_ARG
    assert pc.pc_set_window(t.handle, [0, float("nan"), 0], [1, 1, 1]) == pc.PC_ERR_INVALID_ARG
    assert pc.pc_set_window(t.handle, None) == pc.PC_OK
