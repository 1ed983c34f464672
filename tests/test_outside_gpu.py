"""Queries outside the map's bounding box, or outside a window, along one
axis only, the other two coordinates inside: the lane search's cell box,
clamped to the grid (or to the window), is then empty along that axis
while the other two ranges are not.  The answer must still be the exact k
nearest points of the map (of the window), bit for bit against the oracle,
at offsets from half a cell to far beyond the first trial radius, on both
sides of each axis, for the lane path (k <= 24 and k <= 32) and the warp
path (k > 32), over a map built whole and over one grown by appended
points."""
import numpy as np
import pytest

import oracle
from paper_2308_07173_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

INF = float("inf")
OFFSETS = (0.3, 1.0, 2.5, 6.0, 25.0, 300.0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def beyond(lo, hi, inner_lo, inner_hi, per, seed):
    """Queries outside [lo, hi] along one axis at each offset (both sides of
    every axis), the other coordinates uniform in [inner_lo, inner_hi]."""
    g = W.rng_for(seed)
    out = []
    for a in range(3):
        for side in (-1.0, 1.0):
            for off in OFFSETS:
                q = inner_lo + g.random((per, 3)) * (inner_hi - inner_lo)
                q[:, a] = (hi[a] + off) if side > 0 else (lo[a] - off)
                out.append(q)
    return np.concatenate(out).astype(np.float32)


@pytest.fixture(scope="module", params=["box", "plane"])
def scene(request, gpu_lib):
    if request.param == "box":  # 3-D: 20k points uniform in 40 x 40 x 4 m
        mp = W.uniform_box(20_000, seed=21)
    else:  # a ground plane, 20k points on z = 0 over 40 x 40 m
        mp = W.uniform_box(20_000, seed=22)
        mp[:, 2] = 0.0
    lo, hi = mp.min(axis=0), mp.max(axis=0)
    q = beyond(lo, hi, lo + 0.1 * (hi - lo), hi - 0.1 * (hi - lo), 16, 23)
    t = gpu_lib.Target(dev(mp))
    yield {"map": mp, "q": q, "t": t}
    t.close()


@pytest.mark.parametrize("k", [10, 20, 32, 40])
def test_beyond_the_map_on_one_axis(scene, gpu_lib, k):
    s = scene
    idx, d2, cov = s["t"].knn_cov(dev(s["q"]), k, 1e-3)
    st = s["t"].sync_status()
    assert st == gpu_lib.PC_OK
    wi, wd = oracle.knn_brute(s["q"], s["map"], k)
    np.testing.assert_array_equal(host(idx), wi)
    np.testing.assert_array_equal(host(d2).view(np.uint32), wd.view(np.uint32))
    assert np.isfinite(host(cov)).all()


@pytest.mark.parametrize("k", [10, 20, 32, 40])
def test_beyond_a_window_on_one_axis(scene, gpu_lib, k):
    s = scene
    mp = s["map"]
    lo_m, hi_m = mp.min(axis=0), mp.max(axis=0)
    span = hi_m - lo_m
    # a window over the middle of the map in x and y, open in z
    lo = [float(lo_m[0] + 0.3 * span[0]), float(lo_m[1] + 0.3 * span[1]), -INF]
    hi = [float(hi_m[0] - 0.3 * span[0]), float(hi_m[1] - 0.3 * span[1]), INF]
    w_lo = np.array([lo[0], lo[1], lo_m[2]], np.float32)
    w_hi = np.array([hi[0], hi[1], hi_m[2]], np.float32)
    # queries inside the map but beyond the window along x or y (offsets
    # that stay inside the map), the other coordinates inside the window
    g = W.rng_for(24)
    qs = []
    for a in range(2):
        for side in (-1.0, 1.0):
            for off in (0.3, 1.0, 2.5, 6.0):
                q = w_lo + 0.1 * (w_hi - w_lo) + g.random((16, 3)) * 0.8 * (w_hi - w_lo)
                q[:, a] = (w_hi[a] + off) if side > 0 else (w_lo[a] - off)
                qs.append(q)
    q = np.concatenate(qs).astype(np.float32)
    s["t"].set_window(lo, hi)
    try:
        idx, d2, cov = s["t"].knn_cov(dev(q), k, 1e-3)
        st = s["t"].sync_status()
    finally:
        s["t"].set_window()
    assert st == gpu_lib.PC_OK
    wi, wd = oracle.knn_window(q, mp, k, lo, hi)
    np.testing.assert_array_equal(host(idx), wi)
    np.testing.assert_array_equal(host(d2).view(np.uint32), wd.view(np.uint32))
    inside = oracle.window_mask(mp, lo, hi)
    assert inside[host(idx).ravel()].all()


@pytest.mark.parametrize("k", [10, 20, 32, 40])
def test_beyond_a_grown_map_on_one_axis(scene, gpu_lib, k):
    # half the map in the main grid, half appended: each grid's clamped box
    # can be empty on its own, and the appended half has its own extent
    s = scene
    mp = s["map"]
    half = len(mp) // 2
    order = np.argsort(mp[:, 0], kind="stable")  # main: the low-x half
    grown = np.ascontiguousarray(mp[order])
    t = gpu_lib.Target(dev(grown[:half]))
    t.append(dev(grown[half:]))
    try:
        idx, d2, cov = t.knn_cov(dev(s["q"]), k, 1e-3)
        st = t.sync_status()
        idx, d2, cov = host(idx), host(d2), host(cov)
    finally:
        t.close()
    assert st == gpu_lib.PC_OK
    wi, wd = oracle.knn_brute(s["q"], grown, k)
    np.testing.assert_array_equal(idx, wi)
    np.testing.assert_array_equal(d2.view(np.uint32), wd.view(np.uint32))
    assert np.isfinite(cov).all()
