"""Pins for the oracle's ground filter, clustering and wall fit (Sec.
III-D, Eq. 24-30), against facts fixed outside it.

* voxel centroids of hand-placed points equal their exact means (dyadic
  coordinates, so binary64 sums are exact);
* a flat ground lattice and a vertical wall: with the 2-D cell equal to the
  voxel, ground columns hold one voxel and wall columns one per voxel of
  height, so the vote separates them exactly;
* the clustering equals a pure-Python breadth-first search over the same
  link rule (transitive chains join, a gap wider than tol splits);
* the wall is the longest cluster on the right (negative y), a longer left
  wall notwithstanding;
* the fit recovers a parabola the wall points were placed on, and d_w is
  its value at x = 0.
The paper prints no worked example for this step (parity with its numbers
unpinned).
"""
from collections import deque

import numpy as np

import oracle
from tests import exact_f32 as ex


def _wall(x0, x1, y_of_x, height=1.0, step=0.1):
    xs = np.arange(x0, x1, step)
    zs = np.arange(0.05, height, step)
    X, Z = np.meshgrid(xs, zs, indexing="ij")
    return np.c_[X.ravel(), y_of_x(X.ravel()), Z.ravel()]


def _ground(x0, x1, y0, y1, step=0.2):
    xs = np.arange(x0, x1, step) + 0.1
    ys = np.arange(y0, y1, step) + 0.1
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return np.c_[X.ravel(), Y.ravel(), np.full(X.size, 0.05)]


def test_voxel_centroids_are_exact_means():
    # four points in voxel (0,0,0) and two in voxel (1,0,0) of edge 0.25
    p = np.array([[0.0625, 0.125, 0.0], [0.125, 0.0625, 0.125], [0.1875, 0.0, 0.0625], [0.0, 0.1875, 0.1875],
                  [0.3125, 0.0, 0.0], [0.375, 0.125, 0.0]], np.float32)
    r = oracle.wall_detect(p, voxel=0.25, cell2d=0.25, min_votes=0, tol=0.01, min_cluster=1)
    assert len(r["centroids"]) == 2
    np.testing.assert_array_equal(r["centroids"][0], p[:4].astype(np.float64).mean(0).astype(np.float32))
    np.testing.assert_array_equal(r["centroids"][1], p[4:].astype(np.float64).mean(0).astype(np.float32))


def test_vote_separates_ground_and_wall():
    g = _ground(0, 10, -4, 4)
    w = _wall(0, 10, lambda x: np.full_like(x, -4.05), height=1.0)
    p = np.vstack([g, w]).astype(np.float32)
    r = oracle.wall_detect(p, voxel=0.2, cell2d=0.2, min_votes=2, tol=0.45, min_cluster=5)
    c = r["centroids"]
    is_wall = c[:, 1] < -4.0
    np.testing.assert_array_equal(r["vertical"], is_wall)
    assert (r["labels"][~is_wall] == -1).all()


def test_vote_threshold_is_strict():
    # a kerb two voxels high: its columns hold exactly 2 voxels, which is not
    # more than min_votes = 2 but is more than 1
    kerb = _wall(0, 5, lambda x: np.full_like(x, -3.05), height=0.4)
    p = kerb.astype(np.float32)
    r2 = oracle.wall_detect(p, voxel=0.2, cell2d=0.2, min_votes=2, tol=0.45, min_cluster=1)
    r1 = oracle.wall_detect(p, voxel=0.2, cell2d=0.2, min_votes=1, tol=0.45, min_cluster=1)
    assert not r2["vertical"].any()
    assert r1["vertical"].all()


def _bfs_labels(c, vertical, tol):
    n = len(c)
    t2 = np.float32(tol) * np.float32(tol)
    lab = np.full(n, -1, np.int64)
    for s in range(n):
        if not vertical[s] or lab[s] >= 0:
            continue
        comp, dq = [s], deque([s])
        lab[s] = s
        while dq:
            a = dq.popleft()
            for b in range(n):
                if vertical[b] and lab[b] < 0 and ex.d2_pinned(c[a], c[b]) <= t2:
                    lab[b] = s
                    comp.append(b)
                    dq.append(b)
        lab[comp] = min(comp)
    return lab


def test_clustering_matches_breadth_first_search():
    rng = np.random.default_rng(3)
    chain = np.c_[np.arange(0, 6, 0.4), np.full(15, -2.0), np.full(15, 0.5)]  # links of 0.4 < tol
    blob = rng.normal([3, 3, 0.5], 0.2, (40, 3))
    far = np.array([[20, -5, 0.5], [20.3, -5, 0.5]])
    p = np.vstack([chain, blob, far]).astype(np.float32)
    r = oracle.wall_detect(p, voxel=0.1, cell2d=0.1, min_votes=0, tol=0.45, min_cluster=1)
    want = _bfs_labels(r["centroids"], r["vertical"], 0.45)
    np.testing.assert_array_equal(r["labels"], want)
    assert len(set(r["labels"][r["labels"] >= 0])) >= 3


def test_longest_right_cluster_is_the_wall_and_fit_recovers_the_parabola():
    b0, b1, b2 = -3.0, 0.02, 0.004
    right = _wall(-20, 20, lambda x: b0 + b1 * x + b2 * x * x, height=1.2)
    left = _wall(-30, 30, lambda x: np.full_like(x, 5.0), height=1.2)  # longer, but on the left
    shortr = _wall(30, 34, lambda x: np.full_like(x, -3.0), height=1.2)  # right, shorter
    p = np.vstack([right, left, shortr, _ground(-30, 34, -2.5, 4.5)]).astype(np.float32)
    r = oracle.wall_detect(p, voxel=0.2, cell2d=0.2, min_votes=2, tol=0.45, min_cluster=10)
    assert r["wall_label"] >= 0
    c = r["centroids"][r["labels"] == r["wall_label"]]
    assert c[:, 0].min() < -19 and c[:, 0].max() > 19 and (c[:, 1] < 0).all()
    # voxel centroids sit on the curve only up to the voxel averaging of a
    # curved wall that cuts across voxel rows; the exact least-squares check
    # below pins the fit itself
    assert np.all(np.abs(r["beta"] - [b0, b1, b2]) <= [5e-3, 2e-4, 3e-5]), r["beta"]
    assert abs(r["d_w"] - b0) < 5e-3
    # the fit is the least-squares solution over the wall centroids
    X = np.c_[np.ones(len(c)), c[:, 0], c[:, 0].astype(np.float64) ** 2]
    ref = np.linalg.lstsq(X, c[:, 1].astype(np.float64), rcond=None)[0]
    np.testing.assert_allclose(r["beta"], ref, rtol=1e-8, atol=1e-10)


def test_no_wall_on_the_right_and_empty_input():
    left = _wall(-10, 10, lambda x: np.full_like(x, 4.0))
    r = oracle.wall_detect(left.astype(np.float32), voxel=0.2, cell2d=0.2, min_votes=2, tol=0.45, min_cluster=5)
    assert r["wall_label"] == -1 and np.isnan(r["beta"]).all()
    r = oracle.wall_detect(np.zeros((0, 3), np.float32))
    assert len(r["centroids"]) == 0 and r["wall_label"] == -1
