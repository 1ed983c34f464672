"""Wall detection (pc_wall_*, Sec. III-D) on the GPU against the oracle.

Voxel centroids, vertical flags, cluster labels, the wall's label, size and
length must match bit for bit (the steps are integer decisions on binary32
values both sides compute the same way, and binary64 centroid sums in the
same order); the quadratic fit within 1e-6 m along the wall (the normal
equations are summed in a different order).  Scans: the body-frame ray cast
on a straight and on a bend, with ground, both walls and range noise.
"""
import numpy as np
import pytest

import oracle
from paper_2308_07173_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OPTS = dict(voxel=0.2, cell2d=0.2, min_votes=2, tol=0.45, min_cluster=10)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(pc, pts, **opts):
    o = dict(OPTS, **opts)
    w = pc.WallDetector(max(len(pts), 1), **o)
    w.detect(dev(pts.reshape(-1, 3)))
    r = w.result(arrays=True)
    w.close()
    return r


def compare(r, want):
    assert r["status"] == 0
    assert r["n_voxels"] == len(want["centroids"])
    if r["n_voxels"] == 0:
        assert r["wall_label"] == -1
        return
    np.testing.assert_array_equal(r["centroids"].view(np.uint32), want["centroids"].view(np.uint32))
    np.testing.assert_array_equal(r["vertical"], want["vertical"])
    np.testing.assert_array_equal(r["labels"], want["labels"])
    assert r["n_vertical"] == int(want["vertical"].sum())
    assert r["wall_label"] == want["wall_label"]
    assert r["wall_count"] == want["wall_count"]
    if want["wall_label"] >= 0:
        c = want["centroids"][want["labels"] == want["wall_label"]]
        xs = np.linspace(c[:, 0].min(), c[:, 0].max(), 50)
        yg = np.polyval(r["beta"][::-1], xs)
        yo = np.polyval(want["beta"][::-1], xs)
        assert np.abs(yg - yo).max() < 1e-6
        assert r["wall_length"] == np.float32(c[:, 0].max()) - np.float32(c[:, 0].min())
    else:
        assert np.isnan(r["beta"]).all()


@pytest.mark.parametrize("s0", [130.0, 600.0])
def test_body_frame_scan_matches_oracle(gpu_lib, s0):
    pts = W.body_frame_scan(s0=s0, w0=2.0, seed=int(s0))
    want = oracle.wall_detect(pts, **OPTS)
    r = run(gpu_lib, pts)
    compare(r, want)
    assert want["wall_label"] >= 0 and want["wall_count"] > 100
    # the sensor rides 2 m towards the outer wall, which is the right one
    # when driving the lap: 6 - 2 = 4 m to the right
    assert -4.5 < want["d_w"] < -3.5


def test_repeatable(gpu_lib):
    pts = W.body_frame_scan(s0=300.0, seed=4)
    w = gpu_lib.WallDetector(len(pts), **OPTS)
    outs = []
    for _ in range(2):
        w.detect(dev(pts))
        outs.append(w.result(arrays=True))
    w.close()
    for key in ("centroids", "vertical", "labels"):
        assert outs[0][key].tobytes() == outs[1][key].tobytes()
    assert outs[0]["beta"] == outs[1]["beta"]


def test_dropped_points_and_no_wall(gpu_lib):
    g = np.random.default_rng(5)
    ground = np.c_[g.uniform(-20, 20, 4000), g.uniform(-20, 20, 4000), np.zeros(4000)]
    left = np.c_[g.uniform(-20, 20, 3000), np.full(3000, 6.0), g.uniform(0, 1, 3000)]
    junk = np.array([[np.nan, 0, 0], [0, np.inf, 0], [500.0, 0, 0], [0, 0, 40.0]])
    pts = np.vstack([ground, left, junk]).astype(np.float32)
    want = oracle.wall_detect(pts, **OPTS)
    r = run(gpu_lib, pts)
    compare(r, want)
    assert want["wall_label"] == -1


def test_empty_and_tiny(gpu_lib):
    compare(run(gpu_lib, np.zeros((0, 3), np.float32)), oracle.wall_detect(np.zeros((0, 3), np.float32), **OPTS))
    one = np.array([[1.0, -2.0, 0.5]], np.float32)
    compare(run(gpu_lib, one), oracle.wall_detect(one, **OPTS))


def test_bad_arguments(gpu_lib):
    pc = gpu_lib
    import ctypes
    w = pc.WallDetector(100, **OPTS)
    big = dev(np.zeros((101, 3), np.float32))
    assert pc.load().pc_wall_detect(w._h, big.data_ptr(), 101, pc._stream_handle()) == pc.PC_ERR_INVALID_ARG
    hostbuf = np.zeros((10, 3), np.float32)
    assert pc.load().pc_wall_detect(w._h, hostbuf.ctypes.data, 10, pc._stream_handle()) == pc.PC_ERR_BAD_POINTER
    w.close()
    o = pc.pc_wall_opts()
    pc.load().pc_wall_default_opts(ctypes.byref(o))
    o.voxel = -1.0
    h = ctypes.c_void_p()
    assert pc.load().pc_wall_create(100, ctypes.byref(o), ctypes.byref(h)) == pc.PC_ERR_INVALID_ARG
