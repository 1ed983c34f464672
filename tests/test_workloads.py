"""The seeded synthetic inputs: reproducible, with the stated geometry."""
import numpy as np

from paper_2308_07173_gb300 import workloads as W


def test_uniform_box_is_seeded_and_bounded():
    a, b = W.uniform_box(1000, seed=1), W.uniform_box(1000, seed=1)
    np.testing.assert_array_equal(a, b)
    assert a.dtype == np.float32 and a.shape == (1000, 3)
    assert (a >= 0).all() and (a <= [40, 40, 4]).all()


def test_track_centreline_length_and_closure():
    tr = W.oval_1500()
    assert abs(2 * tr.ls + 2 * np.pi * tr.r - 1500.0) < 1e-9
    s = np.linspace(0, tr.length, 20001)
    pos, tan, nrm = tr.pose(s)
    step = np.linalg.norm(np.diff(pos, axis=0), axis=1)
    assert abs(step.sum() - tr.length) < 1e-3
    np.testing.assert_allclose(pos[0], pos[-1], atol=1e-9)
    np.testing.assert_allclose((tan * nrm).sum(1), 0, atol=1e-12)


def test_map_points_lie_on_track_surfaces():
    tr = W.oval_1500()
    m = tr.sample_map(200_000, seed=2)
    ground = m[:, 2] == 0
    w = tr.lateral(m[:, 0].astype(np.float64), m[:, 1].astype(np.float64))
    assert np.abs(w[ground]).max() <= 6.0 + 1e-4
    assert np.abs(np.abs(w[~ground]) - 6.0).max() < 1e-3
    # area split ground : walls = 18000 : 3000
    assert abs(ground.mean() - 18000 / 21000) < 0.01
    assert ((m[~ground, 2] >= 0) & (m[~ground, 2] <= 1)).all()


def test_raycast_scan_shape_and_hits():
    tr = W.oval_1500()
    g = W.rng_for(3)
    q = tr.raycast(*tr.random_pose(g), g)
    assert 120_000 < len(q) <= 128 * 1024
    assert q.dtype == np.float32
    # the sensor sits at 0.8 m: nothing above the wall top (1 m) + noise
    assert q[:, 2].max() < 1.1
    g2 = W.rng_for(3)
    np.testing.assert_array_equal(q, tr.raycast(*tr.random_pose(g2), g2))


def test_scan_batch_sizes_log_uniform_range():
    scans = W.scan_batch(8, seed=4)
    n = np.array([len(s) for s in scans])
    assert (n >= 20_000).all() and (n <= 130_000).all()
    again = W.scan_batch(8, seed=4)
    for a, b in zip(scans, again):
        np.testing.assert_array_equal(a, b)


def test_arrival_stream_rates():
    arr = W.arrival_stream(duration=1.0, vehicles=2, sensors=3, pool=4, seed=5)
    t = np.array([a.t for a in arr])
    assert (np.diff(t) >= 0).all() and (t < 1.0).all()
    assert 60 <= len(arr) <= 190  # 6 sensors x 20 Hz x 1 s = 120 expected
    assert all(30_000 <= len(a.points) <= 130_000 for a in arr)
