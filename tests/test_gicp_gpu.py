"""GICP linearisation and pose update on the GPU (through the C ABI)
against the binary64 oracle.

Correspondences and the pair count must match bit for bit; H, b and E lie
within tests/helpers.gicp_tolerance (derived from binary32 arithmetic on the
combined covariance).  Inputs are the track workload (map and a ray-cast
scan, seeded) with covariances computed by the oracle, so both sides get
identical inputs.
"""
import numpy as np
import pytest

import oracle
from paper_2308_07173_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from scipy.spatial.transform import Rotation  # noqa: E402

EPS = 1e-3
K = 20
ISO = np.array([1, 0, 0, 1, 0, 1], np.float32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def pose12(R, t):
    return np.concatenate([np.asarray(R, np.float32).ravel(), np.asarray(t, np.float32)]).astype(np.float32)


def unpack(v):
    v = np.asarray(v, np.float64)
    Hm = np.zeros((6, 6))
    Hm[np.triu_indices(6)] = v[:21]
    Hm = Hm + np.triu(Hm, 1).T
    return {"H": Hm, "b": v[21:27], "error": float(v[27]), "pairs": int(v[28])}


@pytest.fixture(scope="module")
def scene(gpu_lib):
    tr = W.oval_1500()
    mp = tr.sample_map(300_000, 2)
    g = W.rng_for(3)
    scan = tr.raycast(*tr.random_pose(g), g)
    src = scan[np.sort(g.choice(len(scan), 20_000, replace=False))]
    tree = oracle.KDTree(mp)
    mi, _ = tree.knn(mp, K)
    mcov = oracle.cov(mp, mi, EPS).astype(np.float32)
    st = oracle.KDTree(src)
    si, _ = st.knn(src, K)
    scov = oracle.cov(src, si, EPS).astype(np.float32)
    st.close()
    t = gpu_lib.Target(dev(mp))
    yield {"map": mp, "src": src, "mcov": mcov, "scov": scov, "tree": tree, "t": t}
    t.close()


POSE = pose12(Rotation.from_rotvec([0.002, -0.003, 0.01]).as_matrix(), [0.1, -0.05, 0.02])


def gpu_lin(pc, t, mcov, src, scov, pose, max_dist, corr=True):
    n = len(src)
    c = torch.empty(n, dtype=torch.int32, device="cuda") if corr else None
    out, c = t.gicp_linearize(dev(mcov), dev(src), dev(scov), dev(pose), max_dist, corr=c)
    st = t.sync_status()
    return unpack(host(out)), (host(c) if corr else None), st


def test_linearize_matches_oracle_regularised(scene, gpu_lib):
    s = scene
    want = oracle.gicp_linearize(s["tree"], s["mcov"], s["src"], s["scov"], POSE, 1.0)
    got, corr, st = gpu_lin(gpu_lib, s["t"], s["mcov"], s["src"], s["scov"], POSE, 1.0)
    assert st == gpu_lib.PC_OK
    np.testing.assert_array_equal(corr, want["corr"])
    assert 0.5 * len(s["src"]) < want["pairs"] <= len(s["src"])
    worst = H.check_gicp(got, want, H.gicp_tolerance(EPS))
    print("worst relative error (regularised):", worst)


def test_linearize_isotropic_tight(scene, gpu_lib):
    # isotropic covariances: S = (a + c) I up to R's rounding, kappa ~ 1
    s = scene
    rng = np.random.default_rng(9)
    mcov = (ISO[None] * rng.uniform(0.5, 2.0, (len(s["map"]), 1))).astype(np.float32)
    scov = (ISO[None] * rng.uniform(0.5, 2.0, (len(s["src"]), 1))).astype(np.float32)
    want = oracle.gicp_linearize(s["tree"], mcov, s["src"], scov, POSE, 1.0)
    got, corr, st = gpu_lin(gpu_lib, s["t"], mcov, s["src"], scov, POSE, 1.0)
    assert st == gpu_lib.PC_OK
    np.testing.assert_array_equal(corr, want["corr"])
    worst = H.check_gicp(got, want, 64 * H.U32)
    print("worst relative error (isotropic):", worst)


def test_linearize_is_bit_reproducible(scene, gpu_lib):
    s = scene
    t = s["t"]
    outs = []
    for _ in range(3):
        out, _ = t.gicp_linearize(dev(s["mcov"]), dev(s["src"]), dev(s["scov"]), dev(POSE), 1.0)
        outs.append(host(out).copy())
    assert outs[0].tobytes() == outs[1].tobytes() == outs[2].tobytes()


@pytest.mark.parametrize("n", [1, 31, 33, 257, 4099])
def test_ragged_sizes(scene, gpu_lib, n):
    s = scene
    src, scov = s["src"][:n], s["scov"][:n]
    want = oracle.gicp_linearize(s["tree"], s["mcov"], src, scov, POSE, 1.0)
    got, corr, st = gpu_lin(gpu_lib, s["t"], s["mcov"], src, scov, POSE, 1.0)
    np.testing.assert_array_equal(corr, want["corr"])
    H.check_gicp(got, want, H.gicp_tolerance(EPS))


def test_max_dist_zero_and_infinite(scene, gpu_lib):
    s = scene
    src, scov = s["src"][:3000], s["scov"][:3000]
    got, corr, _ = gpu_lin(gpu_lib, s["t"], s["mcov"], src, scov, POSE, 0.0)
    want = oracle.gicp_linearize(s["tree"], s["mcov"], src, scov, POSE, 0.0)
    np.testing.assert_array_equal(corr, want["corr"])
    assert got["pairs"] == want["pairs"]
    got, corr, _ = gpu_lin(gpu_lib, s["t"], s["mcov"], src, scov, POSE, float("inf"))
    want = oracle.gicp_linearize(s["tree"], s["mcov"], src, scov, POSE, np.inf)
    np.testing.assert_array_equal(corr, want["corr"])
    assert (corr >= 0).all()
    H.check_gicp(got, want, H.gicp_tolerance(EPS))


def test_far_points_exhaustive_and_search_limit(gpu_lib):
    rng = np.random.default_rng(10)
    mp = (rng.random((5000, 3)) * [20, 20, 2]).astype(np.float32)
    src = np.vstack([mp[:100] + 0.01, np.array([[500.0, 500.0, 50.0], [-300.0, 0.0, 0.0]], np.float32)])
    src = src.astype(np.float32)
    mcov = np.tile(ISO, (5000, 1))
    scov = np.tile(ISO, (len(src), 1))
    pose = pose12(np.eye(3), [0, 0, 0])
    tree = oracle.KDTree(mp)
    want = oracle.gicp_linearize(tree, mcov, src, scov, pose, np.inf)
    t = gpu_lib.Target(dev(mp), max_box_cells=64)
    got, corr, st = gpu_lin(gpu_lib, t, mcov, src, scov, pose, float("inf"))
    assert st == gpu_lib.PC_OK
    np.testing.assert_array_equal(corr, want["corr"])
    H.check_gicp(got, want, 64 * H.U32)
    assert t.stats()["exhaustive"] >= 2
    t.close()
    t = gpu_lib.Target(dev(mp), max_box_cells=64, exhaustive=False)
    got, corr, st = gpu_lin(gpu_lib, t, mcov, src, scov, pose, float("inf"))
    assert st == gpu_lib.PC_ERR_SEARCH_LIMIT
    np.testing.assert_array_equal(corr[:100], want["corr"][:100])
    assert (corr[100:] == -1).all()
    # a finite max_dist bounds the search: the far points end without a pair
    got, corr, st = gpu_lin(gpu_lib, t, mcov, src, scov, pose, 1.0)
    assert st == gpu_lib.PC_OK
    assert (corr[100:] == -1).all()
    t.close()


def test_nonfinite_and_empty(scene, gpu_lib):
    s = scene
    src = s["src"][:64].copy()
    src[5] = np.nan
    src[40, 2] = np.inf
    got, corr, st = gpu_lin(gpu_lib, s["t"], s["mcov"], src, s["scov"][:64], POSE, 1.0)
    assert st == gpu_lib.PC_ERR_NONFINITE
    want = oracle.gicp_linearize(s["tree"], s["mcov"], src, s["scov"][:64], POSE, 1.0)
    np.testing.assert_array_equal(corr, want["corr"])
    assert corr[5] == -1 and corr[40] == -1
    out, _ = s["t"].gicp_linearize(dev(s["mcov"]), torch.empty((0, 3), device="cuda"),
                                   torch.empty((0, 6), device="cuda"), dev(POSE), 1.0)
    assert (host(out) == 0).all()


def test_invalid_arguments(scene, gpu_lib):
    pc = gpu_lib
    s = scene
    t = s["t"]
    mc, sr, sc, po = dev(s["mcov"]), dev(s["src"][:10]), dev(s["scov"][:10]), dev(POSE)
    out = torch.empty(29, dtype=torch.float64, device="cuda")
    work = t.gicp_work()
    h = pc._stream_handle()
    call = lambda **kw: pc.pc_gicp_linearize(
        t.handle, kw.get("mc", mc.data_ptr()), sr.data_ptr(), kw.get("n", 10), sc.data_ptr(), po.data_ptr(),
        kw.get("md", 1.0), kw.get("out", out.data_ptr()), None, kw.get("work", work.data_ptr()),
        kw.get("wb", work.numel()), h)
    assert call() == pc.PC_OK
    assert call(md=-1.0) == pc.PC_ERR_INVALID_ARG
    assert call(md=float("nan")) == pc.PC_ERR_INVALID_ARG
    assert call(n=-1) == pc.PC_ERR_INVALID_ARG
    assert call(wb=work.numel() - 1) == pc.PC_ERR_INVALID_ARG
    assert call(work=work.data_ptr() + 16) == pc.PC_ERR_INVALID_ARG
    assert call(out=out.data_ptr() + 4) == pc.PC_ERR_INVALID_ARG
    assert call(mc=None) == pc.PC_ERR_INVALID_ARG
    hostbuf = np.zeros(64, np.float32)
    assert call(mc=hostbuf.ctypes.data) == pc.PC_ERR_BAD_POINTER
    torch.cuda.synchronize()
    assert pc.pc_gicp_update(None, 0.0, po.data_ptr(), None, h) == pc.PC_ERR_INVALID_ARG
    assert pc.pc_gicp_update(out.data_ptr(), -1.0, po.data_ptr(), None, h) == pc.PC_ERR_INVALID_ARG
    assert pc.pc_gicp_update(out.data_ptr(), 0.0, hostbuf.ctypes.data, None, h) == pc.PC_ERR_BAD_POINTER


@pytest.mark.parametrize("lam", [0.0, 0.5])
def test_update_matches_oracle_step(scene, gpu_lib, lam):
    s = scene
    want = oracle.gicp_linearize(s["tree"], s["mcov"], s["src"], s["scov"], POSE, 1.0)
    lin = np.concatenate([want["H"][np.triu_indices(6)], want["b"], [want["error"], want["pairs"]]])
    new_w, xi_w = oracle.gicp_update(POSE, want["H"], want["b"], lam)
    p = dev(POSE.copy())
    xi = torch.empty(6, dtype=torch.float64, device="cuda")
    rc = gpu_lib.pc_gicp_update(dev(lin).data_ptr(), lam, p.data_ptr(), xi.data_ptr(), gpu_lib._stream_handle())
    assert rc == gpu_lib.PC_OK
    xg, pg = host(xi), host(p)
    np.testing.assert_allclose(xg, xi_w, rtol=1e-9, atol=1e-12 * np.abs(xi_w).max())
    # binary64 on both sides, rounded once to binary32: within 1 ulp
    np.testing.assert_array_less(np.abs(pg.astype(np.float64) - new_w), np.spacing(np.abs(new_w)) * 1.01 + 1e-30)


def test_update_not_positive_definite_keeps_pose(gpu_lib):
    lin = np.zeros(29)
    p = dev(POSE.copy())
    xi = torch.empty(6, dtype=torch.float64, device="cuda")
    assert gpu_lib.pc_gicp_update(dev(lin).data_ptr(), 0.0, p.data_ptr(), xi.data_ptr(),
                                  gpu_lib._stream_handle()) == gpu_lib.PC_OK
    assert np.isnan(host(xi)).all()
    assert host(p).tobytes() == POSE.tobytes()
    assert gpu_lib.pc_gicp_update(dev(lin).data_ptr(), 1.0, p.data_ptr(), xi.data_ptr(),
                                  gpu_lib._stream_handle()) == gpu_lib.PC_OK
    assert (host(xi) == 0).all() and host(p).tobytes() == POSE.tobytes()


@pytest.fixture(scope="module")
def pit_scene(gpu_lib):
    """The pit lane of the 4 km track (garage walls constrain all six
    degrees of freedom; the plain oval's planes and cylinders do not): a
    400k-point map, and 17k points of an independent sample within 40 m of a
    sensor in the pit lane, in that sensor's frame."""
    tr = W.oval_4000_pit()
    mp = tr.sample_map(400_000, 6, noise=0.01)
    o = np.array([0.0, tr.r + tr.half_width + tr.pit_width / 2, 0.8])
    other = tr.sample_map(400_000, 7, noise=0.01)
    near = other[np.linalg.norm(other[:, :2] - o[:2], axis=1) < 40.0]
    Rt = Rotation.from_rotvec([0, 0, 0.3]).as_matrix()
    src = ((near.astype(np.float64) - o) @ Rt).astype(np.float32)
    tree = oracle.KDTree(mp)
    mi, _ = tree.knn(mp, K)
    mcov = oracle.cov(mp, mi, EPS).astype(np.float32)
    st = oracle.KDTree(src)
    si, _ = st.knn(src, K)
    scov = oracle.cov(src, si, EPS).astype(np.float32)
    st.close()
    t = gpu_lib.Target(dev(mp))
    start = pose12(Rotation.from_rotvec([0.003, -0.004, 0.02]).as_matrix() @ Rt, o + [0.2, -0.15, 0.05])
    yield {"map": mp, "src": src, "mcov": mcov, "scov": scov, "tree": tree, "t": t, "Rt": Rt, "tt": o,
           "start": start}
    t.close()


def test_pit_scene_linearize_matches_oracle(pit_scene, gpu_lib):
    s = pit_scene
    want = oracle.gicp_linearize(s["tree"], s["mcov"], s["src"], s["scov"], s["start"], 1.0)
    got, corr, st = gpu_lin(gpu_lib, s["t"], s["mcov"], s["src"], s["scov"], s["start"], 1.0)
    assert st == gpu_lib.PC_OK
    np.testing.assert_array_equal(corr, want["corr"])
    H.check_gicp(got, want, H.gicp_tolerance(EPS))


def test_device_registration_recovers_pose_like_oracle(pit_scene, gpu_lib):
    from paper_2308_07173_gb300 import gicp

    s = pit_scene
    reg = gicp.Registration(dev(s["map"]), map_cov=dev(s["mcov"]), target=s["t"])
    pose = dev(s["start"].copy())
    lin, xi = reg.align(dev(s["src"]), dev(s["scov"]), pose, iters=6, max_dist=1.0)
    pg = host(pose)
    po = s["start"].copy()
    for _ in range(6):
        r = oracle.gicp_linearize(s["tree"], s["mcov"], s["src"], s["scov"], po, 1.0)
        po, _ = oracle.gicp_update(po, r["H"], r["b"])
    Rg = pg[:9].reshape(3, 3).astype(np.float64)
    Ro = po[:9].reshape(3, 3).astype(np.float64)
    # the same fixed point as the oracle's iterations
    assert np.abs(Rotation.from_matrix(Rg @ Ro.T).as_rotvec()).max() < 2e-6
    assert np.abs(pg[9:].astype(np.float64) - po[9:]).max() < 2e-5
    # and the true pose to within the 1 cm surface noise
    assert np.abs(Rotation.from_matrix(Rg @ s["Rt"].T).as_rotvec()).max() < 2e-4
    assert np.abs(pg[9:] - s["tt"]).max() < 5e-3
    e = host(lin)[:, 27] / np.maximum(host(lin)[:, 28], 1)
    assert e[-1] < 0.05 * e[0]


def test_graph_replay_equals_eager(scene, gpu_lib):
    from paper_2308_07173_gb300 import gicp

    s = scene
    reg = gicp.Registration(dev(s["map"]), map_cov=dev(s["mcov"]), target=s["t"])
    src, scov = dev(s["src"]), dev(s["scov"])
    p1 = dev(POSE.copy())
    l1, x1 = reg.align(src, scov, p1, iters=4, max_dist=1.0)
    a = (host(l1).copy(), host(x1).copy(), host(p1).copy())
    p2 = dev(POSE.copy())
    l2, x2 = reg.align(src, scov, p2, iters=4, max_dist=1.0, graph=True)
    b = (host(l2).copy(), host(x2).copy(), host(p2).copy())
    for u, v in zip(a, b):
        assert u.tobytes() == v.tobytes()
    # replaying again continues from the moved pose (same graph, new values)
    p2.copy_(dev(POSE.copy()))
    l3, _ = reg.align(src, scov, p2, iters=4, max_dist=1.0, graph=True)
    assert host(l3).tobytes() == a[0].tobytes()
