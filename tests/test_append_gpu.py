"""Incremental map updates (pc_target_append / pc_target_compact) against
the oracle over all the points at once.

idx and d2 must equal the oracle's kNN over the concatenated map bit for bit
(appended points indexed after the main ones), covariances within the usual
bar, and GICP pairing, pc_cov, windows and kernel weights must see the whole
union.  Compaction keeps every index and answer; batched forms refuse a
target with appended points until it is compacted.
"""
import numpy as np
import pytest

import oracle
from paper_2308_07173_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K = 20


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def scene():
    tr = W.oval_1500()
    mp = tr.sample_map(300_000, 2)
    g = W.rng_for(3)
    scan = tr.raycast(*tr.random_pose(g), g)
    q = scan[np.sort(g.choice(len(scan), 20_000, replace=False))]
    tree = oracle.KDTree(mp)
    idx, d2 = tree.knn(q, K)
    return {"map": mp, "q": q, "tree": tree, "idx": idx, "d2": d2}


def grown_target(pc, mp, n_main, steps):
    t = pc.Target(dev(mp[:n_main]))
    at = n_main
    for n in steps:
        t.append(dev(mp[at:at + n]))
        at += n
    assert at == len(mp)
    return t


def test_append_equals_oracle_over_the_union(scene, gpu_lib):
    s = scene
    t = grown_target(gpu_lib, s["map"], 250_000, [30_000, 20_000])
    assert t.info()["delta_m"] == 50_000
    idx, d2, cov = (host(x) for x in t.knn_cov(dev(s["q"]), K, -1.0))
    assert t.sync_status() == gpu_lib.PC_OK
    np.testing.assert_array_equal(idx, s["idx"])
    np.testing.assert_array_equal(d2.view(np.uint32), s["d2"].view(np.uint32))
    assert (idx >= 250_000).any()  # appended points do answer
    H.check_raw_cov(cov, oracle.cov(s["map"], idx, -1.0))
    # pc_cov takes the global indices
    c2 = host(t.cov(dev(idx), -1.0))
    H.check_raw_cov(c2, oracle.cov(s["map"], idx, -1.0))
    # compaction keeps every answer
    t.compact()
    assert t.info()["delta_m"] == 0 and t.info()["m"] == 300_000
    i2, e2, _ = (host(x) for x in t.knn_cov(dev(s["q"]), K, -1.0))
    np.testing.assert_array_equal(i2, s["idx"])
    np.testing.assert_array_equal(e2.view(np.uint32), s["d2"].view(np.uint32))
    t.close()


@pytest.mark.parametrize("k", [10, 32, 40])
def test_union_search_modes_with_fused_covariance(scene, gpu_lib, k):
    # k = 10 and 32 run the lane path over both grids (32 and 64 survivor
    # slots), k = 40 the warp search; the regularised covariance is fused
    s = scene
    t = grown_target(gpu_lib, s["map"], 240_000, [60_000])
    idx, d2, cov = (host(x) for x in t.knn_cov(dev(s["q"]), k, 1e-3))
    assert t.sync_status() == gpu_lib.PC_OK
    want_i, want_d = s["tree"].knn(s["q"], k)
    np.testing.assert_array_equal(idx, want_i)
    np.testing.assert_array_equal(d2.view(np.uint32), want_d.view(np.uint32))
    assert (idx >= 240_000).any()
    raw = host(t.cov(dev(idx), -1.0))
    H.check_regularised_cov(cov, oracle.cov(s["map"], idx, 1e-3), oracle.cov(s["map"], idx, -1.0), raw, 1e-3)
    t.close()


def test_k_larger_than_the_main_grid(gpu_lib):
    g = np.random.default_rng(3)
    mp = (g.random((60, 3)) * 4).astype(np.float32)
    q = (g.random((500, 3)) * 4).astype(np.float32)
    t = gpu_lib.Target(dev(mp[:10]))
    t.append(dev(mp[10:35]))
    t.append(dev(mp[35:]))
    for k in (5, 25, 60):
        idx, d2 = (host(x) for x in t.knn(dev(q), k))
        want_i, want_d = oracle.knn_brute(q, mp, k)
        np.testing.assert_array_equal(idx, want_i)
        np.testing.assert_array_equal(d2.view(np.uint32), want_d.view(np.uint32))
    with pytest.raises(gpu_lib.PcError):
        t.knn(dev(q), 61)
    t.close()


def test_window_and_kernel_weights_see_appended_points(scene, gpu_lib):
    s = scene
    t = grown_target(gpu_lib, s["map"], 200_000, [100_000])
    c = np.median(s["q"], axis=0)
    lo, hi = [c[0] - 40, c[1] - 40, -np.inf], [c[0] + 40, c[1] + 40, np.inf]
    t.set_window(lo, hi)
    idx, d2 = (host(x) for x in t.knn(dev(s["q"]), K))
    t.set_window()
    wi, wd = oracle.knn_window(s["q"], s["map"], K, lo, hi)
    np.testing.assert_array_equal(idx, wi)
    t.set_cov_kernel("laplacian", sigma=0.1)
    idx, _, cov = (host(x) for x in t.knn_cov(dev(s["q"]), K, -1.0))
    t.set_cov_kernel("none")
    np.testing.assert_array_equal(idx, s["idx"])
    origin = t.info()["origin"]
    H.check_raw_cov(cov, oracle.cov_weighted(s["map"], s["q"], idx, -1.0, "laplacian", sigma=0.1, origin=origin))
    t.close()


def test_gicp_pairs_over_the_union(scene, gpu_lib):
    s = scene
    t = grown_target(gpu_lib, s["map"], 150_000, [150_000])
    iso = np.array([1, 0, 0, 1, 0, 1], np.float32)
    rng = np.random.default_rng(6)
    mcov = (iso[None] * rng.uniform(0.5, 2, (len(s["map"]), 1))).astype(np.float32)
    scov = (iso[None] * rng.uniform(0.5, 2, (len(s["q"]), 1))).astype(np.float32)
    pose = np.concatenate([np.eye(3).ravel(), [0.05, -0.02, 0.01]]).astype(np.float32)
    want = oracle.gicp_linearize(s["tree"], mcov, s["q"], scov, pose, 1.0)
    c = torch.empty(len(s["q"]), dtype=torch.int32, device="cuda")
    out, _ = t.gicp_linearize(dev(mcov), dev(s["q"]), dev(scov), dev(pose), 1.0, corr=c)
    assert t.sync_status() == gpu_lib.PC_OK
    np.testing.assert_array_equal(host(c), want["corr"])
    v = host(out)
    Hm = np.zeros((6, 6))
    Hm[np.triu_indices(6)] = v[:21]
    got = {"H": Hm + np.triu(Hm, 1).T, "b": v[21:27], "error": float(v[27]), "pairs": int(v[28])}
    H.check_gicp(got, want, 64 * H.U32)
    t.close()


def test_nonfinite_append_is_refused_and_batches_wait_for_compaction(scene, gpu_lib):
    pc = gpu_lib
    s = scene
    t = pc.Target(dev(s["map"][:1000]))
    bad = s["map"][1000:1100].copy()
    bad[7, 1] = np.nan
    with pytest.raises(pc.PcError):
        t.append(dev(bad))
    assert t.info()["delta_m"] == 0
    t.append(dev(s["map"][1000:1100]))
    q = dev(s["q"][:256])
    outs = [(q, torch.empty((256, 8), dtype=torch.int32, device="cuda"),
             torch.empty((256, 8), dtype=torch.float32, device="cuda"), None)]
    with pytest.raises(pc.PcError):
        pc.Batch(t, outs, 8, 1e-3)
    t.compact()
    b = pc.Batch(t, outs, 8, 1e-3)
    b.run()
    want_i, _ = oracle.knn_brute(s["q"][:256], s["map"][:1100], 8)
    np.testing.assert_array_equal(host(outs[0][1]), want_i)
    b.close()
    t.close()
