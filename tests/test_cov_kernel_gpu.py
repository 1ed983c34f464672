"""Kernel-descriptor weighted covariances (pc_set_cov_kernel, Table I) on
the GPU against the binary64 oracle.

The neighbours must be bit-identical to the unweighted search (the weights
only enter the covariance); raw weighted covariances within the relative
Frobenius bar of tests/helpers.py, regularised ones within the Davis-Kahan
rule.  Also: the batched form equals the single-scan form bit for bit, a
zero total weight gives NaN rows, clearing restores the plain covariance,
and bad descriptors are refused.
"""
import numpy as np
import pytest

import oracle
from paper_2308_07173_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K = 20
KERNELS = [
    ("rbf", dict(sigma=30.0)),
    ("gaussian", dict(sigma=0.15)),
    ("laplacian", dict(sigma=0.1)),
    ("polynomial", dict(alpha=1e-5, c=1.0, d=2.0)),
    ("hi", dict()),
]


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
    t = gpu_lib.Target(dev(mp))
    plain = [host(x) for x in t.knn_cov(dev(q), K, 1e-3)]
    yield {"map": mp, "q": q, "t": t, "plain": plain, "origin": t.info()["origin"]}
    t.close()


@pytest.mark.parametrize("kind,prm", KERNELS, ids=[k for k, _ in KERNELS])
def test_weighted_covariance_matches_oracle(scene, gpu_lib, kind, prm):
    s = scene
    t = s["t"]
    t.set_cov_kernel(kind, **prm)
    try:
        idx, d2, raw = (host(x) for x in t.knn_cov(dev(s["q"]), K, -1.0))
        _, _, reg = (host(x) for x in t.knn_cov(dev(s["q"]), K, 1e-3))
        st = t.sync_status()
    finally:
        t.set_cov_kernel("none")
    assert st == gpu_lib.PC_OK
    np.testing.assert_array_equal(idx, s["plain"][0])
    np.testing.assert_array_equal(d2.view(np.uint32), s["plain"][1].view(np.uint32))
    want_raw = oracle.cov_weighted(s["map"], s["q"], idx, -1.0, kind, origin=s["origin"], **prm)
    want_reg = oracle.cov_weighted(s["map"], s["q"], idx, 1e-3, kind, origin=s["origin"], **prm)
    H.check_raw_cov(raw, want_raw)
    H.check_regularised_cov(reg, want_reg, want_raw, raw, 1e-3)
    # the weights matter: the raw covariance differs from the plain one
    plain_raw = oracle.cov(s["map"], idx, -1.0)
    assert np.abs(want_raw - plain_raw).max() > 1e-6 * np.abs(plain_raw).max()


@pytest.mark.parametrize("grown", [False, True], ids=["whole", "grown"])
def test_weighted_rows_of_the_warp_search(scene, gpu_lib, grown):
    # k = 40 runs the warp-cooperative search, whose rows take the weighted
    # covariance from the caller-order copies (of both grids when grown)
    s = scene
    k = 40
    q = s["q"][:4000]
    if grown:
        t = gpu_lib.Target(dev(s["map"][:200_000]))
        t.append(dev(s["map"][200_000:]))
    else:
        t = s["t"]
    t.set_cov_kernel("laplacian", sigma=0.1)
    try:
        idx, _, raw = (host(x) for x in t.knn_cov(dev(q), k, -1.0))
        _, _, reg = (host(x) for x in t.knn_cov(dev(q), k, 1e-3))
        st = t.sync_status()
        origin = t.info()["origin"]
    finally:
        t.set_cov_kernel("none")
        if grown:
            t.close()
    assert st == gpu_lib.PC_OK
    want_i, _ = oracle.knn_brute(q, s["map"], k)
    np.testing.assert_array_equal(idx, want_i)
    want_raw = oracle.cov_weighted(s["map"], q, idx, -1.0, "laplacian", origin=origin, sigma=0.1)
    want_reg = oracle.cov_weighted(s["map"], q, idx, 1e-3, "laplacian", origin=origin, sigma=0.1)
    H.check_raw_cov(raw, want_raw)
    H.check_regularised_cov(reg, want_reg, want_raw, raw, 1e-3)


def test_batched_equals_single_and_clear_restores(scene, gpu_lib):
    s = scene
    t = s["t"]
    t.set_cov_kernel("laplacian", sigma=0.1)
    parts = [s["q"][:7000], s["q"][7000:]]
    single = [[host(x) for x in t.knn_cov(dev(p), K, 1e-3)] for p in parts]
    outs = []
    for p in parts:
        outs.append((dev(p), torch.empty((len(p), K), dtype=torch.int32, device="cuda"),
                     torch.empty((len(p), K), dtype=torch.float32, device="cuda"),
                     torch.empty((len(p), 6), dtype=torch.float32, device="cuda")))
    b = gpu_lib.Batch(t, outs, K, 1e-3)
    t.set_cov_kernel("none")
    b.run()  # the plan keeps the kernel set when it was planned
    assert t.sync_status() == gpu_lib.PC_OK
    for o, ref in zip(outs, single):
        for u, v in zip(o[1:], ref):
            assert host(u).tobytes() == v.tobytes()
    b.close()
    again = [host(x) for x in t.knn_cov(dev(s["q"]), K, 1e-3)]
    for u, v in zip(again, s["plain"]):
        assert u.tobytes() == v.tobytes()


def test_zero_total_weight_is_nan(scene, gpu_lib):
    s = scene
    t = s["t"]
    t.set_cov_kernel("polynomial", alpha=0.0, c=0.0, d=1.0)
    _, _, cov = (host(x) for x in t.knn_cov(dev(s["q"][:100]), K, 1e-3))
    t.set_cov_kernel("none")
    assert np.isnan(cov).all()


def test_bad_descriptors(scene, gpu_lib):
    pc = gpu_lib
    h = scene["t"].handle
    bad = [pc.pc_cov_kernel(9, 1, 1, 0, 1), pc.pc_cov_kernel(2, 0.0, 1, 0, 1), pc.pc_cov_kernel(5, -1.0, 1, 0, 1),
           pc.pc_cov_kernel(1, float("nan"), 1, 0, 1), pc.pc_cov_kernel(3, 1, float("inf"), 0, 1)]
    import ctypes
    for kd in bad:
        assert pc.load().pc_set_cov_kernel(h, ctypes.byref(kd)) == pc.PC_ERR_INVALID_ARG
    assert pc.load().pc_set_cov_kernel(h, None) == pc.PC_OK
