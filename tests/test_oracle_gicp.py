"""Pins for the oracle's GICP linearisation (Eq. 18-20), against facts fixed
outside it.

* the binary32 transform against exact rational arithmetic (one rounding
  per fmaf, in the pinned order);
* correspondences against brute force on the moved points and the
  fl(max_dist^2) threshold;
* H, b, E against closed forms: isotropic covariances and a pure
  translation give sums of [p]_x identities; a rank-one source covariance
  under a non-symmetric rotation gives Omega by Sherman-Morrison (so R C R^T
  cannot be confused with R^T C R);
* the Jacobian's signs and column order against central finite differences
  of the residual under a left perturbation exp(xi^) T built by scipy;
* Gauss-Newton steps built from H and b bring a perturbed pose back to the
  true one on plane-regularised data with exact correspondences.

The paper prints no worked example of a registration step, so none of these
can be a paper value.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from tests import exact_f32 as ex

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

ISO = np.array([1, 0, 0, 1, 0, 1], np.float32)


def _pose(R, t):
    return np.concatenate([np.asarray(R, np.float32).ravel(), np.asarray(t, np.float32)]).astype(np.float32)


def _skew(x):
    return np.array([[0, -x[2], x[1]], [x[2], 0, -x[0]], [-x[1], x[0], 0]], np.float64)


def test_transform_matches_exact_rational_fma_chain():
    rng = np.random.default_rng(1)
    R = Rotation.from_rotvec(rng.standard_normal(3)).as_matrix().astype(np.float32)
    t = (rng.standard_normal(3) * 30).astype(np.float32)
    pose = _pose(R, t)
    src = (rng.standard_normal((40, 3)) * rng.choice([1e-2, 1.0, 100.0], (40, 1))).astype(np.float32)
    got = oracle.gicp_transform(pose, src)
    F = ex.F
    naive_differs = 0
    for i in range(src.shape[0]):
        for a in range(3):
            acc = ex.round_f32(F(pose[3 * a]) * F(src[i, 0]) + F(pose[9 + a]))
            acc = ex.round_f32(F(pose[3 * a + 1]) * F(src[i, 1]) + F(acc))
            want = ex.round_f32(F(pose[3 * a + 2]) * F(src[i, 2]) + F(acc))
            assert got[i, a].tobytes() == want.tobytes(), (i, a)
            naive = np.float32(np.float32(R[a] @ src[i]) + t[a])
            naive_differs += naive != want
    assert naive_differs > 0  # the order matters on these inputs


def test_correspondences_are_brute_force_nearest_within_max_dist():
    rng = np.random.default_rng(2)
    mp = (rng.random((700, 3)) * [10, 10, 2]).astype(np.float32)
    src = (rng.random((300, 3)) * [12, 12, 3] - 1).astype(np.float32)
    R = Rotation.from_rotvec([0.02, -0.01, 0.3]).as_matrix()
    pose = _pose(R, [0.3, -0.2, 0.1])
    tree = oracle.KDTree(mp)
    max_dist = 0.35
    r = oracle.gicp_linearize(tree, np.tile(ISO, (700, 1)), src, np.tile(ISO, (300, 1)), pose, max_dist)
    moved = oracle.gicp_transform(pose, src)
    bi, bd = oracle.knn_brute(moved, mp, 1)
    lim = np.float32(max_dist) * np.float32(max_dist)
    want = np.where(bd[:, 0] <= lim, bi[:, 0], -1)
    np.testing.assert_array_equal(r["corr"], want)
    assert r["pairs"] == int((want >= 0).sum())
    assert 0 < r["pairs"] < 300
    # max_dist = inf takes every point; 0 only exact coincidences
    r = oracle.gicp_linearize(tree, np.tile(ISO, (700, 1)), src, np.tile(ISO, (300, 1)), pose, np.inf)
    np.testing.assert_array_equal(r["corr"], bi[:, 0])
    r = oracle.gicp_linearize(tree, np.tile(ISO, (700, 1)), src, np.tile(ISO, (300, 1)), pose, 0.0)
    assert r["pairs"] == 0 and (r["corr"] == -1).all()


def test_translation_with_isotropic_covariances_closed_form():
    # map = source on a 1/64 grid, pose = pure translation by a dyadic delta
    # well below the spacing: p' = p + delta exactly, the pair of p is p itself
    # and every residual is -delta; Omega = I / (a + c).
    rng = np.random.default_rng(3)
    pts = np.unique(rng.integers(0, 64 * 8, (400, 3)), axis=0).astype(np.float32) / 64.0
    pts = pts[: 300]
    a, c = 0.5, 0.25
    delta = np.array([1.0 / 512, -3.0 / 1024, 1.0 / 256], np.float32)
    tree = oracle.KDTree(pts)
    r = oracle.gicp_linearize(tree, np.tile(ISO * a, (len(pts), 1)), pts, np.tile(ISO * c, (len(pts), 1)),
                              _pose(np.eye(3), delta), 1.0)
    n = len(pts)
    np.testing.assert_array_equal(r["corr"], np.arange(n))
    w = 1.0 / (a + c)
    pm = pts.astype(np.float64) + delta
    dl = delta.astype(np.float64)
    S = pm.sum(0)
    H = np.zeros((6, 6))
    H[:3, :3] = w * (np.sum(pm * pm) * np.eye(3) - pm.T @ pm)
    H[:3, 3:] = w * _skew(S)
    H[3:, :3] = H[:3, 3:].T
    H[3:, 3:] = w * n * np.eye(3)
    b = np.concatenate([w * np.cross(S, dl), w * n * dl])
    np.testing.assert_allclose(r["H"], H, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(r["b"], b, rtol=1e-12, atol=1e-12)
    assert r["error"] == pytest.approx(w * n * float(dl @ dl), rel=1e-12)
    assert r["pairs"] == n


def test_omega_sherman_morrison_under_nonsymmetric_rotation():
    # one pair; C_q = I, C_p = v v^T with small integers (exact in binary32):
    # S = I + w w^T with w = R v, so Omega = I - w w^T / (1 + w^T w).
    R = Rotation.from_rotvec([0.4, -0.7, 0.9]).as_matrix().astype(np.float32)
    assert np.abs(R - R.T).max() > 0.1
    v = np.array([1.0, 2.0, 2.0])
    cp = np.outer(v, v)
    cp6 = np.array([[cp[0, 0], cp[0, 1], cp[0, 2], cp[1, 1], cp[1, 2], cp[2, 2]]], np.float32)
    q = np.array([[1.0, 2.0, 0.5]], np.float32)
    p = np.array([[0.2, -0.1, 0.3]], np.float32)
    t = np.array([0.75, 2.125, 0.25], np.float32)
    pose = _pose(R, t)
    r = oracle.gicp_linearize(oracle.KDTree(q), ISO[None], p, cp6, pose, 10.0)
    assert r["pairs"] == 1
    pm = oracle.gicp_transform(pose, p)[0].astype(np.float64)
    d = q[0].astype(np.float64) - pm
    w = R.astype(np.float64) @ v
    Om = np.eye(3) - np.outer(w, w) / (1.0 + w @ w)
    assert r["error"] == pytest.approx(float(d @ Om @ d), rel=1e-12)
    np.testing.assert_allclose(r["b"][3:], -(Om @ d), rtol=1e-12, atol=1e-14)
    Jw = _skew(pm)
    np.testing.assert_allclose(r["H"][:3, :3], Jw.T @ Om @ Jw, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(r["H"][3:, 3:], Om, rtol=1e-12, atol=1e-14)
    # the transposed rotation gives a different answer on these inputs
    wt = R.astype(np.float64).T @ v
    Omt = np.eye(3) - np.outer(wt, wt) / (1.0 + wt @ wt)
    assert abs(float(d @ Omt @ d) - r["error"]) > 1e-3 * r["error"]


def _perturb(xi, P):
    """exp(xi^) applied on the left to already-moved points P (float64)."""
    Rw = Rotation.from_rotvec(xi[:3]).as_matrix()
    return P @ Rw.T + xi[3:]


def test_jacobian_matches_central_differences():
    rng = np.random.default_rng(4)
    mp = (rng.random((600, 3)) * [8, 8, 2]).astype(np.float32)
    src = (mp[rng.choice(600, 150, replace=False)] + rng.normal(0, 0.05, (150, 3))).astype(np.float32)
    R = Rotation.from_rotvec([0.05, 0.02, -0.1]).as_matrix()
    pose = _pose(R, [0.1, 0.05, -0.02])
    # isotropic covariances, different scales per point: Omega_i = I / s_i
    sq = rng.uniform(0.5, 2.0, 600)
    sp = rng.uniform(0.5, 2.0, 150)
    tree = oracle.KDTree(mp)
    r = oracle.gicp_linearize(tree, ISO[None] * sq[:, None].astype(np.float32), src,
                              ISO[None] * sp[:, None].astype(np.float32), pose, np.inf)
    corr = r["corr"]
    assert (corr >= 0).all()
    P = oracle.gicp_transform(pose, src).astype(np.float64)
    Q = mp[corr].astype(np.float64)
    w = 1.0 / (sq[corr].astype(np.float32).astype(np.float64) + sp.astype(np.float32).astype(np.float64))
    h = 1e-6
    J = np.zeros((150, 3, 6))
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        J[:, :, j] = ((Q - _perturb(e, P)) - (Q - _perturb(-e, P))) / (2 * h)
    d = Q - P
    H = np.einsum("n,nar,nac->rc", w, J, J)
    b = np.einsum("n,nar,na->r", w, J, d)
    E = float(np.sum(w * np.sum(d * d, 1)))
    # tolerances: O(h^2) of the differences, and the binary32 R being
    # orthogonal only to ~1e-7 (R (s I) R^T = s I only to that order)
    np.testing.assert_allclose(r["H"], H, rtol=1e-6, atol=1e-6 * np.abs(H).max())
    np.testing.assert_allclose(r["b"], b, rtol=1e-6, atol=1e-6 * np.abs(b).max())
    assert r["error"] == pytest.approx(E, rel=1e-6)


def _plane_scene(rng, n_per=400):
    """Points on three orthogonal-ish planes with the plane-regularised
    covariance I - (1 - eps) n n^T of each plane."""
    eps = 1e-3
    normals = [np.array([0, 0, 1.0]), np.array([1.0, 0.2, 0]), np.array([0.1, 1.0, 0.3])]
    pts, covs = [], []
    for nv in normals:
        nv = nv / np.linalg.norm(nv)
        a = np.cross(nv, [0.3, 0.5, 0.7])
        a /= np.linalg.norm(a)
        bb = np.cross(nv, a)
        uv = rng.uniform(-4, 4, (n_per, 2))
        pts.append(uv[:, :1] * a + uv[:, 1:] * bb + nv * 2.0)
        C = np.eye(3) - (1 - eps) * np.outer(nv, nv)
        covs.append(np.tile([C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]], (n_per, 1)))
    return np.vstack(pts).astype(np.float32), np.vstack(covs).astype(np.float32)


def test_gauss_newton_steps_recover_the_pose():
    rng = np.random.default_rng(5)
    mp, mcov = _plane_scene(rng)
    tree = oracle.KDTree(mp)
    # source: the map seen from the true pose T (p = T^-1 q), with the same
    # covariances rotated into the source frame
    Rt = Rotation.from_rotvec([0.03, -0.02, 0.08]).as_matrix()
    tt = np.array([0.2, -0.1, 0.05])
    sel = rng.choice(len(mp), 600, replace=False)
    src = ((mp[sel].astype(np.float64) - tt) @ Rt).astype(np.float32)
    C = oracle.unpack6(mcov[sel].astype(np.float64))
    Cs = np.einsum("ji,njk,kl->nil", Rt, C, Rt)
    scov = np.stack([Cs[:, 0, 0], Cs[:, 0, 1], Cs[:, 0, 2], Cs[:, 1, 1], Cs[:, 1, 2], Cs[:, 2, 2]], 1)
    scov = scov.astype(np.float32)
    R = Rotation.from_rotvec([0.0, 0.0, 0.05]).as_matrix()
    t = np.zeros(3)
    errs = []
    for _ in range(8):
        r = oracle.gicp_linearize(tree, mcov, src, scov, _pose(R, t), 1.0)
        errs.append(r["error"] / max(r["pairs"], 1))
        xi = np.linalg.solve(r["H"], -r["b"])
        Rw = Rotation.from_rotvec(xi[:3]).as_matrix()
        R, t = Rw @ R, Rw @ t + xi[3:]
    assert errs[-1] < 1e-6 * errs[0] + 1e-9
    assert np.abs(Rotation.from_matrix(R @ Rt.T).as_rotvec()).max() < 1e-4
    assert np.abs(t - tt).max() < 1e-4


def test_singular_combined_covariance_is_skipped():
    # C_q = C_p = 0: S = 0 has no inverse, the pair is matched but not summed
    q = np.array([[0.0, 0.0, 0.0]], np.float32)
    r = oracle.gicp_linearize(oracle.KDTree(q), np.zeros((1, 6), np.float32), q, np.zeros((1, 6), np.float32),
                              _pose(np.eye(3), [0, 0, 0]), 1.0)
    assert r["pairs"] == 0 and r["corr"][0] == 0
    assert not r["H"].any() and not r["b"].any() and r["error"] == 0.0


def test_nonfinite_source_points_are_not_paired():
    q = np.array([[0.0, 0.0, 0.0], [1.0, 0, 0]], np.float32)
    src = np.array([[np.nan, 0, 0], [0.9, 0, 0], [np.inf, 1, 1]], np.float32)
    r = oracle.gicp_linearize(oracle.KDTree(q), np.tile(ISO, (2, 1)), src, np.tile(ISO, (3, 1)),
                              _pose(np.eye(3), [0, 0, 0]), 1.0)
    np.testing.assert_array_equal(r["corr"], [-1, 1, -1])
    assert r["pairs"] == 1


def test_bad_max_dist_is_rejected():
    q = np.zeros((1, 3), np.float32)
    for bad in (-1.0, np.nan):
        with pytest.raises(ValueError):
            oracle.gicp_linearize(oracle.KDTree(q), ISO[None], q, ISO[None], _pose(np.eye(3), [0, 0, 0]), bad)


def test_so3_exp_matches_scipy_rotation():
    rng = np.random.default_rng(7)
    for w in [np.zeros(3), np.array([1e-9, 0, 0]), *rng.standard_normal((6, 3)), np.array([np.pi - 1e-3, 0, 0])]:
        np.testing.assert_allclose(oracle.so3_exp(w), Rotation.from_rotvec(w).as_matrix(), atol=1e-14)


def test_gicp_update_step_solves_the_normal_equations():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((6, 6))
    H = A @ A.T + 0.1 * np.eye(6)
    b = rng.standard_normal(6)
    R = Rotation.from_rotvec([0.1, -0.2, 0.3]).as_matrix()
    pose = _pose(R, [1.0, 2.0, 3.0])
    for lam in (0.0, 0.5):
        new, xi = oracle.gicp_update(pose, H, b, lam)
        np.testing.assert_allclose((H + lam * np.eye(6)) @ xi, -b, atol=1e-12)
        Rw = Rotation.from_rotvec(xi[:3]).as_matrix()
        np.testing.assert_allclose(new[:9].reshape(3, 3), Rw @ pose[:9].reshape(3, 3).astype(np.float64), atol=1e-6)
        np.testing.assert_allclose(new[9:], Rw @ pose[9:].astype(np.float64) + xi[3:], atol=1e-6)
