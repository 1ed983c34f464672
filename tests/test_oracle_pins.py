"""Pins for the CPU oracle, against facts fixed outside it.

Each test is chosen so that a plausible slip in the oracle fails it:
* exact rational arithmetic pins the binary32 d2 order (a missing fmaf or a
  reordered sum changes low bits on the random cases below);
* a tiny pure-Python brute force on integer lattices (exact squared
  distances, many ties) pins the (d2, index) order and the tie-break;
* the k-d tree must equal brute force bit for bit;
* scipy's cKDTree cross-checks neighbour sets where no near-ties exist;
* closed-form covariances (planar grid, cube corners, collinear points),
  trace = mean squared deviation, symmetry, PSD and translation invariance
  pin the 1/k normaliser, centring and index use;
* regularised covariances on exact and rotated planes, and numpy.linalg.eigh,
  pin the eigenvector choice and C' = I - (1 - eps) n n^T.

Covariance follows Sec. III-C1 (per-point Gaussians of Eq. 19); the paper
prints no worked example, so no paper value can pin it.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import exact_f32 as ex

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- d2 order
def test_d2_matches_exact_rational_fma_order():
    rng = np.random.default_rng(11)
    p = (rng.standard_normal((64, 3)) * rng.choice([1e-3, 1.0, 300.0], (64, 1))).astype(np.float32)
    q = (rng.standard_normal((8, 3)) * 50).astype(np.float32)
    idx, d2 = oracle.knn_brute(q, p, k=64, threads=1)
    naive_differs = 0
    for n in range(q.shape[0]):
        for r in range(64):
            j = idx[n, r]
            want = ex.d2_pinned(q[n], p[j])
            assert d2[n, r] == want, (n, r, j)
            # a plain dx*dx + dy*dy + dz*dz in binary32 gives other bits on
            # some of these cases, so this test can tell the orders apart
            d = (q[n].astype(np.float32) - p[j].astype(np.float32)).astype(np.float32)
            naive = np.float32(np.float32(d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
            naive_differs += int(naive != want)
    assert naive_differs > 0


def test_exact_f32_rounding_helper():
    # the helper itself, against numpy's correctly rounded float64 -> float32
    rng = np.random.default_rng(3)
    for v in rng.standard_normal(200) * 10.0 ** rng.integers(-30, 30, 200):
        assert ex.round_f32(Fraction(float(v))) == np.float32(v)
    assert ex.round_f32(Fraction(1) + Fraction(1, 2 ** 24)) == np.float32(1.0)  # tie to even
    assert ex.round_f32(Fraction(1) + Fraction(3, 2 ** 24)) == np.float32(1 + 2 ** -22)  # tie to even, upwards


# ---------------------------------------------------------------- kNN order
def _py_brute(q, p, k):
    """Pure-Python exact brute force (Fractions): the definition, tiny inputs."""
    out_i, out_d = [], []
    for qq in q:
        keys = []
        for j, pp in enumerate(p):
            keys.append((ex.d2_pinned(qq, pp), j))
        keys.sort(key=lambda t: (float(t[0]), t[1]))
        out_i.append([j for _, j in keys[:k]])
        out_d.append([d for d, _ in keys[:k]])
    return np.array(out_i, np.int32), np.array(out_d, np.float32)


def _lattice(nx, ny, nz, scale=1.0, shuffle_seed=None):
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1)
    g = (g.reshape(-1, 3) * scale).astype(np.float32)
    if shuffle_seed is not None:
        g = g[np.random.default_rng(shuffle_seed).permutation(len(g))]
    return g


def test_brute_lattice_ties_against_python():
    p = _lattice(5, 4, 3, shuffle_seed=5)
    q = np.concatenate([p[:6], p[:6] + np.float32(0.5), np.array([[2.0, 1.5, 1.0], [-1, -1, -1]], np.float32)])
    for k in (1, 7, 26, len(p)):
        idx, d2 = oracle.knn_brute(q, p, k, threads=2)
        want_i, want_d = _py_brute(q, p, k)
        np.testing.assert_array_equal(idx, want_i)
        np.testing.assert_array_equal(d2, want_d)
    # query on a target point: that point is rank 0 at d2 = 0
    idx, d2 = oracle.knn_brute(p[:10], p, 3)
    np.testing.assert_array_equal(idx[:, 0], np.arange(10))
    assert (d2[:, 0] == 0).all()


def test_brute_duplicates_tie_break_lower_index():
    p = np.repeat(np.array([[1, 2, 3], [1, 2, 4]], np.float32), 5, axis=0)  # indices 0..4 equal, 5..9 equal
    idx, d2 = oracle.knn_brute(np.array([[1, 2, 3]], np.float32), p, 7)
    np.testing.assert_array_equal(idx[0], [0, 1, 2, 3, 4, 5, 6])
    np.testing.assert_array_equal(d2[0], [0, 0, 0, 0, 0, 1, 1])


def test_brute_rejects_k_above_m():
    with pytest.raises(ValueError):
        oracle.knn_brute(np.zeros((1, 3), np.float32), np.zeros((3, 3), np.float32), 4)


@pytest.mark.parametrize("case", ["uniform", "lattice", "dups", "clustered", "plane"])
def test_kdtree_equals_brute(case):
    rng = np.random.default_rng(hash(case) % 2 ** 32)
    if case == "uniform":
        p = rng.uniform(0, 40, (3000, 3)).astype(np.float32)
        q = rng.uniform(-5, 45, (400, 3)).astype(np.float32)
    elif case == "lattice":
        p = _lattice(12, 10, 6, scale=0.25, shuffle_seed=1)
        q = np.concatenate([p[::7], p[::11] + np.float32(0.125)])
    elif case == "dups":
        base = rng.uniform(0, 3, (200, 3)).astype(np.float32)
        p = base[rng.integers(0, 200, 2000)]
        q = base[:100]
    elif case == "clustered":
        c = rng.uniform(0, 100, (10, 3))
        p = (c[rng.integers(0, 10, 3000)] + rng.standard_normal((3000, 3)) * 0.05).astype(np.float32)
        q = (c[rng.integers(0, 10, 300)] + rng.standard_normal((300, 3)) * 0.5).astype(np.float32)
    else:
        xy = rng.uniform(-500, 500, (3000, 2))
        p = np.c_[xy, np.zeros(3000)].astype(np.float32) + np.float32(1000)
        q = p[rng.integers(0, 3000, 300)] + rng.standard_normal((300, 3)).astype(np.float32) * np.float32(0.1)
    tree = oracle.KDTree(p)
    for k in (1, 10, 33):
        bi, bd = oracle.knn_brute(q, p, k)
        ti, td = tree.knn(q, k)
        np.testing.assert_array_equal(ti, bi)
        np.testing.assert_array_equal(td, bd)


def test_knn_sets_match_scipy_ckdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(7)
    p = rng.uniform(0, 10, (5000, 3)).astype(np.float32)
    q = rng.uniform(0, 10, (300, 3)).astype(np.float32)
    k = 12
    idx, d2 = oracle.knn_brute(q, p, k)
    dd, ii = spatial.cKDTree(p.astype(np.float64)).query(q.astype(np.float64), k=k + 1)
    checked = 0
    for n in range(len(q)):
        # compare only where the k-th and (k+1)-th distances are well apart
        if dd[n, k] - dd[n, k - 1] > 1e-4:
            assert set(idx[n]) == set(ii[n, :k])
            checked += 1
        np.testing.assert_allclose(np.sqrt(d2[n].astype(np.float64)), dd[n, :k], rtol=1e-6, atol=1e-6)
    assert checked > 250


# ---------------------------------------------------------------- covariance
def _cov_of_all(p, eps):
    idx = np.arange(len(p), dtype=np.int32)[None, :]
    return oracle.unpack6(oracle.cov(p, idx, eps))[0]


def test_cov_planar_grid_closed_form():
    s = 0.25
    g = np.array([[i * s, j * s, 0.0] for i in (-1, 0, 1) for j in (-1, 0, 1)], np.float32)
    C = _cov_of_all(g + np.float32(7.0), eps=-1)
    np.testing.assert_allclose(C, np.diag([2 * s * s / 3, 2 * s * s / 3, 0.0]), atol=1e-15)


def test_cov_cube_corners_closed_form():
    a = 0.5
    g = np.array([[x, y, z] for x in (-a, a) for y in (-a, a) for z in (-a, a)], np.float32)
    C = _cov_of_all(g + np.float32(3.0), eps=-1)
    np.testing.assert_allclose(C, a * a * np.eye(3), atol=1e-15)


def test_cov_collinear_rank_one():
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    t = np.arange(-3, 4, dtype=np.float64)  # 7 points, var = 4
    g = (t[:, None] * u[None, :] * 0.375).astype(np.float32)
    C = _cov_of_all(g, eps=-1)
    g64 = g.astype(np.float64)
    d = g64 - g64.mean(0)
    np.testing.assert_allclose(C, d.T @ d / len(g), atol=1e-15)
    w = np.linalg.eigvalsh(C)
    assert abs(w[0]) < 1e-15 and abs(w[1]) < 1e-15 and w[2] > 0.1


def test_cov_invariants_random():
    rng = np.random.default_rng(2)
    # values on a 2^-10 grid, so that the shift below is exact in binary32
    p = (np.round(rng.uniform(-20, 20, (2000, 3)) * 1024) / 1024).astype(np.float32)
    idx = rng.integers(0, 2000, (300, 17)).astype(np.int32)
    C6 = oracle.cov(p, idx, eps=-1)
    C = oracle.unpack6(C6)
    p64 = p.astype(np.float64)
    for n in range(300):
        pts = p64[idx[n]]
        dev = pts - pts.mean(0)
        # trace equals the mean squared deviation from the mean (1/k normaliser)
        assert abs(np.trace(C[n]) - (dev ** 2).sum(1).mean()) <= 1e-12 * max(1.0, np.trace(C[n]))
        w = np.linalg.eigvalsh(C[n])
        assert w[0] >= -1e-12 * w.sum()
    np.testing.assert_array_equal(C, np.swapaxes(C, 1, 2))
    # translation invariance: shift by a power of two, exact in binary32 here
    shift = np.float32(64.0)
    C2 = oracle.cov(p + shift, idx, eps=-1)
    np.testing.assert_allclose(C2, C6, rtol=0, atol=1e-11)


def test_cov_uses_index_rows():
    # swapping two neighbour rows must swap the covariance rows
    rng = np.random.default_rng(4)
    p = rng.uniform(0, 1, (100, 3)).astype(np.float32)
    idx = rng.integers(0, 100, (2, 5)).astype(np.int32)
    a = oracle.cov(p, idx, -1)
    b = oracle.cov(p, idx[::-1].copy(), -1)
    np.testing.assert_array_equal(a[::-1], b)


def test_cov_rejects_out_of_range_index():
    with pytest.raises(ValueError):
        oracle.cov(np.zeros((4, 3), np.float32), np.array([[0, 4]], np.int32), -1)


# ---------------------------------------------------------------- regularised
def test_regularised_exact_plane_is_diag_11eps():
    rng = np.random.default_rng(9)
    xy = rng.uniform(0, 1, (30, 2))
    g = np.c_[xy, np.zeros(30)].astype(np.float32)
    eps = 1e-3
    Cp = _cov_of_all(g, eps)
    np.testing.assert_allclose(Cp, np.diag([1.0, 1.0, eps]), atol=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_regularised_rotated_plane_normal(seed):
    rng = np.random.default_rng(100 + seed)
    nrm = rng.standard_normal(3)
    nrm /= np.linalg.norm(nrm)
    a = np.cross(nrm, [1.0, 0, 0] if abs(nrm[0]) < 0.9 else [0, 1.0, 0])
    a /= np.linalg.norm(a)
    b = np.cross(nrm, a)
    uv = rng.uniform(-1, 1, (40, 2))
    g = (uv[:, :1] * a + uv[:, 1:] * b + 5.0).astype(np.float32)
    eps = 1e-3
    Cp = _cov_of_all(g, eps)
    want = np.eye(3) - (1 - eps) * np.outer(nrm, nrm)
    # binary32 input rounding tilts the plane by ~1e-7
    np.testing.assert_allclose(Cp, want, atol=2e-6)


def test_regularised_matches_numpy_eigh():
    rng = np.random.default_rng(12)
    p = rng.uniform(0, 5, (500, 3)).astype(np.float32)
    p[:, 2] *= 0.1  # flattened, so lambda_min is simple
    idx = rng.integers(0, 500, (200, 20)).astype(np.int32)
    raw = oracle.unpack6(oracle.cov(p, idx, -1))
    reg = oracle.unpack6(oracle.cov(p, idx, 0.01))
    for n in range(200):
        w, V = np.linalg.eigh(raw[n])
        assert (w[1] - w[0]) > 1e-6
        nv = V[:, 0]
        want = np.eye(3) - 0.99 * np.outer(nv, nv)
        np.testing.assert_allclose(reg[n], want, atol=1e-10)
        np.testing.assert_allclose(np.linalg.eigvalsh(reg[n]), [0.01, 1, 1], atol=1e-12)


def test_jacobi_against_eigh():
    rng = np.random.default_rng(13)
    for _ in range(200):
        A = rng.standard_normal((3, 3))
        A = A @ A.T * 10.0 ** rng.integers(-6, 3)
        c6 = np.array([A[0, 0], A[0, 1], A[0, 2], A[1, 1], A[1, 2], A[2, 2]])
        w, V = oracle.eig_sym3(c6)
        we = np.linalg.eigvalsh(A)
        np.testing.assert_allclose(w, we, rtol=1e-10, atol=1e-14 * np.abs(we).max())
        np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-12)
        np.testing.assert_allclose(A @ V, V * w, atol=1e-10 * np.abs(we).max())


def test_degenerate_single_point_neighbourhood():
    g = np.repeat(np.array([[1.5, -2.0, 3.0]], np.float32), 6, 0)
    np.testing.assert_array_equal(_cov_of_all(g, -1), np.zeros((3, 3)))
    np.testing.assert_allclose(_cov_of_all(g, 0.5), np.diag([1, 1, 0.5]), atol=0)


# ---------------------------------------------------------------- windowed search
def test_window_knn_pins():
    rng = np.random.default_rng(41)
    p = rng.integers(0, 6, (60, 3)).astype(np.float32)  # lattice: exact d2, ties
    q = rng.integers(0, 6, (15, 3)).astype(np.float32) + 0.5
    inf = np.float32(np.inf)
    # an infinite window is the whole map
    i0, d0 = oracle.knn_brute(q, p, 7)
    i1, d1 = oracle.knn_window(q, p, 7, [-inf] * 3, [inf] * 3)
    np.testing.assert_array_equal(i0, i1)
    np.testing.assert_array_equal(d0, d1)
    # a half-space window: pure-Python brute force over the kept points
    lo, hi = [-inf, 2.0, -inf], [inf, inf, 3.0]
    iw, dw = oracle.knn_window(q, p, 7, lo, hi)
    for n in range(len(q)):
        keys = sorted((float(((q[n] - p[j]).astype(np.float64) ** 2).sum()), j) for j in range(len(p))
                      if 2.0 <= p[j, 1] and p[j, 2] <= 3.0)
        assert [j for _, j in keys[:7]] == list(iw[n])
        assert all(p[j, 1] >= 2.0 and p[j, 2] <= 3.0 for j in iw[n])
    # fewer than k points in the window
    i2, d2 = oracle.knn_window(q, p, 7, [0, 0, 0], [0.5, 0.5, 0.5])
    assert (i2 == -1).all() and np.isinf(d2).all()
