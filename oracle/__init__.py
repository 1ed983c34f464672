"""CPU oracle for the kNN + covariance step (Sec. III-C1, Eq. 18-20).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module and shares no code with it.

Functions follow the plain definitions:

* ``knn_brute(q, p, k)``   -- every target's binary32 d2 in the pinned order
  ``fmaf(dz,dz,fmaf(dy,dy,dx*dx))``, first k under (d2, index) ascending.
* ``KDTree(p).knn(q, k)``  -- the same answer through a median-split k-d tree
  (pruning by a proven lower bound of the binary32 d2; ties still visited).
* ``cov(p, idx, eps)``     -- binary64 neighbourhood covariance with 1/k, and
  for eps >= 0 the plane regularisation C' = I - (1-eps) n n^T with n the
  smallest-eigenvalue eigenvector (cyclic Jacobi).
* ``eig_sym3(c6)``         -- the Jacobi eigen-solver on its own.
* ``cov_weighted``         -- the covariance with kernel-descriptor weights
  (Table I) on the neighbours.
* ``gicp_transform`` / ``gicp_linearize`` -- one Gauss-Newton linearisation
  of GICP (Eq. 18-20) in binary64 on top of the nearest-point search.
* ``window_mask`` / ``knn_window`` -- the search restricted to a box of the
  map (sliding-window submap, Sec. III-C3).
* ``wall_detect``          -- voxel filter, 2-D vote ground filter, Euclidean
  clustering and the wall's quadratic fit (Sec. III-D).
* ``gicp_update`` / ``so3_exp`` -- the step that follows it: solve
  (H + lam I) xi = -b, move the pose by Exp(omega) on the left.

Parity of the covariance against the paper's own numbers is unpinned: the
paper prints no worked example.  ``cov_weighted`` is also parity unpinned
against the paper, which never says how a kernel descriptor enters the
covariance: it fixes one reading (weights in the moments), pinned only by
closed forms of that reading.  The pins live in ``tests/test_oracle_pins.py``
(closed forms, invariants, exact rational arithmetic, library
cross-checks), ``tests/test_oracle_gicp.py`` (finite differences, a
Sherman-Morrison case, pose recovery), ``tests/test_oracle_kernels.py`` and
``tests/test_oracle_wall.py`` (exact means, vote separation, breadth-first
clustering, parabola recovery).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, no CUDA)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        vp = ctypes.c_void_p
        lib.oracle_knn_brute.argtypes = [vp, i64, vp, i64, i32, vp, vp, i32]
        lib.oracle_knn_brute.restype = i32
        lib.oracle_kdtree_build.argtypes = [vp, i64]
        lib.oracle_kdtree_build.restype = vp
        lib.oracle_kdtree_free.argtypes = [vp]
        lib.oracle_kdtree_free.restype = None
        lib.oracle_kdtree_knn.argtypes = [vp, vp, i64, i32, vp, vp, i32]
        lib.oracle_kdtree_knn.restype = i32
        lib.oracle_cov.argtypes = [vp, i64, vp, i64, i32, f64, vp, i32]
        lib.oracle_cov.restype = i32
        lib.oracle_eig_sym3.argtypes = [vp, vp, vp]
        lib.oracle_eig_sym3.restype = None
        lib.oracle_gicp_linearize.argtypes = [vp, vp, vp, i64, vp, vp, ctypes.c_float, vp, vp, i32]
        lib.oracle_gicp_linearize.restype = i32
        lib.oracle_cov_weighted.argtypes = [vp, i64, vp, vp, i64, i32, f64, i32, vp, vp, vp]
        lib.oracle_cov_weighted.restype = i32
        lib.oracle_wall_detect.argtypes = [vp, i64, ctypes.c_float, ctypes.c_float, i32, ctypes.c_float, i32,
                                           ctypes.c_float, ctypes.c_float, vp, vp, vp, vp, vp, vp]
        lib.oracle_wall_detect.restype = i64
        lib.oracle_gicp_transform.argtypes = [vp, vp, i64, vp]
        lib.oracle_gicp_transform.restype = None
        lib.oracle_default_threads.argtypes = []
        lib.oracle_default_threads.restype = i32
        _lib = lib
    return _lib


def default_threads() -> int:
    return int(_load().oracle_default_threads())


def _f32x3(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("points must be [n,3] float32")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def knn_brute(q, p, k: int, threads: int = 0):
    """Exact kNN by definition: returns (idx int32 [n,k], d2 float32 [n,k])."""
    q, p = _f32x3(q), _f32x3(p)
    n, m = q.shape[0], p.shape[0]
    idx = np.empty((n, k), np.int32)
    d2 = np.empty((n, k), np.float32)
    rc = _load().oracle_knn_brute(_ptr(q), n, _ptr(p), m, int(k), _ptr(idx), _ptr(d2), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_knn_brute: bad arguments (k={k}, m={m})")
    return idx, d2


class KDTree:
    """Median-split k-d tree over p; answers equal knn_brute bit for bit."""

    def __init__(self, p):
        self._p = _f32x3(p)  # the tree keeps a pointer into this array
        self.m = self._p.shape[0]
        self._h = _load().oracle_kdtree_build(_ptr(self._p), self.m)
        if not self._h:
            raise ValueError("empty target")

    def knn(self, q, k: int, threads: int = 0):
        q = _f32x3(q)
        n = q.shape[0]
        idx = np.empty((n, k), np.int32)
        d2 = np.empty((n, k), np.float32)
        rc = _load().oracle_kdtree_knn(self._h, _ptr(q), n, int(k), _ptr(idx), _ptr(d2), int(threads))
        if rc != 0:
            raise ValueError(f"oracle_kdtree_knn: bad arguments (k={k}, m={self.m})")
        return idx, d2

    def close(self):
        if self._h:
            _load().oracle_kdtree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gicp_transform(pose, src) -> np.ndarray:
    """p' = R p + t in binary32 with the pinned order
    fmaf(R_a2, p_z, fmaf(R_a1, p_y, fmaf(R_a0, p_x, t_a))); pose = (R 3x3
    row-major, t 3)."""
    pose = np.ascontiguousarray(pose, dtype=np.float32).reshape(12)
    src = _f32x3(src)
    out = np.empty_like(src)
    _load().oracle_gicp_transform(_ptr(pose), _ptr(src), src.shape[0], _ptr(out))
    return out


def gicp_linearize(tree: "KDTree", map_cov, src, src_cov, pose, max_dist: float, threads: int = 0) -> dict:
    """One Gauss-Newton linearisation of GICP (Eq. 18-20) in binary64: the
    source points moved by pose (gicp_transform), each paired with its nearest
    map point of tree when d2 <= fl(max_dist^2), Omega = (C_q + R C_p R^T)^-1,
    H = sum J^T Omega J, b = sum J^T Omega d, E = sum d^T Omega d with
    d = q - p' and J = [[p']_x, -I] (left perturbation, xi = (omega, v)).
    Returns {H [6,6], b [6], error, pairs, corr [n] (map index or -1)}."""
    map_cov = np.ascontiguousarray(map_cov, dtype=np.float32)
    src = _f32x3(src)
    src_cov = np.ascontiguousarray(src_cov, dtype=np.float32)
    if map_cov.shape != (tree.m, 6) or src_cov.shape != (src.shape[0], 6):
        raise ValueError("covariances must be [m,6] and [n,6]")
    pose = np.ascontiguousarray(pose, dtype=np.float32).reshape(12)
    out = np.empty(29, np.float64)
    corr = np.empty(src.shape[0], np.int32)
    rc = _load().oracle_gicp_linearize(tree._h, _ptr(map_cov), _ptr(src), src.shape[0], _ptr(src_cov), _ptr(pose),
                                       float(max_dist), _ptr(out), _ptr(corr), int(threads))
    if rc != 0:
        raise ValueError("oracle_gicp_linearize: bad arguments")
    H = np.zeros((6, 6))
    H[np.triu_indices(6)] = out[:21]
    H = H + np.triu(H, 1).T
    return {"H": H, "b": out[21:27].copy(), "error": float(out[27]), "pairs": int(out[28]), "corr": corr}


def window_mask(p, lo, hi) -> np.ndarray:
    """Map points inside the box [lo, hi] (componentwise, binary32
    comparisons): the sliding-window submap of Sec. III-C3."""
    p = _f32x3(p)
    lo = np.asarray(lo, np.float32).reshape(3)
    hi = np.asarray(hi, np.float32).reshape(3)
    return np.all((p >= lo) & (p <= hi), axis=1)


def knn_window(q, p, k: int, lo, hi, threads: int = 0):
    """kNN over the submap {p in [lo, hi]} with indices into the whole map:
    the plain definition applied to the submap (its points keep their
    relative order, so ties still go to the lower whole-map index).  Rows
    get -1 / +inf when the submap holds fewer than k points."""
    q, p = _f32x3(q), _f32x3(p)
    sel = np.nonzero(window_mask(p, lo, hi))[0]
    n = q.shape[0]
    if len(sel) < k:
        return np.full((n, k), -1, np.int32), np.full((n, k), np.inf, np.float32)
    sub = p[sel]
    if len(sel) * max(n, 1) <= 50_000_000:
        i, d = knn_brute(q, sub, k, threads)
    else:
        t = KDTree(sub)
        i, d = t.knn(q, k, threads)
        t.close()
    return sel[i].astype(np.int32), d


def wall_detect(pts, voxel: float = 0.2, cell2d: float = 0.5, min_votes: int = 3, tol: float = 0.5,
                min_cluster: int = 10, max_range: float = 128.0, max_height: float = 16.0) -> dict:
    """Ground filter by 2-D voting, Euclidean clustering of the vertical
    voxels and the wall's quadratic fit (Sec. III-D, Eq. 24-30): see
    oracle_wall_detect in oracle.c for the exact definition."""
    pts = _f32x3(pts)
    n = pts.shape[0]
    cent = np.empty((max(n, 1), 3), np.float32)
    vert = np.empty(max(n, 1), np.int32)
    lab = np.empty(max(n, 1), np.int64)
    wl = np.zeros(1, np.int64)
    wc = np.zeros(1, np.int64)
    beta = np.empty(3, np.float64)
    nv = _load().oracle_wall_detect(_ptr(pts), n, voxel, cell2d, int(min_votes), tol, int(min_cluster), max_range,
                                    max_height, _ptr(cent), _ptr(vert), _ptr(lab), _ptr(wl), _ptr(beta), _ptr(wc))
    if nv < 0:
        raise ValueError("oracle_wall_detect: bad arguments")
    return {"centroids": cent[:nv].copy(), "vertical": vert[:nv].astype(bool), "labels": lab[:nv].copy(),
            "wall_label": int(wl[0]), "wall_count": int(wc[0]), "beta": beta.copy(), "d_w": float(beta[0])}


def so3_exp(w) -> np.ndarray:
    """Rotation matrix of the rotation vector w by the Rodrigues formula
    I + sin(th)/th [w]_x + (1 - cos(th))/th^2 [w]_x^2 (binary64)."""
    w = np.asarray(w, np.float64).reshape(3)
    th = float(np.sqrt(w @ w))
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]], np.float64)
    if th == 0.0:
        return np.eye(3)
    return np.eye(3) + np.sin(th) / th * K + (1.0 - np.cos(th)) / (th * th) * (K @ K)


def gicp_update(pose, H, b, lam: float = 0.0):
    """The Gauss-Newton (lam = 0) or Levenberg-Marquardt step after a
    linearisation: xi = (H + lam I)^-1 (-b), then R <- Exp(omega) R,
    t <- Exp(omega) t + v (xi = (omega, v)).  Returns (pose float32 [12],
    xi float64 [6]); pose rounded once from binary64."""
    pose = np.asarray(pose, np.float32).reshape(12).astype(np.float64)
    A = np.asarray(H, np.float64) + float(lam) * np.eye(6)
    xi = np.linalg.solve(A, -np.asarray(b, np.float64))
    E = so3_exp(xi[:3])
    R = pose[:9].reshape(3, 3)
    t = pose[9:]
    return np.concatenate([(E @ R).ravel(), E @ t + xi[3:]]).astype(np.float32), xi


def cov(p, idx, eps: float, threads: int = 0) -> np.ndarray:
    """binary64 covariance (eps < 0) or regularised covariance (eps >= 0) of
    each neighbourhood row of idx over the target p: float64 [n,6] packed
    (xx, xy, xz, yy, yz, zz)."""
    p = _f32x3(p)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if idx.ndim != 2:
        raise ValueError("idx must be [n,k]")
    n, k = idx.shape
    out = np.empty((n, 6), np.float64)
    rc = _load().oracle_cov(_ptr(p), p.shape[0], _ptr(idx), n, k, float(eps), _ptr(out), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_cov: bad arguments (rc={rc})")
    return out


KERNELS = {"none": 0, "rbf": 1, "gaussian": 2, "polynomial": 3, "hi": 4, "laplacian": 5}


def cov_weighted(p, q, idx, eps: float, kernel: str, sigma: float = 1.0, alpha: float = 1.0, c: float = 0.0,
                 d: float = 1.0, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Kernel-descriptor weighted covariance (Sec. III-C1, Table I): weights
    w_j = K(q, p_j) on the neighbours of each row, weighted mean and moments,
    then the plane regularisation for eps >= 0; binary64 [n,6].  Polynomial
    and HI take coordinates relative to `origin` (the target's bounding-box
    minimum).  Rows with a non-positive total weight are NaN."""
    p, q = _f32x3(p), _f32x3(q)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n, k = idx.shape
    if q.shape[0] != n:
        raise ValueError("q and idx rows differ")
    prm = np.array([sigma, alpha, c, d], np.float64)
    o = np.ascontiguousarray(origin, dtype=np.float64).reshape(3)
    out = np.empty((n, 6), np.float64)
    rc = _load().oracle_cov_weighted(_ptr(p), p.shape[0], _ptr(q), _ptr(idx), n, k, float(eps), KERNELS[kernel],
                                     _ptr(prm), _ptr(o), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_cov_weighted: bad arguments (rc={rc})")
    return out


def eig_sym3(c6):
    """Jacobi eigen-decomposition of one packed symmetric 3x3: (w ascending,
    V with eigenvectors as columns)."""
    a = np.ascontiguousarray(c6, dtype=np.float64).reshape(6)
    w = np.empty(3, np.float64)
    V = np.empty((3, 3), np.float64)
    _load().oracle_eig_sym3(_ptr(a), _ptr(w), _ptr(V))
    return w, V


def unpack6(c6) -> np.ndarray:
    """[...,6] packed upper triangle -> [...,3,3] symmetric matrices."""
    c6 = np.asarray(c6)
    xx, xy, xz, yy, yz, zz = (c6[..., i] for i in range(6))
    return np.stack(
        [np.stack([xx, xy, xz], -1), np.stack([xy, yy, yz], -1), np.stack([xz, yz, zz], -1)], -2
    )
