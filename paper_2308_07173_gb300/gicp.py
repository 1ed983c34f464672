"""Scan-to-map GICP registration on the device (Sec. III-C1, Eq. 18-20).

The per-point Gaussians come from the search kernels (map covariances once
per map, source covariances once per scan); each iteration is one
``pc_gicp_linearize`` launch (exact nearest-point correspondences, the
combined covariance and the 6x6 normal equations) and one ``pc_gicp_update``
launch (binary64 Cholesky solve and the pose update on the device).  The
iterations queue on one stream with no host round trip; with ``graph=True``
they are captured once and replayed.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import pc


def unpack_lin(lin) -> dict:
    """29 doubles -> {H [6,6], b [6], error, pairs} (numpy)."""
    v = np.asarray(lin, dtype=np.float64).reshape(29)
    H = np.zeros((6, 6))
    H[np.triu_indices(6)] = v[:21]
    H = H + np.triu(H, 1).T
    return {"H": H, "b": v[21:27].copy(), "error": float(v[27]), "pairs": int(round(v[28]))}


def pose_tensor(R=None, t=None, device="cuda"):
    """A device pose [12] (R row-major, t) from numpy-like R [3,3], t [3]."""
    import torch

    R = np.eye(3) if R is None else np.asarray(R, np.float64)
    t = np.zeros(3) if t is None else np.asarray(t, np.float64)
    return torch.tensor(np.concatenate([R.ravel(), t]).astype(np.float32), device=device)


class Registration:
    """Registers scans against one map: holds the map target, the map
    covariances and the device buffers of a fixed number of iterations."""

    def __init__(self, map_xyz, k: int = 20, eps: float = 1e-3, map_cov=None, target: Optional[pc.Target] = None,
                 **build):
        import torch

        self.k, self.eps = int(k), float(eps)
        self.map = target if target is not None else pc.Target(map_xyz, **build)
        if map_cov is None:
            _, _, map_cov = self.map.knn_cov(map_xyz, self.k, self.eps)
        self.map_cov = map_cov
        self.device = map_xyz.device
        self.work = self.map.gicp_work()
        self._graph = None
        self._graph_key = None

    def source_covariances(self, src):
        """Covariances of the scan's own neighbourhoods (a target built from
        the scan, queried with the scan)."""
        st = pc.Target(src)
        try:
            _, _, cov = st.knn_cov(src, self.k, self.eps)
        finally:
            st.close()
        return cov

    def _queue(self, src, src_cov, pose, lin, xi, max_dist, lam, iters, stream):
        for i in range(iters):
            self.map.gicp_linearize(self.map_cov, src, src_cov, pose, max_dist, out=lin[i], work=self.work,
                                    stream=stream)
            pc._check(pc.pc_gicp_update(lin[i].data_ptr(), float(lam), pose.data_ptr(), xi[i].data_ptr(),
                                        pc._stream_handle(stream)), "pc_gicp_update")

    def align(self, src, src_cov, pose, iters: int = 10, max_dist: float = 1.0, lam: float = 0.0,
              graph: bool = False, stream=None):
        """Runs `iters` Gauss-Newton (lam = 0) or Levenberg-Marquardt
        iterations in place on the device pose [12]; returns (lin [iters,29],
        xi [iters,6]) device tensors (one row per iteration, read them when
        needed)."""
        import torch

        lin = torch.empty((iters, 29), dtype=torch.float64, device=self.device)
        xi = torch.empty((iters, 6), dtype=torch.float64, device=self.device)
        if not graph:
            self._queue(src, src_cov, pose, lin, xi, max_dist, lam, iters, stream)
            return lin, xi
        key = (src.data_ptr(), src_cov.data_ptr(), pose.data_ptr(), iters, float(max_dist), float(lam))
        if self._graph is None or self._graph_key != key:
            self._glin, self._gxi = lin, xi
            s = torch.cuda.Stream(device=self.device)
            s.wait_stream(torch.cuda.current_stream(self.device))
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                g.capture_begin(capture_error_mode="thread_local")
                self._queue(src, src_cov, pose, lin, xi, max_dist, lam, iters, s)
                g.capture_end()
            torch.cuda.current_stream(self.device).wait_stream(s)
            self._graph, self._graph_key = g, key
        self._graph.replay()
        return self._glin, self._gxi

    def close(self):
        self._graph = None
        self.map.close()
