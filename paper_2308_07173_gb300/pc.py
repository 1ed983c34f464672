"""Thin ctypes binding of libpc.so (include/pc.h).

The module-level ``pc_*`` functions mirror the C ABI one to one (argument
marshalling only: pointers, sizes, streams).  ``Target`` and ``Batch`` wrap
them for torch CUDA tensors.  PyTorch only provides device memory and
streams; every step of the computation runs in the library's kernels.

There is no fallback: if libpc.so cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpc.so")

PC_OK = 0
PC_ERR_INVALID_ARG = 1
PC_ERR_K_GT_M = 2
PC_ERR_NONFINITE = 3
PC_ERR_OOM = 4
PC_ERR_CUDA = 5
PC_ERR_SEARCH_LIMIT = 6
PC_ERR_BAD_POINTER = 7
PC_ERR_BAD_INDEX = 8
PC_ERR_DESTROYED = 9
PC_NOALLOC_MAX_SCANS = 256
PC_GICP_OUT = 29

_STATUS_NAMES = {
    0: "PC_OK",
    1: "PC_ERR_INVALID_ARG",
    2: "PC_ERR_K_GT_M",
    3: "PC_ERR_NONFINITE",
    4: "PC_ERR_OOM",
    5: "PC_ERR_CUDA",
    6: "PC_ERR_SEARCH_LIMIT",
    7: "PC_ERR_BAD_POINTER",
    8: "PC_ERR_BAD_INDEX",
    9: "PC_ERR_DESTROYED",
}


class PcError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = int(code)
        msg = _STATUS_NAMES.get(self.code, str(code))
        try:
            msg += ": " + _lib.pc_status_string(self.code).decode()
        except Exception:
            pass
        super().__init__(f"{where}: {msg}" if where else msg)


class pc_build_opts(ctypes.Structure):
    _fields_ = [
        ("cell_size", ctypes.c_float),
        ("occupancy", ctypes.c_float),
        ("hash_load", ctypes.c_float),
        ("max_box_cells", ctypes.c_int),
        ("exhaustive", ctypes.c_int),
    ]


class pc_cov_kernel(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("sigma", ctypes.c_float), ("alpha", ctypes.c_float),
                ("c", ctypes.c_float), ("d", ctypes.c_float)]


PC_KERNELS = {"none": 0, "rbf": 1, "gaussian": 2, "polynomial": 3, "hi": 4, "laplacian": 5}


class pc_wall_opts(ctypes.Structure):
    _fields_ = [("voxel", ctypes.c_float), ("cell2d", ctypes.c_float), ("min_votes", ctypes.c_int),
                ("tol", ctypes.c_float), ("min_cluster", ctypes.c_int), ("max_range", ctypes.c_float),
                ("max_height", ctypes.c_float)]


class pc_wall_result(ctypes.Structure):
    _fields_ = [("n_voxels", ctypes.c_int64), ("n_vertical", ctypes.c_int64), ("wall_label", ctypes.c_int64),
                ("wall_count", ctypes.c_int64), ("wall_length", ctypes.c_float), ("beta", ctypes.c_double * 3),
                ("d_w", ctypes.c_double)]


class pc_window(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3)]


class pc_tune(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("warps", ctypes.c_int), ("rho_scale", ctypes.c_float),
                ("order", ctypes.c_int), ("probe", ctypes.c_int), ("slots", ctypes.c_int)]


class pc_target_info(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64),
        ("ncells", ctypes.c_int64),
        ("table_cap", ctypes.c_int64),
        ("cell_size", ctypes.c_float),
        ("origin", ctypes.c_float * 3),
        ("bbox_max", ctypes.c_float * 3),
        ("dims", ctypes.c_int * 3),
        ("device_bytes", ctypes.c_int64),
        ("rho_hint", ctypes.c_float * 64),
        ("delta_m", ctypes.c_int64),
    ]


class pc_stats(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_int64), ("warp_search", ctypes.c_int64),
                ("exhaustive", ctypes.c_int64), ("candidates", ctypes.c_int64)]


class pc_scan(ctypes.Structure):
    _fields_ = [
        ("q_dev", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("idx_dev", ctypes.c_void_p),
        ("d2_dev", ctypes.c_void_p),
        ("cov_dev", ctypes.c_void_p),
    ]


# (name, restype, argtypes): the C ABI of include/pc.h
_VP, _I64, _INT, _F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float
SIGNATURES = {
    "pc_default_build_opts": (None, [ctypes.POINTER(pc_build_opts)]),
    "pc_build_target": (_INT, [_VP, _I64, ctypes.POINTER(pc_build_opts), _VP, ctypes.POINTER(_VP)]),
    "pc_destroy_target": (None, [_VP]),
    "pc_set_tune": (_INT, [_VP, ctypes.POINTER(pc_tune)]),
    "pc_get_info": (_INT, [_VP, ctypes.POINTER(pc_target_info)]),
    "pc_knn": (_INT, [_VP, _VP, _I64, _INT, _VP, _VP, _VP]),
    "pc_cov": (_INT, [_VP, _VP, _I64, _INT, _F, _VP, _VP]),
    "pc_knn_cov": (_INT, [_VP, _VP, _I64, _INT, _F, _VP, _VP, _VP, _VP]),
    "pc_knn_cov_host": (_INT, [_VP, _VP, _I64, _INT, _F, _VP, _VP, _VP, _VP]),
    "pc_sync_status": (_INT, [_VP, _VP]),
    "pc_get_stats": (_INT, [_VP, _VP, ctypes.POINTER(pc_stats), _INT]),
    "pc_batch_plan": (_INT, [_VP, ctypes.POINTER(pc_scan), _INT, _INT, _F, ctypes.POINTER(_VP)]),
    "pc_batch_run": (_INT, [_VP, _VP]),
    "pc_batch_destroy": (None, [_VP]),
    "pc_batch_run_noalloc": (_INT, [_VP, ctypes.POINTER(pc_scan), _INT, _INT, _F, _VP]),
    "pc_batch_scratch_bytes": (ctypes.c_size_t, [_INT]),
    "pc_batch_run_scratch": (_INT, [_VP, ctypes.POINTER(pc_scan), _INT, _INT, _F, _VP, ctypes.c_size_t, _VP]),
    "pc_set_window": (_INT, [_VP, ctypes.POINTER(pc_window)]),
    "pc_target_append": (_INT, [_VP, _VP, _I64, _VP]),
    "pc_target_compact": (_INT, [_VP, _VP]),
    "pc_set_cov_kernel": (_INT, [_VP, ctypes.POINTER(pc_cov_kernel)]),
    "pc_wall_default_opts": (None, [ctypes.POINTER(pc_wall_opts)]),
    "pc_wall_create": (_INT, [_I64, ctypes.POINTER(pc_wall_opts), ctypes.POINTER(_VP)]),
    "pc_wall_detect": (_INT, [_VP, _VP, _I64, _VP]),
    "pc_wall_get": (_INT, [_VP, _VP, ctypes.POINTER(pc_wall_result), _VP, _VP, _VP]),
    "pc_wall_destroy": (None, [_VP]),
    "pc_gicp_work_bytes": (ctypes.c_size_t, []),
    "pc_gicp_linearize": (_INT, [_VP, _VP, _VP, _I64, _VP, _VP, _F, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "pc_gicp_update": (_INT, [_VP, _F, _VP, _VP, _VP]),
    "pc_status_string": (ctypes.c_char_p, [_INT]),
    "pc_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: Optional[str] = None, build_if_missing: bool = True):
    """Load libpc.so (building it in-tree with nvcc if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"libpc.so not built at {path}")
        from . import _build

        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != PC_OK:
        raise PcError(rc, where)


# ---------------------------------------------------------------- raw ABI
def pc_default_build_opts() -> pc_build_opts:
    o = pc_build_opts()
    load().pc_default_build_opts(ctypes.byref(o))
    return o


def pc_build_target(xyz_dev: int, M: int, opts: Optional[pc_build_opts], stream: int) -> int:
    h = ctypes.c_void_p()
    rc = load().pc_build_target(xyz_dev, M, ctypes.byref(opts) if opts is not None else None, stream, ctypes.byref(h))
    _check(rc, "pc_build_target")
    return h.value


def pc_destroy_target(t: int) -> None:
    load().pc_destroy_target(t)


def pc_set_tune(t: int, tune: Optional[pc_tune]) -> None:
    _check(load().pc_set_tune(t, ctypes.byref(tune) if tune is not None else None), "pc_set_tune")


def pc_get_info(t: int) -> pc_target_info:
    info = pc_target_info()
    _check(load().pc_get_info(t, ctypes.byref(info)), "pc_get_info")
    return info


def pc_knn(t, q_dev, N, k, idx_dev, d2_dev, stream) -> int:
    return load().pc_knn(t, q_dev, N, k, idx_dev, d2_dev, stream)


def pc_cov(t, idx_dev, N, k, eps, cov_dev, stream) -> int:
    return load().pc_cov(t, idx_dev, N, k, eps, cov_dev, stream)


def pc_knn_cov(t, q_dev, N, k, eps, idx_dev, d2_dev, cov_dev, stream) -> int:
    return load().pc_knn_cov(t, q_dev, N, k, eps, idx_dev, d2_dev, cov_dev, stream)


def pc_knn_cov_host(t, q_host, N, k, eps, idx_host, d2_host, cov_host, stream) -> int:
    return load().pc_knn_cov_host(t, q_host, N, k, eps, idx_host, d2_host, cov_host, stream)


def pc_sync_status(t, stream) -> int:
    return load().pc_sync_status(t, stream)


def pc_get_stats(t, stream, reset: bool = False) -> pc_stats:
    st = pc_stats()
    _check(load().pc_get_stats(t, stream, ctypes.byref(st), 1 if reset else 0), "pc_get_stats")
    return st


def pc_batch_plan(t, scans: Sequence[pc_scan], k: int, eps: float) -> int:
    arr = (pc_scan * len(scans))(*scans)
    h = ctypes.c_void_p()
    _check(load().pc_batch_plan(t, arr, len(scans), k, eps, ctypes.byref(h)), "pc_batch_plan")
    return h.value


def pc_batch_run(b, stream) -> int:
    return load().pc_batch_run(b, stream)


def pc_batch_run_noalloc(t, scans: Sequence[pc_scan], k: int, eps: float, stream) -> int:
    arr = (pc_scan * len(scans))(*scans)
    return load().pc_batch_run_noalloc(t, arr, len(scans), k, eps, stream)


def pc_batch_scratch_bytes(n_scans: int) -> int:
    return int(load().pc_batch_scratch_bytes(n_scans))


def pc_batch_run_scratch(t, scans: Sequence[pc_scan], k: int, eps: float, scratch_dev: int,
                         scratch_bytes: int, stream) -> int:
    arr = (pc_scan * len(scans))(*scans)
    return load().pc_batch_run_scratch(t, arr, len(scans), k, eps, scratch_dev, scratch_bytes, stream)


def pc_batch_run_scratch_array(t, arr, n: int, k: int, eps: float, scratch_dev: int, scratch_bytes: int,
                               stream) -> int:
    """pc_batch_run_scratch on a ready ctypes array of n pc_scan."""
    return load().pc_batch_run_scratch(t, arr, n, k, eps, scratch_dev, scratch_bytes, stream)


def pc_set_window(t, lo=None, hi=None) -> int:
    if lo is None:
        return load().pc_set_window(t, None)
    w = pc_window((ctypes.c_float * 3)(*[float(v) for v in lo]), (ctypes.c_float * 3)(*[float(v) for v in hi]))
    return load().pc_set_window(t, ctypes.byref(w))


def pc_set_cov_kernel(t, kernel: str = "none", sigma: float = 1.0, alpha: float = 1.0, c: float = 0.0,
                      d: float = 1.0) -> int:
    if kernel == "none":
        return load().pc_set_cov_kernel(t, None)
    kd = pc_cov_kernel(PC_KERNELS[kernel], sigma, alpha, c, d)
    return load().pc_set_cov_kernel(t, ctypes.byref(kd))


def pc_gicp_work_bytes() -> int:
    return int(load().pc_gicp_work_bytes())


def pc_gicp_linearize(t, map_cov_dev, src_dev, n, src_cov_dev, pose_dev, max_dist, out_dev, corr_dev,
                      work_dev, work_bytes, stream) -> int:
    return load().pc_gicp_linearize(t, map_cov_dev, src_dev, n, src_cov_dev, pose_dev, max_dist, out_dev,
                                    corr_dev, work_dev, work_bytes, stream)


def pc_gicp_update(lin_dev, lam, pose_dev, xi_dev, stream) -> int:
    return load().pc_gicp_update(lin_dev, lam, pose_dev, xi_dev, stream)


def pc_batch_destroy(b) -> None:
    load().pc_batch_destroy(b)


def pc_status_string(code: int) -> str:
    return load().pc_status_string(code).decode()


def pc_version() -> str:
    return load().pc_version().decode()


# ---------------------------------------------------------------- torch layer
def _torch():
    import torch

    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev_tensor(x, dtype, shape_tail, name):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and (x.dim() != 2 or x.shape[1] != shape_tail):
        raise ValueError(f"{name} must be [n,{shape_tail}]")
    return x


class Target:
    """A device-resident target (map) grid: kNN + covariance queries."""

    def __init__(self, xyz, cell_size: float = 0.0, occupancy: float = 0.0, hash_load: float = 0.0,
                 max_box_cells: int = 0, exhaustive: bool = True, stream=None):
        torch = _torch()
        xyz = _dev_tensor(xyz, torch.float32, 3, "xyz")
        o = pc_default_build_opts()
        if cell_size > 0:
            o.cell_size = cell_size
        if occupancy > 0:
            o.occupancy = occupancy
        if hash_load > 0:
            o.hash_load = hash_load
        if max_box_cells > 0:
            o.max_box_cells = max_box_cells
        o.exhaustive = 1 if exhaustive else 0
        self.device = xyz.device
        self.m = xyz.shape[0]
        self._h = None
        self._h = pc_build_target(xyz.data_ptr(), self.m, o, _stream_handle(stream))

    @property
    def handle(self) -> int:
        if self._h is None:
            raise PcError(PC_ERR_DESTROYED, "Target")
        return self._h

    def info(self) -> dict:
        i = pc_get_info(self.handle)
        return {
            "m": i.m,
            "ncells": i.ncells,
            "table_cap": i.table_cap,
            "cell_size": i.cell_size,
            "origin": list(i.origin),
            "bbox_max": list(i.bbox_max),
            "dims": list(i.dims),
            "device_bytes": i.device_bytes,
            "rho_hint": list(i.rho_hint),
            "delta_m": i.delta_m,
        }

    def set_tune(self, tile: int = 0, warps: int = 0, rho_scale: float = 0.0, order: int = 0, probe: int = 0,
                 slots: int = 0):
        pc_set_tune(self.handle, pc_tune(tile, warps, rho_scale, order, probe, slots))

    def knn(self, q, k: int, idx=None, d2=None, stream=None):
        torch = _torch()
        q = _dev_tensor(q, torch.float32, 3, "q")
        n = q.shape[0]
        idx = idx if idx is not None else torch.empty((n, k), dtype=torch.int32, device=q.device)
        d2 = d2 if d2 is not None else torch.empty((n, k), dtype=torch.float32, device=q.device)
        _check(pc_knn(self.handle, q.data_ptr(), n, k, idx.data_ptr(), d2.data_ptr(), _stream_handle(stream)), "pc_knn")
        return idx, d2

    def cov(self, idx, eps: float, cov=None, stream=None):
        torch = _torch()
        idx = _dev_tensor(idx, torch.int32, None, "idx")
        n, k = idx.shape
        cov = cov if cov is not None else torch.empty((n, 6), dtype=torch.float32, device=idx.device)
        _check(pc_cov(self.handle, idx.data_ptr(), n, k, float(eps), cov.data_ptr(), _stream_handle(stream)), "pc_cov")
        return cov

    def knn_cov(self, q, k: int, eps: float, idx=None, d2=None, cov=None, stream=None):
        torch = _torch()
        q = _dev_tensor(q, torch.float32, 3, "q")
        n = q.shape[0]
        dev = q.device
        idx = idx if idx is not None else torch.empty((n, k), dtype=torch.int32, device=dev)
        d2 = d2 if d2 is not None else torch.empty((n, k), dtype=torch.float32, device=dev)
        cov = cov if cov is not None else torch.empty((n, 6), dtype=torch.float32, device=dev)
        rc = pc_knn_cov(self.handle, q.data_ptr(), n, k, float(eps), idx.data_ptr(), d2.data_ptr(),
                        cov.data_ptr(), _stream_handle(stream))
        _check(rc, "pc_knn_cov")
        return idx, d2, cov

    def knn_cov_host(self, q: np.ndarray, k: int, eps: float, out=None, stream=None):
        """Host buffers in and out (pinned torch CPU tensors or numpy arrays)."""
        torch = _torch()
        if isinstance(q, torch.Tensor):
            assert q.device.type == "cpu" and q.dtype == torch.float32 and q.is_contiguous()
            n = q.shape[0]
            qp = q.data_ptr()
            if out is None:
                out = (torch.empty((n, k), dtype=torch.int32), torch.empty((n, k), dtype=torch.float32),
                       torch.empty((n, 6), dtype=torch.float32))
            ptrs = [o.data_ptr() for o in out]
        else:
            q = np.ascontiguousarray(q, dtype=np.float32)
            n = q.shape[0]
            qp = q.ctypes.data
            if out is None:
                out = (np.empty((n, k), np.int32), np.empty((n, k), np.float32), np.empty((n, 6), np.float32))
            ptrs = [o.ctypes.data for o in out]
        rc = pc_knn_cov_host(self.handle, qp, n, k, float(eps), ptrs[0], ptrs[1], ptrs[2], _stream_handle(stream))
        _check(rc, "pc_knn_cov_host")
        return out

    def set_cov_kernel(self, kernel: str = "none", sigma: float = 1.0, alpha: float = 1.0, c: float = 0.0,
                       d: float = 1.0):
        """Weight the covariances of later fused searches by a kernel
        descriptor of Table I ('rbf', 'gaussian', 'polynomial', 'hi',
        'laplacian'); 'none' restores the plain covariance."""
        _check(pc_set_cov_kernel(self.handle, kernel, sigma, alpha, c, d), "pc_set_cov_kernel")

    def append(self, xyz, stream=None):
        """Add points to the map without rebuilding its grid (indices continue
        after the existing ones)."""
        torch = _torch()
        xyz = _dev_tensor(xyz, torch.float32, 3, "xyz")
        _check(load().pc_target_append(self.handle, xyz.data_ptr(), xyz.shape[0], _stream_handle(stream)),
               "pc_target_append")
        self.m_appended = getattr(self, "m_appended", 0) + xyz.shape[0]

    def compact(self, stream=None):
        """Fold appended points into a rebuilt main grid."""
        _check(load().pc_target_compact(self.handle, _stream_handle(stream)), "pc_target_compact")

    def set_window(self, lo=None, hi=None):
        """Restrict later searches to the map points in the box [lo, hi]
        (sliding-window submap); no arguments restore the whole map."""
        _check(pc_set_window(self.handle, lo, hi), "pc_set_window")

    def gicp_work(self):
        """A device workspace for gicp_linearize (kept on the handle; calls
        that share it must not overlap on the GPU)."""
        torch = _torch()
        if getattr(self, "_gicp_work", None) is None:
            nb = pc_gicp_work_bytes()
            if nb <= 0:
                raise PcError(PC_ERR_CUDA, "pc_gicp_work_bytes")
            self._gicp_work = torch.zeros(nb, dtype=torch.uint8, device=self.device)
        return self._gicp_work

    def gicp_linearize(self, map_cov, src, src_cov, pose, max_dist: float, out=None, corr=None, work=None,
                       stream=None):
        """One GICP linearisation against this target (the map): returns the
        f64 [29] device tensor (H upper triangle, b, E, pairs) and corr."""
        torch = _torch()
        map_cov = _dev_tensor(map_cov, torch.float32, 6, "map_cov")
        src = _dev_tensor(src, torch.float32, 3, "src")
        src_cov = _dev_tensor(src_cov, torch.float32, 6, "src_cov")
        pose = _dev_tensor(pose, torch.float32, None, "pose")
        if pose.numel() != 12:
            raise ValueError("pose must hold 12 floats (R row-major, t)")
        n = src.shape[0]
        if map_cov.shape[0] != self.m + getattr(self, "m_appended", 0) or src_cov.shape[0] != n:
            raise ValueError("map_cov must be [M,6] for this target (appended points included) and src_cov [n,6]")
        out = out if out is not None else torch.empty(PC_GICP_OUT, dtype=torch.float64, device=src.device)
        work = work if work is not None else self.gicp_work()
        cp = corr.data_ptr() if corr is not None else None
        rc = pc_gicp_linearize(self.handle, map_cov.data_ptr(), src.data_ptr(), n, src_cov.data_ptr(),
                               pose.data_ptr(), float(max_dist), out.data_ptr(), cp, work.data_ptr(),
                               work.numel(), _stream_handle(stream))
        _check(rc, "pc_gicp_linearize")
        return out, corr

    def stats(self, reset: bool = False, stream=None) -> dict:
        st = pc_get_stats(self.handle, _stream_handle(stream), reset)
        return {"queries": st.queries, "warp_search": st.warp_search, "exhaustive": st.exhaustive,
                "candidates": st.candidates}

    def sync_status(self, stream=None) -> int:
        return pc_sync_status(self.handle, _stream_handle(stream))

    def close(self):
        if self._h is not None:
            pc_destroy_target(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many scans, one launch replayed as a CUDA graph."""

    def __init__(self, target: Target, scans, k: int, eps: float):
        """scans: list of (q [n,3] f32, idx [n,k] i32, d2 [n,k] f32, cov [n,6] f32 or None)."""
        self.target = target
        self._keep = list(scans)
        descs = []
        for q, idx, d2, cov in scans:
            descs.append(pc_scan(q.data_ptr(), q.shape[0], idx.data_ptr(), d2.data_ptr(),
                                 cov.data_ptr() if cov is not None else None))
        self._h = None
        self._h = pc_batch_plan(target.handle, descs, k, eps)

    def run(self, stream=None):
        _check(pc_batch_run(self._h, _stream_handle(stream)), "pc_batch_run")

    def close(self):
        if self._h is not None:
            pc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WallDetector:
    """Ground filter, wall clustering and wall fit for scans in the vehicle
    body frame (pc_wall_*, Sec. III-D)."""

    def __init__(self, max_points: int, **opts):
        o = pc_wall_opts()
        load().pc_wall_default_opts(ctypes.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        h = ctypes.c_void_p()
        _check(load().pc_wall_create(int(max_points), ctypes.byref(o), ctypes.byref(h)), "pc_wall_create")
        self._h = h.value
        self.max_points = int(max_points)

    def detect(self, pts, stream=None):
        torch = _torch()
        pts = _dev_tensor(pts, torch.float32, 3, "pts")
        _check(load().pc_wall_detect(self._h, pts.data_ptr(), pts.shape[0], _stream_handle(stream)), "pc_wall_detect")

    def result(self, arrays: bool = False, stream=None) -> dict:
        r = pc_wall_result()
        st = load().pc_wall_get(self._h, _stream_handle(stream), ctypes.byref(r), None, None, None)
        if st not in (PC_OK, PC_ERR_SEARCH_LIMIT):
            _check(st, "pc_wall_get")
        out = {"n_voxels": r.n_voxels, "n_vertical": r.n_vertical, "wall_label": r.wall_label,
               "wall_count": r.wall_count, "wall_length": r.wall_length, "beta": list(r.beta), "d_w": r.d_w,
               "status": st}
        if arrays and r.n_voxels > 0:
            n = r.n_voxels
            cent = np.empty((n, 3), np.float32)
            vert = np.empty(n, np.int32)
            lab = np.empty(n, np.int32)
            st = load().pc_wall_get(self._h, _stream_handle(stream), ctypes.byref(r), cent.ctypes.data,
                                    vert.ctypes.data, lab.ctypes.data)
            out.update(centroids=cent, vertical=vert.astype(bool), labels=lab, status=st)
        return out

    def close(self):
        if self._h:
            load().pc_wall_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
