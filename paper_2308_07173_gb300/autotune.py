"""Tuner for the search kernel's free parameters, with a JSON cache.

None of the parameters changes a result bit (the search is exact for any
cell size, launch shape or starting radius), so the tuner only times them:

* occupancy -- target mean points per occupied cell, which sets the cell
  edge h of the voxel-hash grid (the target is rebuilt per value);
* rho_scale -- the starting radius as a multiple of the calibrated k-th
  neighbour distance (the lane path's trial radii scale with it);
* warps -- warps per block; tile (queries per warp item) stays 32, one per
  lane of the lane path.

Each configuration is timed with CUDA events on the launching stream, L2
flushed (a 256 MB write) before every timed call, and its outputs are
compared bit for bit with the first configuration's.  The best result is
cached per (GPU, k, target size, query count) in a JSON file.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Iterable, Optional

from . import pc

FLUSH_BYTES = 256 << 20


PKG = os.path.dirname(os.path.abspath(__file__))


def default_cache() -> str:
    """The package's cache of tuned configurations (JSON), consulted by the
    batched and served forms when they are given no configuration."""
    return os.path.join(PKG, "tune_cache.json")


def n_bucket(n: int) -> int:
    """Query counts share a cache entry within a power of two (0: any)."""
    n = int(n)
    return 0 if n <= 0 else 1 << (n - 1).bit_length()


def _key(k: int, m: int, n: int) -> str:
    import torch

    name = torch.cuda.get_device_name().replace(" ", "_")
    return f"{name}|k{k}|m{m}|n{n_bucket(n)}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def lookup(path: str, k: int, m: int, n: int) -> Optional[dict]:
    return load_cache(path).get(_key(k, m, n))


def _time_call(fn, flush, reps: int) -> float:
    import torch

    for _ in range(3):
        fn()
    evs = []
    for _ in range(reps):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    v = sorted(x.elapsed_time(y) for x, y in evs)
    return v[len(v) // 2]


def tune(map_xyz, queries, k: int, eps: float, occupancies: Iterable[float] = (8, 12, 16),
         rho_scales: Iterable[float] = (0.8, 0.9, 1.0), warps: Iterable[int] = (2, 4, 8),
         reps: int = 15, cache: Optional[str] = None) -> dict:
    """Time every combination on (map_xyz [M,3], queries [N,3]) CUDA float32
    tensors; returns the best {occupancy, rho_scale, warps, tile, ms} plus
    the whole grid, and stores the best in `cache` if given."""
    import torch

    n = queries.shape[0]
    dev = queries.device
    idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    d2 = torch.empty((n, k), dtype=torch.float32, device=dev)
    cov = torch.empty((n, 6), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ref = None
    grid = []
    for occ in occupancies:
        t = pc.Target(map_xyz, occupancy=float(occ))
        h = t.info()["cell_size"]
        for rs, w in itertools.product(rho_scales, warps):
            t.set_tune(32, int(w), float(rs))
            ms = _time_call(lambda: t.knn_cov(queries, k, eps, idx, d2, cov), flush, reps)
            out = (idx.clone(), d2.view(torch.int32).clone(), cov.view(torch.int32).clone())
            if ref is None:
                ref = out
            elif not all(torch.equal(a, b) for a, b in zip(ref, out)):
                raise RuntimeError(f"results changed with occupancy={occ} rho_scale={rs} warps={w}")
            grid.append({"occupancy": float(occ), "cell_size": h, "rho_scale": float(rs), "warps": int(w),
                         "tile": 32, "ms": ms})
        t.close()
    best = dict(min(grid, key=lambda r: r["ms"]))
    if cache:
        data = load_cache(cache)
        data[_key(k, int(map_xyz.shape[0]), int(n))] = best
        tmp = cache + ".tmp"
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return {"best": best, "grid": grid}


def apply(map_xyz, cfg: dict) -> "pc.Target":
    """Build a target with a tuned configuration."""
    t = pc.Target(map_xyz, occupancy=cfg["occupancy"])
    t.set_tune(cfg.get("tile", 32), cfg["warps"], cfg["rho_scale"])
    return t
