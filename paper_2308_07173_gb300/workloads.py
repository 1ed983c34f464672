"""Seeded synthetic inputs standing in for the paper's race-track LiDAR data.

The paper's logs and datasets (IAC/HAC runs, the ES dataset, Monza) are not
available, so inputs are generated with the shapes of its workload: a
128-channel spinning LiDAR (Sec. IV-B, Ouster OS2-128; Sec. IV-E1 names
128-channel clouds as the case that needs the GPU) on an oval race track
with a flat ground plane and concrete barrier walls, queried against a map
of the same track.

This module holds geometry and random sampling only -- none of the search
or covariance arithmetic -- so tests can feed the same arrays to the CUDA
path and to the CPU oracle.  Every generator takes an explicit seed and
uses numpy's PCG64.

Track: a stadium oval, two straights of length ``ls`` joined by two
semicircles of centreline radius ``r``; lateral offset w in [-6, 6] m
(positive = away from the oval's centre); ground z = 0 over the band and
vertical walls of height 1 m at w = +-6 m.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- C1
def uniform_box(n: int = 8192, size=(40.0, 40.0, 4.0), seed: int = 1) -> np.ndarray:
    """n points uniform in [0,sx] x [0,sy] x [0,sz], float32 [n,3]."""
    g = rng_for(seed)
    return (g.random((n, 3)) * np.asarray(size)).astype(np.float32)


# ---------------------------------------------------------------- track
@dataclass
class Track:
    r: float = 100.0            # centreline radius of the bends
    length: float = 1500.0      # centreline length
    half_width: float = 6.0
    wall_h: float = 1.0
    pit: bool = False           # add the pit lane and garages (large-map stress case)
    pit_width: float = 15.0
    n_garages: int = 40

    @property
    def ls(self) -> float:
        return (self.length - 2.0 * math.pi * self.r) / 2.0

    # centreline pose at arc length s: position, tangent, outward normal
    def pose(self, s) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        s = np.mod(np.asarray(s, np.float64), self.length)
        ls, r = self.ls, self.r
        pos = np.zeros(s.shape + (2,))
        tan = np.zeros(s.shape + (2,))
        nrm = np.zeros(s.shape + (2,))
        a = s < ls
        pos[a] = np.stack([-ls / 2 + s[a], np.full(a.sum(), -r)], -1)
        tan[a] = [1.0, 0.0]
        nrm[a] = [0.0, -1.0]
        b = (s >= ls) & (s < ls + math.pi * r)
        phi = -math.pi / 2 + (s[b] - ls) / r
        pos[b] = np.stack([ls / 2 + r * np.cos(phi), r * np.sin(phi)], -1)
        tan[b] = np.stack([-np.sin(phi), np.cos(phi)], -1)
        nrm[b] = np.stack([np.cos(phi), np.sin(phi)], -1)
        c = (s >= ls + math.pi * r) & (s < 2 * ls + math.pi * r)
        u = s[c] - ls - math.pi * r
        pos[c] = np.stack([ls / 2 - u, np.full(c.sum(), r)], -1)
        tan[c] = [-1.0, 0.0]
        nrm[c] = [0.0, 1.0]
        d = s >= 2 * ls + math.pi * r
        phi = math.pi / 2 + (s[d] - 2 * ls - math.pi * r) / r
        pos[d] = np.stack([-ls / 2 + r * np.cos(phi), r * np.sin(phi)], -1)
        tan[d] = np.stack([-np.sin(phi), np.cos(phi)], -1)
        nrm[d] = np.stack([np.cos(phi), np.sin(phi)], -1)
        return pos, tan, nrm

    def lateral(self, x, y) -> np.ndarray:
        """Signed lateral offset of ground points from the centreline."""
        ls, r = self.ls, self.r
        w = np.full(np.shape(x), np.inf)
        mid = np.abs(x) <= ls / 2
        wb = -y - r  # bottom straight, outward = -y
        wt = y - r   # top straight, outward = +y
        w = np.where(mid & (np.abs(wb) <= np.abs(wt)), wb, w)
        w = np.where(mid & (np.abs(wt) < np.abs(wb)), wt, w)
        right = x > ls / 2
        w = np.where(right, np.hypot(x - ls / 2, y) - r, w)
        left = x < -ls / 2
        w = np.where(left, np.hypot(x + ls / 2, y) - r, w)
        return w

    # ---------------------------------------------------------------- map
    def sample_surface(self, n: int, g: np.random.Generator, noise: float = 0.0) -> np.ndarray:
        """n points area-uniform on the ground band and both walls."""
        ls, r, hw, wh = self.ls, self.r, self.half_width, self.wall_h
        ground_area = 2 * hw * self.length
        wall_area = 2 * self.length * wh  # inner + outer wall lengths sum to 2 x centreline
        n_ground = int(round(n * ground_area / (ground_area + wall_area)))
        n_wall = n - n_ground
        out = np.empty((n, 3), np.float64)
        # ground: straights by arc length, bends area-uniform in the annulus
        pg = np.empty((n_ground, 3))
        a_str = 2 * hw * 2 * ls
        k_str = g.random(n_ground) < a_str / ground_area
        ns = int(k_str.sum())
        s = g.random(ns) * 2 * ls
        s = np.where(s < ls, s, s - ls + ls + math.pi * r)  # map to the two straights
        pos, _, nrm = self.pose(s)
        w = (g.random(ns) * 2 - 1) * hw
        pg[k_str, :2] = pos + nrm * w[:, None]
        nb = n_ground - ns
        rr = np.sqrt(g.random(nb) * ((r + hw) ** 2 - (r - hw) ** 2) + (r - hw) ** 2)
        side = g.random(nb) < 0.5
        phi = (g.random(nb) - 0.5) * math.pi
        cx = np.where(side, ls / 2, -ls / 2)
        phi = np.where(side, phi, phi + math.pi)
        pg[~k_str, 0] = cx + rr * np.cos(phi)
        pg[~k_str, 1] = rr * np.sin(phi)
        pg[:, 2] = 0.0
        # walls: position along the wall length, both sides
        lin = 2 * ls + math.pi * (r - hw)   # inner wall length
        lout = 2 * ls + math.pi * (r + hw)  # outer wall length
        outer = g.random(n_wall) < lout / (lin + lout)
        t = g.random(n_wall)
        pw = np.empty((n_wall, 3))
        for is_outer, sign in ((True, 1.0), (False, -1.0)):
            sel = outer == is_outer
            rad = r + sign * hw
            L = 2 * ls + math.pi * rad
            u = t[sel] * L
            # walk the wall: straight, bend, straight, bend (same layout as the centreline)
            s_c = np.where(u < ls, u,
                           np.where(u < ls + math.pi * rad, ls + (u - ls) * r / rad,
                                    np.where(u < 2 * ls + math.pi * rad, u - math.pi * rad + math.pi * r,
                                             2 * ls + math.pi * r + (u - 2 * ls - math.pi * rad) * r / rad)))
            pos, _, nrm = self.pose(s_c)
            pw[sel, :2] = pos + nrm * (sign * hw)
        pw[:, 2] = g.random(n_wall) * wh
        out[:n_ground] = pg
        out[n_ground:] = pw
        if noise > 0:
            out += self._surface_normals(out) * g.normal(0.0, noise, (n, 1))
        return out

    def _surface_normals(self, p: np.ndarray) -> np.ndarray:
        nrm = np.zeros_like(p)
        ground = np.abs(p[:, 2]) < 1e-9
        nrm[ground, 2] = 1.0
        w = ~ground
        x, y = p[w, 0], p[w, 1]
        ls = self.ls
        n2 = np.zeros((w.sum(), 2))
        mid = np.abs(x) <= ls / 2
        n2[mid, 1] = 1.0
        right = x > ls / 2
        d = np.stack([x[right] - ls / 2, y[right]], -1)
        n2[right] = d / np.linalg.norm(d, axis=1, keepdims=True)
        left = x < -ls / 2
        d = np.stack([x[left] + ls / 2, y[left]], -1)
        n2[left] = d / np.linalg.norm(d, axis=1, keepdims=True)
        nrm[w, :2] = n2
        return nrm

    def sample_map(self, n: int, seed: int, noise: float = 0.0) -> np.ndarray:
        """Map points area-uniform on track surfaces (and, with pit=True,
        half of them on the pit lane structures); float32 [n,3]."""
        g = rng_for(seed)
        if not self.pit:
            return self.sample_surface(n, g, noise).astype(np.float32)
        n_track = n // 2
        track = self.sample_surface(n_track, g, noise)
        pit = self._sample_pit(n - n_track, g, noise)
        out = np.concatenate([track, pit])
        return out[g.permutation(len(out))].astype(np.float32)

    def _sample_pit(self, n: int, g: np.random.Generator, noise: float) -> np.ndarray:
        """Pit lane beside the top straight: a ground strip behind the outer
        wall, a 1 m pit wall, and garage boxes (back wall + side walls)."""
        ls, r, hw = self.ls, self.r, self.half_width
        y0 = r + hw                     # outer wall of the top straight
        y1 = y0 + self.pit_width        # pit wall
        box_w, box_d, box_h = 8.0, 6.0, 4.0
        span = ls * 0.8
        x0 = -span / 2
        gap = span / self.n_garages
        parts = []
        areas = np.array([span * self.pit_width, span * 1.0,
                          self.n_garages * box_w * box_h, self.n_garages * 2 * box_d * box_h])
        counts = g.multinomial(n, areas / areas.sum())
        # ground strip
        m = counts[0]
        parts.append(np.c_[x0 + g.random(m) * span, y0 + g.random(m) * self.pit_width, np.zeros(m)])
        nrm = [np.tile([0, 0, 1.0], (m, 1))]
        # pit wall (plane y = y1, height 1 m)
        m = counts[1]
        parts.append(np.c_[x0 + g.random(m) * span, np.full(m, y1), g.random(m) * 1.0])
        nrm.append(np.tile([0, 1.0, 0], (m, 1)))
        # garage back walls at y = y1 + box_d
        m = counts[2]
        i = g.integers(0, self.n_garages, m)
        parts.append(np.c_[x0 + i * gap + g.random(m) * box_w, np.full(m, y1 + box_d), g.random(m) * box_h])
        nrm.append(np.tile([0, 1.0, 0], (m, 1)))
        # garage side walls at x = left/right edge of each box
        m = counts[3]
        i = g.integers(0, self.n_garages, m)
        right = g.random(m) < 0.5
        parts.append(np.c_[x0 + i * gap + np.where(right, box_w, 0.0), y1 + g.random(m) * box_d,
                           g.random(m) * box_h])
        nrm.append(np.tile([1.0, 0, 0], (m, 1)))
        p = np.concatenate(parts)
        if noise > 0:
            p += np.concatenate(nrm) * g.normal(0.0, noise, (len(p), 1))
        return p

    # ---------------------------------------------------------------- scans
    def raycast(self, s0: float, w0: float, heading_dev: float, g: np.random.Generator,
                n_beams: int = 128, n_az: int = 1024, el_min_deg: float = -25.0,
                el_max_deg: float = 0.0, height: float = 0.8, max_range: float = 120.0,
                range_noise: float = 0.02) -> np.ndarray:
        """A spinning-LiDAR scan from the pose (arc length s0, lateral w0,
        heading = tangent + heading_dev), ray-cast in closed form against the
        ground band, wall planes (straights) and wall cylinders (bends).
        Returns world-frame float32 points in (beam, azimuth) order; rays
        with no hit within max_range are dropped."""
        ls, r, hw, wh = self.ls, self.r, self.half_width, self.wall_h
        pos, tan, nrm = self.pose(np.array([s0]))
        o = np.array([*(pos[0] + nrm[0] * w0), height])
        yaw0 = math.atan2(tan[0, 1], tan[0, 0]) + heading_dev
        el = np.deg2rad(np.linspace(el_min_deg, el_max_deg, n_beams))
        az = yaw0 + np.arange(n_az) * (2 * math.pi / n_az)
        E, A = np.meshgrid(el, az, indexing="ij")
        d = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
        n = d.shape[0]
        best = np.full(n, np.inf)
        # ground
        with np.errstate(divide="ignore", invalid="ignore"):
            tg = np.where(d[:, 2] < 0, -o[2] / d[:, 2], np.inf)
        hit = o[None, :] + np.where(np.isfinite(tg), tg, 0.0)[:, None] * d
        wg = self.lateral(hit[:, 0], hit[:, 1])
        ok = np.isfinite(tg) & (np.abs(wg) <= hw)
        best = np.where(ok, tg, best)
        # straight walls: planes y = -r -+ hw (bottom) and y = r -+ hw (top), |x| <= ls/2
        with np.errstate(divide="ignore", invalid="ignore"):
            for yw in (-r - hw, -r + hw, r - hw, r + hw):
                t = (yw - o[1]) / d[:, 1]
                p = o[None, :] + t[:, None] * d
                ok = (t > 1e-6) & (np.abs(p[:, 0]) <= ls / 2) & (p[:, 2] >= 0) & (p[:, 2] <= wh)
                best = np.where(ok & (t < best), t, best)
        # bend walls: cylinders of radius r -+ hw around (+-ls/2, 0)
        dxy2 = d[:, 0] ** 2 + d[:, 1] ** 2
        for cx, side in ((ls / 2, 1.0), (-ls / 2, -1.0)):
            ox, oy = o[0] - cx, o[1]
            bq = ox * d[:, 0] + oy * d[:, 1]
            for rad in (r - hw, r + hw):
                cq = ox * ox + oy * oy - rad * rad
                disc = bq * bq - dxy2 * cq
                sq = np.sqrt(np.maximum(disc, 0.0))
                for sgn in (-1.0, 1.0):
                    with np.errstate(divide="ignore", invalid="ignore"):
                        t = (-bq + sgn * sq) / dxy2
                    p = o[None, :] + t[:, None] * d
                    ok = ((disc >= 0) & (t > 1e-6) & (side * (p[:, 0] - cx) >= 0) & (p[:, 2] >= 0)
                          & (p[:, 2] <= wh))
                    best = np.where(ok & (t < best), t, best)
        keep = best <= max_range
        t = best[keep] + g.normal(0.0, range_noise, keep.sum())
        return (o[None, :] + t[:, None] * d[keep]).astype(np.float32)

    def random_pose(self, g: np.random.Generator, lateral: float = 4.0, heading_deg: float = 2.0):
        return (float(g.random() * self.length), float((g.random() * 2 - 1) * lateral),
                float(np.deg2rad((g.random() * 2 - 1) * heading_deg)))


def oval_1500() -> Track:
    return Track(r=100.0, length=1500.0)


def oval_4000_pit() -> Track:
    return Track(r=150.0, length=4000.0, pit=True)


# ---------------------------------------------------------------- workloads
def body_frame_scan(track: Optional[Track] = None, s0: float = 130.0, w0: float = 1.0, heading_dev: float = 0.0,
                    seed: int = 9) -> np.ndarray:
    """A ray-cast scan expressed in the vehicle body frame of its pose (x
    forward along the heading, y left, z up from the ground), float32."""
    tr = track or oval_1500()
    g = rng_for(seed)
    pts = tr.raycast(s0, w0, heading_dev, g).astype(np.float64)
    pos, tan, nrm = tr.pose(np.array([s0]))
    o = pos[0] + nrm[0] * w0
    yaw = math.atan2(tan[0, 1], tan[0, 0]) + heading_dev
    c, s_ = math.cos(yaw), math.sin(yaw)
    dx, dy = pts[:, 0] - o[0], pts[:, 1] - o[1]
    return np.c_[c * dx + s_ * dy, -s_ * dx + c * dy, pts[:, 2]].astype(np.float32)


def scan_vs_map(map_points: int = 2_000_000, map_seed: int = 2, scan_seed: int = 3,
                track: Optional[Track] = None):
    """One 128 x 1024 ray-cast scan at a random pose and the map it is queried
    against (131072 rays; drops make N a little smaller)."""
    tr = track or oval_1500()
    m = tr.sample_map(map_points, map_seed)
    g = rng_for(scan_seed)
    q = tr.raycast(*tr.random_pose(g), g)
    return q, m


def scan_batch(n_scans: int = 64, lo: int = 20_000, hi: int = 130_000, seed: int = 4,
               track: Optional[Track] = None) -> List[np.ndarray]:
    """Scans with log-uniform sizes in [lo, hi]: each a full ray cast at a
    random pose, then a seeded random subset kept in scan order."""
    tr = track or oval_1500()
    g = rng_for(seed)
    sizes = np.exp(g.uniform(math.log(lo), math.log(hi), n_scans)).astype(np.int64)
    out = []
    for sz in sizes:
        full = tr.raycast(*tr.random_pose(g), g)
        sz = min(int(sz), len(full))
        keep = np.sort(g.choice(len(full), sz, replace=False))
        out.append(full[keep])
    return out


@dataclass
class Arrival:
    t: float          # arrival time in seconds
    vehicle: int
    sensor: int
    points: np.ndarray


def arrival_stream(duration: float = 10.0, vehicles: int = 8, sensors: int = 3, rate_hz: float = 20.0,
                   lo: int = 30_000, hi: int = 130_000, seed: int = 5, pool: int = 48,
                   speed: float = 60.0, track: Optional[Track] = None) -> List[Arrival]:
    """Poisson arrivals from vehicles x sensors LiDARs, each at rate_hz.  A
    vehicle drives the lap at `speed` with a random phase; each sensor looks
    along a yaw offset of 0 / +120 / -120 degrees.  To bound generation time
    the ray casts come from a pool of `pool` poses per run (the nearest pool
    pose to the vehicle's position at the arrival time) and each arrival takes
    a uniform-size random subset in scan order."""
    tr = track or oval_1500()
    g = rng_for(seed)
    pool_s = np.sort(g.random(pool) * tr.length)
    yaw_off = [0.0, 2 * math.pi / 3, -2 * math.pi / 3]
    casts = {}

    def cast(pi: int, sensor: int) -> np.ndarray:
        key = (pi, sensor % 3)
        if key not in casts:
            gg = rng_for(seed * 1000 + pi * 3 + sensor % 3)
            casts[key] = tr.raycast(pool_s[pi], 0.0, yaw_off[sensor % 3], gg)
        return casts[key]

    out: List[Arrival] = []
    for v in range(vehicles):
        phase = g.random() * tr.length
        for sn in range(sensors):
            t = 0.0
            while True:
                t += g.exponential(1.0 / rate_hz)
                if t >= duration:
                    break
                s = (phase + speed * t) % tr.length
                pi = int(np.argmin(np.abs(pool_s - s)))
                full = cast(pi, sn)
                sz = min(int(g.integers(lo, hi + 1)), len(full))
                keep = np.sort(g.choice(len(full), sz, replace=False))
                out.append(Arrival(t, v, sn, full[keep]))
    out.sort(key=lambda a: a.t)
    return out


def stress(map_points: int = 20_000_000, n_poses: int = 8, seed: int = 6):
    """Large-map stress case: a 4 km oval with a pit lane and garages, 1 cm
    surface noise, half the points on pit structures (uneven occupancy), and
    queries from ray-cast scans at n_poses poses (scans see the track
    surfaces only)."""
    tr = oval_4000_pit()
    m = tr.sample_map(map_points, seed, noise=0.01)
    g = rng_for(seed + 100)
    q = np.concatenate([tr.raycast(*tr.random_pose(g), g) for _ in range(n_poses)])
    return q, m
