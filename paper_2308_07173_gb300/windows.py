"""Pose-keyed map windows along a race line (Sec. III-C3: each pose on the
race line is associated with its part of the unified map, and scan matching
searches that sliding window instead of the whole map).

Stations are points of the race line at a fixed spacing; each owns the box
of half-extents `half` around it.  The window for a vehicle position is the
box of its nearest station, applied to a Target with ``Target.set_window``
(no grid rebuild: the search clips its boxes to the window's cells).  This
is host-side bookkeeping only; the searches run in the library's kernels.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np


class RaceLineWindows:
    def __init__(self, stations, half: Sequence[float] = (60.0, 60.0, float("inf"))):
        st = np.asarray(stations, np.float64)
        if st.ndim != 2 or st.shape[1] != 3 or len(st) == 0:
            raise ValueError("stations must be [n,3]")
        half = np.asarray(half, np.float64).reshape(3)
        if (half < 0).any() or np.isnan(half).any():
            raise ValueError("half extents must be >= 0")
        self.stations = st
        self.half = half

    @classmethod
    def along(cls, track, spacing: float = 10.0, half=(60.0, 60.0, float("inf")), height: float = 0.0):
        """Stations every `spacing` metres of a Track's centreline."""
        s = np.arange(0.0, track.length, spacing)
        pos, _, _ = track.pose(s)
        return cls(np.c_[pos, np.full(len(s), height)], half)

    def nearest(self, xyz) -> int:
        d = np.sum((self.stations - np.asarray(xyz, np.float64).reshape(1, 3)) ** 2, axis=1)
        return int(np.argmin(d))

    def window(self, i: int) -> Tuple[np.ndarray, np.ndarray]:
        c = self.stations[i]
        return (c - self.half).astype(np.float32), (c + self.half).astype(np.float32)

    def apply(self, target, xyz) -> int:
        """Sets the target's window to the box of the station nearest xyz;
        returns the station index."""
        i = self.nearest(xyz)
        lo, hi = self.window(i)
        target.set_window(lo, hi)
        return i
