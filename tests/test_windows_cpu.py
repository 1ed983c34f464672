"""Host-side bookkeeping of pose-keyed windows (no GPU)."""
import numpy as np
import pytest

from paper_2308_07173_gb300 import windows
from paper_2308_07173_gb300 import workloads as W


def test_stations_along_the_track_and_nearest():
    tr = W.oval_1500()
    rw = windows.RaceLineWindows.along(tr, spacing=10.0, half=(50, 50, 5))
    assert len(rw.stations) == 150
    # every station is its own nearest; a point 3 m off a station maps to it
    for i in (0, 37, 149):
        assert rw.nearest(rw.stations[i]) == i
        assert rw.nearest(rw.stations[i] + [0.0, 3.0, 0.0]) == i
    lo, hi = rw.window(37)
    np.testing.assert_allclose(hi - lo, [100, 100, 10])
    np.testing.assert_allclose((lo + hi) / 2, rw.stations[37], atol=1e-4)


class _FakeTarget:
    def __init__(self):
        self.calls = []

    def set_window(self, lo, hi):
        self.calls.append((np.asarray(lo), np.asarray(hi)))


def test_apply_sets_the_nearest_window():
    rw = windows.RaceLineWindows([[0, 0, 0], [100, 0, 0]], half=(10, 10, np.inf))
    t = _FakeTarget()
    assert rw.apply(t, [90, 1, 0]) == 1
    lo, hi = t.calls[-1]
    np.testing.assert_allclose(lo[:2], [90, -10])
    assert np.isinf(hi[2])


def test_bad_arguments():
    with pytest.raises(ValueError):
        windows.RaceLineWindows(np.zeros((0, 3)))
    with pytest.raises(ValueError):
        windows.RaceLineWindows([[0, 0, 0]], half=(-1, 1, 1))
