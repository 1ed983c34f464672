"""The regularised-covariance bar itself (tests/helpers.py), checked on CPU
with hand-built rows: a rule that accepted a wrong normal, or rejected a
right one, would make every GPU parity test that uses it meaningless."""
import numpy as np
import pytest

from tests import helpers as H


def pack(C):
    C = np.asarray(C, np.float64)
    return np.array([C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]])


def reg_of(n, eps):
    n = np.asarray(n, np.float64)
    n = n / np.linalg.norm(n)
    return pack(np.eye(3) - (1.0 - eps) * np.outer(n, n))


def rot(axis, angle):
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


EPS = 1e-3


def case(evals, normal_tilt):
    """A covariance with eigenvalues `evals` in a rotated frame, its exact C',
    and a C' whose normal is tilted by `normal_tilt` radians."""
    R = rot([1, 2, 3], 0.7)
    C = R @ np.diag(evals) @ R.T
    n = R[:, int(np.argmin(evals))]
    t = np.cross(n, R[:, int(np.argmax(evals))])
    n2 = np.cos(normal_tilt) * n + np.sin(normal_tilt) * t
    return pack(C), reg_of(n, EPS), reg_of(n2, EPS)


def test_well_separated_row_held_to_plain_bar():
    raw, ref, _ = case([1.0, 0.5, 0.001], 0.0)
    _, _, off = case([1.0, 0.5, 0.001], 2e-5)  # ~2.8e-5 relative Frobenius
    raw1 = raw[None]
    b = H.check_regularised_cov(ref[None], ref[None], raw1, raw1, EPS)
    assert b["well"]["rows"] == 1
    with pytest.raises(AssertionError):
        H.check_regularised_cov(off[None], ref[None], raw1, raw1, EPS)


def test_well_band_starts_at_one_percent_gap():
    # gap/tr just above 1e-2: a Davis-Kahan-sized error is no longer accepted
    raw, ref, off = case([1.0, 0.0205, 0.0], 3e-5)
    g = 0.0205 / 1.0205
    assert g >= H.WELL_GAP
    with pytest.raises(AssertionError):
        H.check_regularised_cov(off[None], ref[None], raw[None], raw[None], EPS)


def test_mid_band_uses_davis_kahan_allowance():
    # gap/tr = 1e-4: an error of 1e-5/gap in the normal is within bound ...
    raw, ref, off = case([1.0, 1e-4, 0.0], 2e-3)
    dC = raw * 1e-7  # a measured binary32 covariance error
    b = H.check_regularised_cov(off[None], ref[None], raw[None], (raw + dC)[None], EPS)
    assert b["mid"]["rows"] == 1 and b["mid"]["over_rtol"] == 1
    # ... but not an error far beyond it
    _, _, far = case([1.0, 1e-4, 0.0], 0.3)
    with pytest.raises(AssertionError):
        H.check_regularised_cov(far[None], ref[None], raw[None], (raw + dC)[None], EPS)


def test_degenerate_row_accepts_any_normal_of_the_eigenspace():
    # collinear neighbourhood: lambda2 = lambda3 = 0, any normal orthogonal
    # to the line is right, the line direction itself is wrong
    C = np.diag([1.0, 0.0, 0.0])
    raw = pack(C)[None]
    ref = reg_of([0, 0, 1], EPS)[None]
    ok = reg_of([0, 1, 1], EPS)[None]
    b = H.check_regularised_cov(ok, ref, raw, raw, EPS)
    assert b["degenerate"]["rows"] == 1
    bad = reg_of([1, 0, 0], EPS)[None]
    with pytest.raises(AssertionError):
        H.check_regularised_cov(bad, ref, raw, raw, EPS)
