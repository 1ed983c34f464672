"""Exact binary32 arithmetic with Python Fractions, for pinning the oracle's
squared-distance order independently of any float hardware or libm."""
from fractions import Fraction

import numpy as np


def round_f32(x: Fraction) -> np.float32:
    """Round an exact rational to binary32, round-half-to-even, with
    subnormals and overflow to infinity."""
    if x == 0:
        return np.float32(0.0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    qe = max(e - 23, -149)  # exponent of the last significand bit
    m = a / Fraction(2) ** qe
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    val = Fraction(fl) * Fraction(2) ** qe
    if val >= Fraction(2) ** 128:
        return np.float32(sign * np.inf)
    return np.float32(sign * float(val))


def F(v) -> Fraction:
    return Fraction(float(np.float32(v)))


def d2_pinned(q, p) -> np.float32:
    """fmaf(dz,dz, fmaf(dy,dy, dx*dx)) with dx = q.x - p.x, every step
    rounded once to binary32 (fmaf rounds the exact a*b + c once)."""
    dx = F(round_f32(F(q[0]) - F(p[0])))
    dy = F(round_f32(F(q[1]) - F(p[1])))
    dz = F(round_f32(F(q[2]) - F(p[2])))
    sx = F(round_f32(dx * dx))
    t = F(round_f32(dy * dy + sx))
    return round_f32(dz * dz + t)
