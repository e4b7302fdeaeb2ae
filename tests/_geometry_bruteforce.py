"""Geometric brute force for the dual-cell averages of Eq. 8.

Independent of the oracle's index sets: it places each E-component sample
point on the Yee lattice (Ex at ((i+1/2)D, jD), Ey at (iD, (j+1/2)D), Ez at
(iD, jD) in plane), builds the Yee-cell-sized box around it and integrates
the piecewise-constant subpixel map over that box by exact interval
overlaps.  Outside the design region the subpixel map is extended by the
boundary rule (edge replicate or wrap).
"""

from fractions import Fraction

import numpy as np

CLAMP, PERIODIC = 0, 1


def _ext(f, a, b, bc):
    mx, my = f.shape
    if bc == CLAMP:
        return f[min(max(a, 0), mx - 1), min(max(b, 0), my - 1)]
    return f[a % mx, b % my]


def _overlap(lo, hi, a):
    """Length of [lo, hi] intersected with the unit cell [a, a+1]."""
    return max(Fraction(0), min(hi, Fraction(a + 1)) - max(lo, Fraction(a)))


def sample_point(component, i, j, s):
    half = Fraction(s, 2)
    x = Fraction(s * i) + (half if component == 0 else 0)
    y = Fraction(s * j) + (half if component == 1 else 0)
    return x, y


def box_average(f, component, i, j, s, bc):
    """(1/|box|) * integral over the box of the subpixel map f."""
    x, y = sample_point(component, i, j, s)
    half = Fraction(s, 2)
    xlo, xhi, ylo, yhi = x - half, x + half, y - half, y + half
    total = 0.0
    for a in range(int(np.floor(xlo)) - 1, int(np.ceil(xhi)) + 1):
        ox = _overlap(xlo, xhi, a)
        if ox == 0:
            continue
        for b in range(int(np.floor(ylo)) - 1, int(np.ceil(yhi)) + 1):
            oy = _overlap(ylo, yhi, b)
            if oy == 0:
                continue
            total += float(ox * oy) * float(_ext(f, a, b, bc))
    return total / float(s * s)


def box_members(component, i, j, s):
    """(a, b, weight) of the subpixels that overlap the box (unmapped)."""
    x, y = sample_point(component, i, j, s)
    half = Fraction(s, 2)
    xlo, xhi, ylo, yhi = x - half, x + half, y - half, y + half
    out = []
    for a in range(int(np.floor(xlo)) - 1, int(np.ceil(xhi)) + 1):
        ox = _overlap(xlo, xhi, a)
        for b in range(int(np.floor(ylo)) - 1, int(np.ceil(yhi)) + 1):
            oy = _overlap(ylo, yhi, b)
            if ox * oy > 0:
                out.append((a, b, float(ox * oy) / float(s * s)))
    return out


def all_box_averages(f, component, nx, ny, s, bc):
    out = np.zeros((nx, ny))
    for i in range(nx):
        for j in range(ny):
            out[i, j] = box_average(f, component, i, j, s, bc)
    return out
