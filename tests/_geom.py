"""Geometry helpers for tests: zero-level-set crossings and radius errors."""
import numpy as np


def zero_crossings(phi, h):
    """Points where phi changes sign along a grid edge (zero counts as
    positive), located by linear interpolation.  Returns (n, 3) array of
    (x, y, z) coordinates in a cell-centred grid with spacing h."""
    pts = []
    nz, ny, nx = phi.shape
    neg = phi < 0
    for axis in range(3):
        a = np.take(phi, range(phi.shape[axis] - 1), axis=axis)
        b = np.take(phi, range(1, phi.shape[axis]), axis=axis)
        na = np.take(neg, range(phi.shape[axis] - 1), axis=axis)
        nb = np.take(neg, range(1, phi.shape[axis]), axis=axis)
        m = na != nb
        idx = np.nonzero(m)
        av, bv = a[m], b[m]
        frac = av / (av - bv)
        z, y, x = (np.asarray(i, dtype=np.float64) for i in idx)
        if axis == 0:
            z = z + frac
        elif axis == 1:
            y = y + frac
        else:
            x = x + frac
        pts.append(np.stack([(x + 0.5) * h, (y + 0.5) * h, (z + 0.5) * h], axis=1))
    return np.concatenate(pts, axis=0)


def radius_error(phi, h, centre, radius):
    """(mean, max) of |crossing - centre| - radius over all zero crossings,
    in units of h."""
    p = zero_crossings(phi, h)
    d = np.linalg.norm(p - np.asarray(centre)[None, :], axis=1) - radius
    return float(d.mean() / h), float(np.abs(d).max() / h)
