"""Independent characterisations used to pin the oracle (pure Python/numpy).

Nothing here packs bits the way the oracle does.  A box is described by its
path from the root: the sequence of octants (x-half + 2*y-half + 4*z-half)
met while bisecting the unit cube, computed from exact dyadic comparisons of
the float32 coordinates (float64 holds them exactly).  Ordering boxes by that
tuple is the depth-first order of the octree, which is the Morton order of
Sec. 1.4 of the paper under the x/y/z bit reading.
"""
from __future__ import annotations

import numpy as np


def octant_path(p, levels: int = 21) -> tuple:
    """Octants met while bisecting [0,1]^3 ``levels`` times around point p.

    The upper half is closed at 1.0, so x == 1.0 always takes the upper half.
    """
    lo = [0.0, 0.0, 0.0]
    size = 1.0
    path = []
    for _ in range(levels):
        size /= 2.0
        o = 0
        for d in range(3):
            mid = lo[d] + size
            if float(p[d]) >= mid:
                o |= 1 << d
                lo[d] = mid
        path.append(o)
    return tuple(path)


def path_to_int(path) -> int:
    """Base-8 number whose digits are the octants, coarsest first."""
    v = 0
    for o in path:
        v = v * 8 + o
    return v


def cells(xyz: np.ndarray, level: int) -> np.ndarray:
    """Integer box coordinates of every point at ``level`` (clamped at 1.0)."""
    m = 1 << level
    c = np.floor(np.asarray(xyz, dtype=np.float64) * m).astype(np.int64)
    return np.minimum(c, m - 1)


def cell_path(c, level: int) -> tuple:
    """Octant path of an integer cell at ``level`` (coarsest octant first)."""
    path = []
    for j in range(level - 1, -1, -1):
        o = 0
        for d in range(3):
            if (int(c[d]) >> j) & 1:
                o |= 1 << d
        path.append(o)
    return tuple(path)


def boxes_by_path(xyz: np.ndarray, level: int):
    """Non-empty boxes of ``level`` in octree (depth-first) order.

    Returns (cells as a list of tuples, point counts)."""
    c = cells(xyz, level)
    uniq = {}
    for row in map(tuple, c.tolist()):
        uniq[row] = uniq.get(row, 0) + 1
    order = sorted(uniq, key=lambda t: cell_path(t, level))
    return order, [uniq[t] for t in order]


def cheb(a, b) -> int:
    return max(abs(int(a[d]) - int(b[d])) for d in range(3))


def brute_lists(src_cells, recv_cells):
    """E2 / E4 by the definitions (Sec. 1.4): for each receiver box, the
    ranks of source boxes at max-norm distance <= 1, and of those whose
    parents are at distance <= 1 while they themselves are not."""
    e2, e4 = [], []
    for r in recv_cells:
        pr = tuple(v // 2 for v in r)
        a, b = [], []
        for t, s in enumerate(src_cells):
            if cheb(r, s) <= 1:
                a.append(t)
            elif cheb(pr, tuple(v // 2 for v in s)) <= 1:
                b.append(t)
        e2.append(a)
        e4.append(b)
    return e2, e4
