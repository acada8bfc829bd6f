"""Pins of the oracle's sorted points and Alg. 2 gather, from geometry alone."""
import numpy as np
import pytest

from paper_1301_1704_gb300 import workloads


def _cells(pts, level):
    return np.minimum(np.floor(pts.astype(np.float64) * (1 << level)), (1 << level) - 1).astype(np.int64)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_gather_e2_is_the_neighbourhood(orc, L):
    src = workloads.clumps(3000, 81, nclumps=4, sigma=0.05)
    recv = workloads.uniform(800, 82)
    t = orc.build_tree(src, recv, L=L)
    off, pts = orc.gather_e2(t, src, L)
    sc = _cells(src, L)
    rkeys = t["recv"]["key"][L]
    rc = np.stack([orc.decode(int(k), L) for k in rkeys]) if len(rkeys) else np.zeros((0, 3))
    assert off[0] == 0 and off[-1] == len(pts)
    for i in range(len(rkeys)):
        got = pts[off[i]:off[i + 1]]
        # brute force: every source point whose cell is within max-norm 1
        near = np.all(np.abs(sc - rc[i]) <= 1, axis=1)
        want = src[near]
        assert len(got) == len(want)
        # as multisets of points
        assert np.array_equal(np.unique(got, axis=0), np.unique(want, axis=0))
        # order: neighbour boxes ascending (Morton order of their cells),
        # points inside a box in the build's order
        gk = orc.keys(got) >> np.uint64(3 * (21 - L)) if len(got) else np.zeros(0, np.uint64)
        assert np.all(np.diff(gk.astype(np.int64)) >= 0)


def test_sorted_points_follow_perm(orc):
    p = workloads.sphere(2000, 83)
    t = orc.build_tree(p, p, L=5)
    sp = orc.sorted_points(p, t["src"]["perm"])
    k = orc.keys(sp)
    assert np.all(np.diff(k.astype(np.int64)) >= 0)
    assert np.array_equal(np.sort(sp.view(np.uint32).reshape(-1, 3), axis=0),
                          np.sort(p.view(np.uint32).reshape(-1, 3), axis=0))
