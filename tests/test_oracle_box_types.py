"""Pins of the Alg. 6 box-type oracle (oracle/box_types.py), no GPU."""
import numpy as np
import pytest

from oracle import box_types as BT
from paper_1301_1704_gb300 import workloads


def _tree(orc, n=4000, L=5, seed=31):
    p = workloads.clumps(n, seed, nclumps=6, sigma=0.08)
    return p, orc.build_tree(p, p, L=L)


def _cells(pts, level):
    return np.minimum(np.floor(pts.astype(np.float64) * (1 << level)), (1 << level) - 1).astype(np.int64)


def test_one_node_owns_everything(orc):
    p, t = _tree(orc)
    for lpar in (2, 3, 4):
        own = np.zeros(len(t["src"]["key"][lpar]), np.uint32)
        types = BT.box_types(t, lpar, own, 0)
        assert all(np.all(v == BT.DOMESTIC) for v in types.values())


def test_node_owning_nothing(orc):
    p, t = _tree(orc)
    lpar = 4
    own = np.ones(len(t["src"]["key"][lpar]), np.uint32)
    types = BT.box_types(t, lpar, own, 0)
    lcrit = lpar - 1
    assert np.all(types[2] == BT.DOMESTIC)
    assert np.all(types[lcrit] == BT.IMPORT)
    for l in range(lcrit + 1, t["L"] + 1):
        assert np.all(types[l] == BT.OTHERS)


@pytest.mark.parametrize("lpar", [2, 3, 4])
def test_two_nodes_against_geometry(orc, lpar):
    """Owner = which half of the cube (x < 1/2) a box lies in.  Checked by
    brute force over the boxes' cells: on-J boxes above l_crit are EXPORT iff
    some off-J source box is an M2L neighbour (parents adjacent, boxes not);
    EXPORT for one node is IMPORT for the other; ROOT boxes at l_crit have
    source points on both sides."""
    p, t = _tree(orc, L=5)
    L = t["L"]
    keys_par = t["src"]["key"][lpar]
    cpar = np.array([orc.decode(int(k), lpar) for k in keys_par])
    own = (cpar[:, 0] >= (1 << (lpar - 1))).astype(np.uint32)
    ty = [BT.box_types(t, lpar, own, j) for j in (0, 1)]
    lcrit = max(lpar - 1, 2)
    for l in range(lcrit + 1, L + 1):
        c = np.array([orc.decode(int(k), l) for k in t["src"]["key"][l]])
        side = (c[:, 0] >= (1 << (l - 1))).astype(int)  # node of each box
        d = np.abs(c[:, None, :] - c[None, :, :]).max(axis=2)
        dp = np.abs((c[:, None, :] >> 1) - (c[None, :, :] >> 1)).max(axis=2)
        m2l = (dp <= 1) & (d >= 2)
        for j in (0, 1):
            mine = side == j
            exp = mine & (m2l & (side[None, :] != j)).any(axis=1)
            imp = ~mine & (m2l & (side[None, :] == j)).any(axis=1)
            want = np.where(exp, BT.EXPORT, np.where(mine, BT.DOMESTIC,
                                                    np.where(imp, BT.IMPORT, BT.OTHERS)))
            assert np.array_equal(ty[j][l], want), (lpar, l, j)
        assert np.array_equal(ty[0][l] == BT.EXPORT, ty[1][l] == BT.IMPORT)
    if lcrit < lpar:
        c = np.array([orc.decode(int(k), lcrit) for k in t["src"]["key"][lcrit]])
        pc = _cells(p, lcrit)
        for k in range(len(c)):
            inside = np.all(pc == c[k], axis=1)
            sides = set((_cells(p[inside], lpar)[:, 0] >= (1 << (lpar - 1))).astype(int))
            assert (ty[0][lcrit][k] == BT.ROOT) == (sides == {0, 1})
    for l in range(2, lcrit):
        assert np.all(ty[0][l] == BT.DOMESTIC)


@pytest.mark.parametrize("lpar,seed", [(3, 37), (4, 38), (5, 39)])
def test_split_through_lcrit_boxes_against_geometry(orc, lpar, seed):
    """Owner = whether a box's x cell at l_par is >= s with s odd, so the
    split cuts the l_crit boxes of one x column in two and leaves the others
    whole on one side.  Every type of every level l_crit..L, for both nodes,
    is checked against geometry alone: a box's children on / off J are the
    l_par cells of the source points inside it and the side each lies on; the
    M2L neighbours of a box are the boxes whose parents are adjacent to its
    parent (max-norm distance <= 1) and that are not adjacent to it.  At
    l_crit: no child on J -> IMPORT; children on both sides -> ROOT; else
    EXPORT when some M2L neighbour has a child off J, else DOMESTIC."""
    p, t = _tree(orc, n=3000, L=6, seed=seed)
    L = t["L"]
    lcrit = lpar - 1
    s = (1 << (lpar - 1)) + 1
    cpar = np.array([orc.decode(int(k), lpar) for k in t["src"]["key"][lpar]])
    own = (cpar[:, 0] >= s).astype(np.uint32)
    ty = [BT.box_types(t, lpar, own, j) for j in (0, 1)]
    # point sides (the node owning each point's l_par cell)
    pside = (_cells(p, lpar)[:, 0] >= s).astype(int)
    seen = set()
    for l in range(lcrit, L + 1):
        c = np.array([orc.decode(int(k), l) for k in t["src"]["key"][l]])
        pcl = _cells(p, l)
        # the boxes are exactly the cells that hold points
        assert {tuple(r) for r in c} == {tuple(r) for r in pcl}
        d = np.abs(c[:, None, :] - c[None, :, :]).max(axis=2)
        dp = np.abs((c[:, None, :] >> 1) - (c[None, :, :] >> 1)).max(axis=2)
        m2l = (dp <= 1) & (d >= 2)
        for j in (0, 1):
            if l == lcrit:
                on = np.zeros(len(c), bool)
                off = np.zeros(len(c), bool)
                for k in range(len(c)):
                    sides = pside[np.all(pcl == c[k], axis=1)]
                    on[k] = (sides == j).any()
                    off[k] = (sides != j).any()
                exp = on & ~off & (m2l & off[None, :]).any(axis=1)
                want = np.where(~on, BT.IMPORT, np.where(on & off, BT.ROOT,
                                                         np.where(exp, BT.EXPORT, BT.DOMESTIC)))
            else:
                side = ((c[:, 0] >> (l - lpar)) >= s).astype(int)
                mine = side == j
                exp = mine & (m2l & (side[None, :] != j)).any(axis=1)
                imp = ~mine & (m2l & (side[None, :] == j)).any(axis=1)
                want = np.where(exp, BT.EXPORT, np.where(mine, BT.DOMESTIC,
                                                        np.where(imp, BT.IMPORT, BT.OTHERS)))
            assert np.array_equal(ty[j][l], want), (lpar, l, j)
            if l == lcrit:
                seen |= set(int(v) for v in want)
    # the split exercises every branch at l_crit (at level 2 every box that
    # is not adjacent is an M2L neighbour, so no box there is DOMESTIC)
    want_seen = {BT.IMPORT, BT.ROOT, BT.EXPORT} | ({BT.DOMESTIC} if lcrit >= 3 else set())
    assert seen == want_seen, seen
