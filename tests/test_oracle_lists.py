"""Pins of the oracle's E2 / E4 lists (Sec. 1.4 items 2 and 4, Alg. 4).

* a hand-worked example (tests/golden/worked_example_L2.json);
* all-pairs brute force written here from box cells found by bisection;
* the oracle's stencil route against its brute-force route;
* the identity: the non-empty source children of the level l-1 boxes that
  touch parent(r) are exactly E2(r) + E4(r), disjoint;
* symmetry when sources and receivers are the same set;
* bounds 27 and 189 (6^3 - 3^3), and level 2: E4 = every source box not in E2;
* closed forms on a full lattice (every box non-empty): per-box E2 count is
  a product of 2 (wall) or 3 (inside) per axis, total E2 = (3n-2)^3 and
  total E2 + E4 = (6n-8)^3 ... see _lattice_totals.
"""
import json
import os

import numpy as np
import pytest

from paper_1301_1704_gb300 import workloads
from tests import geom_ref

GOLD = os.path.join(os.path.dirname(__file__), "golden", "worked_example_L2.json")


def _rows(off, idx):
    off = off.astype(np.int64)
    return [list(idx[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


def test_worked_example(orc):
    g = json.load(open(GOLD))
    t = orc.build_tree(np.array(g["src"], np.float32), np.array(g["recv"], np.float32), L=g["L"])
    for side in ("src", "recv"):
        e = g["expect"][side]
        assert list(t[side]["perm"]) == e["perm"]
        for l in range(g["L"] + 1):
            assert list(t[side]["key"][l]) == e["key"][l]
            assert list(t[side]["off"][l]) == e["off"][l]
            assert list(t[side]["parent"][l]) == e["parent"][l]
            assert list(t[side]["child"][l]) == e["child"][l]
    for nm in ("e2_off", "e2_idx", "e4_off", "e4_idx"):
        assert list(t[nm][2]) == g["expect"][nm]


def _tiny_cases():
    return [
        (workloads.uniform(60, 41), workloads.uniform(50, 42), 3),
        (workloads.clumps(80, 43, nclumps=3, sigma=0.05), workloads.uniform(40, 44), 4),
        (workloads.uniform(25, 45), workloads.clumps(70, 46, nclumps=2, sigma=0.04), 4),
        (np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [0.99, 0.01, 0.5]], np.float32),
         np.array([[0.01, 0.0, 0.02], [1, 1, 0.9], [0.49, 0.51, 0.5]], np.float32), 3),
    ]


@pytest.mark.parametrize("src,recv,L", _tiny_cases())
def test_lists_match_python_brute_force(orc, src, recv, L):
    t = orc.build_tree(src, recv, L=L, mode=orc.MODE_STENCIL)
    for l in range(2, L + 1):
        sc, _ = geom_ref.boxes_by_path(src, l)
        rc, _ = geom_ref.boxes_by_path(recv, l)
        e2, e4 = geom_ref.brute_lists(sc, rc)
        assert _rows(t["e2_off"][l], t["e2_idx"][l]) == e2
        assert _rows(t["e4_off"][l], t["e4_idx"][l]) == e4


def _random_cases():
    return [
        (workloads.uniform(3000, 51), workloads.uniform(3000, 52), 4),
        (workloads.clumps(3000, 53, nclumps=6, sigma=0.03), workloads.sphere(3000, 54), 5),
        (workloads.sphere(2000, 55), workloads.sphere(2000, 55), 5),
    ]


@pytest.mark.parametrize("src,recv,L", _random_cases())
def test_stencil_equals_brute(orc, src, recv, L):
    a = orc.build_tree(src, recv, L=L, mode=orc.MODE_STENCIL)
    b = orc.build_tree(src, recv, L=L, mode=orc.MODE_BRUTE)
    for l in range(2, L + 1):
        for nm in ("e2_off", "e2_idx", "e4_off", "e4_idx"):
            assert np.array_equal(a[nm][l], b[nm][l]), (nm, l)


@pytest.mark.parametrize("src,recv,L", _random_cases())
def test_parent_neighbourhood_identity(orc, src, recv, L):
    t = orc.build_tree(src, recv, L=L)
    S, R = t["src"], t["recv"]
    for l in range(2, L + 1):
        e2 = _rows(t["e2_off"][l], t["e2_idx"][l])
        e4 = _rows(t["e4_off"][l], t["e4_idx"][l])
        if l >= 3:
            e2up = _rows(t["e2_off"][l - 1], t["e2_idx"][l - 1])
        for r in range(len(R["key"][l])):
            assert len(e2[r]) <= 27 and len(e4[r]) <= 189
            assert not set(e2[r]) & set(e4[r])
            assert e2[r] == sorted(e2[r]) and e4[r] == sorted(e4[r])
            if l == 2:
                parents = range(len(S["key"][1]))  # all level-1 boxes touch
            else:
                parents = e2up[int(R["parent"][l][r])]
            kids = []
            ch = S["child"][l - 1].astype(np.int64)
            for q in parents:
                kids.extend(range(ch[q], ch[q + 1]))
            assert sorted(e2[r] + e4[r]) == kids
        if l == 2:
            for r in range(len(R["key"][l])):
                assert sorted(e2[r] + e4[r]) == list(range(len(S["key"][2])))


def test_symmetry_same_set(orc):
    p = workloads.clumps(4000, 61, nclumps=8, sigma=0.04)
    t = orc.build_tree(p, p, L=5)
    for l in range(2, 6):
        for nm in ("e2", "e4"):
            rows = _rows(t[nm + "_off"][l], t[nm + "_idx"][l])
            pairs = {(r, s) for r, row in enumerate(rows) for s in row}
            assert pairs == {(s, r) for r, s in pairs}


def _lattice_totals(l):
    n = 1 << l
    e2 = (3 * n - 2) ** 3
    return e2, (6 * n - 8) ** 3 - e2


@pytest.mark.parametrize("level", [2, 3, 4])
def test_full_lattice_closed_forms(orc, level):
    p = workloads.lattice(level)
    t = orc.build_tree(p, p, L=level)
    n = 1 << level
    for l in range(2, level + 1):
        m = 1 << l
        assert len(t["src"]["key"][l]) == m ** 3
        e2tot, e4tot = _lattice_totals(l)
        assert len(t["e2_idx"][l]) == e2tot
        assert len(t["e4_idx"][l]) == e4tot
        c2 = np.diff(t["e2_off"][l].astype(np.int64))
        c4 = np.diff(t["e4_off"][l].astype(np.int64))
        for r, k in enumerate(t["recv"]["key"][l]):
            c = orc.decode(int(k), l)
            want = 1
            for v in c:
                want *= 2 if v in (0, m - 1) else 3
            assert c2[r] == want
            pc = [v // 2 for v in c]
            if l >= 3 and all(0 < v < m // 2 - 1 for v in pc):
                assert c4[r] == 189  # interior parent: full 6x6x6 block minus 27
        assert c2.max() == 27 if l >= 2 else True
    assert n == 1 << level


def test_totals_formula_matches_brute_small(orc):
    """The closed form itself, counted by brute force in 1D per axis."""
    for l in (2, 3):
        m = 1 << l
        e2 = sum(1 for a in range(m) for b in range(m) if abs(a - b) <= 1) ** 3
        blk = sum(1 for a in range(m) for b in range(m) if abs(a // 2 - b // 2) <= 1) ** 3
        assert (e2, blk - e2) == _lattice_totals(l)
