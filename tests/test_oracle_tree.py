"""Pins of the oracle's order, boxes and cluster-size mode (Alg. 1, Alg. 3,
Sec. 2.1 and the bookmark definitions of Sec. 2.2).

* order: numpy's stable argsort of the keys (a different sort from the
  oracle's std::sort of pairs) must give the same permutation;
* boxes: the bookmarks partition the sorted points, every point of a box
  has the box's key, parent ranges contain child ranges, counts are bounded,
  and the boxes in order equal the octree's non-empty cells in depth-first
  order found by geometric bisection;
* cluster-size mode: brute-force occupancy per level.
"""
import numpy as np
import pytest

from paper_1301_1704_gb300 import workloads
from tests import geom_ref


def _sets():
    return [
        ("uniform", workloads.uniform(3000, 21), workloads.uniform(2500, 22), 4),
        ("clumps", workloads.clumps(3000, 23, nclumps=5, sigma=0.02), workloads.sphere(2000, 24), 6),
        ("dups", np.repeat(workloads.uniform(7, 25), 40, axis=0), workloads.uniform(100, 26), 5),
        ("faces", np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [1, 0, 0.25], [0.75, 1, 0]] * 3,
                           np.float32), workloads.uniform(9, 27), 3),
    ]


@pytest.mark.parametrize("name,src,recv,L", _sets())
def test_order_matches_stable_argsort(orc, name, src, recv, L):
    t = orc.build_tree(src, recv, L=L, mode=orc.MODE_NOLISTS)
    for side, pts in (("src", src), ("recv", recv)):
        k = orc.keys(pts)
        ref = np.argsort(k, kind="stable")
        assert np.array_equal(t[side]["perm"], ref.astype(np.uint32))
        assert np.array_equal(t[side]["sorted_keys"], k[ref])
        assert np.all(np.diff(t[side]["sorted_keys"].astype(np.float64)) >= 0) or len(k) < 2
        assert np.array_equal(np.sort(t[side]["perm"]), np.arange(len(pts), dtype=np.uint32))


@pytest.mark.parametrize("name,src,recv,L", _sets())
def test_box_invariants(orc, name, src, recv, L):
    t = orc.build_tree(src, recv, L=L, mode=orc.MODE_NOLISTS)
    for side, pts in (("src", src), ("recv", recv)):
        d = t[side]
        n = len(pts)
        sk = d["sorted_keys"]
        prev_nb = 0
        for l in range(L + 1):
            key, off = d["key"][l], d["off"][l].astype(np.int64)
            nb = len(key)
            assert nb <= min(n, 8 ** l)
            assert nb >= prev_nb
            prev_nb = nb
            assert off[0] == 0 and off[-1] == n
            assert np.all(np.diff(off) > 0)
            # every point of box b carries the box's level-l key
            lk = sk >> np.uint64(3 * (21 - l))
            rep = np.repeat(np.arange(nb), np.diff(off))
            assert np.array_equal(lk, key[rep])
            assert np.all(np.diff(key.astype(np.float64)) > 0)
            if l >= 1:
                par = d["parent"][l].astype(np.int64)
                pk = d["key"][l - 1]
                assert np.array_equal(pk[par], key >> np.uint64(3))
                poff = d["off"][l - 1].astype(np.int64)
                assert np.all(poff[par] <= off[:-1]) and np.all(off[1:] <= poff[par + 1])
            if l < L:
                ch = d["child"][l].astype(np.int64)
                assert len(ch) == nb + 1 and ch[0] == 0 and ch[-1] == len(d["key"][l + 1])
                cpar = d["parent"][l + 1]
                for b in range(nb):
                    assert np.all(cpar[ch[b]:ch[b + 1]] == b)
                    assert 1 <= ch[b + 1] - ch[b] <= 8
        assert len(d["key"][0]) == 1


@pytest.mark.parametrize("name,src,recv,L", _sets()[:2])
def test_boxes_match_octree_bisection(orc, name, src, recv, L):
    t = orc.build_tree(src, recv, L=L, mode=orc.MODE_NOLISTS)
    for side, pts in (("src", src), ("recv", recv)):
        for l in range(1, L + 1):
            cells, counts = geom_ref.boxes_by_path(pts, l)
            keys = t[side]["key"][l]
            assert len(keys) == len(cells)
            assert np.array_equal(np.diff(t[side]["off"][l].astype(np.int64)), np.array(counts))
            for k, c in zip(keys, cells):
                assert int(k) == geom_ref.path_to_int(geom_ref.cell_path(c, l))


def test_empty_sets(orc):
    z = np.zeros((0, 3), np.float32)
    t = orc.build_tree(z, z, L=3)
    for side in ("src", "recv"):
        for l in range(4):
            assert len(t[side]["key"][l]) == 0
            assert list(t[side]["off"][l]) == [0]
    for l in (2, 3):
        assert list(t["e2_off"][l]) == [0] and len(t["e4_idx"][l]) == 0
    t = orc.build_tree(z, workloads.uniform(50, 1), L=3)
    for l in (2, 3):
        assert len(t["e2_idx"][l]) == 0 and len(t["e4_idx"][l]) == 0
        assert np.all(t["e2_off"][l] == 0)


def test_bad_arguments(orc):
    p = workloads.uniform(10, 1)
    for L, s in ((22, 0), (-1, 0), (-2, 5)):
        with pytest.raises(orc.OracleError) as e:
            orc.build_tree(p, p, L=L, s=s)
        assert e.value.code == orc.ORC_ERR_LEVEL


@pytest.mark.parametrize("s", [1, 3, 16, 64, 500])
def test_cluster_size_mode_brute(orc, s):
    src = workloads.clumps(2000, 31, nclumps=4, sigma=0.03)
    recv = workloads.uniform(1500, 32)
    t = orc.build_tree(src, recv, L=-1, s=s, mode=orc.MODE_NOLISTS)
    want, unmet = 21, 1
    for l in range(2, 22):
        occ = max(max(np.unique(geom_ref.cells(p, l), axis=0, return_counts=True)[1])
                  for p in (src, recv))
        if occ <= s:
            want, unmet = l, 0
            break
    assert t["L"] == want and t["s_unmet"] == unmet
    assert len(t["src"]["key"]) == want + 1


def test_cluster_size_unmet(orc):
    same = np.repeat(np.array([[0.3, 0.3, 0.3]], np.float32), 10, axis=0)
    t = orc.build_tree(same, same, L=-1, s=4, mode=orc.MODE_NOLISTS)
    assert t["L"] == 21 and t["s_unmet"] == 1


@pytest.mark.parametrize("L", [0, 1, 3, 5])
def test_box_key_order(orc, L):
    """(level-L key, index) order: a stable argsort of the level-L keys (a
    different sort), ascending indices inside every level-L box, the same
    boxes as the full-key order, and permuted points that stay inside the
    boxes the full-key order gives them."""
    from paper_1301_1704_gb300 import workloads
    src = workloads.clumps(6000, 51, nclumps=5, sigma=0.03)
    recv = workloads.uniform(3000, 52)
    full = orc.build_tree(src, recv, L=L)
    box = orc.build_tree(src, recv, L=L, order=orc.ORDER_BOX)
    for side, pts in (("src", src), ("recv", recv)):
        k = orc.keys(pts) >> np.uint64(3 * (21 - L))
        assert np.array_equal(box[side]["perm"], np.argsort(k, kind="stable"))
        off = box[side]["off"][L]
        for b in range(len(off) - 1):
            seg = box[side]["perm"][off[b]:off[b + 1]]
            assert np.all(np.diff(seg.astype(np.int64)) > 0)
            assert set(seg) == set(full[side]["perm"][off[b]:off[b + 1]])
        for l in range(L + 1):
            for nm in ("key", "off", "parent", "child"):
                assert np.array_equal(box[side][nm][l], full[side][nm][l])
    for l in range(2, L + 1):
        for nm in ("e2_off", "e2_idx", "e4_off", "e4_idx"):
            assert np.array_equal(box[nm][l], full[nm][l])


def test_box_key_order_cluster_size(orc):
    from paper_1301_1704_gb300 import workloads
    p = workloads.clumps(5000, 53, nclumps=3, sigma=0.02)
    box = orc.build_tree(p, p, L=-1, s=16, order=orc.ORDER_BOX)
    full = orc.build_tree(p, p, L=-1, s=16)
    assert box["L"] == full["L"]
    k = orc.keys(p) >> np.uint64(3 * (21 - box["L"]))
    assert np.array_equal(box["src"]["perm"], np.argsort(k, kind="stable"))


def test_parallel_build_equals_serial(orc):
    """The OpenMP build of the oracle (key loop, parallel sort, list blocks)
    gives exactly the single-threaded result."""
    from paper_1301_1704_gb300 import workloads
    src = workloads.clumps(60000, 57, nclumps=8, sigma=0.03)
    recv = workloads.uniform(50000, 58)
    a = orc.build_tree(src, recv, L=5)
    b = orc.build_tree(src, recv, L=5, parallel=True)
    assert a["L"] == b["L"]
    for side in ("src", "recv"):
        assert np.array_equal(a[side]["perm"], b[side]["perm"])
        for nm in ("key", "off", "parent", "child"):
            for x, y in zip(a[side][nm], b[side][nm]):
                assert np.array_equal(x, y)
    for nm in ("e2_off", "e2_idx", "e4_off", "e4_idx"):
        for l in a[nm]:
            assert np.array_equal(a[nm][l], b[nm][l])
    bad = src.copy()
    bad[777, 1] = np.nan
    with pytest.raises(orc.OracleError):
        orc.build_tree(bad, recv, L=3, parallel=True)
