"""GPU path vs the CPU oracle, element by element, through the C ABI.

All of this is integer and index work, so the bar is bit-exact equality of
every output array.  Small and medium cases compare whole trees (several
sort, box and scan tiles plus ragged tails); the full-size workloads compare
keys, permutations and boxes in full and the lists on sampled receiver boxes
that the oracle computes one by one.
"""
import numpy as np
import pytest

from paper_1301_1704_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_1704_gb300 import build, fmmds
    build.build()
    c = fmmds.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def compare_full(got, want, L):
    assert got["L"] == want["L"] == L
    for side in ("src", "recv"):
        assert np.array_equal(got[side]["perm"], want[side]["perm"]), f"{side} perm"
        for l in range(L + 1):
            for nm in ("key", "off", "parent", "child"):
                g, w = got[side][nm][l], want[side][nm][l]
                assert np.array_equal(g, w), f"{side} {nm} level {l}: {g[:8]} vs {w[:8]}"
    for l in range(2, L + 1):
        for nm in ("e2_off", "e2_idx", "e4_off", "e4_idx"):
            assert np.array_equal(got[nm][l], want[nm][l]), f"{nm} level {l}"


def run_both(ctx, orc, src, recv, L, mode=None, aliased=False):
    s = _dev(src)
    r = s if aliased else _dev(recv)
    got = ctx.build(s, r, L=L).numpy()
    want = orc.build_tree(src, src if aliased else recv, L=L,
                          mode=orc.MODE_STENCIL if mode is None else mode)
    return got, want


def test_morton_keys_match_oracle(ctx, orc):
    rng = np.random.default_rng(3)
    pts = [rng.random((100003, 3)).astype(np.float32),
           np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.25, 1.0], [1 - 2 ** -21, 2 ** -21, 0.75]],
                    np.float32)]
    for p in pts:
        got = ctx.morton_keys(_dev(p)).cpu().numpy().view(np.uint64)
        assert np.array_equal(got, orc.keys(p))


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_sort_kinds_agree(ctx, orc, kind):
    from paper_1301_1704_gb300 import fmmds
    src = workloads.clumps(150000, 30, nclumps=10, sigma=0.03)
    recv = workloads.uniform(90001, 31)
    ctx.set_tuning(kind)
    try:
        got, want = run_both(ctx, orc, src, recv, 6)
        compare_full(got, want, 6)
        p = workloads.clumps(40000, 32, nclumps=3, sigma=0.01)  # long boxes: full 63-bit sort
        got, want = run_both(ctx, orc, p, p[:5000].copy(), 2)
        compare_full(got, want, 2)
    finally:
        ctx.set_tuning(fmmds.FMM_SORT_BUCKET)


def test_config1_full_tree_brute(ctx, orc):
    src, recv, L = workloads.config_inputs(1)
    got, want = run_both(ctx, orc, src, recv, L, mode=orc.MODE_BRUTE)
    compare_full(got, want, L)


@pytest.mark.parametrize("N,M,L", [
    (1, 1, 3), (2, 7, 2), (31, 1000, 4), (4095, 4097, 5), (4096, 8191, 3), (12345, 23456, 6),
    (100000, 77777, 5), (70001, 50000, 8),
])
def test_uniform_ragged_sizes(ctx, orc, N, M, L):
    src = workloads.uniform(N, 100 + N)
    recv = workloads.uniform(M, 200 + M)
    got, want = run_both(ctx, orc, src, recv, L)
    compare_full(got, want, L)


@pytest.mark.parametrize("L", [0, 1, 2, 3, 9, 10, 12, 21])
def test_levels_edge(ctx, orc, L):
    src = workloads.clumps(20000, 7, nclumps=5, sigma=0.02)
    recv = workloads.sphere(15000, 8)
    got, want = run_both(ctx, orc, src, recv, L)
    compare_full(got, want, L)


def test_empty_sets(ctx, orc):
    z = np.zeros((0, 3), np.float32)
    p = workloads.uniform(5000, 9)
    for src, recv in ((z, p), (p, z), (z, z)):
        got, want = run_both(ctx, orc, src, recv, 4)
        compare_full(got, want, 4)


def test_identical_points(ctx, orc):
    same = np.repeat(np.array([[0.3, 0.7, 0.1]], np.float32), 5000, axis=0)
    got, want = run_both(ctx, orc, same, workloads.uniform(3000, 4), 5)
    compare_full(got, want, 5)


def test_long_boxes_take_the_full_sort(ctx, orc):
    # 60000 points in 2 boxes at the sort depth: boxes far longer than the
    # finishing sort's window, distinct full keys inside them.
    rng = np.random.default_rng(5)
    p = (0.25 + 0.01 * rng.random((60000, 3))).astype(np.float32)
    p[:30000, 0] += 0.5
    got, want = run_both(ctx, orc, p, p[::-1].copy(), 3)
    compare_full(got, want, 3)


def test_faces_and_corners(ctx, orc):
    vals = np.array([0.0, 1.0, 0.5, 0.25, 0.75, 2.0 ** -21, 1 - 2.0 ** -24], np.float32)
    rng = np.random.default_rng(12)
    p = vals[rng.integers(0, len(vals), size=(9000, 3))]
    got, want = run_both(ctx, orc, p, workloads.uniform(4000, 13), 6)
    compare_full(got, want, 6)


def test_unaligned_coordinates(ctx, orc):
    """Coordinates starting 4 bytes past a 16-byte boundary take the plain-load path."""
    src = workloads.uniform(50001, 40)
    recv = workloads.clumps(30000, 41, nclumps=4, sigma=0.03)
    buf = torch.zeros(3 * 50001 + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(src.ravel()).cuda()
    s_dev = buf[1:].view(50001, 3)
    assert s_dev.data_ptr() % 16 == 4
    got = ctx.build(s_dev, _dev(recv), L=6).numpy()
    compare_full(got, orc.build_tree(src, recv, L=6), 6)


def test_aliased_sets(ctx, orc):
    p = workloads.clumps(30000, 14, nclumps=6, sigma=0.03)
    got, want = run_both(ctx, orc, p, p, 6, aliased=True)
    compare_full(got, want, 6)
    assert np.array_equal(got["src"]["perm"], got["recv"]["perm"])


def test_host_input_flag(ctx, orc):
    from paper_1301_1704_gb300 import fmmds
    src = workloads.uniform(20000, 15)
    recv = workloads.sphere(17000, 16)
    hs = torch.from_numpy(src).pin_memory()
    hr = torch.from_numpy(recv).pin_memory()
    got = ctx.build(hs, hr, L=5, flags=fmmds.FMM_FLAG_HOST_INPUT).numpy()
    compare_full(got, orc.build_tree(src, recv, L=5), 5)
    # pageable host memory too; and with the sorted points and onesweep passes
    got = ctx.build(torch.from_numpy(src), torch.from_numpy(recv), L=5,
                    flags=fmmds.FMM_FLAG_HOST_INPUT).numpy()
    compare_full(got, orc.build_tree(src, recv, L=5), 5)
    try:
        ctx.set_tuning(fmmds.FMM_SORT_ONESWEEP)
        t = ctx.build(hs, hr, L=5, flags=fmmds.FMM_FLAG_HOST_INPUT | fmmds.FMM_FLAG_SORTED_XYZ).numpy()
        want = orc.build_tree(src, recv, L=5)
        compare_full(t, want, 5)
        assert np.array_equal(t["sorted_src"], orc.sorted_points(src, want["src"]["perm"]))
    finally:
        ctx.set_tuning(fmmds.FMM_SORT_BUCKET)
    # the bucket path, each set boxed as soon as it has landed: with the
    # sorted points, and next to a set too dense for one sub-cell's block
    # (the build is redone on the radix path, copies included)
    t = ctx.build(hs, hr, L=5, flags=fmmds.FMM_FLAG_HOST_INPUT | fmmds.FMM_FLAG_SORTED_XYZ).numpy()
    want = orc.build_tree(src, recv, L=5)
    compare_full(t, want, 5)
    assert np.array_equal(t["sorted_recv"], orc.sorted_points(recv, want["recv"]["perm"]))
    tight = workloads.clumps(60000, 80, nclumps=2, sigma=0.002)
    ht = torch.from_numpy(tight).pin_memory()
    for a, b, ha, hb, L in ((src, tight, hs, ht, 6), (tight, src, ht, hs, 4)):
        got = ctx.build(ha, hb, L=L, flags=fmmds.FMM_FLAG_HOST_INPUT).numpy()
        compare_full(got, orc.build_tree(a, b, L=L), L)
    # sets copied in several pieces, the last one ragged: pinned (issued at
    # once) and pageable (issued piece by piece), bucket and radix paths
    bs = workloads.uniform(300001, 25)
    br = workloads.clumps(200003, 26, nclumps=4, sigma=0.05)
    want = orc.build_tree(bs, br, L=6)
    pinned = (torch.from_numpy(bs).pin_memory(), torch.from_numpy(br).pin_memory())
    for a, b in (pinned, (torch.from_numpy(bs), torch.from_numpy(br))):
        compare_full(ctx.build(a, b, L=6, flags=fmmds.FMM_FLAG_HOST_INPUT).numpy(), want, 6)
    try:
        ctx.set_tuning(fmmds.FMM_SORT_RTS)
        compare_full(ctx.build(*pinned, L=6, flags=fmmds.FMM_FLAG_HOST_INPUT).numpy(), want, 6)
    finally:
        ctx.set_tuning(fmmds.FMM_SORT_BUCKET)


@pytest.mark.parametrize("s", [1, 8, 64, 300])
def test_cluster_size_mode(ctx, orc, s):
    src = workloads.clumps(40000, 17, nclumps=8, sigma=0.02)
    recv = workloads.uniform(30000, 18)
    got = ctx.build(_dev(src), _dev(recv), s=s).numpy()
    want = orc.build_tree(src, recv, L=-1, s=s)
    assert (got["L"], got["s_unmet"]) == (want["L"], want["s_unmet"])
    compare_full(got, want, want["L"])


def test_domain_error_then_recovery(ctx, orc):
    from paper_1301_1704_gb300 import fmmds
    p = workloads.uniform(10000, 19)
    for bad in (np.nan, -0.5, 1.5):
        q = p.copy()
        q[1234, 1] = bad
        with pytest.raises(fmmds.FmmError) as e:
            ctx.build(_dev(q), _dev(p), L=4)
        assert e.value.code == fmmds.FMM_ERR_DOMAIN
    got, want = run_both(ctx, orc, p, p[:777].copy(), 4)
    compare_full(got, want, 4)


def test_allocator_failure_then_recovery(orc):
    """An allocator that returns NULL makes the build fail with FMM_ERR_OOM
    before any work; once it allocates again, the same context builds
    correctly."""
    import ctypes as C
    from paper_1301_1704_gb300 import fmmds
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = fmmds._load()
    state = {"fail": True, "live": {}}

    def _alloc(nbytes, stream, user):
        if state["fail"]:
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        state["live"][t.data_ptr()] = t
        return t.data_ptr()

    def _free(ptr, nbytes, stream, user):
        state["live"].pop(ptr, None)

    a_cb, f_cb = fmmds.ALLOC_FN(_alloc), fmmds.FREE_FN(_free)
    h = C.c_void_p()
    assert lib.fmm_create(C.byref(h), 0, a_cb, f_cb, None) == fmmds.FMM_OK
    try:
        p, q = workloads.uniform(5000, 3), workloads.uniform(4000, 4)
        dp, dq = _dev(p), _dev(q)
        torch.cuda.synchronize()

        def build():
            tc = fmmds.TreeC()
            st = lib.fmm_build(h, C.c_void_p(dp.data_ptr()), len(p), C.c_void_p(dq.data_ptr()),
                               len(q), fmmds.Params(4, 0, 0, 0), C.byref(tc), C.c_void_p(0))
            return st, tc

        st, _ = build()
        assert st == fmmds.FMM_ERR_OOM
        state["fail"] = False
        st, tc = build()
        assert st == fmmds.FMM_OK
        compare_full(fmmds._tree_from(tc, len(p), len(q)).numpy(), orc.build_tree(p, q, L=4), 4)
    finally:
        lib.fmm_destroy(h)


def test_bounded_wait_reports_timeout(ctx, orc):
    """One sort tile never publishes (test flag): the bounded look-back must
    give up with FMM_ERR_TIMEOUT, and the context must stay usable."""
    from paper_1301_1704_gb300 import fmmds
    p = workloads.uniform(200000, 20)
    with pytest.raises(fmmds.FmmError) as e:
        ctx.build(_dev(p), _dev(p[:1000].copy()), L=5, flags=fmmds.FMM_FLAG_TEST_STALL, wait_ms=100)
    assert e.value.code == fmmds.FMM_ERR_TIMEOUT
    got, want = run_both(ctx, orc, p[:50000].copy(), p[:1000].copy(), 5)
    compare_full(got, want, 5)


def test_bad_arguments(ctx):
    from paper_1301_1704_gb300 import fmmds
    p = _dev(workloads.uniform(10, 1))
    with pytest.raises(fmmds.FmmError) as e:
        ctx.build(p, p, L=22)
    assert e.value.code == fmmds.FMM_ERR_LEVEL
    with pytest.raises(ValueError):
        ctx.build(p, p)
    # more points than 32-bit offsets can index: refused before any work
    import ctypes as C
    lib = fmmds._load()
    tc = fmmds.TreeC()
    st = lib.fmm_build(ctx._h, C.c_void_p(p.data_ptr()), 1 << 31, C.c_void_p(p.data_ptr() + 4),
                       1 << 31, fmmds.Params(5, 0, 0, 0), C.byref(tc), C.c_void_p(0))
    assert st == fmmds.FMM_ERR_ARG


# ---------------------------------------------------------------------------
# Full-size workloads, in the launch configuration the benchmark times (the
# autotuner's choice on the same inputs): every output array of the whole
# tree -- permutations, boxes of every level, every E2 / E4 list -- against
# the oracle's build of the same inputs (its OpenMP build: the same source,
# pinned equal to the single-threaded one).

@pytest.mark.slow
@pytest.mark.parametrize("cfg", [2, 3])
def test_full_size_configs(ctx, orc, cfg):
    from paper_1301_1704_gb300 import fmmds
    src, recv, L = workloads.config_inputs(cfg)
    s, r = _dev(src), _dev(recv)
    ctx.autotune([(s, r)], L=L, trials=1)
    try:
        got = ctx.build(s, r, L=L).numpy()
    finally:
        ctx.set_tuning(fmmds.FMM_SORT_BUCKET)
    del s, r
    want = orc.build_tree(src, recv, L=L, mode=orc.MODE_STENCIL, parallel=True)
    compare_full(got, want, L)


# ---------------------------------------------------------------------------
# Box-key order (FMM_FLAG_BOX_ORDER): points ordered by (level-L key, index).

@pytest.mark.parametrize("L", [0, 1, 2, 5, 7, 12, 21])
def test_box_key_order_fixed_level(ctx, orc, L):
    from paper_1301_1704_gb300 import fmmds
    src = workloads.clumps(60000, 60 + L, nclumps=6, sigma=0.02)
    recv = workloads.uniform(40001, 61)
    got = ctx.build(_dev(src), _dev(recv), L=L, flags=fmmds.FMM_FLAG_BOX_ORDER).numpy()
    compare_full(got, orc.build_tree(src, recv, L=L, order=orc.ORDER_BOX), L)


def test_box_key_order_cluster_size_and_batched(ctx, orc):
    from paper_1301_1704_gb300 import fmmds
    pts = [workloads.clumps(30000, 70, nclumps=4, sigma=0.02), workloads.uniform(5000, 71),
           np.repeat(np.array([[0.5, 0.5, 0.5]], np.float32), 300, axis=0)]
    got = ctx.build(_dev(pts[0]), _dev(pts[1]), s=32, flags=fmmds.FMM_FLAG_BOX_ORDER).numpy()
    want = orc.build_tree(pts[0], pts[1], L=-1, s=32, order=orc.ORDER_BOX)
    assert got["L"] == want["L"]
    compare_full(got, want, want["L"])
    devs = [_dev(p) for p in pts]
    trees = ctx.build_batched([(d, d) for d in devs], s=16, flags=fmmds.FMM_FLAG_BOX_ORDER)
    for p, t in zip(pts, trees):
        want = orc.build_tree(p, p, L=-1, s=16, order=orc.ORDER_BOX)
        g = t.numpy()
        assert (g["L"], g["s_unmet"]) == (want["L"], want["s_unmet"])
        compare_full(g, want, want["L"])


# ---------------------------------------------------------------------------
# Sorted points (FMM_FLAG_SORTED_XYZ) and Alg. 2 over whole levels.

def test_sorted_points_and_e2_gather(ctx, orc):
    from paper_1301_1704_gb300 import fmmds
    src = workloads.clumps(40000, 90, nclumps=6, sigma=0.03)
    recv = workloads.uniform(9000, 91)
    L = 5
    tree = ctx.build(_dev(src), _dev(recv), L=L, flags=fmmds.FMM_FLAG_SORTED_XYZ)
    got = tree.numpy()
    want = orc.build_tree(src, recv, L=L)
    compare_full(got, want, L)
    assert np.array_equal(got["sorted_src"], orc.sorted_points(src, want["src"]["perm"]))
    assert np.array_equal(got["sorted_recv"], orc.sorted_points(recv, want["recv"]["perm"]))
    for level in (2, 4, L):
        off, pts = ctx.gather_e2(tree, level)
        woff, wpts = orc.gather_e2(want, src, level)
        assert np.array_equal(off.cpu().numpy().view(np.uint32).astype(np.uint64), woff)
        assert np.array_equal(pts.cpu().numpy(), wpts)


def test_sorted_points_aliased_and_long_boxes(ctx, orc):
    from paper_1301_1704_gb300 import fmmds
    rng = np.random.default_rng(92)
    p = (0.25 + 0.01 * rng.random((30000, 3))).astype(np.float32)  # boxes past the window
    t = ctx.build(_dev(p), _dev(p), L=3, flags=fmmds.FMM_FLAG_SORTED_XYZ).numpy()
    w = orc.build_tree(p, p, L=3)
    compare_full(t, w, 3)
    assert np.array_equal(t["sorted_src"], orc.sorted_points(p, w["src"]["perm"]))


@pytest.mark.parametrize("items", [4, 7, 8])
def test_sort_tile_sizes_agree(ctx, orc, items):
    """The tile-size knob (points per thread of a radix tile) changes no result."""
    from paper_1301_1704_gb300 import fmmds
    src = workloads.clumps(100003, 95, nclumps=10, sigma=0.03)
    recv = workloads.uniform(70001, 96)
    try:
        for kind in (fmmds.FMM_SORT_RTS, fmmds.FMM_SORT_FIXED_GRID):
            ctx.set_tuning(kind, items)
            assert ctx.tuning() == {"sort_kind": kind, "sort_items": items}
            got, want = run_both(ctx, orc, src, recv, 6)
            compare_full(got, want, 6)
        ctx.set_tuning(fmmds.FMM_SORT_RTS, items)
        got = ctx.build(_dev(src), _dev(recv), s=40).numpy()
        want = orc.build_tree(src, recv, L=-1, s=40)
        compare_full(got, want, want["L"])
    finally:
        ctx.set_tuning(fmmds.FMM_SORT_BUCKET, 6)


def test_autotune_picks_a_candidate(ctx, orc):
    from paper_1301_1704_gb300 import fmmds
    pts = [workloads.uniform(200000, 97), workloads.clumps(50000, 98, nclumps=4, sigma=0.02)]
    devs = [_dev(p) for p in pts]
    try:
        best = ctx.autotune([(d, d) for d in devs], s=64, trials=2)
        assert (best["sort_kind"], best["sort_items"]) in {
            (0, 4), (0, 6), (0, 7), (0, 8), (1, 6), (2, 4), (2, 6), (2, 7), (2, 8)}
        assert best["median_ms"] > 0
        assert ctx.tuning() == {"sort_kind": best["sort_kind"], "sort_items": best["sort_items"]}
        trees = ctx.build_batched([(d, d) for d in devs], s=64)
        for p, t in zip(pts, trees):
            want = orc.build_tree(p, p, L=-1, s=64)
            compare_full(t.numpy(), want, want["L"])
    finally:
        ctx.set_tuning(fmmds.FMM_SORT_BUCKET, 6)
    with pytest.raises(fmmds.FmmError):
        ctx.set_tuning(fmmds.FMM_SORT_RTS, 5)


# ---------------------------------------------------------------------------
# Alg. 6 source-box types.

@pytest.mark.parametrize("lpar", [2, 3, 4])
def test_box_types_match_oracle(ctx, orc, lpar):
    from oracle import box_types as BT
    p = workloads.clumps(50000, 100 + lpar, nclumps=8, sigma=0.06)
    L = 6
    d = _dev(p)
    tree = ctx.build(d, d, L=L)
    want_tree = orc.build_tree(p, p, L=L)
    compare_full(tree.numpy(), want_tree, L)
    rng = np.random.default_rng(lpar)
    nparts = 3
    owner = rng.integers(0, nparts, size=tree.src.nbox[lpar]).astype(np.uint32)
    od = torch.from_numpy(owner.view(np.int32)).cuda()
    for node in range(nparts):
        got = ctx.box_types(tree, lpar, od, node)
        want = BT.box_types(want_tree, lpar, owner, node)
        for l in range(2, L + 1):
            assert np.array_equal(got[l].cpu().numpy(), want[l]), (lpar, node, l)


# ---------------------------------------------------------------------------
# The bucket path (the default sort kind): cases that reach its rare branches.

def test_bucket_ties_below_the_kept_key_bits(ctx, orc):
    """An item keeps the key bits down to about level 18 (the rest of its 64
    bits hold the point index); points tied there but apart further down are
    ordered by their full keys recomputed from the coordinates, and runs of
    more tied points than one thread orders fall back to a full sort."""
    rng = np.random.default_rng(77)
    base = workloads.uniform(120000, 78)
    h = 2.0 ** -21
    parts = [base]
    for run in (2, 3, 17, 300):  # tied runs within one level-19 cell
        c = np.floor(rng.random(3) * 2 ** 19) / 2 ** 19
        off = rng.integers(0, 4, size=(run, 3)) * h
        parts.append((c + off).astype(np.float32))
    src = np.ascontiguousarray(np.concatenate(parts)[rng.permutation(sum(len(p) for p in parts))])
    recv = workloads.uniform(50000, 79)
    got, want = run_both(ctx, orc, src, recv, 6)
    compare_full(got, want, 6)
    # a run longer than one thread's share: the full-sort fallback
    c = np.floor(rng.random(3) * 2 ** 19) / 2 ** 19
    long_run = (c + rng.integers(0, 4, size=(3000, 3)) * h).astype(np.float32)
    src2 = np.ascontiguousarray(np.concatenate([base, long_run]))
    got, want = run_both(ctx, orc, src2, recv, 5)
    compare_full(got, want, 5)


def test_bucket_overflow_falls_back_to_radix(ctx, orc):
    """A cell holding more points than one block sorts sends its set to the
    radix path (the build is redone), alone or next to a set that fits."""
    tight = workloads.clumps(60000, 80, nclumps=2, sigma=0.002)
    loose = workloads.uniform(60000, 81)
    for src, recv, L in ((tight, loose, 6), (loose, tight, 4), (tight, tight, 8)):
        got, want = run_both(ctx, orc, src, recv, L)
        compare_full(got, want, L)


@pytest.mark.parametrize("n,L", [(1, 0), (5, 3), (4608, 2), (4609, 5), (36865, 1), (300001, 9),
                                 (2359297, 6)])
def test_bucket_cell_levels(ctx, orc, n, L):
    """Bucket cell levels 0..4 (the level follows n), box depths above and
    below the cell level, ragged tails of the count and scatter tiles."""
    src = workloads.uniform(n, 1000 + n)
    recv = workloads.sphere(max(1, n // 3), 2000 + n)
    got, want = run_both(ctx, orc, src, recv, L)
    compare_full(got, want, L)


def test_bucket_batched_sets_of_every_size(ctx, orc):
    """One batched fixed-level build whose sets sit at different bucket cell
    levels (and one too full for a block, on the radix path), all in the same
    launches."""
    pts = [workloads.uniform(n, 3000 + n) for n in (1, 700, 5000, 40000, 330000)]
    pts.append(workloads.clumps(50000, 3100, nclumps=1, sigma=0.001))
    devs = [_dev(p) for p in pts]
    trees = ctx.build_batched([(d, d) for d in devs], L=6)
    for p, t in zip(pts, trees):
        compare_full(t.numpy(), orc.build_tree(p, p, L=6), 6)


def test_workspace_bound_holds():
    """fmm_query_workspace bounds the arena a build needs: a fresh context's
    arena, sized from that bound, does not grow during the build -- also
    where the bucket path's sub-cells (room for one block's points each)
    outgrow the radix arrays, and where a set overflows and is redone."""
    from paper_1301_1704_gb300 import fmmds
    cases = [(workloads.uniform(5, 90), 2), (workloads.uniform(294913, 91), 2),
             (workloads.uniform(294913, 92), 7), (workloads.uniform(1 << 20, 93), 3),
             (workloads.clumps(300000, 94, nclumps=2, sigma=0.002), 4)]
    for pts, L in cases:
        d = _dev(pts)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        c = fmmds.Context(0)
        try:
            c.build(d, d, L=L, raw=True)
            torch.cuda.synchronize()
            used = torch.cuda.memory_allocated() - before
        finally:
            c.close()
        # torch's allocator rounds a block up (to 2 MiB for large ones); an
        # arena that grew would have added a chunk of 64 MiB or more
        bound = fmmds.query_workspace(len(pts), len(pts), L=L)
        assert used <= (bound + (2 << 20) - 1) // (2 << 20) * (2 << 20), (len(pts), L, used, bound)
