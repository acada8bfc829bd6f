"""Graph mode (fmm_set_graphs): fixed-depth builds after a context's first
one record their launches into a CUDA graph that is updated and launched.
Every result must equal the oracle's, bit for bit, including time steps that
rebuild from the same device buffers with new coordinates, changes of shape,
batched builds, cluster-size builds (which run eagerly), the full-key re-sort
of long boxes after the graph, and a failing build in the middle."""
import numpy as np
import pytest

from paper_1301_1704_gb300 import workloads
from tests.test_gpu_parity import compare_full

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture()
def gctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_1704_gb300 import build, fmmds
    build.build()
    c = fmmds.Context(0)
    c.set_graphs(True)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_time_steps_from_the_same_buffers(gctx, orc):
    n, m, L = 30000, 20000, 5
    s_dev = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    r_dev = torch.empty((m, 3), dtype=torch.float32, device="cuda")
    inst = []
    for step in range(4):
        src = workloads.uniform(n, 100 + step)
        recv = workloads.clumps(m, 200 + step, nclumps=5, sigma=0.03)
        s_dev.copy_(torch.from_numpy(src))
        r_dev.copy_(torch.from_numpy(recv))
        got = gctx.build(s_dev, r_dev, L=L).numpy()
        compare_full(got, orc.build_tree(src, recv, L=L), L)
        inst.append(gctx.graph_stats()["instantiations"])
    st = gctx.graph_stats()
    assert st["launches"] > 0  # builds after the first ran as graphs
    assert inst[0] == 0 and inst[1] > 0
    assert inst[3] == inst[2] == inst[1]  # same shape: updated, not rebuilt


def test_shape_changes_and_batched_fixed_levels(gctx, orc):
    for k, (n, m, L) in enumerate(((20000, 9000, 4), (45000, 45000, 6), (20000, 9000, 4))):
        src = workloads.sphere(n, 300 + k)
        recv = workloads.uniform(m, 400 + k)
        got = gctx.build(_dev(src), _dev(recv), L=L).numpy()
        compare_full(got, orc.build_tree(src, recv, L=L), L)
    sets = [workloads.uniform(7000, 501), workloads.clumps(12000, 502, nclumps=3, sigma=0.02),
            workloads.sphere(3000, 503)]
    devs = [_dev(p) for p in sets]
    for _ in range(2):
        trees = gctx.build_batched([(d, d) for d in devs], levels=[3, 5, 4])
        for p, t, L in zip(sets, trees, (3, 5, 4)):
            compare_full(t.numpy(), orc.build_tree(p, p, L=L), L)


def test_cluster_size_builds_run_eagerly(gctx, orc):
    sets = [workloads.clumps(25000, 601, nclumps=6, sigma=0.02), workloads.uniform(9000, 602)]
    devs = [_dev(p) for p in sets]
    for step in range(3):
        if step:
            for p, d in zip(sets, devs):
                p[:] = np.clip(p + np.float32(1e-3) * step, 0.0, 1.0)
                d.copy_(torch.from_numpy(p))
        before = gctx.graph_stats()["launches"]
        trees = gctx.build_batched([(d, d) for d in devs], s=48)
        assert gctx.graph_stats()["launches"] == before
        for p, t in zip(sets, trees):
            w = orc.build_tree(p, p, L=-1, s=48)
            assert t.L == w["L"]
            compare_full(t.numpy(), w, w["L"])


def test_long_boxes_and_a_failing_build(gctx, orc):
    from paper_1301_1704_gb300 import fmmds
    rng = np.random.default_rng(7)
    p = (0.25 + 0.01 * rng.random((60000, 3))).astype(np.float32)
    p[:30000, 0] += 0.5
    q = p[::-1].copy()
    for _ in range(2):  # boxes longer than the finishing window: full-key re-sort
        got = gctx.build(_dev(p), _dev(q), L=3).numpy()
        compare_full(got, orc.build_tree(p, q, L=3), 3)
    bad = p.copy()
    bad[17, 2] = np.nan
    with pytest.raises(fmmds.FmmError) as e:
        gctx.build(_dev(bad), _dev(q), L=3)
    assert e.value.code == fmmds.FMM_ERR_DOMAIN
    u = workloads.uniform(40000, 8)
    got = gctx.build(_dev(u), _dev(q), L=4).numpy()
    compare_full(got, orc.build_tree(u, q, L=4), 4)
