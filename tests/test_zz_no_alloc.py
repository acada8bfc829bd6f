"""fmm_exclusive_scan_noalloc through the C ABI.

Callers that must not allocate device memory while they run (a loop that
reserved all device memory up front, code where the CUDA allocator may not be
called) get the CSR row starts of per-box counts from this entry point.  The
tests check it three ways:

* against a host prefix sum (numpy) at the edge sizes -- no counts, one
  count, a single partial tile, one tile plus or minus one, the largest size
  the fixed scratch takes -- and with totals past 2^32 (the 64-bit total);
* against the row starts of an ordinary fmm_build: its E2 / E4 row starts are
  turned back into counts and rescanned twice in a row (different sizes, the
  shared scratch reused), and must come back bit for bit;
* for what it is for: a call leaves both PyTorch's allocator and the
  device's free memory (cudaMemGetInfo) exactly as they were.

This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_1301_1704_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_1704_gb300 import build, fmmds
    build.build()
    return fmmds


def _scan(fm, counts_np):
    """Device scan of host counts; returns (offsets as uint32, 64-bit total)."""
    n = len(counts_np)
    counts = torch.from_numpy(counts_np.astype(np.uint32).view(np.int32)).cuda()
    offsets = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    fm.exclusive_scan_noalloc(counts, offsets, total)
    torch.cuda.synchronize()
    return offsets.cpu().numpy().view(np.uint32), int(total.cpu().numpy().view(np.uint64)[0])


def _want(counts_np):
    c = np.concatenate([np.zeros(1, np.uint64),
                        np.cumsum(counts_np.astype(np.uint64), dtype=np.uint64)])
    return (c & np.uint64(0xffffffff)).astype(np.uint32), int(c[-1])


@pytest.mark.parametrize("n", [0, 1, 5, 4095, 4096, 4097, 3 * 4096 + 17, None])
def test_noalloc_scan_matches_host_prefix_sum(fm, n):
    if n is None:
        n = fm.FMM_NOALLOC_SCAN_MAX  # the largest size the fixed scratch takes
    rng = np.random.default_rng(n + 1)
    counts = rng.integers(0, 200, size=n).astype(np.uint32)
    got, tot = _scan(fm, counts)
    want, wtot = _want(counts)
    assert np.array_equal(got, want)
    assert tot == wtot


def test_noalloc_scan_totals_past_32_bits(fm):
    rng = np.random.default_rng(7)
    for n in (1, 17, 4097, 70000):
        counts = rng.integers(1 << 30, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        got, tot = _scan(fm, counts)
        want, wtot = _want(counts)
        assert wtot >= (1 << 32) or n == 1
        assert np.array_equal(got, want), n
        assert tot == wtot, n


def test_noalloc_scan_matches_build_offsets(fm):
    ctx = fm.Context(0)
    try:
        src = torch.from_numpy(workloads.uniform(300000, 71)).cuda()
        recv = torch.from_numpy(workloads.clumps(250000, 72, nclumps=8, sigma=0.03)).cuda()
        tree = ctx.build(src, recv, L=6)
        cases = [tree.e4_off[6], tree.e2_off[5]]  # two calls in a row, different sizes
        for off in cases:
            want = off.clone()
            counts = (want[1:] - want[:-1]).contiguous()
            got = torch.full_like(want, -1)
            total = torch.zeros(1, dtype=torch.int64, device="cuda")
            fm.exclusive_scan_noalloc(counts, got, total)
            torch.cuda.synchronize()
            assert torch.equal(got, want)
            assert int(total.item()) == int(want[-1].item())
    finally:
        ctx.close()


def test_noalloc_scan_allocates_nothing(fm):
    n = 1 << 20
    counts = torch.randint(0, 1000, (n,), dtype=torch.int32, device="cuda")
    offsets = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    # a first call loads the kernel and looks the scratch up
    fm.exclusive_scan_noalloc(counts, offsets, total)
    torch.cuda.synchronize()
    before_torch = torch.cuda.memory_allocated()
    before_free = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        fm.exclusive_scan_noalloc(counts, offsets, total)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before_torch
    assert torch.cuda.mem_get_info()[0] == before_free
    want, wtot = _want(counts.cpu().numpy().view(np.uint32))
    assert np.array_equal(offsets.cpu().numpy().view(np.uint32), want)
    assert int(total.item()) == wtot


def test_noalloc_scan_refuses_bad_arguments(fm):
    out = torch.zeros(2, dtype=torch.int32, device="cuda")
    # sizes beyond the fixed scratch are refused before anything runs
    st = fm.library().fmm_exclusive_scan_noalloc(
        out.data_ptr(), fm.FMM_NOALLOC_SCAN_MAX + 1, out.data_ptr(), None, None)
    assert st == fm.FMM_ERR_ARG
    cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        fm.exclusive_scan_noalloc(cnt, torch.zeros(4, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        fm.exclusive_scan_noalloc(cnt.cpu(), torch.zeros(5, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        fm.exclusive_scan_noalloc(cnt, torch.zeros(5, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        fm.exclusive_scan_noalloc(cnt, torch.zeros(5, dtype=torch.int32, device="cuda"),
                                  torch.zeros(1, dtype=torch.int32, device="cuda"))
