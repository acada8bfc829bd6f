"""fmm_exclusive_scan_noalloc through the C ABI.

Callers that must not allocate device memory while they run (a loop that
reserved all device memory up front, code where the CUDA allocator may not be
called) get the CSR row starts of per-box counts from this entry point.  The
test turns the E2 / E4 row starts of an ordinary fmm_build back into counts,
rescans them with the no-allocation entry point twice in a row (different
sizes, the shared scratch reused) and requires the same row starts, bit for
bit, as fmm_build produced.  This file sorts last so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1301_1704_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_scan_matches_build_offsets():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_1704_gb300 import build, fmmds
    build.build()
    ctx = fmmds.Context(0)
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
            fmmds.exclusive_scan_noalloc(counts, got, total)
            torch.cuda.synchronize()
            assert torch.equal(got, want)
            assert int(total.item()) == int(want[-1].item())
        # sizes beyond the fixed scratch are refused before anything runs
        out = torch.zeros(2, dtype=torch.int32, device="cuda")
        st = fmmds.library().fmm_exclusive_scan_noalloc(
            out.data_ptr(), fmmds.FMM_NOALLOC_SCAN_MAX + 1, out.data_ptr(), None, None)
        assert st == fmmds.FMM_ERR_ARG
    finally:
        ctx.close()
