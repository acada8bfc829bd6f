"""The seeded inputs have the shapes the workloads state: uniform in the unit
cube, a sphere surface of radius 0.4 with 1e-3 radial jitter, 64 Gaussian
clumps of sigma 0.01 with centres in [0.1, 0.9]^3, log-uniform batch sizes.
CPU only."""
import numpy as np

from paper_1301_1704_gb300 import workloads


def _common(p, n):
    assert p.dtype == np.float32 and p.shape == (n, 3) and p.flags.c_contiguous
    assert np.all(p >= 0.0) and np.all(p < 1.0)


def test_uniform():
    p = workloads.uniform(200000, 3)
    _common(p, 200000)
    assert np.allclose(p.mean(axis=0), 0.5, atol=5e-3)
    assert np.allclose(p.var(axis=0), 1.0 / 12.0, atol=2e-3)
    counts = np.histogram(p[:, 0], bins=16, range=(0.0, 1.0))[0]
    assert counts.min() > 0.9 * 200000 / 16
    assert np.array_equal(p, workloads.uniform(200000, 3))  # seeded
    assert not np.array_equal(p, workloads.uniform(200000, 4))


def test_sphere():
    p = workloads.sphere(100000, 5)
    _common(p, 100000)
    r = np.linalg.norm(p.astype(np.float64) - 0.5, axis=1)
    assert abs(r.mean() - 0.4) < 1e-4 and abs(r.std() - 1e-3) < 1e-4
    d = (p.astype(np.float64) - 0.5) / r[:, None]
    assert np.allclose(d.mean(axis=0), 0.0, atol=1e-2)  # directions isotropic


def test_clumps():
    p = workloads.clumps(200000, 6)
    _common(p, 200000)
    rng = np.random.Generator(np.random.PCG64(6))
    centres = 0.1 + 0.8 * rng.random((64, 3))  # the generator's own first draw
    dist = np.linalg.norm(p[:, None, :].astype(np.float64) - centres[None], axis=2)
    near = dist.argmin(axis=1)
    off = p.astype(np.float64) - centres[near]
    assert abs(off.std() - 0.01) < 1e-3
    assert len(np.unique(near)) == 64
    assert np.bincount(near, minlength=64).min() > 0.5 * 200000 / 64


def test_batch_sets():
    sets, kinds = workloads.batch_sets(workloads.CONFIG_SEEDS[4])
    n = np.array([len(s) for s in sets])
    assert len(sets) == 512 and n.min() >= 1000 and n.max() <= 1000000
    logn = np.log(n)
    assert abs(logn.mean() - 0.5 * (np.log(1e3) + np.log(1e6))) < 0.3  # log-uniform
    counts = np.bincount(np.asarray(kinds), minlength=3)  # uniform / sphere / clumps, 1/3 each
    assert len(counts) == 3 and counts.min() > 512 / 3 - 45
