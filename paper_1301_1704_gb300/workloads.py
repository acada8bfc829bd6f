"""Seeded synthetic point sets shaped like the paper's workloads.

This module only draws points: it holds none of the structure-building
arithmetic, so both the GPU tests and the CPU oracle take their inputs from
here.  Every generator returns a C-contiguous float32 array of shape
``[n, 3]`` with every coordinate in [0, 1) (samples that fall outside are
redrawn), drawn from numpy's PCG64 with the given seed.

Workload shapes (Sec. 4 of the paper):
  * ``uniform``: i.i.d. uniform in the unit cube (the single-node table);
  * ``sphere``: points on a sphere surface (the second single-node test),
    radius 0.4 about the cube centre with Gaussian radial jitter;
  * ``clumps``: Gaussian clumps, a strongly non-uniform octree.
"""
from __future__ import annotations

import numpy as np

CONFIG_SEEDS = {1: (1, 2), 2: (3, 4), 3: (5, 6), 4: 7, 5: 8}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _clip_redraw(pts: np.ndarray, redraw) -> np.ndarray:
    """Cast to float32 and redraw any row with a coordinate outside [0, 1)."""
    out = pts.astype(np.float32)
    bad = ~np.all((out >= 0.0) & (out < 1.0), axis=1)
    while bad.any():
        out[bad] = redraw(int(bad.sum())).astype(np.float32)
        bad = ~np.all((out >= 0.0) & (out < 1.0), axis=1)
    return np.ascontiguousarray(out)


def uniform(n: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    return _clip_redraw(rng.random((n, 3)), lambda k: rng.random((k, 3)))


def sphere(n: int, seed: int, radius: float = 0.4, jitter: float = 1e-3) -> np.ndarray:
    rng = _rng(seed)

    def draw(k):
        d = rng.standard_normal((k, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        r = radius + jitter * rng.standard_normal((k, 1))
        return 0.5 + r * d

    return _clip_redraw(draw(n), draw)


def clumps(n: int, seed: int, nclumps: int = 64, sigma: float = 0.01) -> np.ndarray:
    rng = _rng(seed)
    centres = 0.1 + 0.8 * rng.random((nclumps, 3))

    def draw(k):
        c = centres[rng.integers(0, nclumps, size=k)]
        return c + sigma * rng.standard_normal((k, 3))

    return _clip_redraw(draw(n), draw)


def sphere_and_clumps(n: int, seed: int) -> np.ndarray:
    """First half on the sphere surface, second half in 64 clumps."""
    h = n // 2
    return np.ascontiguousarray(np.concatenate([sphere(h, seed), clumps(n - h, seed + 1000)]))


def lattice(level: int) -> np.ndarray:
    """One point at the centre of every box of ``level`` (a full octree)."""
    m = 1 << level
    g = (np.arange(m, dtype=np.float64) + 0.5) / m
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.ascontiguousarray(np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32))


def config_inputs(cfg: int, scale: float = 1.0):
    """(src, recv, L) of configurations 1-3; ``scale`` shrinks n for tests."""
    if cfg == 1:
        n, L, gen = 16384, 4, uniform
    elif cfg == 2:
        n, L, gen = 1 << 24, 7, uniform
    elif cfg == 3:
        n, L, gen = 1 << 24, 9, sphere_and_clumps
    else:
        raise ValueError("configs 1-3 are single builds")
    n = max(1, int(round(n * scale)))
    s1, s2 = CONFIG_SEEDS[cfg]
    return gen(n, s1), gen(n, s2), L


def batch_sets(seed: int = 7, nsets: int = 512, lo: float = 1e3, hi: float = 1e6):
    """Batched workload: ``nsets`` sets with log-uniform sizes in [lo, hi],
    each uniform, sphere-surface or Gaussian clumps with probability 1/3."""
    rng = _rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=nsets))).astype(np.int64)
    kinds = rng.integers(0, 3, size=nsets)
    sets = []
    for i, (n, k) in enumerate(zip(sizes, kinds)):
        sub = seed * 100003 + i
        gen = (uniform, sphere, clumps)[int(k)]
        sets.append(gen(int(n), sub))
    return sets, kinds
