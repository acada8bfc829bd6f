"""CPU oracle of one served time step: the counter-based Gaussian
displacement of every point, with reflection at the cube walls.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use it.

The paper rebuilds its structures every time step of a dynamic simulation
(Sec. 1, Sec. 6) but fixes no motion; the served workload moves each point by
an independent N(0, sigma^2) step per axis and reflects it at the walls of
the unit cube.  The random numbers come from a counter-based generator so
that a point's step depends only on (system seed, step number, point index),
never on which other systems share a batched build:

  * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
    easy as 1, 2, 3", SC'11, Sec. 4.1): a 4 x 32-bit counter and a 2 x 32-bit
    key; ten rounds, each multiplying counter words 0 and 2 by the two
    Philox multipliers, swapping in the high / low halves xor-ed with the
    other counter words and the key; the key is bumped by the two Weyl
    constants between rounds.
  * counter = (point index, step low word, step high word, 0), key = (seed
    low word, seed high word); the four output words r0..r3 become uniforms
    u_k = (floor(r_k / 2^9) + 1/2) * 2^-23 in (0, 1) (exact in float32);
  * Box-Muller: z_x = sqrt(-2 ln u0) cos(2 pi u1), z_y = sqrt(-2 ln u0)
    sin(2 pi u1), z_z = sqrt(-2 ln u2) cos(2 pi u3);
  * x' = x + sigma z per axis, then x' < 0 -> -x', x' > 1 -> 2 - x'.

Arithmetic here is float64 (the GPU path computes in float32; tests compare
within a stated tolerance).
"""
from __future__ import annotations

import numpy as np

PHILOX_M = (0xD2511F53, 0xCD9E8D57)   # round multipliers
PHILOX_W = (0x9E3779B9, 0xBB67AE85)   # key increments (Weyl sequence)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of counters ``[n, 4]`` (uint32) under key (k0, k1)."""
    c = np.asarray(counter, dtype=np.uint64).reshape(-1, 4)
    k0, k1 = np.uint64(int(key[0]) & 0xFFFFFFFF), np.uint64(int(key[1]) & 0xFFFFFFFF)
    m0, m1 = np.uint64(PHILOX_M[0]), np.uint64(PHILOX_M[1])
    w0, w1 = np.uint64(PHILOX_W[0]), np.uint64(PHILOX_W[1])
    for _ in range(10):
        p0 = m0 * c[:, 0]  # 32 x 32 -> 64-bit products
        p1 = m1 * c[:, 2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
        k0 = (k0 + w0) & _MASK
        k1 = (k1 + w1) & _MASK
    return c.astype(np.uint32)


def uniforms(words: np.ndarray) -> np.ndarray:
    """32-bit words -> uniforms in (0, 1): (floor(r / 2^9) + 1/2) * 2^-23."""
    return ((np.asarray(words, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def normals(n: int, seed: int, step: int) -> np.ndarray:
    """The [n, 3] standard normal draws of points 0..n-1 at `step`."""
    i = np.arange(n, dtype=np.uint64)
    ctr = np.stack([i & _MASK,
                    np.full(n, step & 0xFFFFFFFF, np.uint64),
                    np.full(n, (step >> 32) & 0xFFFFFFFF, np.uint64),
                    np.zeros(n, np.uint64)], axis=1)
    r = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    u = uniforms(r)
    rad0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    rad1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    return np.stack([rad0 * np.cos(2.0 * np.pi * u[:, 1]),
                     rad0 * np.sin(2.0 * np.pi * u[:, 1]),
                     rad1 * np.cos(2.0 * np.pi * u[:, 3])], axis=1)


def reflect(x: np.ndarray) -> np.ndarray:
    """Mirror at the walls of [0, 1] (one reflection: steps are far below 1)."""
    x = np.where(x < 0.0, -x, x)
    return np.where(x > 1.0, 2.0 - x, x)


def displace(xyz: np.ndarray, seed: int, step: int, sigma: float) -> np.ndarray:
    """One time step of the points ``xyz`` [n, 3] (float64 result)."""
    x = np.asarray(xyz, dtype=np.float64)
    return reflect(x + sigma * normals(x.shape[0], seed, step))


def sigma_of(level: int, scale: float = 0.1) -> float:
    """Step size: scale times the finest box size 2^-L, rounded to float32
    (the value the device receives)."""
    return float(np.float32(scale * 2.0 ** -level))
