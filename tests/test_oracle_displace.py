"""Pins of the served-step oracle (oracle/displace.py) against what the
generator's publication and the mathematics fix, with no GPU."""
import json
import os

import numpy as np
import pytest

from oracle import displace as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")


def test_philox_known_answers():
    kat = json.load(open(GOLDEN))
    for v in kat["vectors"]:
        ctr = np.array([[int(x, 16) for x in v["counter"]]], dtype=np.uint64)
        key = [int(x, 16) for x in v["key"]]
        got = D.philox4x32_10(ctr, key)[0]
        assert [int(x) for x in got] == [int(x, 16) for x in v["out"]]


def test_philox_is_a_function_of_counter_and_key_only():
    ctr = np.array([[7, 1, 0, 0], [8, 1, 0, 0], [7, 2, 0, 0]], dtype=np.uint64)
    a = D.philox4x32_10(ctr, (5, 0))
    b = D.philox4x32_10(ctr[::-1].copy(), (5, 0))[::-1]
    assert np.array_equal(a, b)                    # no state carried between counters
    assert not np.array_equal(a[0], a[1]) and not np.array_equal(a[0], a[2])
    assert not np.array_equal(a, D.philox4x32_10(ctr, (6, 0)))


def test_uniforms_open_interval_and_float32_exact():
    w = np.array([0, 1, 511, 512, 0xFFFFFFFF], dtype=np.uint64)
    u = D.uniforms(w)
    assert u[0] == u[1] == u[2] == 2.0 ** -24 and u[3] == 3 * 2.0 ** -24
    assert u[-1] == 1.0 - 2.0 ** -24
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_normals_statistics():
    # 2^20 points x 3 axes: mean, variance, fourth moment and tail mass of a
    # standard normal, and no correlation between the axes.
    z = D.normals(1 << 20, seed=12345, step=3)
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs((z ** 4).mean() - 3.0) < 5 * np.sqrt(96.0 / n)
    tail = np.mean(np.abs(z) > 1.959963984540054)
    assert abs(tail - 0.05) < 5 * np.sqrt(0.05 * 0.95 / n)
    c = np.corrcoef(z.T)
    assert np.all(np.abs(c - np.eye(3)) < 5 / np.sqrt(z.shape[0]))


def test_quantiles_match_the_normal_distribution():
    st = pytest.importorskip("scipy.stats")
    z = D.normals(200000, seed=9, step=0).ravel()
    assert st.kstest(z, "norm").pvalue > 1e-4


def test_steps_differ_and_repeat():
    a = D.normals(1000, 1, 5)
    assert np.array_equal(a, D.normals(1000, 1, 5))
    assert not np.allclose(a, D.normals(1000, 1, 6))
    assert not np.allclose(a, D.normals(1000, 2, 5))
    # a point's draw does not depend on how many points the set has
    assert np.array_equal(a[:10], D.normals(10, 1, 5))
    # the step counter's high word is used
    assert not np.allclose(D.normals(10, 1, 5), D.normals(10, 1, 5 + (1 << 32)))


def test_reflection_keeps_points_in_the_cube():
    e = 2.0 ** -30
    x = np.array([-0.25, -e, 0.0, 0.5, 1.0, 1.0 + e, 1.25])
    assert np.array_equal(D.reflect(x), [0.25, e, 0.0, 0.5, 1.0, 1.0 - e, 0.75])
    rng = np.random.default_rng(0)
    p = rng.random((50000, 3))
    q = D.displace(p, seed=4, step=1, sigma=0.05)
    assert np.all((q >= 0) & (q <= 1))
    # away from the walls the step is exactly sigma * z
    z = D.normals(p.shape[0], 4, 1)
    far = np.all((p + 0.05 * z > 0) & (p + 0.05 * z < 1), axis=1)
    assert far.mean() > 0.5
    assert np.array_equal(q[far], p[far] + 0.05 * z[far])


def test_sigma_of_level():
    assert D.sigma_of(0) == float(np.float32(0.1))
    assert D.sigma_of(10) == float(np.float32(0.1 / 1024))
