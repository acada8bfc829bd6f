"""Pins of the oracle's quantisation and Morton encoding (Sec. 1.4, Sec. 2:
"BoxIndex", interleave / deinterleave).

* bisection: the key's base-8 digits must be the octants met while bisecting
  the cube around the point (an independent, geometric definition of the
  Morton index, with 1.0 in the last cell);
* closed forms: a coordinate of all ones spreads to the geometric series
  sum_k 8^k = (2^63 - 1) / 7, times 1, 2, 4 for x, y, z;
* round trip encode/decode on random cells and every 0/max corner pattern;
* on x86 with BMI2, equality with the parallel-bit-deposit instruction.
"""
import ctypes
import os
import platform
import subprocess
import tempfile

import numpy as np
import pytest

from tests import geom_ref

MAXQ = (1 << 21) - 1


def _edge_points():
    vals = [0.0, 1.0, 0.5, 0.25, 0.75, 0.125, 1.0 / 1024, 1.0 - 2.0 ** -21, 2.0 ** -21,
            np.nextafter(np.float32(0.5), np.float32(0)), np.nextafter(np.float32(1), np.float32(0)),
            np.nextafter(np.float32(0.25), np.float32(1)), 3.0 * 2.0 ** -21]
    vals = np.array(vals, dtype=np.float32)
    rng = np.random.default_rng(11)
    pts = [[vals[i], vals[j], vals[k]] for i, j, k in rng.integers(0, len(vals), size=(60, 3))]
    return np.array(pts, dtype=np.float32)


def test_keys_match_geometric_bisection(orc):
    rng = np.random.default_rng(5)
    pts = np.concatenate([rng.random((200, 3)).astype(np.float32), _edge_points()])
    keys = orc.keys(pts)
    for p, k in zip(pts, keys):
        assert int(k) == geom_ref.path_to_int(geom_ref.octant_path(p, 21)), p


def test_level_keys_are_path_prefixes(orc):
    rng = np.random.default_rng(6)
    pts = rng.random((64, 3)).astype(np.float32)
    keys = orc.keys(pts)
    for p, k in zip(pts, keys):
        path = geom_ref.octant_path(p, 21)
        for l in (1, 2, 5, 9, 20):
            assert int(k) >> (3 * (21 - l)) == geom_ref.path_to_int(path[:l])


def test_corner_closed_forms(orc):
    series = ((1 << 63) - 1) // 7  # sum_{k<21} 8^k
    assert series == 0x1249249249249249
    assert orc.encode(MAXQ, 0, 0) == series
    assert orc.encode(0, MAXQ, 0) == 2 * series
    assert orc.encode(0, 0, MAXQ) == 4 * series
    assert orc.encode(MAXQ, MAXQ, MAXQ) == (1 << 63) - 1
    assert orc.encode(0, 0, 0) == 0
    # single bits: bit k of x/y/z lands at 3k/3k+1/3k+2
    for k in range(21):
        assert orc.encode(1 << k, 0, 0) == 1 << (3 * k)
        assert orc.encode(0, 1 << k, 0) == 1 << (3 * k + 1)
        assert orc.encode(0, 0, 1 << k) == 1 << (3 * k + 2)


def test_encode_decode_round_trip(orc):
    rng = np.random.default_rng(7)
    cases = [tuple(int(v) for v in rng.integers(0, MAXQ + 1, size=3)) for _ in range(300)]
    for m in range(8):
        cases.append(tuple(MAXQ if (m >> d) & 1 else 0 for d in range(3)))
    for c in cases:
        assert orc.decode(orc.encode(*c, 21), 21) == c
    for bits in (1, 2, 4, 7, 9):
        for _ in range(50):
            c = tuple(int(v) for v in rng.integers(0, 1 << bits, size=3))
            key = orc.encode(*c, bits)
            assert key < (1 << (3 * bits))
            assert orc.decode(key, bits) == c


def test_domain_and_boundary(orc):
    assert int(orc.keys(np.array([[1.0, 1.0, 1.0]], np.float32))[0]) == (1 << 63) - 1
    assert int(orc.keys(np.array([[-0.0, 0.0, 0.0]], np.float32))[0]) == 0
    for bad in (np.nan, -1e-7, 1.0000001, np.inf, -np.inf):
        with pytest.raises(orc.OracleError) as e:
            orc.keys(np.array([[0.5, bad, 0.5]], np.float32))
        assert e.value.code == orc.ORC_ERR_DOMAIN


@pytest.mark.skipif(platform.machine() not in ("x86_64", "AMD64"), reason="BMI2 is x86 only")
def test_keys_match_pdep_instruction(orc):
    flags = open("/proc/cpuinfo").read() if os.path.exists("/proc/cpuinfo") else ""
    if " bmi2" not in flags:
        pytest.skip("no BMI2 on this host")
    src = r"""
    #include <immintrin.h>
    #include <stdint.h>
    uint64_t dep(uint32_t x, uint32_t y, uint32_t z) {
      return _pdep_u64(x, 0x1249249249249249ull) | _pdep_u64(y, 0x2492492492492492ull)
           | _pdep_u64(z, 0x4924924924924924ull);
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c, so = os.path.join(d, "pdep.c"), os.path.join(d, "pdep.so")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-O1", "-mbmi2", "-shared", "-fPIC", c, "-o", so])
        lib = ctypes.CDLL(so)
        lib.dep.argtypes = [ctypes.c_uint32] * 3
        lib.dep.restype = ctypes.c_uint64
        rng = np.random.default_rng(8)
        for _ in range(2000):
            x, y, z = (int(v) for v in rng.integers(0, MAXQ + 1, size=3))
            assert orc.encode(x, y, z, 21) == lib.dep(x, y, z)
