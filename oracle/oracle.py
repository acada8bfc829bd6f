"""Python access to the CPU oracle (``fmm_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may use this module; the library never
does.  It compiles ``fmm_oracle.cpp`` with the host C++ compiler on first use
(or via :func:`build`) and returns plain numpy arrays.

Status codes are the oracle's own: 0 ok, 1 bad argument, 2 a coordinate
outside [0, 1] or NaN, 3 bad level / cluster size.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle_fmm.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_ERR_ARG, ORC_ERR_DOMAIN, ORC_ERR_LEVEL = 0, 1, 2, 3
MODE_STENCIL, MODE_BRUTE, MODE_NOLISTS = 0, 1, 2
ORDER_KEY, ORDER_BOX = 0, 16  # point order: (full key, index) or (level-L key, index)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


_LIB_OMP = os.path.join(_HERE, "liboracle_fmm_omp.so")
_lib_omp = None


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle_fmm.so`` (plain -O2, one
    core), or with ``parallel`` the same source with OpenMP and libstdc++'s
    parallel mode (all cores: key loop, sort, per-box list blocks) into
    ``oracle/liboracle_fmm_omp.so``.  Both compute the same result."""
    lib = _LIB_OMP if parallel else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        cxx = os.environ.get("CXX", "g++")
        tmp = lib + f".tmp{os.getpid()}"
        extra = ["-fopenmp", "-D_GLIBCXX_PARALLEL"] if parallel else []
        subprocess.check_call([cxx, "-std=c++17", "-O2", "-fPIC", "-shared", *extra, _SRC,
                               "-o", tmp])
        os.replace(tmp, lib)
    return lib


def _load(parallel: bool = False):
    global _lib, _lib_omp
    with _lock:
        if parallel and _lib_omp is not None:
            return _lib_omp
        if not parallel and _lib is not None:
            return _lib
        lib = C.CDLL(build(parallel=parallel))
        u32p, u64p, f32p = C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), C.POINTER(C.c_float)
        lib.orc_keys.argtypes = [f32p, C.c_uint32, u64p]
        lib.orc_keys.restype = C.c_int
        lib.orc_encode.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_int]
        lib.orc_encode.restype = C.c_uint64
        lib.orc_decode.argtypes = [C.c_uint64, C.c_int, C.POINTER(C.c_int64)]
        lib.orc_decode.restype = None
        lib.orc_build.argtypes = [f32p, C.c_uint32, f32p, C.c_uint32, C.c_int, C.c_uint32, C.c_int,
                                  C.POINTER(C.c_void_p)]
        lib.orc_build.restype = C.c_int
        lib.orc_free.argtypes = [C.c_void_p]
        lib.orc_free.restype = None
        for name in ("orc_level", "orc_s_unmet"):
            getattr(lib, name).argtypes = [C.c_void_p]
            getattr(lib, name).restype = C.c_int
        lib.orc_perm.argtypes = [C.c_void_p, C.c_int]
        lib.orc_perm.restype = u32p
        lib.orc_sorted_keys.argtypes = [C.c_void_p, C.c_int]
        lib.orc_sorted_keys.restype = u64p
        lib.orc_nbox.argtypes = [C.c_void_p, C.c_int, C.c_int]
        lib.orc_nbox.restype = C.c_uint32
        lib.orc_box_keys.argtypes = [C.c_void_p, C.c_int, C.c_int]
        lib.orc_box_keys.restype = u64p
        for name in ("orc_box_off", "orc_box_parent", "orc_box_child"):
            getattr(lib, name).argtypes = [C.c_void_p, C.c_int, C.c_int]
            getattr(lib, name).restype = u32p
        lib.orc_box_child_len.argtypes = [C.c_void_p, C.c_int, C.c_int]
        lib.orc_box_child_len.restype = C.c_uint32
        lib.orc_nnz.argtypes = [C.c_void_p, C.c_int, C.c_int]
        lib.orc_nnz.restype = C.c_uint64
        lib.orc_list_off.argtypes = [C.c_void_p, C.c_int, C.c_int]
        lib.orc_list_off.restype = u32p
        lib.orc_list_idx.argtypes = [C.c_void_p, C.c_int, C.c_int]
        lib.orc_list_idx.restype = u32p
        lib.orc_box_lists.argtypes = [u64p, C.c_uint32, C.c_int, C.c_uint64, C.c_int, u32p, u32p,
                                      u32p, u32p]
        lib.orc_box_lists.restype = C.c_int
        if parallel:
            _lib_omp = lib
        else:
            _lib = lib
        return lib


def _f32(xyz) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
    return a


def _copy(ptr, n: int, dtype) -> np.ndarray:
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def keys(xyz) -> np.ndarray:
    """Morton keys (uint64) of the points, in input order."""
    lib = _load()
    a = _f32(xyz)
    out = np.zeros(a.shape[0], dtype=np.uint64)
    st = lib.orc_keys(a.ctypes.data_as(C.POINTER(C.c_float)), a.shape[0],
                      out.ctypes.data_as(C.POINTER(C.c_uint64)))
    if st != ORC_OK:
        raise OracleError(st, "keys")
    return out


def encode(qx: int, qy: int, qz: int, bits: int = 21) -> int:
    return int(_load().orc_encode(qx, qy, qz, bits))


def decode(key: int, bits: int = 21) -> tuple:
    c = (C.c_int64 * 3)()
    _load().orc_decode(C.c_uint64(key), bits, c)
    return (int(c[0]), int(c[1]), int(c[2]))


def build_tree(src, recv, L: int = -1, s: int = 0, mode: int = MODE_STENCIL,
               order: int = ORDER_KEY, parallel: bool = False) -> dict:
    """The whole structure as a dict of numpy arrays.

    Keys: ``L``, ``s_unmet``; per side (``"src"``, ``"recv"``): ``perm``,
    ``sorted_keys``, ``key[l]``, ``off[l]``, ``parent[l]`` (l >= 1),
    ``child[l]`` (l < L); lists: ``e2_off[l]``, ``e2_idx[l]``, ``e4_off[l]``,
    ``e4_idx[l]`` for l in 2..L (absent with ``mode=MODE_NOLISTS``).
    ``order=ORDER_BOX`` orders the points by (level-L key, index) instead of
    (full key, index); only ``perm`` differs.  ``parallel`` runs the OpenMP
    build of the same source on all host cores.
    """
    lib = _load(parallel)
    a, b = _f32(src), _f32(recv)
    h = C.c_void_p()
    fp = C.POINTER(C.c_float)
    st = lib.orc_build(a.ctypes.data_as(fp), a.shape[0], b.ctypes.data_as(fp), b.shape[0], L, s,
                       mode | order, C.byref(h))
    if st != ORC_OK:
        raise OracleError(st, "build")
    try:
        Lr = lib.orc_level(h)
        out = {"L": Lr, "s_unmet": lib.orc_s_unmet(h)}
        for k, name, n in ((0, "src", a.shape[0]), (1, "recv", b.shape[0])):
            d = {
                "n": n,
                "perm": _copy(lib.orc_perm(h, k), n, np.uint32),
                "sorted_keys": _copy(lib.orc_sorted_keys(h, k), n, np.uint64),
                "key": [], "off": [], "parent": [], "child": [],
            }
            for l in range(Lr + 1):
                nb = lib.orc_nbox(h, k, l)
                d["key"].append(_copy(lib.orc_box_keys(h, k, l), nb, np.uint64))
                d["off"].append(_copy(lib.orc_box_off(h, k, l), nb + 1, np.uint32))
                d["parent"].append(_copy(lib.orc_box_parent(h, k, l), nb if l >= 1 else 0,
                                         np.uint32))
                d["child"].append(_copy(lib.orc_box_child(h, k, l), lib.orc_box_child_len(h, k, l),
                                        np.uint32))
            out[name] = d
        if mode != MODE_NOLISTS:
            for which, nm in ((0, "e2"), (1, "e4")):
                offs, idxs = {}, {}
                for l in range(2, Lr + 1):
                    nr = lib.orc_nbox(h, 1, l)
                    offs[l] = _copy(lib.orc_list_off(h, which, l), nr + 1, np.uint32)
                    idxs[l] = _copy(lib.orc_list_idx(h, which, l), lib.orc_nnz(h, which, l),
                                    np.uint32)
                out[nm + "_off"] = offs
                out[nm + "_idx"] = idxs
        return out
    finally:
        lib.orc_free(h)


def time_build(src, recv, L: int = -1, s: int = 0, mode: int = MODE_STENCIL,
               parallel: bool = False) -> float:
    """Seconds the oracle takes to build the whole structure of (src, recv)
    (what ``build_tree`` computes, without copying it out): the timed CPU
    baseline."""
    import time
    lib = _load(parallel)
    a, b = _f32(src), _f32(recv)
    h = C.c_void_p()
    fp = C.POINTER(C.c_float)
    t0 = time.perf_counter()
    st = lib.orc_build(a.ctypes.data_as(fp), a.shape[0], b.ctypes.data_as(fp), b.shape[0], L, s,
                       mode, C.byref(h))
    dt = time.perf_counter() - t0
    if st != ORC_OK:
        raise OracleError(st, "build")
    lib.orc_free(h)
    return dt


def box_lists(src_keys_l, level: int, recv_key: int, mode: int = MODE_STENCIL):
    """E2 and E4 lists (ascending source ranks) of one receiver box."""
    lib = _load()
    sk = np.ascontiguousarray(np.asarray(src_keys_l, dtype=np.uint64))
    e2 = np.zeros(27, dtype=np.uint32)
    e4 = np.zeros(189, dtype=np.uint32)
    n2, n4 = C.c_uint32(), C.c_uint32()
    u32p = C.POINTER(C.c_uint32)
    st = lib.orc_box_lists(sk.ctypes.data_as(C.POINTER(C.c_uint64)), sk.shape[0], level,
                           C.c_uint64(int(recv_key)), mode, e2.ctypes.data_as(u32p), C.byref(n2),
                           e4.ctypes.data_as(u32p), C.byref(n4))
    if st != ORC_OK:
        raise OracleError(st, "box_lists")
    return e2[: n2.value].copy(), e4[: n4.value].copy()


def sorted_points(xyz, perm) -> np.ndarray:
    """SortedSrc / SortedRecv (Sec. 2.1): the points in the build's order,
    point j = xyz[perm[j]]."""
    return np.ascontiguousarray(np.asarray(xyz, dtype=np.float32)[np.asarray(perm, dtype=np.int64)])


def gather_e2(tree: dict, src_xyz, level: int):
    """Alg. 2 (Access-Source-E2-neighborhood) for every receiver box of
    `level`, in receiver order: for box i, the entries j of its neighbour
    list give source boxes v, and the source points of v are read from
    SortedSrc[SrcBookmark[v] .. SrcBookmark[v+1]).  Returns (offsets [nbox+1],
    points [total, 3]); box i's points are points[offsets[i]:offsets[i+1]]."""
    sorted_src = sorted_points(src_xyz, tree["src"]["perm"])
    book = tree["src"]["off"][level].astype(np.int64)
    nb_off = tree["e2_off"][level].astype(np.int64)
    nb_list = tree["e2_idx"][level].astype(np.int64)
    nrecv = len(nb_off) - 1
    out, offsets = [], [0]
    for i in range(nrecv):
        temp = []
        for j in range(nb_off[i], nb_off[i + 1]):
            v = nb_list[j]
            for k in range(book[v], book[v + 1]):
                temp.append(sorted_src[k])
        out.extend(temp)
        offsets.append(offsets[-1] + len(temp))
    pts = np.array(out, dtype=np.float32).reshape(-1, 3)
    return np.array(offsets, dtype=np.uint64), pts
