"""ctypes binding of ``libfmmds.so`` (the C ABI in ``include/fmmds.h``).

Argument marshalling only: every step of the build runs in the library's
CUDA kernels.  PyTorch supplies device memory (its caching allocator backs
the context's arena) and streams.  If the shared library is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmmds.so")

FMM_LEVELS = 22
FMM_MAX_LEVEL = 21

FMM_OK, FMM_ERR_ARG, FMM_ERR_DOMAIN, FMM_ERR_LEVEL = 0, 1, 2, 3
FMM_ERR_OOM, FMM_ERR_TIMEOUT, FMM_ERR_CUDA, FMM_ERR_CAPACITY = 4, 5, 6, 7
FMM_PENDING = 8

FMM_FLAG_HOST_INPUT = 0x1
FMM_FLAG_BOX_ORDER = 0x2
FMM_FLAG_SORTED_XYZ = 0x4
FMM_FLAG_TEST_STALL = 0x80000000

_u32p = C.POINTER(C.c_uint32)
_u64p = C.POINTER(C.c_uint64)
_L = FMM_LEVELS


class Params(C.Structure):
    _fields_ = [("L", C.c_int), ("s", C.c_uint32), ("flags", C.c_uint32), ("wait_ms", C.c_uint32)]


class TreeC(C.Structure):
    _fields_ = [
        ("L", C.c_int), ("s_unmet", C.c_uint32), ("n_src", C.c_uint32), ("n_recv", C.c_uint32),
        ("perm_src", C.c_void_p), ("perm_recv", C.c_void_p),
        ("nbox_src", C.c_uint32 * _L), ("nbox_recv", C.c_uint32 * _L),
        ("key_src", C.c_void_p * _L), ("key_recv", C.c_void_p * _L),
        ("off_src", C.c_void_p * _L), ("off_recv", C.c_void_p * _L),
        ("parent_src", C.c_void_p * _L), ("parent_recv", C.c_void_p * _L),
        ("child_src", C.c_void_p * _L), ("child_recv", C.c_void_p * _L),
        ("nnz_e2", C.c_uint64 * _L), ("nnz_e4", C.c_uint64 * _L),
        ("e2_off", C.c_void_p * _L), ("e2_idx", C.c_void_p * _L),
        ("e4_off", C.c_void_p * _L), ("e4_idx", C.c_void_p * _L),
        ("sorted_src", C.c_void_p), ("sorted_recv", C.c_void_p),
    ]


class SizesC(C.Structure):
    _fields_ = [("workspace_bytes", C.c_uint64),
                ("max_nbox_src", C.c_uint32 * _L), ("max_nbox_recv", C.c_uint32 * _L),
                ("max_nnz_e2", C.c_uint64 * _L), ("max_nnz_e4", C.c_uint64 * _L)]


class SetC(C.Structure):
    _fields_ = [("src", C.c_void_p), ("N", C.c_uint32), ("recv", C.c_void_p), ("M", C.c_uint32),
                ("L", C.c_int32)]


class Batch:
    """fmm_set array (and result array) of a list of (src, recv) tensor pairs,
    with optional per-pair depths ``levels`` (None or -1: the call's L or s)."""

    def __init__(self, sets, levels=None):
        self.k = len(sets)
        if levels is not None and len(levels) != self.k:
            raise ValueError("one level per set")
        self.arr = (SetC * max(self.k, 1))()
        self.outs = (TreeC * max(self.k, 1))()
        self.sizes = []
        self._keep = list(sets)
        for i, (a, b) in enumerate(sets):
            for t in (a, b):
                if t.dtype.itemsize != 4 or (t.numel() and not t.is_contiguous()):
                    raise ValueError("points must be contiguous float32 [n, 3]")
            lv = -1 if levels is None or levels[i] is None else int(levels[i])
            self.arr[i] = SetC(a.data_ptr() if a.shape[0] else 0, a.shape[0],
                               b.data_ptr() if b.shape[0] else 0, b.shape[0], lv)
            self.sizes.append((a.shape[0], b.shape[0]))


class ServerParams(C.Structure):
    _fields_ = [("workers", C.c_uint32), ("max_batch", C.c_uint32), ("mem_budget", C.c_uint64),
                ("flags", C.c_uint32)]


class RequestInfo(C.Structure):
    _fields_ = [("id", C.c_uint64), ("system", C.c_uint32), ("status", C.c_uint32),
                ("step", C.c_uint64), ("t_arrival", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double), ("batch_size", C.c_uint32), ("worker", C.c_uint32),
                ("points", C.c_uint64), ("nnz_e2", C.c_uint64), ("nnz_e4", C.c_uint64),
                ("digest", C.c_uint64)]


FMM_SERVER_DIGEST = 0x1
_INFO_FIELDS = [f for f, _ in RequestInfo._fields_]


def _info_dict(x: RequestInfo) -> dict:
    return {f: getattr(x, f) for f in _INFO_FIELDS}


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("total_ms", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

# Every function declared in include/fmmds.h.
EXPORTS = (
    "fmm_create", "fmm_destroy", "fmm_build", "fmm_build_batched", "fmm_morton_keys",
    "fmm_query_workspace", "fmm_query_sizes", "fmm_server_poll",
    "fmm_set_tuning", "fmm_get_tuning", "fmm_set_timing", "fmm_get_timing", "fmm_reset_timing",
    "fmm_last_launch_count", "fmm_status_string", "fmm_exclusive_scan_noalloc",
    "fmm_autotune", "fmm_e2_source_offsets", "fmm_gather_e2_sources", "fmm_box_types",
    "fmm_displace", "fmm_server_create", "fmm_server_destroy", "fmm_server_add_system",
    "fmm_server_submit", "fmm_server_wait", "fmm_server_run_trace", "fmm_server_points",
    "fmm_server_tree", "fmm_set_graphs", "fmm_graph_stats",
)
FMM_NOALLOC_SCAN_MAX = 1 << 26

FMM_SORT_RTS = 0
FMM_SORT_ONESWEEP = 1
FMM_SORT_FIXED_GRID = 2
FMM_SORT_BUCKET = 3


class Tuning(C.Structure):
    _fields_ = [("sort_kind", C.c_uint32), ("sort_items", C.c_uint32)]

_lib = None


class FmmError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = _load().fmm_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} (status {code})")
        self.code = code


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1301_1704_gb300.build`"
                           " (or __graft_entry__.build()); there is no fallback path")
    lib = C.CDLL(LIB_PATH)
    lib.fmm_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, ALLOC_FN, FREE_FN, C.c_void_p]
    lib.fmm_create.restype = C.c_int
    lib.fmm_destroy.argtypes = [C.c_void_p]
    lib.fmm_destroy.restype = C.c_int
    lib.fmm_build.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, Params,
                              C.POINTER(TreeC), C.c_void_p]
    lib.fmm_build.restype = C.c_int
    lib.fmm_build_batched.argtypes = [C.c_void_p, C.POINTER(SetC), C.c_uint32, Params,
                                      C.POINTER(TreeC), C.c_void_p]
    lib.fmm_build_batched.restype = C.c_int
    lib.fmm_morton_keys.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p]
    lib.fmm_morton_keys.restype = C.c_int
    lib.fmm_query_workspace.argtypes = [C.c_uint32, C.c_uint32, Params, _u64p]
    lib.fmm_query_workspace.restype = C.c_int
    lib.fmm_query_sizes.argtypes = [C.c_uint32, C.c_uint32, Params, C.POINTER(SizesC)]
    lib.fmm_query_sizes.restype = C.c_int
    lib.fmm_set_tuning.argtypes = [C.c_void_p, C.POINTER(Tuning)]
    lib.fmm_set_tuning.restype = C.c_int
    lib.fmm_get_tuning.argtypes = [C.c_void_p, C.POINTER(Tuning)]
    lib.fmm_get_tuning.restype = C.c_int
    lib.fmm_set_timing.argtypes = [C.c_void_p, C.c_int]
    lib.fmm_set_timing.restype = C.c_int
    lib.fmm_reset_timing.argtypes = [C.c_void_p]
    lib.fmm_reset_timing.restype = C.c_int
    lib.fmm_get_timing.argtypes = [C.c_void_p, C.POINTER(KernelTime), C.c_int, C.POINTER(C.c_int)]
    lib.fmm_get_timing.restype = C.c_int
    lib.fmm_last_launch_count.argtypes = [C.c_void_p, _u64p]
    lib.fmm_last_launch_count.restype = C.c_int
    lib.fmm_set_graphs.argtypes = [C.c_void_p, C.c_int]
    lib.fmm_set_graphs.restype = C.c_int
    lib.fmm_graph_stats.argtypes = [C.c_void_p, _u64p, _u64p]
    lib.fmm_graph_stats.restype = C.c_int
    lib.fmm_exclusive_scan_noalloc.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p,
                                               C.c_void_p]
    lib.fmm_exclusive_scan_noalloc.restype = C.c_int
    lib.fmm_status_string.argtypes = [C.c_int]
    lib.fmm_status_string.restype = C.c_char_p
    lib.fmm_autotune.argtypes = [C.c_void_p, C.POINTER(SetC), C.c_uint32, Params, C.c_uint32,
                                 C.POINTER(Tuning), C.POINTER(C.c_double), C.c_void_p]
    lib.fmm_autotune.restype = C.c_int
    lib.fmm_box_types.argtypes = [C.c_void_p, C.POINTER(TreeC), C.c_int, C.c_void_p, C.c_uint32,
                                  C.POINTER(C.c_void_p), C.c_void_p]
    lib.fmm_box_types.restype = C.c_int
    lib.fmm_e2_source_offsets.argtypes = [C.c_void_p, C.POINTER(TreeC), C.c_int, C.c_void_p,
                                          _u64p, C.c_void_p]
    lib.fmm_e2_source_offsets.restype = C.c_int
    lib.fmm_gather_e2_sources.argtypes = [C.c_void_p, C.POINTER(TreeC), C.c_int, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
    lib.fmm_gather_e2_sources.restype = C.c_int
    lib.fmm_displace.argtypes = [C.c_void_p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_float,
                                 C.c_void_p]
    lib.fmm_displace.restype = C.c_int
    lib.fmm_server_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(ServerParams)]
    lib.fmm_server_create.restype = C.c_int
    lib.fmm_server_destroy.argtypes = [C.c_void_p]
    lib.fmm_server_destroy.restype = C.c_int
    lib.fmm_server_add_system.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_int, C.c_int,
                                          C.c_float, C.c_uint64, C.POINTER(C.c_uint32)]
    lib.fmm_server_add_system.restype = C.c_int
    lib.fmm_server_submit.argtypes = [C.c_void_p, C.c_uint32, _u64p]
    lib.fmm_server_submit.restype = C.c_int
    lib.fmm_server_wait.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(RequestInfo)]
    lib.fmm_server_wait.restype = C.c_int
    lib.fmm_server_poll.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(RequestInfo)]
    lib.fmm_server_poll.restype = C.c_int
    lib.fmm_server_run_trace.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32,
                                         C.POINTER(RequestInfo)]
    lib.fmm_server_run_trace.restype = C.c_int
    lib.fmm_server_points.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p]
    lib.fmm_server_points.restype = C.c_int
    lib.fmm_server_tree.argtypes = [C.c_void_p, C.c_uint32, C.POINTER(TreeC)]
    lib.fmm_server_tree.restype = C.c_int
    _lib = lib
    return lib


def library():
    return _load()


class _DevArray:
    """Zero-copy view of a device array for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {
            "shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False), "version": 3,
        }


def _view(ptr, n: int, typestr: str):
    import torch
    if n == 0 or not ptr:
        return torch.zeros(0, dtype=torch.int64 if typestr.endswith("8") else torch.int32,
                           device="cuda")
    return torch.as_tensor(_DevArray(ptr, n, typestr), device="cuda")


@dataclass
class Side:
    """Per-set arrays of a build (device tensors; int32/int64 carry the uint32/uint64 bits)."""
    n: int
    perm: object
    nbox: list
    key: list = field(default_factory=list)
    off: list = field(default_factory=list)
    parent: list = field(default_factory=list)
    child: list = field(default_factory=list)


@dataclass
class Tree:
    """Result of :meth:`Context.build`; valid until the context's next build."""
    L: int
    s_unmet: int
    src: Side
    recv: Side
    nnz_e2: list
    nnz_e4: list
    e2_off: dict
    e2_idx: dict
    e4_off: dict
    e4_idx: dict
    sorted_src: object = None   # float32 [N, 3] with FMM_FLAG_SORTED_XYZ
    sorted_recv: object = None
    raw: object = None          # the fmm_tree struct (for calls that take it)

    def numpy(self) -> dict:
        """Host copy with the oracle's layout (uint32 / uint64 numpy arrays)."""
        def u32(t):
            return t.cpu().numpy().view(np.uint32).copy()

        def u64(t):
            return t.cpu().numpy().view(np.uint64).copy()

        out = {"L": self.L, "s_unmet": self.s_unmet}
        for name, sd in (("src", self.src), ("recv", self.recv)):
            out[name] = {
                "n": sd.n, "perm": u32(sd.perm),
                "key": [u64(k) for k in sd.key], "off": [u32(o) for o in sd.off],
                "parent": [u32(p) for p in sd.parent], "child": [u32(c) for c in sd.child],
            }
        for nm in ("e2_off", "e2_idx", "e4_off", "e4_idx"):
            out[nm] = {l: u32(t) for l, t in getattr(self, nm).items()}
        for nm in ("sorted_src", "sorted_recv"):
            t = getattr(self, nm)
            if t is not None:
                out[nm] = t.cpu().numpy().copy()
        return out


def _side(tc: TreeC, which: str, L: int, n: int) -> Side:
    nbox = [int(v) for v in getattr(tc, "nbox_" + which)]
    sd = Side(n=n, perm=_view(getattr(tc, "perm_" + which), n, "<i4"), nbox=nbox)
    for l in range(L + 1):
        nb = nbox[l]
        sd.key.append(_view(getattr(tc, "key_" + which)[l], nb, "<i8"))
        sd.off.append(_view(getattr(tc, "off_" + which)[l], nb + 1, "<i4"))
        sd.parent.append(_view(getattr(tc, "parent_" + which)[l], nb if l >= 1 else 0, "<i4"))
        sd.child.append(_view(getattr(tc, "child_" + which)[l], nb + 1 if l < L else 0, "<i4"))
    return sd


def _tree_from(tc: TreeC, n: int, m: int) -> Tree:
    Lr = tc.L
    tree = Tree(L=Lr, s_unmet=tc.s_unmet, src=_side(tc, "src", Lr, n),
                recv=_side(tc, "recv", Lr, m), nnz_e2=list(tc.nnz_e2), nnz_e4=list(tc.nnz_e4),
                e2_off={}, e2_idx={}, e4_off={}, e4_idx={})
    import torch
    for nm, cnt in (("sorted_src", n), ("sorted_recv", m)):
        ptr = getattr(tc, nm)
        if ptr:
            setattr(tree, nm, _view(ptr, 3 * cnt, "<i4").view(torch.float32).view(cnt, 3))
    tree.raw = tc
    for l in range(2, Lr + 1):
        nr = tc.nbox_recv[l]
        tree.e2_off[l] = _view(tc.e2_off[l], nr + 1, "<i4")
        tree.e4_off[l] = _view(tc.e4_off[l], nr + 1, "<i4")
        tree.e2_idx[l] = _view(tc.e2_idx[l], tc.nnz_e2[l], "<i4")
        tree.e4_idx[l] = _view(tc.e4_idx[l], tc.nnz_e4[l], "<i4")
    return tree


class Context:
    """One fmm_ctx on one CUDA device, its arena backed by torch's allocator."""

    def __init__(self, device: int = 0, torch_allocator: bool = True):
        import torch
        lib = _load()
        self.device = device
        self._h = C.c_void_p()
        if torch_allocator:
            def _alloc(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
                except Exception:
                    return None

            def _free(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
        else:
            self._alloc_cb = C.cast(None, ALLOC_FN)
            self._free_cb = C.cast(None, FREE_FN)
        st = lib.fmm_create(C.byref(self._h), device, self._alloc_cb, self._free_cb, None)
        if st != FMM_OK:
            raise FmmError(st, "fmm_create")

    def close(self):
        if self._h:
            _load().fmm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream) -> int:
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)

    def build(self, src, recv, L: int | None = None, s: int | None = None, stream=None,
              flags: int = 0, wait_ms: int = 0, raw: bool = False):
        """fmm_build.  ``src``/``recv``: float32 [n, 3] CUDA tensors (or pinned
        CPU tensors with ``flags=FMM_FLAG_HOST_INPUT``).  Give ``L`` (0..21) or
        ``s`` (cluster size).  Returns a :class:`Tree` (or the raw ``TreeC``)."""
        lib = _load()
        if (L is None) == (s is None):
            raise ValueError("give exactly one of L or s")
        p = Params(L if L is not None else -1, s if s is not None else 0, flags, wait_ms)
        for t in (src, recv):
            if t.dtype.itemsize != 4 or (t.numel() and not t.is_contiguous()):
                raise ValueError("points must be contiguous float32 [n, 3]")
        tc = TreeC()
        n, m = src.shape[0], recv.shape[0]
        st = lib.fmm_build(self._h, C.c_void_p(src.data_ptr() if n else 0), n,
                           C.c_void_p(recv.data_ptr() if m else 0), m, p, C.byref(tc),
                           C.c_void_p(self._stream(stream)))
        if st != FMM_OK:
            raise FmmError(st, "fmm_build")
        if raw:
            return tc
        return _tree_from(tc, n, m)

    def batch(self, sets, levels=None) -> "Batch":
        """The fmm_set array of a list of (src, recv) pairs of float32 [n, 3]
        CUDA tensors, built once for repeated fmm_build_batched calls on the
        same tensors (the tensors must stay alive and in place)."""
        return Batch(sets, levels)

    def build_batched(self, sets, L: int | None = None, s: int | None = None, stream=None,
                      flags: int = 0, raw: bool = False, levels=None):
        """fmm_build_batched.  ``sets``: list of (src, recv) pairs of float32
        [n, 3] CUDA tensors (the same tensor twice for an aliased set), or a
        :class:`Batch` of them; ``levels``: optional per-set depths that
        override L / s.  Returns one :class:`Tree` per set (or the raw
        ``TreeC`` array)."""
        lib = _load()
        b = sets if isinstance(sets, Batch) else Batch(sets, levels)
        if L is None and s is None and levels is not None and all(
                v is not None and v >= 0 for v in levels):
            L = 0  # every set carries its own depth
        if (L is None) == (s is None):
            raise ValueError("give exactly one of L or s")
        p = Params(L if L is not None else -1, s if s is not None else 0, flags, 0)
        st = lib.fmm_build_batched(self._h, b.arr, b.k, p, b.outs, C.c_void_p(self._stream(stream)))
        if st != FMM_OK:
            raise FmmError(st, "fmm_build_batched")
        if raw:
            return b.outs
        return [_tree_from(b.outs[i], b.sizes[i][0], b.sizes[i][1]) for i in range(b.k)]

    def box_types(self, tree: "Tree", lpar: int, owner, node: int, stream=None) -> dict:
        """fmm_box_types (Alg. 6): uint8 CUDA tensors per level 2..L of the
        source boxes' types for `node`; `owner`: uint32-valued CUDA tensor of
        the owners of the source boxes at level `lpar`.  The tree must come
        from a build of the sources against themselves."""
        import torch
        types = {l: torch.empty(tree.src.nbox[l], dtype=torch.uint8, device="cuda")
                 for l in range(2, tree.L + 1)}
        arr = (C.c_void_p * FMM_LEVELS)()
        for l, t in types.items():
            arr[l] = t.data_ptr() if t.numel() else 0
        st = _load().fmm_box_types(self._h, C.byref(tree.raw), lpar,
                                   C.c_void_p(owner.data_ptr() if owner.numel() else 0), node, arr,
                                   C.c_void_p(self._stream(stream)))
        if st != FMM_OK:
            raise FmmError(st, "fmm_box_types")
        return types

    def gather_e2(self, tree: "Tree", level: int, sorted_src=None, stream=None):
        """Alg. 2 for every receiver box of `level` (fmm_e2_source_offsets +
        fmm_gather_e2_sources): returns (offsets int32-carrying-uint32 [nbox+1],
        points float32 [total, 3]) on the device."""
        import torch
        lib = _load()
        if sorted_src is None:
            sorted_src = tree.sorted_src
        if sorted_src is None:
            raise ValueError("build with FMM_FLAG_SORTED_XYZ or pass sorted_src")
        nb = tree.recv.nbox[level]
        off = torch.empty(nb + 1, dtype=torch.int32, device="cuda")
        total = C.c_uint64()
        h = C.c_void_p(self._stream(stream))
        st = lib.fmm_e2_source_offsets(self._h, C.byref(tree.raw), level, C.c_void_p(off.data_ptr()),
                                       C.byref(total), h)
        if st != FMM_OK:
            raise FmmError(st, "fmm_e2_source_offsets")
        out = torch.empty((int(total.value), 3), dtype=torch.float32, device="cuda")
        st = lib.fmm_gather_e2_sources(self._h, C.byref(tree.raw), level,
                                       C.c_void_p(sorted_src.data_ptr() if sorted_src.numel() else 0),
                                       C.c_void_p(off.data_ptr()),
                                       C.c_void_p(out.data_ptr() if out.numel() else 0), h)
        if st != FMM_OK:
            raise FmmError(st, "fmm_gather_e2_sources")
        return off, out

    def morton_keys(self, xyz, out=None, stream=None):
        """fmm_morton_keys: int64 CUDA tensor carrying the uint64 keys."""
        import torch
        lib = _load()
        n = xyz.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.int64, device=xyz.device)
        st = lib.fmm_morton_keys(self._h, C.c_void_p(xyz.data_ptr() if n else 0), n,
                                 C.c_void_p(out.data_ptr() if n else 0),
                                 C.c_void_p(self._stream(stream)))
        if st != FMM_OK:
            raise FmmError(st, "fmm_morton_keys")
        return out

    def set_tuning(self, sort_kind: int, sort_items: int = 0):
        t = Tuning(sort_kind, sort_items)
        st = _load().fmm_set_tuning(self._h, C.byref(t))
        if st != FMM_OK:
            raise FmmError(st, "fmm_set_tuning")

    def tuning(self) -> dict:
        t = Tuning()
        _load().fmm_get_tuning(self._h, C.byref(t))
        return {"sort_kind": int(t.sort_kind), "sort_items": int(t.sort_items)}

    def autotune(self, sets, L: int | None = None, s: int | None = None, trials: int = 3,
                 flags: int = 0, stream=None) -> dict:
        """fmm_autotune over (sort kind, items per thread) on the given pairs
        (a list of (src, recv) CUDA tensors, or a Batch); keeps the fastest."""
        lib = _load()
        b = sets if isinstance(sets, Batch) else Batch(sets)
        if (L is None) == (s is None):
            raise ValueError("give exactly one of L or s")
        p = Params(L if L is not None else -1, s if s is not None else 0, flags, 0)
        best = Tuning()
        ms = C.c_double()
        st = lib.fmm_autotune(self._h, b.arr, b.k, p, trials, C.byref(best), C.byref(ms),
                              C.c_void_p(self._stream(stream)))
        if st != FMM_OK:
            raise FmmError(st, "fmm_autotune")
        return {"sort_kind": int(best.sort_kind), "sort_items": int(best.sort_items),
                "median_ms": ms.value}

    def set_timing(self, on: bool):
        _load().fmm_set_timing(self._h, 1 if on else 0)

    def reset_timing(self):
        _load().fmm_reset_timing(self._h)

    def timing(self) -> dict:
        lib = _load()
        n = C.c_int()
        buf = (KernelTime * 64)()
        lib.fmm_get_timing(self._h, buf, 64, C.byref(n))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
                for i in range(min(n.value, 64))}

    def last_launch_count(self) -> int:
        v = C.c_uint64()
        _load().fmm_last_launch_count(self._h, C.byref(v))
        return int(v.value)

    def set_graphs(self, on: bool):
        """Graph mode: builds after the first record their stream work into
        CUDA graphs that are updated and launched (see fmm_set_graphs)."""
        st = _load().fmm_set_graphs(self._h, 1 if on else 0)
        if st != 0:
            raise FmmError(st, "fmm_set_graphs")

    def graph_stats(self) -> dict:
        a, b = C.c_uint64(), C.c_uint64()
        st = _load().fmm_graph_stats(self._h, C.byref(a), C.byref(b))
        if st != 0:
            raise FmmError(st, "fmm_graph_stats")
        return {"launches": int(a.value), "instantiations": int(b.value)}


def exclusive_scan_noalloc(counts, offsets, total=None, stream=None) -> None:
    """fmm_exclusive_scan_noalloc: offsets[0..n] from counts[0..n) (CUDA
    tensors of 4-byte integers, offsets one longer); allocates nothing."""
    import torch
    dev = torch.cuda.current_device()
    for name, t in (("counts", counts), ("offsets", offsets)):
        if (not t.is_cuda or t.device.index != dev or not t.is_contiguous()
                or t.element_size() != 4 or t.dtype.is_floating_point):
            raise ValueError(f"{name} must be a contiguous 4-byte integer CUDA tensor "
                             "on the current device")
    n = counts.numel()
    if offsets.numel() != n + 1:
        raise ValueError("offsets needs n + 1 entries")
    if total is not None and (not total.is_cuda or total.device.index != dev
                              or total.dtype not in (torch.int64, torch.uint64)
                              or total.numel() < 1):
        raise ValueError("total must be an int64 CUDA tensor of at least one element "
                         "on the current device")
    st = _load().fmm_exclusive_scan_noalloc(
        C.c_void_p(counts.data_ptr() if n else 0), n, C.c_void_p(offsets.data_ptr()),
        C.c_void_p(total.data_ptr() if total is not None else 0),
        C.c_void_p(Context._stream(stream)))
    if st != FMM_OK:
        raise FmmError(st, "fmm_exclusive_scan_noalloc")


def query_workspace(N: int, M: int, L: int | None = None, s: int | None = None, flags: int = 0) -> int:
    v = C.c_uint64()
    p = Params(L if L is not None else -1, s if s is not None else 0, flags, 0)
    st = _load().fmm_query_workspace(N, M, p, C.byref(v))
    if st != FMM_OK:
        raise FmmError(st, "fmm_query_workspace")
    return int(v.value)


def query_sizes(N: int, M: int, L: int | None = None, s: int | None = None,
                flags: int = 0) -> dict:
    """fmm_query_sizes: the workspace bound and the per-level box and list
    size bounds of a build of N sources and M receivers."""
    v = SizesC()
    p = Params(L if L is not None else -1, s if s is not None else 0, flags, 0)
    st = _load().fmm_query_sizes(N, M, p, C.byref(v))
    if st != FMM_OK:
        raise FmmError(st, "fmm_query_sizes")
    return {"workspace_bytes": int(v.workspace_bytes),
            "max_nbox_src": list(v.max_nbox_src), "max_nbox_recv": list(v.max_nbox_recv),
            "max_nnz_e2": list(v.max_nnz_e2), "max_nnz_e4": list(v.max_nnz_e4)}


def status_string(code: int) -> str:
    return _load().fmm_status_string(code).decode()


def displace(xyz, seed: int, step: int, sigma: float, stream=None) -> None:
    """fmm_displace: one time step of the float32 [n, 3] CUDA tensor in place."""
    import torch
    lib = _load()
    if xyz.dtype != torch.float32 or not xyz.is_contiguous() or not xyz.is_cuda:
        raise ValueError("points must be a contiguous float32 CUDA tensor [n, 3]")
    n = xyz.shape[0]
    h = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    st = lib.fmm_displace(C.c_void_p(xyz.data_ptr() if n else 0), n, seed, step, sigma,
                          C.c_void_p(h))
    if st != FMM_OK:
        raise FmmError(st, "fmm_displace")


class Server:
    """Served dynamic rebuilds (fmm_server_*): resident time-stepped systems,
    continuous batching over ``workers`` concurrent batched builds."""

    def __init__(self, device: int = 0, workers: int = 2, max_batch: int = 8,
                 mem_budget: int = 0, digest: bool = False):
        lib = _load()
        self._h = C.c_void_p()
        prm = ServerParams(workers, max_batch, mem_budget, FMM_SERVER_DIGEST if digest else 0)
        st = lib.fmm_server_create(C.byref(self._h), device, C.byref(prm))
        if st != FMM_OK:
            raise FmmError(st, "fmm_server_create")
        self.sizes = []

    def add_system(self, xyz, L: int, sigma_scale: float = 0.1, seed: int = 0) -> int:
        """Copies the points (numpy float32 [n, 3], or a CUDA tensor) in."""
        lib = _load()
        sid = C.c_uint32()
        if isinstance(xyz, np.ndarray):
            a = np.ascontiguousarray(xyz, dtype=np.float32)
            ptr, host, n = a.ctypes.data, 1, a.shape[0]
        else:
            a = xyz.contiguous()
            ptr, host, n = a.data_ptr(), 0, a.shape[0]
        st = lib.fmm_server_add_system(self._h, C.c_void_p(ptr if n else 0), n, host, L,
                                       sigma_scale, seed, C.byref(sid))
        if st != FMM_OK:
            raise FmmError(st, "fmm_server_add_system")
        self.sizes.append(n)
        return sid.value

    def submit(self, system: int) -> int:
        rid = C.c_uint64()
        st = _load().fmm_server_submit(self._h, system, C.byref(rid))
        if st != FMM_OK:
            raise FmmError(st, "fmm_server_submit")
        return rid.value

    def wait(self, request_id: int) -> dict:
        inf = RequestInfo()
        st = _load().fmm_server_wait(self._h, request_id, C.byref(inf))
        if st != FMM_OK:
            raise FmmError(st, "fmm_server_wait")
        return _info_dict(inf)

    def poll(self, request_id: int):
        """The request's info once it is done, else None (does not block)."""
        inf = RequestInfo()
        st = _load().fmm_server_poll(self._h, request_id, C.byref(inf))
        if st == FMM_PENDING:
            return None
        if st != FMM_OK:
            raise FmmError(st, "fmm_server_poll")
        return _info_dict(inf)

    def step(self, system: int) -> dict:
        return self.wait(self.submit(system))

    def run_trace(self, arrival_s, systems) -> list:
        t = np.ascontiguousarray(arrival_s, dtype=np.float64)
        y = np.ascontiguousarray(systems, dtype=np.uint32)
        k = t.shape[0]
        out = (RequestInfo * max(k, 1))()
        st = _load().fmm_server_run_trace(self._h, C.c_void_p(t.ctypes.data),
                                          C.c_void_p(y.ctypes.data), k, out)
        if st != FMM_OK:
            raise FmmError(st, "fmm_server_run_trace")
        return [_info_dict(out[i]) for i in range(k)]

    def points(self, system: int) -> np.ndarray:
        n = self.sizes[system]
        a = np.empty((n, 3), np.float32)
        st = _load().fmm_server_points(self._h, system, C.c_void_p(a.ctypes.data))
        if st != FMM_OK:
            raise FmmError(st, "fmm_server_points")
        return a

    def tree(self, system: int) -> "Tree":
        tc = TreeC()
        st = _load().fmm_server_tree(self._h, system, C.byref(tc))
        if st != FMM_OK:
            raise FmmError(st, "fmm_server_tree")
        n = self.sizes[system]
        return _tree_from(tc, n, n)

    def close(self):
        if self._h:
            _load().fmm_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
