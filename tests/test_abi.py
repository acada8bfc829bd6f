"""The C-ABI library builds, loads and exports every function that
include/fmmds.h declares (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "fmmds.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1301_1704_gb300 import build, fmmds
    build.build()
    return fmmds.library()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(fmm_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("fmm_create", "fmm_destroy", "fmm_build", "fmm_morton_keys",
                 "fmm_query_workspace", "fmm_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1301_1704_gb300 import fmmds
    names = _declared()
    assert set(names) <= set(fmmds.EXPORTS) | set(names)
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_status_strings(lib):
    from paper_1301_1704_gb300 import fmmds
    for code in range(9):
        s = fmmds.status_string(code)
        assert s and s != "unknown status"
    assert fmmds.status_string(99) == "unknown status"


def test_query_workspace_host_only(lib):
    from paper_1301_1704_gb300 import fmmds
    a = fmmds.query_workspace(1 << 20, 1 << 20, L=7)
    b = fmmds.query_workspace(1 << 24, 1 << 24, L=7)
    assert 0 < a < b
    # lists dominate: at least the E4 bound of the finest level for 2^24 receivers
    assert b >= 189 * 4 * (1 << 21)
    with pytest.raises(fmmds.FmmError) as e:
        fmmds.query_workspace(10, 10, L=22)
    assert e.value.code == fmmds.FMM_ERR_LEVEL
    with pytest.raises(fmmds.FmmError):
        fmmds.query_workspace(10, 10, s=0)


def test_query_sizes_host_only(lib):
    from paper_1301_1704_gb300 import fmmds
    q = fmmds.query_sizes(1 << 24, 1000, L=7)
    assert q["workspace_bytes"] == fmmds.query_workspace(1 << 24, 1000, L=7)
    assert q["max_nbox_src"][:8] == [1, 8, 64, 512, 4096, 32768, 262144, 2097152]
    assert q["max_nbox_recv"][:8] == [1, 8, 64, 512, 1000, 1000, 1000, 1000]
    assert q["max_nbox_src"][8] == 0 and q["max_nnz_e2"][1] == 0
    assert q["max_nnz_e2"][7] == 27 * 1000 and q["max_nnz_e4"][7] == 189 * 1000
    assert q["max_nnz_e4"][2] == 189 * 64
    q = fmmds.query_sizes(5, 5, s=1)  # cluster-size mode: bounds of every level
    assert q["max_nbox_src"][21] == 5
    with pytest.raises(fmmds.FmmError):
        fmmds.query_sizes(10, 10, L=22)


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    from paper_1301_1704_gb300 import fmmds
    monkeypatch.setattr(fmmds, "_lib", None)
    monkeypatch.setattr(fmmds, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        fmmds.library()
