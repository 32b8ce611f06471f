"""The C-ABI library loads and exports every entry point include/gpusparse.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpusparse.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("gs_index_build", "gs_search", "gs_search_workspace_size", "gs_index_free", "gs_status_str"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    from paper_2606_26441_gb300 import _build, gpusparse
    path = _build.build()
    lib = ctypes.CDLL(path)  # loads without a GPU: no CUDA call at load time
    for name in declared():
        assert hasattr(lib, name), name
    assert set(declared()) == set(gpusparse.EXPORTED)
    L = gpusparse.load()
    assert L.gs_version() >= 100
    assert L.gs_status_str(0) == b"ok"
