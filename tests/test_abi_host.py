"""C ABI checks that need no GPU: the library loads, exports every function
that include/mocd.h declares, and rejects malformed graphs before touching
the device; the product path fails loudly when the library is missing."""
import os
import re

import numpy as np
import pytest

import paper_2506_01752_gb300 as mocd
from paper_2506_01752_gb300 import build as cuda_build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mocd.h")


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return mocd.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mocd_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "mocd_graph_upload" in names and "mocd_generation" in names
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert mocd.status_string(0) == "ok"
    assert "symmetric" in mocd.status_string(-2)
    assert mocd.status_string(-99) == "unknown status"


def _upload_status(rp, ci):
    import ctypes
    ctx = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    rc = mocd.load().mocd_graph_upload(ctypes.byref(ctx), rp.size - 1, rp.ctypes.data_as(ctypes.c_void_p),
                                       ci.ctypes.data_as(ctypes.c_void_p), None)
    if rc == 0:
        mocd.destroy(ctx)
    return rc


@pytest.mark.parametrize("rp,ci,status", [
    ([0, 1, 1], [1], -2),                 # 0->1 without 1->0
    ([0, 1, 2], [0, 1], -3),              # self loops
    ([0, 2, 4], [1, 1, 0, 0], -4),        # repeated edge
    ([0, 0, 0], [], -5),                  # no edges
    ([0, 1, 2], [1, 5], -1),              # neighbour out of range
    ([0, 2, 1], [1, 0], -1),              # row_ptr decreasing
])
def test_graph_validation_before_device(lib, rp, ci, status):
    assert _upload_status(rp, ci) == status


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(mocd, "_lib", None)
    monkeypatch.setattr(mocd, "library_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        mocd.load()
