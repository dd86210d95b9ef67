"""CPU checks of the boundary: the library builds, loads without a GPU and
exports every entry point include/hnv.h declares; the binding refuses to
run without the library (no CPU fallback)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hnv.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(hnv_[a-z0-9_]+)\s*\(", text))
    # typedef'd function-pointer names are not functions
    names -= set(re.findall(r"\(\*\s*(hnv_[a-z0-9_]+)\)", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2103_09660_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hnv_build_incidence", "hnv_coarsen", "hnv_project", "hnv_refine",
                     "hnv_vcycle", "hnv_graph_free", "hnv_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_error_strings_without_gpu(libpath):
    import paper_2103_09660_gb300 as H
    L = H.lib()
    assert L.hnv_error_string(0) == b"HNV_OK"
    assert L.hnv_error_string(-7) == b"HNV_ERR_UNSUPPORTED_D"
    assert L.hnv_set_allocator(None, None, None) == 0
    # one hook without the other is rejected
    cb = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)(lambda a, b, c: None)
    assert L.hnv_set_allocator(ctypes.cast(cb, ctypes.c_void_p), None, None) == -1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2103_09660_gb300 as H
    monkeypatch.setattr(H, "_lib", None)
    monkeypatch.setattr(H, "library_path", str(tmp_path / "missing.so"))
    with pytest.raises(H.HNVLibraryMissing):
        H.lib()
