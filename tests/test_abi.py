"""The C-ABI library builds for sm_103a, loads on a host without a GPU, and
exports every function include/qfca.h declares.  Only host-side calls here
(status strings, version); compute calls need a GPU (tests marked gpu)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "qfca.h")).read()
    return sorted(set(re.findall(r"\b(qfca_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_15602_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = _header_functions()
    for n in ["qfca_create", "qfca_destroy", "qfca_fit_pca", "qfca_quantize", "qfca_score"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _header_functions():
        assert hasattr(lib, n), n


def test_status_strings_and_version(lib):
    lib.qfca_status_string.restype = ctypes.c_char_p
    lib.qfca_status_string.argtypes = [ctypes.c_int]
    assert lib.qfca_status_string(0) == b"QFCA_OK"
    assert lib.qfca_status_string(-1) == b"QFCA_ERR_INVALID_ARG"
    assert lib.qfca_status_string(-4) == b"QFCA_ERR_CUDA"
    lib.qfca_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.qfca_version()


def test_null_context_rejected(lib):
    lib.qfca_destroy.argtypes = [ctypes.c_void_p]
    assert lib.qfca_destroy(None) == -1
    lib.qfca_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p]
    assert lib.qfca_create(0, 0, None) == -1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    # the binding refuses to import when libqfca.so is absent (no CPU fallback)
    import importlib.util
    import shutil
    pkg = tmp_path / "pkgcopy"
    pkg.mkdir()
    src = os.path.join(ROOT, "paper_2510_15602_gb300", "qfca.py")
    shutil.copy(src, pkg / "qfca.py")
    spec = importlib.util.spec_from_file_location("qfca_nolib", pkg / "qfca.py")
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
