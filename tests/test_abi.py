"""The C-ABI library builds, loads and exports every symbol include/sqd.h
declares; the binding refuses to run without a GPU (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sqd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sqd_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2601_16169_gb300 import build
    return build.build()


def test_header_declares_the_five_calls():
    names = declared_symbols()
    for n in ("sqd_build_strings", "sqd_excitation_tables", "sqd_sigma", "sqd_davidson",
              "sqd_rdm"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(L, name), name
    L.sqd_version.restype = ctypes.c_char_p
    assert L.sqd_version().startswith(b"sqd-gb300")


def test_binding_symbol_list_matches_header(libpath):
    import paper_2601_16169_gb300 as sqd
    assert sorted(sqd.EXPORTED) == declared_symbols()


def test_status_on_null_arguments(libpath):
    # host-side validation, no GPU work
    L = ctypes.CDLL(libpath)
    L.sqd_last_error.restype = ctypes.c_char_p
    L.sqd_last_error.argtypes = [ctypes.c_void_p]
    assert L.sqd_create(None, 0, None) == -1
    assert b"NULL" in L.sqd_last_error(None)
    assert L.sqd_sigma(None, None, None, None, 1) == -1


def test_no_cpu_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2601_16169_gb300 as sqd
    with pytest.raises(RuntimeError):
        sqd.Context()
