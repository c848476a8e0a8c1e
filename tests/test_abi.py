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


def test_every_declaration_is_documented():
    # each declared call is preceded by a comment that cites its passage of
    # the paper (a Section, Table or Appendix) or says it is not in the paper
    src = open(os.path.join(ROOT, "include", "sqd.h")).read()
    pieces = re.split(r"(/\*.*?\*/)", src, flags=re.S)
    last_comment = ""
    seen = {}
    for piece in pieces:
        if piece.startswith("/*"):
            last_comment += piece
            continue
        for name in re.findall(r"\b(sqd_[a-z_0-9]+)\s*\(", piece):
            seen.setdefault(name, last_comment)
        if re.search(r"\b(sqd_[a-z_0-9]+)\s*\(", piece):
            last_comment = ""
    assert sorted(seen) == declared_symbols()
    cites = re.compile(r"Section|Table|App\.|Appendix|not in the paper|paper has no|"
                       r"no counterpart|\(not in\b", re.I)
    undocumented = [n for n, c in seen.items() if not c.strip()]
    assert not undocumented, undocumented
    uncited = [n for n, c in seen.items() if not cites.search(c)]
    # calls grouped under one comment share its citation; a group comment
    # without one must be a housekeeping call (context, errors, version)
    housekeeping = {"sqd_set_stream", "sqd_last_error", "sqd_version"}
    assert set(uncited) <= housekeeping, sorted(set(uncited) - housekeeping)
