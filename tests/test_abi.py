"""The C-ABI library loads and exports every entry point include/tsqr.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_0808_2664_gb300 import build

    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("tsqr_factor", "tsqr_apply_qt", "tsqr_apply_q", "tsqr_form_q", "caqr_factor", "caqr_apply_qt"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_0808_2664_gb300._lib import SIGNATURES

    assert set(declared_functions()) <= set(SIGNATURES)


def test_status_strings_and_version(libpath):
    from paper_0808_2664_gb300._lib import lib

    L = lib()
    assert L.tsqr_version() >= 100
    assert L.tsqr_status_string(0) == b"ok"
    assert L.tsqr_status_string(-3) == b"invalid argument"
    assert b"non-finite" in L.tsqr_status_string(4)


def test_oracle_and_library_share_nothing():
    """The oracle and the CUDA path import / include nothing from each other."""
    pkg = os.path.join(ROOT, "paper_0808_2664_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|from|#include)\s+[\"<]?([\w./]+)", src), f
    for f in ("householder.c", "__init__.py"):
        src = open(os.path.join(ROOT, "oracle", f)).read()
        deps = re.findall(r"(?:^|\n)\s*(?:import|from|#include)\s+[\"<]?([\w./]+)", src)
        assert not [d for d in deps if "paper_0808_2664_gb300" in d or "tsqr" in d], (f, deps)


def test_binding_exports_every_public_name():
    import paper_0808_2664_gb300 as tq

    for name in tq.__all__:
        assert hasattr(tq, name), name
