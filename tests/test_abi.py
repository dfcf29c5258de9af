"""The C ABI library builds, loads and exports every entry point declared in
include/dfm.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dfm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
    return sorted(set(re.findall(r"^[ \t]*(?!typedef)[A-Za-z_][\w \t\*]*?\b(dfm_\w+)[ \t]*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dfm_mesh_create", "dfm_assemble", "dfm_solve", "dfm_apply", "dfm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1608_04607_gb300 import build, dfm

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the whole header
    assert set(declared_functions()) == set(dfm.SIGNATURES)
    assert lib.dfm_version
