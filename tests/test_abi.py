"""The C-ABI library builds, loads without a GPU, and exports every function
declared in include/drt.h (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "drt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(drt_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("drt_create", "drt_scene_upload", "drt_render", "drt_render_backward", "drt_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1904_12228_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.drt_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.drt_version()


def test_binding_lists_every_declared_symbol():
    from paper_1904_12228_gb300 import drt
    assert sorted(drt.EXPORTED) == declared_functions()
