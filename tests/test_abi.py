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


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the Python binding passes by pointer has the size and field
    offsets the C compiler gives the header's declaration (host-only check:
    gcc compiles a probe that prints sizeof and offsetof)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("no C compiler")
    from paper_1904_12228_gb300 import drt
    pairs = [("drt_scene_desc", drt.SceneDesc), ("drt_render_opts", drt.RenderOpts), ("drt_grads", drt.Grads),
             ("drt_batch_item", drt.BatchItem), ("drt_batch_info", drt.BatchInfo),
             ("drt_mlp_weights", drt.MlpWeights), ("drt_mlp_grads", drt.MlpGrads), ("drt_mlp_log", drt.MlpLog),
             ("drt_mlp_state", drt.MlpState), ("drt_mlp_train_opts", drt.MlpTrainOpts)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "drt.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                               text=True).stdout.splitlines())
    for cname, py in pairs:
        assert int(out["%s size" % cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out["%s.%s" % (cname, fname)]) == getattr(py, fname).offset, (cname, fname)
