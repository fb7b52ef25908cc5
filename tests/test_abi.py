"""The C ABI library builds, loads and exports every symbol include/curast.h
declares (no device calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "curast.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(curast_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_21749_gb300.build import build_library
    return ctypes.CDLL(build_library())


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ["curast_upload_mesh", "curast_add_instance", "curast_render", "curast_resolve",
              "curast_render_batch", "curast_interpolate", "curast_interpolate_backward"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2604_21749_gb300 import api
    assert set(declared_functions()) <= set(api.EXPORTS)


def test_status_strings(lib):
    f = lib.curast_status_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int32]
    assert f(0) == b"ok"
    assert b"2^36" in f(-3)
    assert f(12345) == b"unknown status"


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2604_21749_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in src.replace("no oracle", ""), fn


def test_renderer_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2604_21749_gb300 import api
    with pytest.raises(RuntimeError):
        api.Renderer(0)


_STRUCTS = {"View": "curast_view", "Config": "curast_config", "Stats": "curast_stats",
            "MeshInfo": "curast_mesh_info", "FrameInfo": "curast_frame_info"}


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and the field
    offsets the C compiler gives the header's struct."""
    import subprocess
    from paper_2604_21749_gb300 import api
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "curast.h"', "int main(void) {"]
    for py, c in _STRUCTS.items():
        lines.append(f'    printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(api, py)._fields_:
            lines.append(f'    printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            py, name, v = ln.split()
            got[(py, name)] = int(v)
    for py in _STRUCTS:
        cls = getattr(api, py)
        assert got[(py, "size")] == ctypes.sizeof(cls), py
        for name, _ in cls._fields_:
            assert got[(py, name)] == getattr(cls, name).offset, (py, name)


def test_set_config_rejects_unknown_keys():
    from paper_2604_21749_gb300 import api
    r = object.__new__(api.Renderer)
    with pytest.raises(KeyError):
        api.Renderer.set_config(r, stage3_raycats=1)
