"""The C ABI library loads without a GPU and exports every entry point gsp.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from conftest import build_gsp
    return ctypes.CDLL(build_gsp())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gsp_edge_map", "gsp_render_fwd", "gsp_render_bwd", "gsp_las_split"):
        assert required in names
    assert len(names) >= 14


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_bounds_checked_build_exports_the_same_symbols(lib):
    dbg = ctypes.CDLL(os.path.join(ROOT, "paper_2603_08661_gb300", "libgsp_debug.so"))
    for name in declared_functions():
        assert hasattr(dbg, name), name


def test_binding_declares_exactly_the_header(lib):
    from paper_2603_08661_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_host_side_queries_without_gpu(lib):
    from paper_2603_08661_gb300 import _lib
    L = _lib.load()
    assert L.gsp_status_string(_lib.GSP_ERR_CAPACITY).startswith(b"capacity")
    assert L.gsp_version() >= 100
    d = (_lib.ImageDesc * 2)()
    d[0] = _lib.ImageDesc(1, 1237, 822, 3712, 0)
    d[1] = _lib.ImageDesc(1, 640, 480, 1920, 1237 * 822)
    opts = _lib.EdgeOpts()
    L.gsp_edge_opts_default(ctypes.byref(opts))
    assert opts.sigma == 1.0 and opts.mode == _lib.GSP_EDGE_FUSED
    assert L.gsp_edge_map_workspace_size(d, 2, ctypes.byref(opts)) > 0
    # invalid: pitch smaller than a row
    d[1] = _lib.ImageDesc(1, 640, 480, 100, 0)
    assert L.gsp_edge_map_workspace_size(d, 2, ctypes.byref(opts)) == 0
    cams = (_lib.Camera * 1)()
    cams[0].fx = cams[0].fy = 100.0
    cams[0].width, cams[0].height = 128, 128
    ro = _lib.RenderOpts(1 << 20)
    assert L.gsp_render_workspace_size(2000, 0, cams, 1, ctypes.byref(ro)) > 0
    assert L.gsp_las_workspace_size(1000) > 0
    p = _lib.LasParams()
    L.gsp_las_params_paper(ctypes.byref(p))
    assert (p.k_off, p.long_factor, p.beta) == (0.5, 0.5, pytest.approx(0.6))


def test_argument_errors_are_returned_before_any_launch(lib):
    from paper_2603_08661_gb300 import _lib
    L = _lib.load()
    d = (_lib.ImageDesc * 1)()
    d[0] = _lib.ImageDesc(None, 10, 10, 30, 0)
    st = L.gsp_edge_map(d, 1, 1, 1, None, None, None, 0, 1, None)
    assert st == _lib.GSP_ERR_INVALID_ARG
    assert L.gsp_edge_map(d, 0, 1, 1, None, None, None, 0, 1, None) == _lib.GSP_ERR_INVALID_ARG
    g = _lib.Gaussians()
    assert L.gsp_las_split(ctypes.byref(g), None, None, 0, None, None, 0, None, None) == _lib.GSP_ERR_INVALID_ARG


STRUCTS = {"ImageDesc": "gsp_image_desc", "EdgeOpts": "gsp_edge_opts", "Gaussians": "gsp_gaussians",
           "Camera": "gsp_camera", "RenderOpts": "gsp_render_opts", "LrSchedule": "gsp_lr_schedule",
           "SelectOpts": "gsp_select_opts", "LasParams": "gsp_las_params"}


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes mirror of a gsp.h struct has the C struct's size and, field
    by field, its names and offsets (a C program compiled against the header
    prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2603_08661_gb300 import _lib as L
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gsp.h"', "int main(void) {"]
    for py, c in STRUCTS.items():
        lines.append(f'printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(L, py)._fields_:
            lines.append(f'printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for py in STRUCTS:
        cls = getattr(L, py)
        assert c_layout[(py, "size")] == ctypes.sizeof(cls), py
        for name, _ in cls._fields_:
            assert c_layout[(py, name)] == getattr(cls, name).offset, (py, name)
    # every field of every C struct is mirrored (the header's member names)
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for py, c in STRUCTS.items():
        body = re.search(r"typedef struct " + c + r"\s*\{(.*?)\}\s*" + c + ";", text, flags=re.S).group(1)
        members = []
        for decl in body.split(";"):
            decl = re.sub(r"\[[^\]]*\]", "", decl).strip()
            if decl:  # "type a, b" declares a and b: the last identifier of each declarator
                members += [re.findall(r"[A-Za-z_]\w*", d)[-1] for d in decl.split(",")]
        assert members == [n for n, _ in getattr(L, py)._fields_], (c, members)
