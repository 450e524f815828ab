"""The binding's ctypes structures have the memory layout of the C structures
in include/hx.h: a small C program compiled with gcc against the header prints
sizeof and offsetof of every field, and the ctypes layout must agree (a field
out of order or of the wrong width would pass garbage to the library)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2408_12479_gb300 import hx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# ctypes structure -> (C type name, {ctypes field name: C field name})
STRUCTS = {
    hx.hx_material: ("hx_material", {"lambda_": "lambda"}),
    hx.hx_mesh_desc: ("hx_mesh_desc", {}),
    hx.hx_cg_options: ("hx_cg_options", {}),
    hx.hx_newton_options: ("hx_newton_options", {}),
    hx.hx_mg_options: ("hx_mg_options", {}),
    hx.hx_newton_report: ("hx_newton_report", {}),
}


def _c_layouts(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hx.h"', "int main(void) {"]
    for py, (cname, rename) in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            cf = rename.get(f, f)
            lines.append(f'  printf("{cname} {f} %zu %zu\\n", offsetof({cname}, {cf}), '
                         f'sizeof((({cname} *)0)->{cf}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                           str(exe)])
    out = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        parts = ln.split()
        if parts[1] == "sizeof":
            out[(parts[0], None)] = (int(parts[2]),)
        else:
            out[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    return out


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_ctypes_structs_match_the_header(tmp_path):
    c = _c_layouts(tmp_path)
    for py, (cname, _) in STRUCTS.items():
        assert c[(cname, None)] == (ctypes.sizeof(py),), cname
        for f, _t in py._fields_:
            desc = getattr(py, f)
            assert c[(cname, f)] == (desc.offset, desc.size), (cname, f)
