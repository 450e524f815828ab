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


_SCALARS = {"int32_t": ctypes.c_int32, "int": ctypes.c_int, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
            "double": ctypes.c_double, "hx_status": ctypes.c_int32}


def _prototypes():
    import re
    inc = os.path.join(ROOT, "include")
    src = "\n".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = {}
    for ret, name, params in re.findall(r"(hx_status|void|const char \*|uint64_t)\s*\b(hx_\w+)\s*\(([^;{]*?)\)\s*;",
                                        src, flags=re.S):
        ps = [p.strip() for p in params.split(",")] if params.strip() not in ("", "void") else []
        protos[name] = (ret.strip(), ps)
    return protos


def _base_type(param):
    toks = param.replace("*", " * ").replace("[", " [ ").split()
    toks = [t for t in toks if t not in ("const", "*", "[", "]") and not t.rstrip("]").isdigit()]
    return toks[0]


def _matches(param, ct):
    base = _base_type(param)
    n_ptr = param.count("*") + param.count("[")
    if n_ptr == 0:
        return ct is _SCALARS[base]
    if ct in (ctypes.c_void_p, ctypes.c_char_p):
        return True  # any pointer may travel as an untyped address
    if n_ptr == 2 or (n_ptr == 1 and base.startswith("hx_") and base not in STRUCT_NAMES):
        # a pointer to an opaque handle, or an array of handles/addresses
        return ct is ctypes.POINTER(ctypes.c_void_p)
    pointee = getattr(ct, "_type_", None)
    if base in STRUCT_NAMES:
        return pointee is STRUCT_NAMES[base]
    return pointee is _SCALARS[base]


STRUCT_NAMES = {cname: py for py, (cname, _) in STRUCTS.items()}


def test_ctypes_signatures_match_the_header():
    if not os.path.exists(hx.LIB_PATH):
        from paper_2408_12479_gb300 import build
        build.build()
    L = hx.lib()
    protos = _prototypes()
    assert sorted(protos) == sorted(hx.EXPORTS)
    rets = {"hx_status": ctypes.c_int32, "void": None, "const char *": ctypes.c_char_p, "uint64_t": ctypes.c_uint64}
    for name, (ret, params) in protos.items():
        f = getattr(L, name)
        assert f.restype is rets[ret], name
        assert len(f.argtypes) == len(params), (name, params)
        for p, ct in zip(params, f.argtypes):
            assert _matches(p, ct), (name, p, ct)
