"""CPU checks of the C-ABI library: it builds, loads and exports every symbol
that the headers in include/ declare (no GPU compute is called here)."""
import ctypes
import os
import re

import pytest

from paper_2408_12479_gb300 import hx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libhx():
    if not os.path.exists(hx.LIB_PATH):
        from paper_2408_12479_gb300 import build
        build.build()
    return hx.lib()


def header_sources():
    inc = os.path.join(ROOT, "include")
    return "\n".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))


def declared_symbols():
    src = re.sub(r"/\*.*?\*/", "", header_sources(), flags=re.S)
    return sorted(set(re.findall(r"\b(hx_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(libhx):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libhx, n), n
    assert sorted(names) == sorted(hx.EXPORTS)


def test_fibre_dispersion_matches_table1(libhx):
    """Host-side constants (no device call): Table 1 of the paper prints
    H = (0.9168, 0.0759, 0.0073) for (a, b) = (3.62, 34.3)."""
    H = hx.hx_fibre_dispersion(3.62, 34.3)
    assert [round(h, 4) for h in H] == [0.9168, 0.0759, 0.0073]
    assert abs(sum(H) - 1.0) < 1e-14
    from oracle import oracle as O
    Ho = O.dispersion_H(3.62, 34.3)
    assert max(abs(a - b) for a, b in zip(H, Ho)) < 1e-14


def test_bad_arguments_are_statuses(libhx):
    H = (ctypes.c_double * 3)()
    assert libhx.hx_fibre_dispersion(3.62, -1.0, H) == hx.HX_ERR_ARG
    assert libhx.hx_sync(None, 0) == hx.HX_ERR_ARG
    assert libhx.hx_tangent_apply(None, None, None, 0) == hx.HX_ERR_ARG
    assert libhx.hx_setup_mesh(None, None, None, None) == hx.HX_ERR_ARG
