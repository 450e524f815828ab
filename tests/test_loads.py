"""Neumann load vectors (hx_traction_load, host code in libhx) against the
FP64 oracle on the CPU: constant tractions on every side of jittered cubes
(structured and connectivity numbering), reference-normal pressure on the
curved tube, accumulation into the output, and argument errors."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import inputs as I

TOL = 1e-13


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(hx.LIB_PATH):
        from paper_2408_12479_gb300 import build
        build.build()
    hx.lib()


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("structured", [True, False])
def test_constant_traction_on_every_box_side(p, structured):
    n = 3
    m = I.box_mesh(n, p, jitter=0.1, seed=20 + p)
    M = O.OracleMesh(m)
    rng = np.random.Generator(np.random.PCG64(p))
    for side in range(6):
        t = rng.uniform(-1.0, 1.0, 3)
        faces = I.box_boundary_faces(n, n, n, side)
        ref = O.traction_load(M, faces, lambda X, N: np.tile(t, (len(X), 1)))
        got = hx.hx_traction_load(m, faces, traction=t, structured=structured)
        assert _rel(got, ref) < TOL, (side, _rel(got, ref))


@pytest.mark.parametrize("which", ["inner", "outer", "bottom", "top"])
def test_pressure_on_the_tube_surfaces(which):
    m = I.tube_mesh(3, n_r=2, n_theta=8, n_z=3)
    M = O.OracleMesh(m)
    faces = I.tube_boundary_faces(2, 8, 3, which)
    ref = O.traction_load(M, faces, lambda X, N: -1.7 * N)
    got = hx.hx_traction_load(m, faces, pressure=1.7)
    assert _rel(got, ref) < TOL


def test_loads_accumulate_and_the_sides_of_a_box_sum_to_zero_under_pressure():
    m = I.box_mesh(2, 3, jitter=0.1, seed=3)
    f = np.zeros(3 * m.n_nodes)
    for side in range(6):
        hx.hx_traction_load(m, I.box_boundary_faces(2, 2, 2, side), pressure=2.0, out=f)
    # uniform pressure on a closed surface has no resultant
    assert np.abs(f.reshape(-1, 3).sum(axis=0)).max() < 1e-14
    one = hx.hx_traction_load(m, I.box_boundary_faces(2, 2, 2, 1), pressure=2.0)
    assert np.allclose(one.reshape(-1, 3).sum(axis=0), [-2.0, 0.0, 0.0], rtol=0, atol=1e-14)


def test_no_faces_and_argument_errors():
    m = I.box_mesh(2, 2)
    assert not hx.hx_traction_load(m, np.zeros((0, 2)), traction=[1.0, 0, 0]).any()
    for bad in ([[8, 1]], [[0, 6]], [[-1, 0]]):
        with pytest.raises(hx.HxError) as e:
            hx.hx_traction_load(m, bad, traction=[1.0, 0, 0])
        assert e.value.status == hx.HX_ERR_ARG
    with pytest.raises(ValueError):
        hx.hx_traction_load(m, [[0, 0]], traction=[1.0, 0, 0], pressure=1.0)
    import ctypes as C
    assert hx.lib().hx_traction_load(None, 0, None, 0, None, None) == hx.HX_ERR_ARG
    d, keep = hx._mesh_desc(m)
    v = (C.c_double * 3)(1.0, 0.0, 0.0)
    f = np.zeros(3 * m.n_nodes)
    assert hx.lib().hx_traction_load(C.byref(d), 1, None, 0, v, f.ctypes.data) == hx.HX_ERR_ARG   # faces missing
    fc = np.array([[0, 0]], dtype=np.int32)
    assert hx.lib().hx_traction_load(C.byref(d), 1, fc.ctypes.data, 2, v, f.ctypes.data) == hx.HX_ERR_ARG  # mode
