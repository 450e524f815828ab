"""The host-buffer tangent apply (hx_tangent_apply_host) against the device
apply on the same state and direction.

On a structured box it runs in z-slabs of element layers with overlapped
copies; elsewhere (connectivity meshes, the fibre law, ordered assembly, boxes
with too few layers or without a 16-byte aligned slab split) it copies whole
vectors. Both give the device apply's result up to the order of the atomic
additions at a node: relative max-norm 1e-12 in FP64 and 2e-6 in FP32 (two
summation orders of at most eight contributions differ by at most
2 (8 - 1) u sum |x_j|, with u = 2^-24 in FP32).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import inputs as I
from tests import cases
from tests._util import rel_inf

pytestmark = pytest.mark.gpu

TOL = {hx.HX_FP64: 1e-12, hx.HX_FP32: 2e-6}
DT = {hx.HX_FP64: torch.float64, hx.HX_FP32: torch.float32}


def _host_vs_device(G, m, prec, storage, seed, slabs=1):
    M_state = cases.state_for(m, "cNH" if G.input.frames is None else "fiber", seed=seed)
    u = M_state[2].copy()
    u[m.dirichlet.astype(bool)] = 0.0
    G.precompute(torch.tensor(u, dtype=torch.float64, device="cuda"), prec, storage)
    du = torch.tensor(I.random_direction(m.n_dofs, seed + 1), dtype=DT[prec])
    ref = G.apply(du.cuda())
    hx.hx_set_host_apply_slabs(G.ctx, G.handle, slabs)
    du_h = du.pin_memory()
    outs = []
    for _ in range(2):  # the second call reuses the streams, events and staging buffers
        out_h = torch.full_like(du_h, float("nan")).pin_memory()
        hx.hx_tangent_apply_host(G.ctx, G.handle, du_h, out_h, prec)
        outs.append(out_h.double().numpy())
    G.sync(60000)
    r = ref.double().cpu().numpy()
    return max(rel_inf(o, r) for o in outs)


@pytest.mark.parametrize("n,p,slabs", [(4, 4, 1), (6, 2, 1), (8, 3, 1), (5, 1, 1), (8, 2, 3)])
@pytest.mark.parametrize("storage", [hx.HX_RECOMPUTE, hx.HX_CACHE_F, hx.HX_SPATIAL_TENSORS])
@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_slabbed_host_apply_matches_device_apply(n, p, slabs, storage, prec):
    """Jittered boxes clamped on x = 0 (constrained rows: out = du), with 4 to
    8 element layers, so the slab split, the per-slab views of the point
    arrays (strategies with and without geometry, and the recompute strategy's
    node vector) and the constrained-row fix per copied layer range all run."""
    m = cases.small_cube(n, p, "cNH", seed=221 + p, clamp=True)
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        assert _host_vs_device(G, m, prec, storage, seed=222 + n, slabs=slabs) < TOL[prec]
    finally:
        G.close()


@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_whole_vector_host_apply_matches_device_apply(prec):
    """The whole-vector path: switched off on a box, and taken by itself on a
    box without an aligned split (5^3, p = 2: the only split puts a slab
    boundary at element layer 3, 3 * 25 * 27 points in, not a multiple of 16
    bytes in either precision), on ordered assembly, and on the fibre tube
    (connectivity numbering)."""
    m = cases.small_cube(4, 3, "cNH", seed=231, clamp=True)
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        assert _host_vs_device(G, m, prec, hx.HX_SPATIAL_TENSORS, seed=232, slabs=0) < TOL[prec]
        hx.hx_set_scatter_mode(G.ctx, G.handle, hx.HX_SCATTER_ORDERED)
        assert _host_vs_device(G, m, prec, hx.HX_CACHE_TENSORS, seed=233) < TOL[prec]
    finally:
        G.close()
    m = cases.small_cube(5, 2, "cNH", seed=234, clamp=True)
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        assert _host_vs_device(G, m, prec, hx.HX_SPATIAL_TENSORS, seed=235) < TOL[prec]
    finally:
        G.close()
    t = I.tube_mesh(2, n_r=2, n_theta=8, n_z=4, clamp=True)
    T = hx.Mesh(t, dict(I.MAT_FIBER))
    try:
        assert _host_vs_device(T, t, prec, hx.HX_SPATIAL_TENSORS, seed=236) < TOL[prec]
    finally:
        T.close()


def test_host_apply_slabs_rejects_other_values():
    m = cases.small_cube(1, 2, "cNH")
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        with pytest.raises(hx.HxError) as e:
            hx.hx_set_host_apply_slabs(G.ctx, G.handle, 9)
        assert e.value.status == hx.HX_ERR_ARG
    finally:
        G.close()
