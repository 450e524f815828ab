"""Assembly order of the element contributions.

Ordered mode (hx_set_scatter_mode(HX_SCATTER_ORDERED)): every element stores
its local vector and a second pass sums each node's contributions in
ascending element order, so repeated calls are bitwise identical; the result
matches the oracle to the parity tolerance like the atomic path.

Atomic mode (default): the order of the additions at a node changes between
runs. A node of a hexahedral box belongs to at most m = 8 elements; two
summation orders of the same m terms differ by at most 2 (m - 1) u sum|x_j|
<= 112 u max_e |r_e| (u the unit roundoff, r_e the element contributions;
recursive-summation bound, Higham, Accuracy and Stability, Sec. 4.2), which
the test checks over repeated applies, with max_e |r_e| from the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import inputs as I
from tests import cases
from tests._util import rel_inf

pytestmark = pytest.mark.gpu

TOL = {hx.HX_FP64: 1e-12, hx.HX_FP32: 1e-5}
DT = {hx.HX_FP64: torch.float64, hx.HX_FP32: torch.float32}
UNIT_ROUNDOFF = {hx.HX_FP64: 2.0 ** -53, hx.HX_FP32: 2.0 ** -24}


def cuda(x, prec=hx.HX_FP64):
    return torch.tensor(np.asarray(x), dtype=DT[prec], device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("p", [2, 4])
@pytest.mark.parametrize("storage", [hx.HX_RECOMPUTE, hx.HX_CACHE_F, hx.HX_SPATIAL_TENSORS])
@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_ordered_apply_is_bitwise_repeatable(p, storage, prec):
    """Every launching variant, on a clamped jittered cube with a ragged last
    tile: two ordered applies are identical bit for bit and match the oracle
    (constrained rows: identity)."""
    m = cases.small_cube(3, p, "iNH", seed=181 + p, clamp=True)
    M, X, u = cases.state_for(m, "iNH", seed=182 + p)
    u[M.dirichlet] = 0.0
    mat = cases.oracle_material("iNH")
    du = I.random_direction(m.n_dofs, 183 + p)
    G = hx.Mesh(m, cases.MATS["iNH"])
    try:
        G.precompute(cuda(u), prec, storage)
        du_t = cuda(du, prec)
        ref = O.apply_constrained(M, mat, u, host(du_t))
        hx.hx_set_scatter_mode(G.ctx, G.handle, hx.HX_SCATTER_ORDERED)
        ran = []
        for variant in range(6):
            hx.hx_set_apply_variant(G.ctx, G.handle, prec, storage, variant)
            try:
                a = G.apply(du_t)
            except hx.HxError as e:
                assert variant >= 2 and e.status == hx.HX_ERR_CUDA, (variant, str(e))
                continue
            b = G.apply(du_t)
            G.sync(60000)
            assert torch.equal(a, b), variant
            assert rel_inf(host(a), ref) < TOL[prec], variant
            ran.append(variant)
        assert 0 in ran and 1 in ran
    finally:
        G.close()


@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_ordered_residual_diagonal_and_connectivity_mesh(prec):
    """Residual and diagonal in ordered mode on a box, and the tangent apply
    on the tube (connectivity numbering, node -> element lists), each
    repeated bit for bit and against the oracle."""
    m = cases.small_cube(3, 3, "cNH", seed=191)
    M, X, u = cases.state_for(m, "cNH", seed=192)
    mat = cases.oracle_material("cNH")
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        hx.hx_set_scatter_mode(G.ctx, G.handle, hx.HX_SCATTER_ORDERED)
        u_t = cuda(u, prec)
        r1, r2 = G.residual(u_t), G.residual(u_t)
        G.precompute(cuda(u), prec, hx.HX_CACHE_TENSORS)
        d1, d2 = G.diagonal(prec), G.diagonal(prec)
        G.sync(60000)
        assert torch.equal(r1, r2) and torch.equal(d1, d2)
        assert rel_inf(host(r1), O.residual(M, mat, host(u_t))) < TOL[prec]
        assert rel_inf(host(d1), O.diagonal(M, mat, u)) < TOL[prec]
    finally:
        G.close()
    t = I.tube_mesh(2, n_r=2, n_theta=16, n_z=3)
    mat_d = dict(I.MAT_FIBER)
    Mt = O.OracleMesh(t)
    ut = I.inflation_field(193)(O.node_coords(Mt)).ravel()
    dut = I.random_direction(t.n_dofs, 194)
    T = hx.Mesh(t, mat_d)
    try:
        T.precompute(cuda(ut), prec, hx.HX_SPATIAL_TENSORS)
        hx.hx_set_scatter_mode(T.ctx, T.handle, hx.HX_SCATTER_ORDERED)
        du_t = cuda(dut, prec)
        a, b = T.apply(du_t), T.apply(du_t)
        T.sync(60000)
        assert torch.equal(a, b)
        assert rel_inf(host(a), O.apply(Mt, cases.oracle_material(mat_d), ut, host(du_t))) < TOL[prec]
    finally:
        T.close()


def test_ordered_cg_solve_is_bitwise_repeatable():
    """FP64 CG with the FP32 Chebyshev-Jacobi preconditioner in ordered
    mode: two solves give the same iterate bit for bit (the CG dot products
    use a fixed reduction order), and the solution solves the system."""
    m = cases.small_cube(3, 3, "cNH", seed=201, clamp=True)
    M, X, u = cases.state_for(m, "cNH", seed=202, strain=0.02)
    u[M.dirichlet] = 0.0
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        hx.hx_set_scatter_mode(G.ctx, G.handle, hx.HX_SCATTER_ORDERED)
        u_t = cuda(u)
        for pr in (hx.HX_FP64, hx.HX_FP32):
            G.precompute(u_t, pr, hx.HX_CACHE_TENSORS)
        rhs = cuda(I.random_direction(m.n_dofs, 203))
        rhs[torch.tensor(M.dirichlet, device="cuda")] = 0.0
        dinv = 1.0 / G.diagonal(hx.HX_FP64)
        lam = hx.hx_estimate_lambda_max(G.ctx, G.handle, dinv, iters=30, seed=3)
        xs = []
        for _ in range(2):
            x = torch.zeros_like(rhs)
            it, rel, st = hx.hx_cg_solve(G.ctx, G.handle, rhs, x, 1e-10, 5000, 3, 1.2 * lam, 15.0, hx.HX_FP32)
            assert st == hx.HX_OK and rel < 1e-10
            xs.append((x, it))
        G.sync(60000)
        assert xs[0][1] == xs[1][1] and torch.equal(xs[0][0], xs[1][0])
        K = O.apply_constrained(M, cases.oracle_material("cNH"), u, host(xs[0][0]))
        assert np.abs(K - host(rhs)).max() <= 1e-8 * np.abs(host(rhs)).max()
    finally:
        G.close()


@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_atomic_apply_run_to_run_difference_is_within_the_reordering_bound(prec):
    """The default atomic scatter, 20 applies: every pair differs by at most
    112 u max_e |r_e| (see the module docstring); the ordered mode's result
    lies within the same bound of each of them."""
    m = cases.small_cube(4, 4, "cNH", seed=211)
    M, X, u = cases.state_for(m, "cNH", seed=212)
    mat = cases.oracle_material("cNH")
    du = I.random_direction(m.n_dofs, 213)
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        G.precompute(cuda(u), prec, hx.HX_SPATIAL_TENSORS)
        du_t = cuda(du, prec)
        du_h = host(du_t)
        r_max = max(np.abs(O.apply(M, mat, u, du_h, elems=np.array([e], dtype=np.int32))).max()
                    for e in range(m.n_elem))
        bound = 112.0 * UNIT_ROUNDOFF[prec] * r_max * 1.01  # 1 % for the device's own rounding of r_e
        outs = [host(G.apply(du_t)) for _ in range(20)]
        hx.hx_set_scatter_mode(G.ctx, G.handle, hx.HX_SCATTER_ORDERED)
        ordered = host(G.apply(du_t))
        G.sync(60000)
        spread = max(np.abs(o - outs[0]).max() for o in outs)
        assert spread <= bound, (spread, bound)
        assert max(np.abs(o - ordered).max() for o in outs) <= bound
    finally:
        G.close()
