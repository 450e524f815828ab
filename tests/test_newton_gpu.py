"""GPU Newton's method (Alg. 1) and the body-force load vector through the C
ABI, against the oracle's plain Newton (direct solves) and the closed form of
homogeneous uniaxial tension."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import inputs as I
from tests import cases
from tests._util import rel_inf

pytestmark = pytest.mark.gpu


def cuda(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_body_force_matches_oracle(p):
    m = I.box_mesh(3, p, jitter=0.1, seed=31 + p, clamp=True)
    M = O.OracleMesh(m)
    b = [0.3, -0.2, 0.5]
    ref = O.body_force(M, b)
    ref[M.dirichlet] = 0.0
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        f = torch.empty(m.n_dofs, dtype=torch.float64, device="cuda")
        hx.hx_body_force(G.ctx, G.handle, b, f)
        G.sync(60000)
        assert rel_inf(f.cpu().numpy(), ref) < 1e-12
    finally:
        G.close()


def _lateral_stretch(law, mat, l1):
    from scipy.optimize import brentq

    def s22(l2):
        J = l1 * l2 * l2
        if law == "cNH":
            return mat["mu"] - (mat["mu"] - 2.0 * mat["lam"] * np.log(J)) / l2 ** 2
        j = J ** (-2.0 / 3.0)
        I1 = l1 ** 2 + 2 * l2 ** 2
        c1 = 0.5 * mat["kappa"] * (J * J - 1.0) - mat["mu"] / 3.0 * j * I1
        return mat["mu"] * j + c1 / l2 ** 2
    return brentq(s22, 0.5, 1.5)


@pytest.mark.parametrize("law", ["cNH", "iNH"])
@pytest.mark.parametrize("storage", [hx.HX_CACHE_TENSORS, hx.HX_SPATIAL_TENSORS, hx.HX_RECOMPUTE])
@pytest.mark.parametrize("pp", [hx.HX_FP64, hx.HX_FP32])
def test_newton_uniaxial_load_steps_match_closed_form(law, storage, pp):
    """Stretch 1.2 reached in ten load steps (each step starts from the last
    solution plus the affine increment of the prescribed stretch, where the
    tangent stays positive definite); the result is the homogeneous state."""
    l1, steps = 1.2, 10
    m, _ = I.workload_uniaxial(2, 3, 1.0)
    mat = dict(cases.MATS[law])
    G = hx.Mesh(m, mat)
    try:
        X = G.node_coords().cpu().numpy().reshape(-1, 3)
        inc = np.zeros_like(X)
        inc[:, 0] = (l1 - 1.0) / steps * X[:, 0]
        u = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
        for _ in range(steps):
            u += cuda(inc.ravel())
            rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, None, eps_abs=1e-11, eps_rel=1e-12, max_newton=15,
                                         storage=storage, precond_prec=pp, cg_tol=1e-11, cg_max_iter=20000)
            assert st == hx.HX_OK and rep["converged"] and rep["newton_iters"] <= 8, rep
        l2 = _lateral_stretch(law, mat, l1)
        exact = X * (np.array([l1, l2, l2]) - 1.0)
        assert np.abs(u.cpu().numpy().reshape(-1, 3) - exact).max() < 1e-9, rep
    finally:
        G.close()


@pytest.mark.parametrize("law", ["cNH", "iNH"])
def test_newton_under_body_force_matches_oracle_newton(law):
    m = I.box_mesh(2, 3, jitter=0.1, seed=41, clamp=True)
    M = O.OracleMesh(m)
    mat_o = cases.oracle_material(law)
    b = [0.0, 0.0, -0.05]
    f = O.body_force(M, b)
    u_ref, norms = O.newton(M, mat_o, np.zeros(m.n_dofs), f_ext=f, eps_rel=1e-13)
    assert norms[-1] < 1e-10 * norms[0]
    G = hx.Mesh(m, cases.MATS[law])
    try:
        u = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
        fg = torch.empty_like(u)
        hx.hx_body_force(G.ctx, G.handle, b, fg)
        rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, fg, eps_abs=1e-14, eps_rel=1e-11, max_newton=15,
                                     storage=hx.HX_CACHE_TENSORS, precond_prec=hx.HX_FP32, cg_tol=1e-12,
                                     cg_max_iter=20000)
        assert st == hx.HX_OK, rep
        assert rel_inf(u.cpu().numpy(), u_ref) < 1e-8, rep
    finally:
        G.close()


@pytest.mark.parametrize("law", ["cNH", "iNH"])
def test_newton_under_traction_matches_oracle_newton(law):
    """Newton's method (Alg. 1) under a Neumann load: the 2^3 Q3 jittered cube
    clamped on x = 0 with a dead traction (0, 0, -0.03) on x = 1. f_ext comes
    from the library's hx_traction_load on the GPU side and from the oracle's
    traction_load on the oracle side; the oracle's Newton (direct solves)
    converges quadratically to about 1e-10 of the initial residual, so the
    two solutions agree to 1e-8."""
    m = I.box_mesh(2, 3, jitter=0.1, seed=41, clamp=True)
    M = O.OracleMesh(m)
    mat_o = cases.oracle_material(law)
    faces = I.box_boundary_faces(2, 2, 2, 1)
    t = np.array([0.0, 0.0, -0.03])
    f_ref = O.traction_load(M, faces, lambda X, N: np.tile(t, (len(X), 1)))
    u_ref, norms = O.newton(M, mat_o, np.zeros(m.n_dofs), f_ext=f_ref, eps_rel=1e-14, max_it=30)
    assert norms[-1] < 1e-9 * norms[0]
    f = hx.hx_traction_load(m, faces, traction=t)
    assert rel_inf(f, f_ref) < 1e-13
    G = hx.Mesh(m, cases.MATS[law])
    try:
        u = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
        fg = torch.tensor(f, dtype=torch.float64, device="cuda")
        rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, fg, eps_abs=1e-14, eps_rel=1e-11, max_newton=20,
                                     storage=hx.HX_CACHE_TENSORS, precond_prec=hx.HX_FP32, cg_tol=1e-12,
                                     cg_max_iter=20000)
        assert st == hx.HX_OK, rep
        assert rel_inf(u.cpu().numpy(), u_ref) < 1e-8, rep
    finally:
        G.close()


def test_newton_reports_iteration_limit():
    m, u0 = I.workload_uniaxial(2, 2, 1.02)
    G = hx.Mesh(m, dict(cases.MATS["cNH"]))
    try:
        u = cuda(u0)
        rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, None, eps_abs=0.0, eps_rel=0.0, max_newton=1)
        assert st == hx.HX_ERR_NOT_CONVERGED and rep["newton_iters"] == 1 and not rep["converged"]
        assert rep["res"] < rep["res0"]
    finally:
        G.close()


@pytest.mark.parametrize("law", ["cNH", "iNH"])
def test_newton_with_multigrid_matches_closed_form(law):
    """The same load-stepped uniaxial problem with p-multigrid-preconditioned
    linear solves."""
    l1, steps = 1.2, 10
    m, _ = I.workload_uniaxial(2, 4, 1.0)
    mat = dict(cases.MATS[law])
    G = hx.Mesh(m, mat)
    mg = hx.Multigrid(G, precond_prec=hx.HX_FP32)
    try:
        assert mg.levels() == [4, 2, 1]
        X = G.node_coords().cpu().numpy().reshape(-1, 3)
        inc = np.zeros_like(X)
        inc[:, 0] = (l1 - 1.0) / steps * X[:, 0]
        u = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
        for _ in range(steps):
            u += cuda(inc.ravel())
            rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, None, eps_abs=1e-11, eps_rel=1e-12, max_newton=15,
                                         storage=hx.HX_CACHE_TENSORS, cg_tol=1e-11, cg_max_iter=2000, mg=mg)
            assert st == hx.HX_OK and rep["converged"] and rep["newton_iters"] <= 8, rep
        l2 = _lateral_stretch(law, mat, l1)
        exact = X * (np.array([l1, l2, l2]) - 1.0)
        assert np.abs(u.cpu().numpy().reshape(-1, 3) - exact).max() < 1e-9, rep
    finally:
        mg.close()
        G.close()


def test_newton_triaxial_compression_with_hp_multigrid_matches_closed_form():
    """The compressed cube as a boundary-value problem (iNH, kappa = 1e3 mu,
    4^3 jittered cube, p = 4): symmetry clamps and the far faces' normal
    displacements prescribed to J = 0.9999. Its solution is the homogeneous
    compression u = (J^(1/3) - 1) X, which the discretisation holds exactly
    (trilinear geometry; Gauss points integrate the constant stress's
    boundary terms exactly). Newton from u = 0 inside, with linear solves by
    FP64 CG and the FP32 hp-multigrid (p 4 -> 2 -> 1, then h-levels to the
    coarse FP64 CG), reaches it to the solver tolerance."""
    m, delta = I.workload_triaxial_compression(n=4, p=4)
    G = hx.Mesh(m, dict(I.MAT_INH))
    mg = hx.Multigrid(G, precond_prec=hx.HX_FP32, storage=hx.HX_SPATIAL_TENSORS, h_levels=1,
                      coarse_cg_iters=200, coarse_cg_tol=1e-10)
    try:
        assert [mg.level(l) for l in range(len(mg.levels()))] == [(4, 4, 4, 4), (2, 4, 4, 4), (1, 4, 4, 4),
                                                                 (1, 2, 2, 2)]
        X = G.node_coords().cpu().numpy().reshape(-1)
        exact = delta * X
        u0 = np.where(m.dirichlet.astype(bool), exact, 0.0)
        u = cuda(u0)
        rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, None, eps_abs=1e-16, eps_rel=1e-11, max_newton=10,
                                     storage=hx.HX_SPATIAL_TENSORS, cg_tol=1e-12, cg_max_iter=2000, mg=mg)
        assert st == hx.HX_OK and rep["converged"] and rep["newton_iters"] <= 4, rep
        err = np.abs(u.cpu().numpy() - exact).max() / abs(delta)
        assert err < 1e-7, (err, rep)
    finally:
        mg.close()
        G.close()


def test_tube_inflation_newton_matches_oracle_newton():
    """The fibre tube (here 2 x 8 x 3 elements, p = 2, Q2 geometry,
    connectivity numbering) inflated by a dead inner pressure of 0.02 in two
    load steps, with the mirror-plane constraints that leave its axisymmetric
    deformations free: GPU Newton (FP64 CG, FP32 Chebyshev-Jacobi) against
    the oracle's Newton (direct solves). Both start from a small inflation,
    where every fibre is stretched (I* > 1 at every point), so the two sides
    take the same branch of the fibre term from the first step on."""
    m, faces, pressure = I.workload_tube_inflation(p=2, n_r=2, n_theta=8, n_z=3)
    M = O.OracleMesh(m)
    mat_d = dict(I.MAT_FIBER)
    mat_o = cases.oracle_material(mat_d)
    f = hx.hx_traction_load(m, faces, pressure=pressure)
    f_ref = O.traction_load(M, faces, lambda X, N: -pressure * N)
    assert rel_inf(f, f_ref) < 1e-13
    X = O.node_coords(M)
    u0 = (1e-3 * X * np.array([1.0, 1.0, 0.0])).ravel()
    u0[M.dirichlet] = 0.0
    u_ref = u0.copy()
    for k in (1, 2):
        u_ref, norms = O.newton(M, mat_o, u_ref, f_ext=f_ref * (k / 2), eps_abs=1e-12, eps_rel=1e-14, max_it=30)
        assert norms[-1] < 1e-11 * norms[0]
    R = np.hypot(X[:, 0], X[:, 1])
    U = u_ref.reshape(-1, 3)
    u_r = (U[:, 0] * X[:, 0] + U[:, 1] * X[:, 1]) / R
    assert u_r[R < 1.0 + 1e-9].min() > 2e-3  # the inner surface moved out beyond the start
    G = hx.Mesh(m, mat_d)
    try:
        u = cuda(u0)
        fg = cuda(f)
        for k in (1, 2):
            rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, fg * (k / 2), eps_abs=1e-12, eps_rel=1e-14,
                                         max_newton=20, storage=hx.HX_SPATIAL_TENSORS, precond_prec=hx.HX_FP32,
                                         cg_tol=1e-12, cg_max_iter=20000)
            assert st == hx.HX_OK and rep["converged"], rep
        assert rel_inf(u.cpu().numpy(), u_ref) < 1e-8
    finally:
        G.close()
