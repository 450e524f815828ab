"""GPU checks of the solver layer (Sec. 6): power-iteration eigenvalue bound,
FP64 CG with an FP32 (or FP64) Chebyshev-Jacobi preconditioner captured as a
CUDA graph, and the autograd wrapper whose backward is the tangent kernel."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import inputs as I
from tests import cases
from tests._util import rel_inf

pytestmark = pytest.mark.gpu


def cuda(x, dt=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dt, device="cuda")


def _problem(law="iNH", n=3, p=3, seed=201):
    """Clamped iNH cube at 1% strain: the constrained tangent is SPD here (at 3%
    random strain with kappa = 50 the compressive stresses exceed mu and the
    tangent turns indefinite, where CG rightly reports non-positive curvature)."""
    m = cases.small_cube(n, p, law, seed=seed, clamp=True)
    M, X, u = cases.state_for(m, law, seed=seed + 1, strain=0.01)
    u[M.dirichlet] = 0.0
    return m, M, u, cases.oracle_material(law)


def test_lambda_max_power_iteration():
    m, M, u, mat = _problem()
    K = O.constrain_matrix(O.assemble_sparse(M, mat, u), M.dirichlet).toarray()
    dinv = 1.0 / O.diagonal_constrained(M, mat, u)
    lam_true = np.abs(np.linalg.eigvals(K * dinv[:, None])).max()
    G = hx.Mesh(m, cases.MATS["iNH"])
    try:
        G.precompute(cuda(u), hx.HX_FP64, hx.HX_CACHE_TENSORS)
        est = hx.hx_estimate_lambda_max(G.ctx, G.handle, cuda(dinv), iters=200, seed=3)
        assert 0.9 * lam_true < est <= lam_true * (1 + 1e-9)
    finally:
        G.close()


@pytest.mark.parametrize("pp", [hx.HX_FP32, hx.HX_FP64])
@pytest.mark.parametrize("graph", [True, False])
def test_cg_solves_newton_step(pp, graph):
    import scipy.sparse.linalg as spla
    m, M, u, mat = _problem()
    K = O.constrain_matrix(O.assemble_sparse(M, mat, u), M.dirichlet)
    b = -O.residual_constrained(M, mat, u)
    x_ref = spla.spsolve(K.tocsc(), b)
    dinv = 1.0 / O.diagonal_constrained(M, mat, u)
    lam = np.abs(np.linalg.eigvals(K.toarray() * dinv[:, None])).max()
    G = hx.Mesh(m, cases.MATS["iNH"])
    try:
        u_t = cuda(u)
        G.precompute(u_t, hx.HX_FP64, hx.HX_CACHE_TENSORS)
        G.precompute(u_t, hx.HX_FP32, hx.HX_CACHE_TENSORS)
        x = torch.zeros_like(u_t)
        it, rel, st = hx.hx_cg_solve(G.ctx, G.handle, cuda(b), x, 1e-10, 2000, 5, 1.1 * lam, 15.0, pp, graph)
        assert st == hx.HX_OK, (it, rel)
        assert rel < 1e-10 and it > 0
        assert rel_inf(x.cpu().numpy(), x_ref) < 1e-7
        # the oracle's plain PCG with the same preconditioner takes a similar count
        Kop = lambda v: O.apply_constrained(M, mat, u, v)
        Mop = lambda r: O.chebyshev_smooth(Kop, r, np.zeros_like(r), dinv, 5, 1.1 * lam, 15.0, zero_initial=True)
        _, it_ref, rel_ref, _ = O.pcg(Kop, b, Mop, tol=1e-10)
        assert abs(it - it_ref) <= max(3, 0.2 * it_ref)
    finally:
        G.close()


def test_cg_not_converged_status():
    m, M, u, mat = _problem()
    b = -O.residual_constrained(M, mat, u)
    G = hx.Mesh(m, cases.MATS["iNH"])
    try:
        u_t = cuda(u)
        G.precompute(u_t, hx.HX_FP64, hx.HX_CACHE_F)
        x = torch.zeros_like(u_t)
        it, rel, st = hx.hx_cg_solve(G.ctx, G.handle, cuda(b), x, 1e-12, 2, 0, 1.0, 2.0, hx.HX_FP64, True)
        assert st == hx.HX_ERR_NOT_CONVERGED and it == 2 and rel > 1e-12
    finally:
        G.close()


@pytest.mark.parametrize("prec", [torch.float64, torch.float32])
def test_autograd_backward_is_tangent(prec):
    """Tube with the fibre law (quadratic geometry, p = 3): the backward of
    w.R(u) is K(u) w; checked against the oracle's assembled matrix and, in
    FP64, against central differences of w.R(u) (h = 1e-6)."""
    m = I.tube_mesh(3, n_r=2, n_theta=16, n_z=2)
    mat_d = dict(I.MAT_FIBER)
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    u = I.inflation_field(301)(X).ravel()
    w = I.random_direction(m.n_dofs, 302)
    mat = cases.oracle_material(mat_d)
    G = hx.Mesh(m, mat_d)
    try:
        u_t = cuda(u, prec).requires_grad_(True)
        r = hx.residual_autograd(G, u_t)
        loss = (r * cuda(w, prec)).sum()
        loss.backward()
        grad = u_t.grad.double().cpu().numpy()
        K = O.assemble_sparse(M, mat, u_t.detach().double().cpu().numpy())
        tol = 1e-12 if prec == torch.float64 else 1e-5
        assert rel_inf(grad, K @ cuda(w, prec).double().cpu().numpy()) < tol
        if prec == torch.float64:
            g = np.random.Generator(np.random.PCG64(303))
            v = g.uniform(-1, 1, size=m.n_dofs)
            h = 1e-6
            def f(x):
                with torch.no_grad():
                    return float((hx.residual_autograd(G, cuda(x)) * cuda(w)).sum())
            fd = (f(u + h * v) - f(u - h * v)) / (2 * h)
            assert abs(fd - grad @ v) < 1e-6 * abs(grad @ v)
    finally:
        G.close()


def test_cg_reports_indefinite_tangent_under_high_pressure():
    """iNH with kappa = 1e3 mu compressed to J ~ 0.9: the pressure (~95 mu)
    makes rotation-dominated modes unstable, so p.Kp <= 0 appears and CG must
    stop with HX_ERR_NAN instead of returning a wrong solution."""
    m, field, seed = I.workload_compressed_cube(n=4, p=3, J_target=0.9, sine_amp=0.005)
    G = hx.Mesh(m, dict(I.MAT_INH))
    try:
        u = torch.tensor(field(G.node_coords().cpu().numpy()).ravel(), dtype=torch.float64, device="cuda")
        G.precompute(u, hx.HX_FP64, hx.HX_CACHE_TENSORS)
        # the constrained tangent has a negative eigenvalue (oracle, dense)
        M = O.OracleMesh(m)
        K = O.constrain_matrix(O.assemble_sparse(M, O.Material.from_dict(dict(I.MAT_INH)), u.cpu().numpy()),
                               M.dirichlet).toarray()
        assert np.linalg.eigvalsh(K).min() < 0
        x = torch.zeros_like(u)
        with pytest.raises(hx.HxError) as e:
            hx.hx_cg_solve(G.ctx, G.handle, -G.residual(u), x, 1e-10, 500, 0, 1.0, 2.0, hx.HX_FP64)
        assert e.value.status == hx.HX_ERR_NAN and "curvature" in str(e.value)
    finally:
        G.close()
