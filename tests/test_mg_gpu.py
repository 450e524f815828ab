"""p-multigrid (Sec. 6) through the C ABI: level transfers against the
oracle's dense transfer matrices, and the V-cycle-preconditioned CG against
a direct solve of the oracle's assembled constrained tangent."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import inputs as I
from tests import cases
from tests._util import rel_inf

pytestmark = pytest.mark.gpu


def cuda(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("p", [2, 4, 5, 6])
def test_level_transfers_match_oracle_matrices(p):
    n = 2
    m = I.box_mesh(n, p, jitter=0.1, seed=3, clamp=True)
    G = hx.Mesh(m, cases.MATS["cNH"])
    mg = hx.Multigrid(G, precond_prec=hx.HX_FP64)
    try:
        degs = mg.levels()
        assert degs[0] == p and degs[-1] == 1 and all(b == a // 2 for a, b in zip(degs, degs[1:]))
        rng = np.random.Generator(np.random.PCG64(5 + p))
        for lvl in range(len(degs) - 1):
            pf, pc = degs[lvl], degs[lvl + 1]
            P = O.box_transfer_matrix(n, n, n, pc, pf)      # coarse -> fine
            S = O.box_transfer_matrix(n, n, n, pf, pc)      # fine function at coarse nodes
            nf, nc = P.shape
            vc = rng.uniform(-1, 1, size=(nc, 3))
            rf = rng.uniform(-1, 1, size=(nf, 3))
            out_f = torch.empty(3 * nf, dtype=torch.float64, device="cuda")
            out_c = torch.empty(3 * nc, dtype=torch.float64, device="cuda")
            mg.transfer(lvl, 0, cuda(vc.ravel()), out_f)
            assert rel_inf(out_f.cpu().numpy().reshape(-1, 3), P @ vc) < 1e-13
            mg.transfer(lvl, 1, cuda(rf.ravel()), out_c)
            assert rel_inf(out_c.cpu().numpy().reshape(-1, 3), P.T @ rf) < 1e-13
            mg.transfer(lvl, 2, cuda(rf.ravel()), out_c)
            assert rel_inf(out_c.cpu().numpy().reshape(-1, 3), S @ rf) < 1e-13
    finally:
        mg.close()
        G.close()


@pytest.mark.parametrize("law", ["cNH", "iNH"])
@pytest.mark.parametrize("pp", [hx.HX_FP64, hx.HX_FP32])
def test_mg_cg_matches_direct_solve_in_few_iterations(law, pp):
    m = cases.small_cube(4, 4, law, clamp=True, seed=17)
    # a small strain keeps the tangent positive definite (at 1 % the iNH
    # state's compressive regions already give negative curvature here)
    M, X, u = cases.state_for(m, law, seed=18, strain=0.002)
    mat = cases.oracle_material(law)
    K = O.constrain_matrix(O.assemble_sparse(M, mat, u), M.dirichlet)
    rhs = I.random_direction(m.n_dofs, 19)
    rhs[M.dirichlet] = 0.0
    import scipy.sparse.linalg as spla
    ref = spla.spsolve(K.tocsc(), rhs)
    G = hx.Mesh(m, cases.MATS[law])
    mg = hx.Multigrid(G, precond_prec=pp, storage=hx.HX_CACHE_TENSORS)
    try:
        u_t = cuda(u)
        G.precompute(u_t, hx.HX_FP64, hx.HX_CACHE_TENSORS)
        mg.setup(u_t)
        x = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
        it, rel, st = mg.cg_solve(cuda(rhs), x, 1e-10, 500)
        assert st == hx.HX_OK and rel <= 1e-10, (it, rel)
        assert rel_inf(x.cpu().numpy(), ref) < 1e-8
        # single-level Chebyshev(5)-Jacobi CG needs many more iterations
        G.precompute(u_t, pp, hx.HX_CACHE_TENSORS)
        dinv = 1.0 / G.diagonal(hx.HX_FP64)
        lam = hx.hx_estimate_lambda_max(G.ctx, G.handle, dinv, iters=30, seed=3)
        x2 = torch.zeros_like(x)
        it2, rel2, st2 = hx.hx_cg_solve(G.ctx, G.handle, cuda(rhs), x2, 1e-10, 5000, 5, 1.2 * lam, 15.0, pp)
        assert st2 == hx.HX_OK
        assert it * 3 < it2, (it, it2)
    finally:
        mg.close()
        G.close()


def test_mg_rejects_unsupported_meshes():
    m = I.tube_mesh(2, n_r=1, n_theta=8, n_z=2)
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        with pytest.raises(hx.HxError) as e:
            hx.Multigrid(G)
        assert e.value.status == hx.HX_ERR_UNSUPPORTED
    finally:
        G.close()


# --------------------------------------------------------------------------
# h-levels and the coarse FP64 CG
# --------------------------------------------------------------------------

def test_h_levels_and_their_transfers_match_oracle_matrices():
    """4^3 Q2 jittered box: p-levels 2, 1, then h-levels 2^3 and 1^3; the
    h-prolongation, its transpose and the state injection against the
    oracle's dense h-transfer matrix (1e-13)."""
    m = I.box_mesh(4, 2, jitter=0.1, seed=3, clamp=True)
    G = hx.Mesh(m, cases.MATS["cNH"])
    mg = hx.Multigrid(G, precond_prec=hx.HX_FP64, h_levels=8, coarse_cg_iters=50, coarse_cg_tol=1e-10)
    try:
        assert mg.levels() == [2, 1, 1, 1]
        assert [mg.level(l) for l in range(4)] == [(2, 4, 4, 4), (1, 4, 4, 4), (1, 2, 2, 2), (1, 1, 1, 1)]
        rng = np.random.Generator(np.random.PCG64(29))
        for lvl in (1, 2):
            _, nxc, nyc, nzc = mg.level(lvl + 1)
            P = O.box_h_transfer_matrix(nxc, nyc, nzc)
            nf, nc = P.shape
            Mf = (2 * nxc + 1, 2 * nyc + 1)
            S = np.zeros((nc, nf))  # injection: coarse node (i, j, k) <- fine node (2i, 2j, 2k)
            for J in range(nc):
                i, j, k = J % (nxc + 1), (J // (nxc + 1)) % (nyc + 1), J // ((nxc + 1) * (nyc + 1))
                S[J, 2 * i + Mf[0] * (2 * j + Mf[1] * 2 * k)] = 1.0
            vc = rng.uniform(-1, 1, size=(nc, 3))
            rf = rng.uniform(-1, 1, size=(nf, 3))
            out_f = torch.empty(3 * nf, dtype=torch.float64, device="cuda")
            out_c = torch.empty(3 * nc, dtype=torch.float64, device="cuda")
            mg.transfer(lvl, 0, cuda(vc.ravel()), out_f)
            assert rel_inf(out_f.cpu().numpy().reshape(-1, 3), P @ vc) < 1e-13
            mg.transfer(lvl, 1, cuda(rf.ravel()), out_c)
            assert rel_inf(out_c.cpu().numpy().reshape(-1, 3), P.T @ rf) < 1e-13
            mg.transfer(lvl, 2, cuda(rf.ravel()), out_c)
            assert rel_inf(out_c.cpu().numpy().reshape(-1, 3), S @ rf) < 1e-15
    finally:
        mg.close()
        G.close()


@pytest.mark.parametrize("pp", [hx.HX_FP64, hx.HX_FP32])
def test_hmg_cg_matches_direct_solve(pp):
    """hp-multigrid (p 4 -> 2 -> 1, then 4^3 -> 2^3 -> 1^3) with the coarse
    FP64 CG preconditions CG to the oracle's direct solution."""
    m = cases.small_cube(4, 4, "cNH", clamp=True, seed=31)
    M, X, u = cases.state_for(m, "cNH", seed=32, strain=0.01)
    mat = cases.oracle_material("cNH")
    K = O.constrain_matrix(O.assemble_sparse(M, mat, u), M.dirichlet)
    rhs = I.random_direction(m.n_dofs, 33)
    rhs[M.dirichlet] = 0.0
    import scipy.sparse.linalg as spla
    ref = spla.spsolve(K.tocsc(), rhs)
    G = hx.Mesh(m, cases.MATS["cNH"])
    mg = hx.Multigrid(G, precond_prec=pp, storage=hx.HX_CACHE_TENSORS, h_levels=8, coarse_cg_iters=100,
                      coarse_cg_tol=1e-8)
    try:
        assert mg.levels() == [4, 2, 1, 1, 1]
        u_t = cuda(u)
        G.precompute(u_t, hx.HX_FP64, hx.HX_CACHE_TENSORS)
        mg.setup(u_t)
        x = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
        it, rel, st = mg.cg_solve(cuda(rhs), x, 1e-10, 500)
        assert st == hx.HX_OK and rel <= 1e-10, (it, rel)
        assert rel_inf(x.cpu().numpy(), ref) < 1e-8
        c_it = mg.coarse_iters()
        assert 1 <= c_it <= 100, c_it
    finally:
        mg.close()
        G.close()


def test_hmg_cg_iterations_stay_flat_from_8_to_32_cubed():
    """Jittered clamped cNH cubes of 8^3, 16^3 and 32^3 Q2 elements at 2 %
    strain: the hp-multigrid preconditioned CG reaches 1e-8 in about the same
    number of iterations at every size, while the p-only hierarchy (its
    degree-1 level smoothed by Chebyshev) needs more and more."""
    its, its_p = {}, {}
    for n in (8, 16, 32):
        m = cases.small_cube(n, 2, "cNH", clamp=True, seed=41)
        M, X, u = cases.state_for(m, "cNH", seed=42, strain=0.02)
        rhs = I.random_direction(m.n_dofs, 43)
        rhs[M.dirichlet] = 0.0
        G = hx.Mesh(m, cases.MATS["cNH"])
        try:
            u_t = cuda(u)
            G.precompute(u_t, hx.HX_FP64, hx.HX_CACHE_TENSORS)
            for h_levels, store in ((10, its), (0, its_p)):
                mg = hx.Multigrid(G, precond_prec=hx.HX_FP32, storage=hx.HX_CACHE_TENSORS, h_levels=h_levels,
                                  coarse_cg_iters=200 if h_levels else 0, coarse_cg_tol=1e-6)
                try:
                    mg.setup(u_t)
                    x = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
                    it, rel, st = mg.cg_solve(cuda(rhs), x, 1e-8, 2000)
                    assert st == hx.HX_OK and rel <= 1e-8, (n, h_levels, it, rel)
                    store[n] = it
                finally:
                    mg.close()
        finally:
            G.close()
    assert its[32] <= 1.5 * its[8] + 2, its
    assert its_p[32] > 1.5 * its[32], (its, its_p)
