"""Batched persistent launch: many meshes of mixed degree, size and Newton
state applied in one launch, each checked against the oracle and against the
single-mesh kernel."""
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


def _meshes(law, specs, ctx):
    out = []
    for k, (n, p) in enumerate(specs):
        m = cases.small_cube(n, p, law, seed=500 + k, clamp=(k == 1))
        M, X, u = cases.state_for(m, law, seed=600 + k)
        if k == 1:
            u[M.dirichlet] = 0.0
        G = hx.Mesh(m, cases.MATS[law], ctx=ctx)
        out.append((m, M, u, G))
    return out


@pytest.mark.parametrize("law", cases.LAWS)
@pytest.mark.parametrize("storage", [hx.HX_CACHE_F, hx.HX_CACHE_TENSORS, hx.HX_SPATIAL_TENSORS])
@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_batch_matches_oracle_and_single_mesh(law, storage, prec):
    ctx = hx.hx_create(0)
    specs = [(3, 4), (2, 6), (4, 2), (3, 3), (2, 5), (5, 1), (3, 4)]
    items = _meshes(law, specs, ctx)
    batch = None
    try:
        dus, outs = [], []
        for k, (m, M, u, G) in enumerate(items):
            G.precompute(torch.tensor(u, dtype=torch.float64, device="cuda"), prec, storage)
            dus.append(torch.tensor(I.random_direction(m.n_dofs, 700 + k), dtype=DT[prec], device="cuda"))
            outs.append(torch.full_like(dus[-1], 7.0))  # stale values must be overwritten
        batch = hx.hx_batch_create(ctx, [it[3] for it in items])
        for rep in range(2):
            hx.hx_batch_tangent_apply(ctx, batch, dus, outs)
            hx.hx_sync(ctx, 60000)
            mat = cases.oracle_material(law)
            for k, (m, M, u, G) in enumerate(items):
                du = dus[k].double().cpu().numpy()
                ref = O.apply_constrained(M, mat, u, du) if k == 1 else O.apply(M, mat, u, du)
                got = outs[k].double().cpu().numpy()
                assert rel_inf(got, ref) < TOL[prec], (k, rel_inf(got, ref))
                single = G.apply(dus[k]).double().cpu().numpy()
                assert rel_inf(got, single) < (1e-14 if prec == hx.HX_FP64 else 1e-6)
    finally:
        if batch is not None:
            hx.hx_batch_destroy(batch)
        for it in items:
            it[3].close()
        hx.hx_destroy(ctx)


def test_batch_statuses():
    ctx = hx.hx_create(0)
    items = _meshes("cNH", [(2, 2), (2, 3)], ctx)
    other = hx.Mesh(cases.small_cube(2, 2, "iNH"), cases.MATS["iNH"], ctx=ctx)
    try:
        with pytest.raises(hx.HxError) as e:
            hx.hx_batch_create(ctx, [items[0][3], other])
        assert e.value.status == hx.HX_ERR_ARG
        batch = hx.hx_batch_create(ctx, [it[3] for it in items])
        dus = [it[3].zeros() for it in items]
        outs = [torch.zeros_like(d) for d in dus]
        with pytest.raises(hx.HxError) as e:
            hx.hx_batch_tangent_apply(ctx, batch, dus, outs)
        assert e.value.status == hx.HX_ERR_NOT_READY
        for it in items:
            it[3].precompute(torch.tensor(it[2], device="cuda"), hx.HX_FP64, hx.HX_RECOMPUTE)
        with pytest.raises(hx.HxError) as e:
            hx.hx_batch_tangent_apply(ctx, batch, dus, outs)
        assert e.value.status == hx.HX_ERR_UNSUPPORTED
        hx.hx_batch_destroy(batch)
    finally:
        other.close()
        for it in items:
            it[3].close()
        hx.hx_destroy(ctx)


@pytest.mark.parametrize("law", ["cNH", "fiber"])
@pytest.mark.parametrize("storage", [hx.HX_CACHE_F, hx.HX_SPATIAL_TENSORS])
@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_batch_many_items_per_cta(law, storage, prec):
    """Meshes large enough that every CTA of the persistent launch takes many
    work items of several degrees in turn (the staged items alternate the
    parity of the CTA's bulk-copy barrier): the batch must equal the
    single-mesh apply of every mesh (itself checked against the oracle)."""
    ctx = hx.hx_create(0)
    specs = [(16, 4), (20, 2), (12, 3), (8, 5), (6, 6)]
    Gs, batch = [], None
    try:
        dus, outs = [], []
        for k, (n, p) in enumerate(specs):
            G = hx.Mesh(cases.small_cube(n, p, law, seed=900 + k), cases.MATS[law], ctx=ctx)
            X = G.node_coords().cpu().numpy()
            u = I.sine_field(910 + k, strain=0.05)(X)
            if law == "fiber":
                u = u + X @ np.diag([0.0, 0.08, 0.08])
            G.precompute(torch.tensor(u.ravel(), dtype=torch.float64, device="cuda"), prec, storage)
            Gs.append(G)
            dus.append(torch.tensor(I.random_direction(3 * X.shape[0], 920 + k), dtype=DT[prec], device="cuda"))
            outs.append(torch.full_like(dus[-1], 7.0))
        batch = hx.hx_batch_create(ctx, Gs)
        for rep in range(2):
            hx.hx_batch_tangent_apply(ctx, batch, dus, outs)
            hx.hx_sync(ctx, 60000)
            for k, G in enumerate(Gs):
                single = G.apply(dus[k]).double().cpu().numpy()
                got = outs[k].double().cpu().numpy()
                assert rel_inf(got, single) < (1e-14 if prec == hx.HX_FP64 else 1e-6), (k, rel_inf(got, single))
    finally:
        if batch is not None:
            hx.hx_batch_destroy(batch)
        for G in Gs:
            G.close()
        hx.hx_destroy(ctx)


@pytest.mark.parametrize("pp", [hx.HX_FP32, hx.HX_FP64])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_cg_matches_direct_solves_and_single_mesh_cg(pp, use_graph):
    """Six clamped jittered cubes of mixed size, degree and state: the
    batched CG (lockstep, per-mesh Chebyshev(3)-Jacobi, one graph per
    iteration) solves every mesh's constrained system to the oracle's direct
    solution, and each mesh's iteration count is that of the single-mesh
    hx_cg_solve on the same system (same eigenvalue estimate) up to the
    rounding differences of the two operator kernels (3 + 5 %)."""
    import scipy.sparse.linalg as spla
    ctx = hx.hx_create(0)
    specs = [(3, 2), (2, 4), (4, 1), (2, 3), (3, 3), (2, 5)]
    items, batch = [], None
    try:
        for k, (n, p) in enumerate(specs):
            m = cases.small_cube(n, p, "cNH", seed=700 + k, clamp=True)
            M, X, u = cases.state_for(m, "cNH", seed=710 + k, strain=0.01)
            u[M.dirichlet] = 0.0
            K = O.constrain_matrix(O.assemble_sparse(M, cases.oracle_material("cNH"), u), M.dirichlet)
            # CG needs an SPD tangent (stronger sine states on these small high-degree cubes are indefinite)
            assert spla.eigsh(K.tocsc(), k=1, which="SA", return_eigenvectors=False)[0] > 0
            G = hx.Mesh(m, cases.MATS["cNH"], ctx=ctx)
            u_t = torch.tensor(u, dtype=torch.float64, device="cuda")
            G.precompute(u_t, hx.HX_FP64, hx.HX_CACHE_TENSORS)
            G.precompute(u_t, pp, hx.HX_CACHE_TENSORS)
            rhs = I.random_direction(m.n_dofs, 720 + k)
            rhs[M.dirichlet] = 0.0
            ref = spla.spsolve(K.tocsc(), rhs)
            items.append((G, torch.tensor(rhs, dtype=torch.float64, device="cuda"), ref))
        batch = hx.hx_batch_create(ctx, [G for G, _, _ in items])
        xs = [torch.zeros_like(r) for _, r, _ in items]
        its, rels, st = hx.hx_batch_cg_solve(ctx, batch, [r for _, r, _ in items], xs, 1e-10, 3000, 3, 15.0, pp,
                                             use_graph)
        assert st == hx.HX_OK, (its, rels)
        for (G, rhs, ref), x, it, rel in zip(items, xs, its, rels):
            assert rel <= 1e-10 and it > 0
            assert rel_inf(x.cpu().numpy(), ref) < 1e-8
            # the same system through the single-mesh solver
            dinv = 1.0 / G.diagonal(hx.HX_FP64)
            lam = hx.hx_estimate_lambda_max(G.ctx, G.handle, dinv, iters=20, seed=7)
            x1 = torch.zeros_like(rhs)
            it1, rel1, st1 = hx.hx_cg_solve(G.ctx, G.handle, rhs, x1, 1e-10, 3000, 3, 1.2 * lam, 15.0, pp)
            assert st1 == hx.HX_OK
            assert abs(it - it1) <= 3 + 0.05 * it1, (it, it1)
    finally:
        if batch is not None:
            hx.hx_batch_destroy(batch)
        for G, _, _ in items:
            G.close()
        hx.hx_destroy(ctx)


def test_batch_cg_reports_a_mesh_that_misses_the_tolerance():
    ctx = hx.hx_create(0)
    items, batch = [], None
    try:
        for k, (n, p) in enumerate([(3, 2), (3, 4)]):
            m = cases.small_cube(n, p, "cNH", seed=730 + k, clamp=True)
            M, X, u = cases.state_for(m, "cNH", seed=740 + k, strain=0.01)
            u[M.dirichlet] = 0.0
            G = hx.Mesh(m, cases.MATS["cNH"], ctx=ctx)
            u_t = torch.tensor(u, dtype=torch.float64, device="cuda")
            G.precompute(u_t, hx.HX_FP64, hx.HX_CACHE_F)
            G.precompute(u_t, hx.HX_FP32, hx.HX_CACHE_F)
            rhs = torch.tensor(I.random_direction(m.n_dofs, 750 + k), dtype=torch.float64, device="cuda")
            rhs[torch.tensor(M.dirichlet, device="cuda")] = 0.0
            items.append((G, rhs))
        batch = hx.hx_batch_create(ctx, [G for G, _ in items])
        xs = [torch.zeros_like(r) for _, r in items]
        its, rels, st = hx.hx_batch_cg_solve(ctx, batch, [r for _, r in items], xs, 1e-12, 3, 2, 15.0, hx.HX_FP32)
        assert st == hx.HX_ERR_NOT_CONVERGED
        assert its == [3, 3] and all(r > 1e-12 for r in rels)
    finally:
        if batch is not None:
            hx.hx_batch_destroy(batch)
        for G, _ in items:
            G.close()
        hx.hx_destroy(ctx)
