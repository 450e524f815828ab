"""Multi-rank paths on CPU ranks (gloo, world size 2): the element partition
with its interface sum reproduces the full tangent apply, and the benchmark's
max-over-ranks timing and weak-scaling aggregate."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _dd_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2408_12479_gb300 import dd
        from paper_2408_12479_gb300 import inputs as I
        from tests import cases
        n, p = 3, 2
        m = I.box_mesh(n, p, jitter=0.1, seed=5, clamp=False)
        M = O.OracleMesh(m)
        mat = cases.oracle_material("cNH")
        X = O.node_coords(M)
        u = I.sine_field(7, strain=0.02)(X).ravel()
        du = I.random_direction(m.n_dofs, 8)
        slabs = dd.slab_partition(n, world)
        z0, z1 = slabs[rank]
        part = O.apply(M, mat, u, du, elems=dd.slab_elements(n, n, z0, z1))
        v = dd.interface_sum(torch.tensor(part), n, n, p, slabs, rank)
        n0, n1 = dd.slab_node_range(n, n, p, z0, z1)
        full = O.apply(M, mat, u, du)
        err = float(np.abs(v.numpy()[3 * n0:3 * n1] - full[3 * n0:3 * n1]).max() / np.abs(full).max())
        out[rank] = err
    finally:
        dist.destroy_process_group()


def test_slab_partition_interface_sum_matches_full_apply():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_dd_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert len(out) == world
    assert max(out.values()) < 1e-13


def _timing_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [1.5, 2.5][rank]
        t_max = bench.max_over_ranks(ms, world)
        out[rank] = (t_max, bench.weak_value(1000, t_max, world))
    finally:
        dist.destroy_process_group()


def test_bench_max_over_ranks_and_weak_aggregate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_timing_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        t_max, value = out[r]
        assert t_max == 2.5
        assert abs(value - 2 * 1000 / 2.5e-3 / 1e9) < 1e-15


def _slab_case(world, rank):
    """Clamped 3^3 jittered Q2 cube (cNH, 2 % sine state) split into `world`
    slabs; returns the oracle pieces and this rank's SlabSystem."""
    from oracle import oracle as O
    from paper_2408_12479_gb300 import dd
    from paper_2408_12479_gb300 import inputs as I
    from tests import cases
    n, p = 3, 2
    m = I.box_mesh(n, p, jitter=0.1, seed=5, clamp=True)
    M = O.OracleMesh(m)
    mat = cases.oracle_material("cNH")
    u = I.sine_field(7, strain=0.02)(O.node_coords(M)).ravel()
    slabs = dd.slab_partition(n, world)
    sl = dd.local_slice(n, n, p, slabs[rank])
    Ms = O.OracleMesh(dd.slab_mesh(m, slabs[rank]))
    u_loc = u[sl].copy()

    def apply_local(v):
        return torch.tensor(O.apply(Ms, mat, u_loc, v.numpy()))

    S = dd.SlabSystem(n, n, p, slabs, rank, apply_local, m.dirichlet[sl].astype(bool))
    d_loc = torch.tensor(O.diagonal(Ms, mat, u_loc))
    return O, M, mat, u, sl, S, d_loc


def _direct(O, M, mat, u, b):
    import scipy.sparse.linalg as spla
    K = O.constrain_matrix(O.assemble_sparse(M, mat, u), M.dirichlet.astype(bool))
    return spla.spsolve(K.tocsc(), b)


def _solve_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2408_12479_gb300 import inputs as I
        O, M, mat, u, sl, S, d_loc = _slab_case(world, rank)
        res = {}
        # the operator, the global dot and the diagonal over slabs
        v = I.random_direction(M.n_dofs, 8)
        ref = O.apply_constrained(M, mat, u, v)
        res["apply"] = float(np.abs(S.apply(torch.tensor(v[sl])).numpy() - ref[sl]).max() / np.abs(ref).max())
        res["dot"] = abs(S.dot(torch.tensor(v[sl]), torch.tensor(ref[sl])) - v @ ref) / abs(v @ ref)
        dref = O.diagonal_constrained(M, mat, u)
        inv_d = 1.0 / S.diagonal(d_loc)
        res["diag"] = float(np.abs(1.0 / inv_d.numpy() - dref[sl]).max() / np.abs(dref).max())
        # the Chebyshev-Jacobi smoother against the oracle's on the whole mesh
        lam = S.lambda_max(inv_d)
        b = O.apply_constrained(M, mat, u, I.random_direction(M.n_dofs, 9))
        x0 = I.random_direction(M.n_dofs, 10)

        def Kc(x):
            return O.apply_constrained(M, mat, u, x)

        y_ref = O.chebyshev_smooth(Kc, b, x0, 1.0 / dref, 4, lam, 15.0)
        y = S.chebyshev(torch.tensor(b[sl]), torch.tensor(x0[sl]), inv_d, 4, lam, 15.0).numpy()
        res["cheb"] = float(np.abs(y - y_ref[sl]).max() / np.abs(y_ref).max())
        res["lam"] = lam
        # CG over the slabs against a direct solve of the assembled system
        x_dir = _direct(O, M, mat, u, b)
        bl = torch.tensor(b[sl])
        x, it, rel = S.cg(bl, precond=lambda r: inv_d * r, tol=1e-11, max_iter=3000)
        res["jacobi"] = (it, rel, float(np.abs(x.numpy() - x_dir[sl]).max() / np.abs(x_dir).max()))
        cheb = lambda r: S.chebyshev(r, torch.zeros_like(r), inv_d, 3, lam, 15.0, zero_initial=True)
        x, it, rel = S.cg(bl, precond=cheb, tol=1e-11, max_iter=3000)
        res["chebcg"] = (it, rel, float(np.abs(x.numpy() - x_dir[sl]).max() / np.abs(x_dir).max()))
        out[rank] = res
    finally:
        dist.destroy_process_group()


def _one_slab_iterations():
    """The same solves with one slab and no process group."""
    from paper_2408_12479_gb300 import inputs as I
    O, M, mat, u, sl, S, d_loc = _slab_case(1, 0)
    inv_d = 1.0 / S.diagonal(d_loc)
    lam = S.lambda_max(inv_d)
    b = torch.tensor(O.apply_constrained(M, mat, u, I.random_direction(M.n_dofs, 9)))
    _, it_j, _ = S.cg(b, precond=lambda r: inv_d * r, tol=1e-11, max_iter=3000)
    cheb = lambda r: S.chebyshev(r, torch.zeros_like(r), inv_d, 3, lam, 15.0, zero_initial=True)
    _, it_c, _ = S.cg(b, precond=cheb, tol=1e-11, max_iter=3000)
    return lam, it_j, it_c


def test_slab_mesh_and_owner_rule_partition_the_dofs():
    from paper_2408_12479_gb300 import dd
    from paper_2408_12479_gb300 import inputs as I
    n, p = 4, 3
    m = I.box_mesh(n, p, jitter=0.1, seed=3)
    slabs = dd.slab_partition(n, 3)
    count = np.zeros(m.n_dofs, dtype=int)
    for r, sl in enumerate(slabs):
        sub = dd.slab_mesh(m, sl)
        rng = dd.local_slice(n, n, p, sl)
        assert sub.n_dofs == rng.stop - rng.start
        # local numbering is the global range: connectivity maps onto the same nodes
        e = dd.slab_elements(n, n, *sl)
        n0 = rng.start // 3
        assert np.array_equal(sub.dof_conn + n0, m.dof_conn[e])
        assert np.array_equal(sub.geo_nodes[sub.geo_conn], m.geo_nodes[m.geo_conn[e]])
        count[rng][dd.owned_mask(n, n, p, slabs, r)] += 1
    assert (count == 1).all()  # every DoF owned by exactly one rank


@pytest.mark.parametrize("world", [2, 3])
def test_cg_over_slabs_matches_direct_solve(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_solve_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert len(out) == world
    lam1, it_j1, it_c1 = _one_slab_iterations()
    for r in range(world):
        res = out[r]
        assert res["apply"] < 1e-13 and res["dot"] < 1e-13 and res["diag"] < 1e-13, res
        assert res["cheb"] < 1e-12, res
        assert abs(res["lam"] - lam1) < 1e-10 * lam1
        for key, it1 in (("jacobi", it_j1), ("chebcg", it_c1)):
            it, rel, err = res[key]
            assert rel < 1e-10 and err < 1e-9, (key, res[key])
            assert abs(it - it1) <= 1, (key, it, it1)  # the partition changes only round-off
        # the smoother preconditions: fewer iterations than plain Jacobi
        assert res["chebcg"][0] < res["jacobi"][0]


def _newton_case(world, rank):
    """Clamped 2^3 Q2 jittered cube (cNH) under a body force, split into
    slabs: the rank's SlabSystem with oracle callables for its elements."""
    from oracle import oracle as O
    from paper_2408_12479_gb300 import dd
    from paper_2408_12479_gb300 import inputs as I
    from tests import cases
    n, p = 2, 2
    m = I.box_mesh(n, p, jitter=0.1, seed=41, clamp=True)
    mat = cases.oracle_material("cNH")
    slabs = dd.slab_partition(n, world)
    sl = dd.local_slice(n, n, p, slabs[rank])
    Ms = O.OracleMesh(dd.slab_mesh(m, slabs[rank]))
    state = {"u": np.zeros(Ms.n_dofs)}

    def apply_local(v):
        return torch.tensor(O.apply(Ms, mat, state["u"], v.numpy()))

    S = dd.SlabSystem(n, n, p, slabs, rank, apply_local, m.dirichlet[sl].astype(bool))
    f = S.assemble(torch.tensor(O.body_force(Ms, [0.0, 0.0, -0.05])))
    calls = dict(residual_local=lambda u: torch.tensor(O.residual(Ms, mat, u.numpy())),
                 set_state=lambda u: state.update(u=u.numpy().copy()),
                 diagonal_local=lambda: torch.tensor(O.diagonal(Ms, mat, state["u"])))
    return m, mat, sl, S, f, calls


def _newton_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        O.set_threads(2)  # the ranks share the host's cores
        m, mat, sl, S, f, calls = _newton_case(world, rank)
        u0 = torch.zeros(sl.stop - sl.start, dtype=torch.float64)
        u, rep = S.newton(u0, f_ext=f, eps_rel=1e-11, cg_tol=1e-12, **calls)
        uc, repc = S.newton(u0, f_ext=f, eps_rel=1e-11, cg_tol=1e-12, cheb_degree=3, **calls)
        out[rank] = (u.numpy(), rep, uc.numpy(), repc, (sl.start, sl.stop))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_newton_over_slabs_matches_oracle_newton(world):
    """Alg. 1 over slabs (residual and load assembled by interface sums,
    norms by owned-DoF reductions, updates by slab CG) reaches the oracle's
    global Newton solution, with the iteration count of the one-slab run."""
    from oracle import oracle as O
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_newton_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    m, mat, sl1, S1, f1, calls1 = _newton_case(1, 0)
    M = O.OracleMesh(m)
    u_ref, norms = O.newton(M, mat, np.zeros(m.n_dofs), f_ext=O.body_force(M, [0.0, 0.0, -0.05]), eps_rel=1e-13)
    _, rep1 = S1.newton(torch.zeros(m.n_dofs, dtype=torch.float64), f_ext=f1, eps_rel=1e-11, cg_tol=1e-12, **calls1)
    assert rep1["converged"] and rep1["newton_iters"] >= 3
    for r in range(world):
        u, rep, uc, repc, (a, b) = out[r]
        for uu, rr in ((u, rep), (uc, repc)):
            assert rr["converged"], rr
            assert np.abs(uu - u_ref[a:b]).max() / np.abs(u_ref).max() < 1e-8
        assert rep["newton_iters"] == rep1["newton_iters"]
        assert repc["cg_iters"] < rep["cg_iters"]  # the Chebyshev preconditioner pays off
