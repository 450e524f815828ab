"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs. Tolerances (relative, max-norm against the oracle's
max entry): 1e-12 in FP64 and 1e-5 in FP32. FP32 runs feed the oracle the
FP32-rounded direction so that only arithmetic differences are measured."""
import math

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
STORAGES = [hx.HX_RECOMPUTE, hx.HX_CACHE_F, hx.HX_CACHE_TENSORS, hx.HX_SPATIAL_TENSORS]


def cuda(x, prec=hx.HX_FP64):
    return torch.tensor(np.asarray(x), dtype=DT[prec], device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hx.lib()


# --------------------------------------------------------------------------
# small meshes: every degree, law, storage strategy and precision
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("law", cases.LAWS)
@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_tangent_apply_matches_oracle(p, law, storage, prec):
    """Every apply variant: three tile shapes, with per-thread loads or with
    the tile's fields staged in shared memory by bulk copies (a staged variant
    may be unavailable where its chunks would be misaligned or too large)."""
    n = 3 if p >= 4 else 4   # 27 or 64 elements: several CTA tiles plus a ragged tail
    m = cases.small_cube(n, p, law, seed=10 + p)
    M, X, u = cases.state_for(m, law, seed=20 + p)
    mat = cases.oracle_material(law)
    if law == "fiber":
        assert cases.fibre_switch_margin(M, mat, u) > 1e-3
    du = I.random_direction(m.n_dofs, 30 + p)
    G = hx.Mesh(m, cases.MATS[law])
    try:
        G.precompute(cuda(u), prec, storage)
        du_t = cuda(du, prec)
        ref = O.apply(M, mat, u, host(du_t))
        ran = []
        for variant in range(6):
            hx.hx_set_apply_variant(G.ctx, G.handle, prec, storage, variant)
            try:
                out = G.apply(du_t)
            except hx.HxError as e:
                assert variant >= 2 and e.status == hx.HX_ERR_CUDA, (variant, str(e))
                continue
            G.sync(60000)
            err = rel_inf(host(out), ref)
            assert err < TOL[prec], (variant, err)
            ran.append(variant)
        assert 0 in ran and 1 in ran
        if prec == hx.HX_FP32 and p <= 4:
            assert any(v >= 3 for v in ran), ran
    finally:
        G.close()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("law", cases.LAWS)
@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_residual_matches_oracle(p, law, prec):
    n = 3 if p >= 4 else 4
    m = cases.small_cube(n, p, law, seed=40 + p)
    M, X, u = cases.state_for(m, law, seed=50 + p)
    mat = cases.oracle_material(law)
    G = hx.Mesh(m, cases.MATS[law])
    try:
        u_t = cuda(u, prec)
        r = G.residual(u_t)
        G.sync(60000)
        ref = O.residual(M, mat, host(u_t))
        assert rel_inf(host(r), ref) < TOL[prec]
    finally:
        G.close()


@pytest.mark.parametrize("p", [1, 2, 4, 6])
@pytest.mark.parametrize("law", cases.LAWS)
@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_diagonal_matches_oracle(p, law, storage, prec):
    m = cases.small_cube(2, p, law, seed=60 + p)
    M, X, u = cases.state_for(m, law, seed=70 + p)
    mat = cases.oracle_material(law)
    G = hx.Mesh(m, cases.MATS[law])
    try:
        G.precompute(cuda(u), prec, storage)
        d = G.diagonal(prec)
        G.sync(60000)
        ref = O.diagonal(M, mat, u)
        assert rel_inf(host(d), ref) < TOL[prec]
    finally:
        G.close()


# --------------------------------------------------------------------------
# the 4^3 affine Q2 cube with the x = 0 face clamped (~1.9k free DoFs)
# --------------------------------------------------------------------------

def test_small_affine_cube_constrained():
    m, field, seed = I.workload_small_cube()
    assert int((m.dirichlet == 0).sum()) == 1944
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    u = field(X).ravel()
    u[M.dirichlet] = 0.0
    du = I.random_direction(m.n_dofs, seed + 1)
    mat = cases.oracle_material("cNH")
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        for storage in STORAGES:
            G.precompute(cuda(u), hx.HX_FP64, storage)
            out = G.apply(cuda(du))
            ref = O.apply_constrained(M, mat, u, du)
            assert rel_inf(host(out), ref) < 1e-12
        r = G.residual(cuda(u))
        assert rel_inf(host(r), O.residual_constrained(M, mat, u)) < 1e-12
        d = G.diagonal()
        assert rel_inf(host(d), O.diagonal_constrained(M, mat, u)) < 1e-12
        G.sync(60000)
    finally:
        G.close()


# --------------------------------------------------------------------------
# connectivity path, node coordinates, tube with a quadratic geometry
# --------------------------------------------------------------------------

def test_structured_and_connectivity_paths_agree():
    m = cases.small_cube(4, 3, "iNH", seed=81)
    M, X, u = cases.state_for(m, "iNH", seed=82)
    du = cuda(I.random_direction(m.n_dofs, 83))
    A = hx.Mesh(m, cases.MATS["iNH"], structured=True)
    B = hx.Mesh(m, cases.MATS["iNH"], structured=False)
    try:
        for G in (A, B):
            G.precompute(cuda(u), hx.HX_FP64, hx.HX_CACHE_F)
        a, b = host(A.apply(du)), host(B.apply(du))
        assert rel_inf(a, b) < 1e-14
        assert np.abs(host(A.node_coords()) - X).max() < 1e-14
        assert np.abs(host(B.node_coords()) - X).max() < 1e-14
    finally:
        A.close()
        B.close()


@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
def test_tube_fiber_quadratic_geometry(prec):
    m = I.tube_mesh(3, n_r=2, n_theta=16, n_z=4)
    mat_d = dict(I.MAT_FIBER)
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    u = I.inflation_field(91)(X).ravel()
    du = I.random_direction(m.n_dofs, 92)
    mat = cases.oracle_material(mat_d)
    G = hx.Mesh(m, mat_d)
    try:
        assert np.abs(host(G.node_coords()) - X).max() < 1e-13
        for storage in STORAGES:
            G.precompute(cuda(u), prec, storage)
            du_t = cuda(du, prec)
            out = G.apply(du_t)
            ref = O.apply(M, mat, u, host(du_t))
            assert rel_inf(host(out), ref) < TOL[prec]
        G.sync(60000)
    finally:
        G.close()


# --------------------------------------------------------------------------
# full-size 32^3 jittered cube: sampled outputs against the oracle
# --------------------------------------------------------------------------

def _adjacent_elements(conn, nodes):
    return np.where(np.isin(conn, nodes).any(axis=1))[0].astype(np.int32)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_full_size_cube_sampled(p):
    m, field, seed = I.workload_jittered_cube(p)
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    u = field(X).ravel()
    du = I.random_direction(m.n_dofs, seed + 3)
    mat = cases.oracle_material("cNH")
    g = np.random.Generator(np.random.PCG64(seed + 5))
    # random nodes plus the 8 corners and a few face nodes: interior residuals
    # are small cancelled sums, so the max-norm scale must include boundary rows
    Np = 32 * p + 1
    corners = [i + Np * (j + Np * k) for i in (0, Np - 1) for j in (0, Np - 1) for k in (0, Np - 1)]
    faces = [Np // 2 + Np * (Np // 3), 7 + Np * Np * (Np // 2), Np - 1 + Np * (5 + Np * 9)]
    nodes = np.unique(np.concatenate([g.choice(m.n_nodes, size=48, replace=False), corners, faces]))
    elems = _adjacent_elements(m.dof_conn, nodes)
    dofs = (3 * nodes[:, None] + np.arange(3)).ravel()
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        for prec in (hx.HX_FP64, hx.HX_FP32):
            G.precompute(cuda(u), prec, hx.HX_CACHE_F)
            du_t = cuda(du, prec)
            out = host(G.apply(du_t))
            ref = O.apply(M, mat, u, host(du_t), elems=elems)
            scale = np.abs(ref[dofs]).max()
            assert np.abs(out[dofs] - ref[dofs]).max() / scale < TOL[prec]
        r = host(G.residual(cuda(u)))
        ref = O.residual(M, mat, u, elems=elems)
        assert np.abs(r[dofs] - ref[dofs]).max() / np.abs(ref[dofs]).max() < 1e-12
        G.sync(120000)
    finally:
        G.close()


# --------------------------------------------------------------------------
# Chebyshev-Jacobi smoother
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [hx.HX_FP64, hx.HX_FP32])
@pytest.mark.parametrize("zero_initial", [True, False])
def test_chebyshev_matches_oracle(prec, zero_initial):
    m = cases.small_cube(3, 3, "iNH", seed=101, clamp=True)
    M, X, u = cases.state_for(m, "iNH", seed=102, strain=0.03)
    u[M.dirichlet] = 0.0
    mat = cases.oracle_material("iNH")
    G = hx.Mesh(m, cases.MATS["iNH"])
    try:
        G.precompute(cuda(u), prec, hx.HX_CACHE_TENSORS)
        dinv = 1.0 / O.diagonal_constrained(M, mat, u)
        rhs = I.random_direction(m.n_dofs, 103)
        rhs[M.dirichlet] = 0.0
        x0 = np.zeros(m.n_dofs) if zero_initial else 0.1 * I.random_direction(m.n_dofs, 104)
        x0[M.dirichlet] = 0.0
        rhs_t, dinv_t, x_t = cuda(rhs, prec), cuda(dinv, prec), cuda(x0, prec)
        lmax, rng = 2.0, 15.0
        hx.hx_chebyshev_smooth(G.ctx, G.handle, rhs_t, x_t, dinv_t, 5, lmax, rng, zero_initial)
        G.sync(60000)
        Kop = lambda v: O.apply_constrained(M, mat, u, v)
        ref = O.chebyshev_smooth(Kop, host(rhs_t), host(cuda(x0, prec)), host(dinv_t), 5, lmax, rng,
                                 zero_initial=zero_initial)
        assert rel_inf(host(x_t), ref) < TOL[prec]
    finally:
        G.close()


# --------------------------------------------------------------------------
# error paths
# --------------------------------------------------------------------------

def test_not_ready_and_noninvertible_statuses():
    m = cases.small_cube(2, 2, "cNH", seed=111)
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        du = G.zeros()
        with pytest.raises(hx.HxError) as e:
            G.apply(du)
        assert e.value.status == hx.HX_ERR_NOT_READY
        X = host(G.node_coords())
        u_bad = cuda((-1.5 * X).ravel())  # F = -0.5 I: J < 0
        G.precompute(u_bad, hx.HX_FP64, hx.HX_CACHE_F)
        with pytest.raises(hx.HxError) as e:
            G.sync(60000)
        assert e.value.status == hx.HX_ERR_NONINVERTIBLE
        G.sync(60000)  # flag cleared once reported
        u_nan = cuda(np.full(m.n_dofs, np.nan))
        G.residual(u_nan)
        with pytest.raises(hx.HxError) as e:
            G.sync(60000)
        assert e.value.status == hx.HX_ERR_NAN
    finally:
        G.close()


def test_empty_mesh_gives_zero():
    m = cases.small_cube(1, 2, "cNH")
    m.geo_conn = m.geo_conn[:0]
    m.dof_conn = m.dof_conn[:0]
    m.box = None
    G = hx.Mesh(m, cases.MATS["cNH"], structured=False)
    try:
        u = G.zeros()
        G.precompute(u, hx.HX_FP64, hx.HX_CACHE_TENSORS)
        out = G.apply(torch.ones_like(u))
        assert torch.count_nonzero(out).item() == 0
        G.sync(60000)
    finally:
        G.close()


def test_autotune_keeps_results():
    """Every tile shape the autotuner may pick computes the same operator."""
    m = cases.small_cube(5, 4, "cNH", seed=121)
    M, X, u = cases.state_for(m, "cNH", seed=122)
    du = cuda(I.random_direction(m.n_dofs, 123), hx.HX_FP32)
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        G.precompute(cuda(u), hx.HX_FP32, hx.HX_CACHE_F)
        out = torch.empty_like(du)
        best, times = hx.hx_autotune(G.ctx, G.handle, du, out, reps=2)
        assert best in range(6) and times[best] > 0
        res = host(G.apply(du))
        ref = O.apply(M, cases.oracle_material("cNH"), u, host(du))
        assert rel_inf(res, ref) < 1e-5
    finally:
        G.close()


def test_full_size_headline_configuration_sampled():
    """The benchmark's timed configuration at its full size: 32^3 jittered
    cube, p = 4, FP32, spatial-tensors cache, the variant the autotuner keeps
    and then every variant that launches (staged ones included), checked on
    sampled DoFs (random nodes, corners, face nodes) against the oracle."""
    p = 4
    m, field, seed = I.workload_jittered_cube(p)
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    u = field(X).ravel()
    du = I.random_direction(m.n_dofs, seed + 3)
    mat = cases.oracle_material("cNH")
    g = np.random.Generator(np.random.PCG64(seed + 7))
    Np = 32 * p + 1
    corners = [i + Np * (j + Np * k) for i in (0, Np - 1) for j in (0, Np - 1) for k in (0, Np - 1)]
    faces = [Np // 2 + Np * (Np // 3), 7 + Np * Np * (Np // 2), Np - 1 + Np * (5 + Np * 9)]
    nodes = np.unique(np.concatenate([g.choice(m.n_nodes, size=64, replace=False), corners, faces]))
    elems = _adjacent_elements(m.dof_conn, nodes)
    dofs = (3 * nodes[:, None] + np.arange(3)).ravel()
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        G.precompute(cuda(u), hx.HX_FP32, hx.HX_SPATIAL_TENSORS)
        du_t = cuda(du, hx.HX_FP32)
        out = torch.empty_like(du_t)
        best, times = hx.hx_autotune(G.ctx, G.handle, du_t, out, reps=2)
        assert best in range(6) and times[best] > 0
        ref = O.apply(M, mat, u, host(du_t), elems=elems)
        scale = np.abs(ref[dofs]).max()
        res = host(G.apply(du_t))
        G.sync(120000)
        assert np.abs(res[dofs] - ref[dofs]).max() / scale < TOL[hx.HX_FP32], best
        ran = []
        for variant in range(6):
            hx.hx_set_apply_variant(G.ctx, G.handle, hx.HX_FP32, hx.HX_SPATIAL_TENSORS, variant)
            try:
                res = host(G.apply(du_t))
            except hx.HxError as e:
                assert variant >= 2 and e.status == hx.HX_ERR_CUDA, (variant, str(e))
                continue
            G.sync(120000)
            assert np.abs(res[dofs] - ref[dofs]).max() / scale < TOL[hx.HX_FP32], variant
            ran.append(variant)
        assert 0 in ran and any(v >= 3 for v in ran), ran
    finally:
        G.close()
