"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every oracle function is checked here against something other than itself:
printed values (Tables 1 and 3), closed forms, invariants (objectivity, rigid
motions, patch test, symmetry), finite differences of the energy and of the
residual, and an independently coded linear-elastic stiffness.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2408_12479_gb300 import inputs as I
from tests._util import rel_inf, rotation
from tests import linear_elastic_ref as LE

GOLD = os.path.join(os.path.dirname(__file__), "golden")

CNH = O.Material(law=0, mu=1.0, lam=10.0)
INH = O.Material(law=1, mu=1.0, kappa=50.0)


def fiber_mat(phi_deg=40.0, k1=1.0, k2=10.0, kappa=3084.3 / 62.1):
    return O.Material(law=2, mu=1.0, kappa=kappa, k1=k1, k2=k2, Hd=O.dispersion_H(3.62, 34.3),
                      phi=math.radians(phi_deg))


ALL_LAWS = [("cNH", CNH), ("iNH", INH), ("fiber", fiber_mat())]
FRAME = np.array([0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 1.0, 0.0, 0.0])  # E1=y, E2=z, E3=x


# --------------------------------------------------------------------------
# 1D rules, Table 1 dispersion constants, Table 3 mesh sizes
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nq", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_gauss_exactness(nq):
    x, w = O.gauss_rule(nq)
    for k in range(2 * nq):
        assert abs((w * x ** k).sum() - 1.0 / (k + 1)) < 1e-14
    # degree 2n is integrated with the classical Gauss error on [0, 1]:
    # int x^{2n} - Q(x^{2n}) = (n!)^4 / ((2n+1) ((2n)!)^2)
    k = 2 * nq
    err = 1.0 / (k + 1) - (w * x ** k).sum()
    exact = math.factorial(nq) ** 4 / ((2 * nq + 1) * math.factorial(2 * nq) ** 2)
    assert abs(err - exact) < 1e-15 + 1e-6 * exact


def test_gll_closed_forms():
    for p, ref in LE.GLL_CLOSED_FORM.items():
        assert np.allclose(O.gll_points(p), ref, atol=1e-15, rtol=0)
    x4 = O.gll_points(4)
    assert np.allclose(x4, [0, 0.5 * (1 - math.sqrt(3 / 7)), 0.5, 0.5 * (1 + math.sqrt(3 / 7)), 1], atol=1e-15)
    for p in range(2, 9):
        x = O.gll_points(p)
        assert np.allclose(x + x[::-1], 1.0, atol=1e-14) and np.all(np.diff(x) > 0)


def test_table1_dispersion():
    g = json.load(open(os.path.join(GOLD, "table1_fibre_parameters.json")))
    H = O.dispersion_H(g["a"], g["b"])
    assert round(H[0], 4) == g["H11"] and round(H[1], 4) == g["H22"] and round(H[2], 4) == g["H33"]
    assert abs(sum(H) - 1.0) < 1e-14


def test_table3_dof_counts():
    g = json.load(open(os.path.join(GOLD, "table3_meshes.json")))
    for row in g["rows"]:
        n = row["N0"] * 2 ** row["l"]
        assert n ** 3 == row["N_el"]
        if row["N_el"] <= 200000:
            m = I.box_mesh(n, row["p"])
            assert m.dof_conn.max() + 1 == m.n_nodes
            assert np.unique(m.dof_conn).size == m.n_nodes
            assert round(3 * m.n_nodes / 1e6, 2) == row["MDoFs"]
        else:
            assert round(3 * (n * row["p"] + 1) ** 3 / 1e6, 2) == row["MDoFs"]


# --------------------------------------------------------------------------
# material laws, pointwise
# --------------------------------------------------------------------------

def _rand_F(seed, scale=0.15):
    g = np.random.Generator(np.random.PCG64(seed))
    return np.eye(3) + scale * g.uniform(-1, 1, size=(3, 3))


def _fd_P(mat, F, frame, h=1e-6):
    P = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            P[i, j] = (O.material_point(mat, F + E, frame=frame)["psi"] -
                       O.material_point(mat, F - E, frame=frame)["psi"]) / (2 * h)
    return P


def _stretch_fibres(seed):
    """F stretching along both fibre families (I* > 1 for both) plus noise."""
    F = _rand_F(seed, 0.03)
    F[1, 1] += 0.12
    F[2, 2] += 0.12
    return F


@pytest.mark.parametrize("name,mat", ALL_LAWS)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_P_is_dPsi_dF(name, mat, seed):
    F = _stretch_fibres(seed) if name == "fiber" else _rand_F(seed)
    r = O.material_point(mat, F, frame=FRAME)
    if name == "fiber":
        assert r["aux"][4] == 1 and r["aux"][5] == 1
    assert rel_inf(r["P"], _fd_P(mat, F, FRAME)) < 1e-7
    assert np.allclose(r["S"], r["S"].T, atol=1e-13)
    assert np.allclose(r["P"], F @ r["S"], atol=1e-13)


@pytest.mark.parametrize("name,mat", ALL_LAWS)
@pytest.mark.parametrize("seed", [4, 5])
def test_dP_is_directional_derivative(name, mat, seed):
    F = _stretch_fibres(seed) if name == "fiber" else _rand_F(seed)
    g = np.random.Generator(np.random.PCG64(seed + 100))
    H = g.uniform(-1, 1, size=(3, 3))
    h = 1e-6
    r = O.material_point(mat, F, H=H, frame=FRAME)
    fd = (O.material_point(mat, F + h * H, frame=FRAME)["P"] - O.material_point(mat, F - h * H, frame=FRAME)["P"]) / (2 * h)
    assert rel_inf(r["dP"], fd) < 1e-7
    # major symmetry of dP/dF (hyperelasticity)
    H2 = g.uniform(-1, 1, size=(3, 3))
    a = (H2 * r["dP"]).sum()
    b = (H * O.material_point(mat, F, H=H2, frame=FRAME)["dP"]).sum()
    assert abs(a - b) < 1e-11 * max(1.0, abs(a))


@pytest.mark.parametrize("name,mat", ALL_LAWS)
def test_objectivity(name, mat):
    F = _stretch_fibres(7) if name == "fiber" else _rand_F(7)
    Q = rotation(8)
    g = np.random.Generator(np.random.PCG64(9))
    H = g.uniform(-1, 1, size=(3, 3))
    r = O.material_point(mat, F, H=H, frame=FRAME)
    rq = O.material_point(mat, Q @ F, H=Q @ H, frame=FRAME)
    assert abs(rq["psi"] - r["psi"]) < 1e-13 * max(1, abs(r["psi"]))
    assert rel_inf(rq["P"], Q @ r["P"]) < 1e-12
    assert rel_inf(rq["dP"], Q @ r["dP"]) < 1e-12


@pytest.mark.parametrize("name,mat,lam_lin", [("cNH", CNH, 20.0), ("iNH", INH, 50.0 - 2.0 / 3.0),
                                              ("fiber", fiber_mat(), 3084.3 / 62.1 - 2.0 / 3.0)])
def test_undeformed_state_is_linear_elasticity(name, mat, lam_lin):
    g = np.random.Generator(np.random.PCG64(11))
    H = g.uniform(-1, 1, size=(3, 3))
    r = O.material_point(mat, np.eye(3), H=H, frame=FRAME)
    assert abs(r["psi"]) < 1e-15 and np.abs(r["S"]).max() < 1e-13
    if name == "fiber":
        assert r["aux"][4] == 0 and r["aux"][5] == 0  # I* = 1 is not > 1
    lin = mat.mu * (H + H.T) + lam_lin * np.trace(H) * np.eye(3)
    assert rel_inf(r["dP"], lin) < 1e-13


@pytest.mark.parametrize("name,mat", [("cNH", CNH), ("iNH", INH)])
def test_simple_shear_energy(name, mat):
    gam = 0.3
    F = np.eye(3)
    F[0, 1] = gam
    assert abs(O.material_point(mat, F)["psi"] - 0.5 * mat.mu * gam ** 2) < 1e-14


def test_fibre_uniaxial_closed_form():
    """Isochoric-free check of the fibre part: stretch lam along M1 of family 4
    gives I*_4 = lam^2 and E_4 = (lam^2 - 1) H11 (M1 is orthogonal to M2, M3)."""
    mat = fiber_mat(phi_deg=27.47, k1=1.4, k2=22.1)
    ph = mat.phi
    E1, E2, E3 = FRAME[:3], FRAME[3:6], FRAME[6:]
    M1 = math.cos(ph) * E1 + math.sin(ph) * E2
    lam = 1.07
    F = np.eye(3) + (lam - 1.0) * np.outer(M1, M1)
    r = O.material_point(mat, F, frame=FRAME)
    assert abs(r["aux"][2] - lam ** 2) < 1e-14
    assert abs(r["aux"][0] - (lam ** 2 - 1) * mat.Hd[0]) < 1e-14
    # family 6 (angle -Phi): M1_6 . C M1_6 = 1 + (lam^2-1) cos^2(2 Phi)
    assert abs(r["aux"][3] - (1 + (lam ** 2 - 1) * math.cos(2 * ph) ** 2)) < 1e-13
    # the fibre energy adds k1/(2k2)(exp(k2 E^2) - 1) per active family
    base = O.material_point(O.Material(law=1, mu=mat.mu, kappa=mat.kappa), F)["psi"]
    extra = sum(mat.k1 / (2 * mat.k2) * (math.exp(mat.k2 * E ** 2) - 1) for E in r["aux"][:2])
    assert abs(r["psi"] - base - extra) < 1e-14


def test_fibre_switch_compression():
    """Fibres under compression (I* < 1) carry nothing (Sec. 3, fiber_Psi)."""
    mat = fiber_mat()
    F = np.diag([1.0, 0.93, 0.95])  # shortens E1 (y) and E2 (z)
    r = O.material_point(mat, F, H=np.ones((3, 3)), frame=FRAME)
    base = O.material_point(O.Material(law=1, mu=mat.mu, kappa=mat.kappa), F, H=np.ones((3, 3)))
    assert r["aux"][4] == 0 and r["aux"][5] == 0
    assert np.allclose(r["P"], base["P"], atol=1e-15) and np.allclose(r["dP"], base["dP"], atol=1e-15)


# --------------------------------------------------------------------------
# meshes and geometry
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p", [2, 3])
def test_node_coords_affine_lattice(p):
    m = I.box_mesh(2, p, lengths=(1.0, 0.7, 1.3))
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    x1 = np.asarray(LE.GLL_CLOSED_FORM[p])
    Nx = 2 * p + 1
    lat = np.concatenate([x1[:-1], 1 + x1])  # two elements per direction
    idx = np.arange(m.n_nodes)
    I_, J_, K_ = idx % Nx, (idx // Nx) % Nx, idx // (Nx * Nx)
    ref = np.stack([0.5 * lat[I_], 0.35 * lat[J_], 0.65 * lat[K_]], axis=1)
    assert np.abs(X - ref).max() < 1e-15


def test_volume_jittered_cube_and_tube():
    m = I.box_mesh(4, 3, jitter=0.1, seed=5)
    M = O.OracleMesh(m)
    JxW, J0, F = O.qp_fields(M, np.zeros(m.n_dofs), np.arange(m.n_elem))
    assert abs(JxW.sum() - 1.0) < 1e-14 and JxW.min() > 0
    t = I.tube_mesh(2, n_r=2, n_theta=16, n_z=4)
    Mt = O.OracleMesh(t)
    JxW, J0, F = O.qp_fields(Mt, np.zeros(t.n_dofs), np.arange(t.n_elem))
    exact = math.pi * (1.3 ** 2 - 1.0) * 10.0
    assert abs(JxW.sum() / exact - 1.0) < 2e-4 and JxW.min() > 0


# --------------------------------------------------------------------------
# global operators
# --------------------------------------------------------------------------

def _small(law_name, jitter=0.1, n=2, p=2, seed=3):
    if law_name == "fiber":
        m = I.box_mesh(n, p, jitter=jitter, seed=seed)
        m.frames = np.tile(FRAME, (m.n_elem, 1))
        return m, fiber_mat()
    return I.box_mesh(n, p, jitter=jitter, seed=seed), dict(ALL_LAWS)[law_name]


def _state(M, seed, strain=0.05, fibre=False):
    X = O.node_coords(M)
    f = I.sine_field(seed, strain=strain)
    u = f(X)
    if fibre:  # stretch both fibre families everywhere (|I* - 1| well above 1e-3)
        u += X @ np.diag([0.0, 0.08, 0.08])
    return u.ravel()


@pytest.mark.parametrize("law", ["cNH", "iNH", "fiber"])
def test_residual_zero_and_rigid(law):
    m, mat = _small(law)
    M = O.OracleMesh(m)
    assert np.abs(O.residual(M, mat, np.zeros(m.n_dofs))).max() < 1e-14
    X = O.node_coords(M)
    Q = rotation(21)
    u = (X @ (Q - np.eye(3)).T).ravel()
    r_rot = O.residual(M, mat, u)
    r_def = O.residual(M, mat, _state(M, 22, fibre=law == "fiber"))
    assert np.abs(r_rot).max() < 1e-12 * np.abs(r_def).max()
    assert abs(O.energy(M, mat, u)) < 1e-13


@pytest.mark.parametrize("law", ["cNH", "iNH", "fiber"])
def test_patch_test_homogeneous_deformation(law):
    """Affine u on a jittered mesh gives constant F, so every interior node's
    residual is zero (Gauss rule exact for the trilinear cofactors)."""
    m, mat = _small(law, n=3)
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    A = np.array([[0.04, 0.01, -0.02], [0.0, 0.09, 0.015], [0.01, -0.01, 0.1]])
    r = O.residual(M, mat, (X @ A.T).ravel()).reshape(-1, 3)
    on_bnd = np.any((np.abs(X) < 1e-12) | (np.abs(X - 1) < 1e-12), axis=1)
    assert np.abs(r[~on_bnd]).max() < 1e-13 * np.abs(r[on_bnd]).max()
    assert np.abs(r[on_bnd]).max() > 1e-3


@pytest.mark.parametrize("law", ["cNH", "iNH", "fiber"])
def test_residual_is_energy_gradient(law):
    m, mat = _small(law)
    M = O.OracleMesh(m)
    u = _state(M, 31, fibre=law == "fiber")
    r = O.residual(M, mat, u)
    g = np.random.Generator(np.random.PCG64(32))
    for _ in range(3):
        v = g.uniform(-1, 1, size=m.n_dofs) * 1e-2
        h = 1e-4
        fd = (O.energy(M, mat, u + h * v) - O.energy(M, mat, u - h * v)) / (2 * h)
        assert abs(fd - r @ v) < 1e-7 * abs(r @ v) + 1e-14


@pytest.mark.parametrize("law", ["cNH", "iNH", "fiber"])
def test_tangent_is_residual_derivative_and_symmetric(law):
    m, mat = _small(law)
    M = O.OracleMesh(m)
    u = _state(M, 41, fibre=law == "fiber")
    g = np.random.Generator(np.random.PCG64(42))
    du = g.uniform(-1, 1, size=m.n_dofs)
    h = 1e-6
    fd = (O.residual(M, mat, u + h * du) - O.residual(M, mat, u - h * du)) / (2 * h)
    Kdu = O.apply(M, mat, u, du)
    assert rel_inf(Kdu, fd) < 1e-7
    w = g.uniform(-1, 1, size=m.n_dofs)
    a, b = w @ Kdu, du @ O.apply(M, mat, u, w)
    assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("law", ["cNH", "iNH", "fiber"])
def test_spatial_form_tangent_is_residual_derivative(law):
    """The spatial-configuration tangent (Sec. 2 Eq. stress_term_in_Ot_with_JC
    with the Sec. 5 tau and Jc, iNH moduli pushed forward from App. A) is the
    derivative of the material residual and equals the material-form tangent."""
    m, mat = _small(law)
    M = O.OracleMesh(m)
    u = _state(M, 43, fibre=law == "fiber")
    g = np.random.Generator(np.random.PCG64(44))
    du = g.uniform(-1, 1, size=m.n_dofs)
    h = 1e-6
    fd = (O.residual(M, mat, u + h * du) - O.residual(M, mat, u - h * du)) / (2 * h)
    Ks = O.apply_spatial(M, mat, u, du)
    assert rel_inf(Ks, fd) < 1e-7
    assert rel_inf(Ks, O.apply(M, mat, u, du)) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("name,mat,lam_lin", [("cNH", CNH, 20.0), ("iNH", INH, 50.0 - 2.0 / 3.0)])
def test_tangent_at_rest_is_linear_elastic_stiffness(p, name, mat, lam_lin):
    L = (1.0, 0.7, 1.3)
    m = I.box_mesh(2, p, lengths=L)
    M = O.OracleMesh(m)
    K_lin = LE.global_stiffness(m, L, mat.mu, lam_lin)
    K = O.assemble_sparse(M, mat, np.zeros(m.n_dofs))
    assert abs(K - K_lin).max() < 1e-12 * abs(K_lin).max()
    g = np.random.Generator(np.random.PCG64(51))
    du = g.uniform(-1, 1, size=m.n_dofs)
    assert rel_inf(O.apply(M, mat, np.zeros(m.n_dofs), du), K_lin @ du) < 1e-13
    assert rel_inf(O.diagonal(M, mat, np.zeros(m.n_dofs)), K_lin.diagonal()) < 1e-13


@pytest.mark.parametrize("law", ["cNH", "iNH"])
def test_tangent_after_rigid_rotation(law):
    """K(u_rot) (Q v) = Q (K(0) v) node by node, for u_rot = (Q - I) X."""
    m, mat = _small(law)
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    Q = rotation(61)
    u = (X @ (Q - np.eye(3)).T).ravel()
    g = np.random.Generator(np.random.PCG64(62))
    v = g.uniform(-1, 1, size=(m.n_nodes, 3))
    lhs = O.apply(M, mat, u, (v @ Q.T).ravel()).reshape(-1, 3)
    rhs = O.apply(M, mat, np.zeros(m.n_dofs), v.ravel()).reshape(-1, 3) @ Q.T
    assert rel_inf(lhs, rhs) < 1e-12


@pytest.mark.parametrize("law", ["cNH", "iNH", "fiber"])
def test_assembled_matrix_consistency(law):
    m, mat = _small(law)
    M = O.OracleMesh(m)
    u = _state(M, 71, fibre=law == "fiber")
    K = O.assemble_sparse(M, mat, u)
    g = np.random.Generator(np.random.PCG64(72))
    du = g.uniform(-1, 1, size=m.n_dofs)
    assert rel_inf(K @ du, O.apply(M, mat, u, du)) < 1e-13
    assert abs(K - K.T).max() < 1e-12 * abs(K).max()
    assert rel_inf(O.diagonal(M, mat, u), K.diagonal()) < 1e-13


def test_element_subset_matches_full():
    m, mat = _small("cNH", n=3)
    M = O.OracleMesh(m)
    u = _state(M, 81)
    full = O.residual(M, mat, u)
    node = m.dof_conn[13, 13]  # interior node of the centre element
    adj = np.where((m.dof_conn == node).any(axis=1))[0]
    part = O.residual(M, mat, u, elems=adj)
    assert np.array_equal(part[3 * node:3 * node + 3], full[3 * node:3 * node + 3]) or \
        rel_inf(part[3 * node:3 * node + 3], full[3 * node:3 * node + 3]) < 1e-15


# --------------------------------------------------------------------------
# smoother and solver
# --------------------------------------------------------------------------

def test_chebyshev_closed_form_on_diagonal_operator():
    """On K = diag(l_i), D = I, x0 = 0, the Chebyshev iteration leaves the error
    e_k = T_k((theta - K)/delta) / T_k(theta/delta) e_0 with e_0 = -K^-1 b."""
    g = np.random.Generator(np.random.PCG64(91))
    lam = g.uniform(0.05, 1.0, size=50)
    b = g.uniform(-1, 1, size=50)
    lmax, rng_ = 1.0, 20.0
    a = lmax / rng_
    theta, delta = 0.5 * (lmax + a), 0.5 * (lmax - a)
    for k in range(1, 8):
        x = O.chebyshev_smooth(lambda v: lam * v, b, np.zeros(50), np.ones(50), k, lmax, rng_, zero_initial=True)
        Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
        ek = Tk((theta - lam) / delta) / Tk(theta / delta) * (-b / lam)
        assert np.abs((x - b / lam) - ek).max() < 1e-12
    # a nonzero start gives the same error polynomial acting on x0 - x*
    x0 = g.uniform(-1, 1, size=50)
    x = O.chebyshev_smooth(lambda v: lam * v, b, x0, np.ones(50), 4, lmax, rng_)
    T4 = np.polynomial.chebyshev.Chebyshev.basis(4)
    assert np.abs((x - b / lam) - T4((theta - lam) / delta) / T4(theta / delta) * (x0 - b / lam)).max() < 1e-12


def test_pcg_solves_constrained_system():
    import scipy.sparse.linalg as spla
    m = I.box_mesh(3, 2, jitter=0.1, seed=4, clamp=True)
    M = O.OracleMesh(m)
    u = _state(M, 95, strain=0.03)
    u[M.dirichlet] = 0.0
    K = O.constrain_matrix(O.assemble_sparse(M, CNH, u), M.dirichlet)
    b = -O.residual_constrained(M, CNH, u)
    dinv = 1.0 / O.diagonal_constrained(M, CNH, u)
    Kop = lambda v: O.apply_constrained(M, CNH, u, v)
    lmax = np.abs(np.linalg.eigvals(K.toarray() * dinv[:, None])).max()
    Mop = lambda r: O.chebyshev_smooth(Kop, r, np.zeros_like(r), dinv, 3, 1.1 * lmax, 15.0, zero_initial=True)
    x, it, rel, hist = O.pcg(Kop, b, Mop, tol=1e-10)
    xs = spla.spsolve(K.tocsc(), b)
    assert rel < 1e-10 and rel_inf(x, xs) < 1e-8
    assert np.all(x[M.dirichlet] == 0.0) or np.abs(x[M.dirichlet]).max() < 1e-14


# --------------------------------------------------------------------------
# external loads and Newton's method (Alg. 1)
# --------------------------------------------------------------------------

def test_body_force_partition_of_unity_and_first_moment():
    """sum_j f_j = b |Omega| (the basis sums to one) and sum_j X_j f_j =
    b int X dV (linear fields are reproduced), on a jittered box."""
    m = I.box_mesh(3, 2, jitter=0.1, seed=9, lengths=(1.0, 0.7, 1.3))
    M = O.OracleMesh(m)
    b = np.array([0.3, -0.2, 0.5])
    f = O.body_force(M, b).reshape(-1, 3)
    vol = 1.0 * 0.7 * 1.3   # the jitter moves interior vertices only
    assert np.abs(f.sum(axis=0) - b * vol).max() < 1e-13
    X = O.node_coords(M)
    centroid = np.array([0.5, 0.35, 0.65])
    assert np.abs(X.reshape(-1, 3).T @ f - np.outer(centroid * vol, b)).max() < 1e-12


def _lateral_stretch(law, mat, l1):
    """Lateral stretch of homogeneous uniaxial tension with free lateral
    faces: S_22 = 0 with F = diag(l1, l2, l2) (Sec. 3 stresses, C^-1_22 = 1/l2^2)."""
    from scipy.optimize import brentq

    def s22(l2):
        J = l1 * l2 * l2
        if law == "cNH":
            return mat.mu - (mat.mu - 2.0 * mat.lam * np.log(J)) / l2 ** 2
        j = J ** (-2.0 / 3.0)
        I1 = l1 ** 2 + 2 * l2 ** 2
        c1 = 0.5 * mat.kappa * (J * J - 1.0) - mat.mu / 3.0 * j * I1
        return mat.mu * j + c1 / l2 ** 2
    return brentq(s22, 0.5, 1.5)


@pytest.mark.parametrize("law,mat", [("cNH", CNH), ("iNH", INH)])
def test_newton_uniaxial_matches_homogeneous_closed_form(law, mat):
    l1 = 1.2
    m, u0 = I.workload_uniaxial(2, 2, l1)
    M = O.OracleMesh(m)
    u, norms = O.newton(M, mat, u0)
    assert norms[-1] < 1e-10 and len(norms) < 12
    # quadratic convergence once close
    tail = [b / a ** 2 for a, b in zip(norms[:-1], norms[1:]) if a < 1e-2 and b > 1e-12]  # above round-off
    assert all(t < 1e3 for t in tail)
    l2 = _lateral_stretch(law, mat, l1)
    X = O.node_coords(M).reshape(-1, 3)
    exact = X * (np.array([l1, l2, l2]) - 1.0)
    assert np.abs(u.reshape(-1, 3) - exact).max() < 1e-10


@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 4), (3, 6), (2, 5)])
def test_transfer_matrix_reproduces_coarse_polynomials(pc, pf):
    """Prolongation is exact on the coarse space: a tensor polynomial of
    degree pc per coordinate sampled at the coarse nodes maps to its samples
    at the fine nodes (unit box, reference = physical up to scaling)."""
    nx, ny, nz = 2, 1, 2
    P = O.box_transfer_matrix(nx, ny, nz, pc, pf)

    def lattice(p):
        x = np.concatenate([[0.0], *[(e + O.gll_points(p)[1:]) / nx for e in range(nx)]])
        y = np.concatenate([[0.0], *[(e + O.gll_points(p)[1:]) / ny for e in range(ny)]])
        z = np.concatenate([[0.0], *[(e + O.gll_points(p)[1:]) / nz for e in range(nz)]])
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X.ravel(), Y.ravel(), Z.ravel()
    f = lambda X, Y, Z: (1 + X ** pc - 0.5 * X) * (0.3 + Y ** pc) * (Z ** pc - 2 * Z + 0.7)
    vc = f(*lattice(pc))
    vf = f(*lattice(pf))
    assert np.abs(P @ vc - vf).max() < 1e-12
    # rows sum to one (partition of unity)
    assert np.abs(P.sum(axis=1) - 1.0).max() < 1e-13


@pytest.mark.parametrize("J", [0.8, 0.9, 0.95, 1.05, 1.1, 1.2])
def test_jpow_newton_converges_quadratically_to_the_power(J):
    """Alg. 2 (Sec. 4): Newton on x^-3 = J^2 from x = 1 reaches J^(-2/3)
    (closed form by the library cube root) and its error squares each step
    with Newton's constant |f''/(2 f')| = 2/x at the root."""
    exact = 1.0 / np.cbrt(J) ** 2
    errs = [abs(O.jpow_newton(J, n) - exact) for n in range(0, 7)]
    assert errs[6] <= 4e-16 * exact
    for k in range(len(errs) - 1):
        if errs[k] > 1e-6:  # above rounding: the quadratic model holds
            ratio = errs[k + 1] / errs[k] ** 2
            assert abs(ratio / (2.0 / exact) - 1.0) < 0.25 + 3.0 * errs[k], (k, ratio)


def test_jpow_newton_exact_at_rest():
    for n in range(0, 5):
        assert O.jpow_newton(1.0, n) == 1.0


def test_traction_partition_of_unity_and_first_moment():
    """On the planar unit face x = 1 of a jittered cube (boundary vertices are
    not jittered): sum_i f_i = t * area and sum_i f_i y_i = t * int y dA."""
    n, p = 3, 3
    m = I.box_mesh(n, p, jitter=0.1, seed=9)
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    t = np.array([0.3, -1.2, 0.7])
    f = O.traction_load(M, I.box_boundary_faces(n, n, n, 1), lambda Xq, Nq: np.tile(t, (len(Xq), 1)))
    F = f.reshape(-1, 3)
    assert np.allclose(F.sum(axis=0), t, rtol=0, atol=1e-14)
    assert np.allclose((F * X[:, 1:2]).sum(axis=0), 0.5 * t, rtol=0, atol=1e-14)
    # only nodes on the face carry load
    assert np.abs(F[np.abs(X[:, 0] - 1.0) > 1e-12]).max() == 0.0


def _boundary_faces_all(m):
    if m.box is not None:
        return np.concatenate([I.box_boundary_faces(*m.box, s) for s in range(6)])
    e = m.extra
    return np.concatenate([I.tube_boundary_faces(e["n_r"], e["n_theta"], e["n_z"], w)
                           for w in ("inner", "outer", "bottom", "top")])


@pytest.mark.parametrize("case", ["cube_p2", "cube_p3", "tube_p3"])
def test_traction_divergence_theorem_against_residual(case):
    """A homogeneous state (u = A X, constant P): the residual equals the
    traction load of h = P N over the whole boundary, the divergence theorem
    applied to each basis function (both quadratures are exact here)."""
    if case.startswith("cube"):
        m = I.box_mesh(3, int(case[-1]), jitter=0.1, seed=11)
    else:
        m = I.tube_mesh(3, n_r=2, n_theta=8, n_z=2)
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    A = 0.04 * np.random.Generator(np.random.PCG64(12)).uniform(-1, 1, (3, 3))
    u = (X @ A.T).ravel()
    mat = CNH
    P = O.material_point(mat, np.eye(3) + A)["P"]
    R = O.residual(M, mat, u)
    f = O.traction_load(M, _boundary_faces_all(m), lambda Xq, Nq: Nq @ P.T)
    # interior rows of R are sums of cancelling element contributions: round-off
    # there is ~1e-12 of max |R| on the curved tube; a wrong normal, sign or area
    # element would be of order one
    assert np.abs(R - f).max() / np.abs(R).max() < 1e-11


def test_pressure_on_a_closed_surface_has_no_resultant():
    """h = -p N over the tube's whole boundary: the resultant is -p times the
    integral of N over a closed surface, i.e. zero; over the inner surface
    alone the axial component vanishes (the normals are radial)."""
    m = I.tube_mesh(3, n_r=2, n_theta=8, n_z=2)
    M = O.OracleMesh(m)
    press = lambda Xq, Nq: -2.5 * Nq
    f = O.traction_load(M, _boundary_faces_all(m), press).reshape(-1, 3)
    inner = O.traction_load(M, I.tube_boundary_faces(2, 8, 2, "inner"), press).reshape(-1, 3)
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * np.abs(f).sum()
    assert abs(inner.sum(axis=0)[2]) < 1e-13 * np.abs(inner).sum()


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 3), (2, 2, 2)])
def test_h_transfer_reproduces_coarse_trilinear_functions(dims):
    """The h-prolongation is exact on the coarse degree-1 space: on an
    unjittered box (nested levels) a trilinear function sampled at the coarse
    vertices maps to its samples at the fine vertices, each fine vertex's
    value being the coarse trilinear interpolant there, computed here through
    the coarse element that contains it (physical coordinates, an independent
    route); rows sum to one."""
    nxc, nyc, nzc = dims
    P = O.box_h_transfer_matrix(nxc, nyc, nzc)

    def lattice(nx, ny, nz):
        x, y, z = np.linspace(0, 1, nx + 1), np.linspace(0, 2, ny + 1), np.linspace(0, 0.5, nz + 1)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X.ravel(), Y.ravel(), Z.ravel()
    f = lambda X, Y, Z: (1.0 + 0.7 * X) * (2.0 - Y) * (0.3 + Z) + 0.2 * X * Z
    assert np.abs(P @ f(*lattice(nxc, nyc, nzc)) - f(*lattice(2 * nxc, 2 * nyc, 2 * nzc))).max() < 1e-13
    assert np.abs(P.sum(axis=1) - 1.0).max() < 1e-14
    # a function that is not trilinear on the coarse cells is not reproduced
    g = lambda X, Y, Z: X ** 2 + Y * Z
    if nxc >= 1:
        assert np.abs(P @ g(*lattice(nxc, nyc, nzc)) - g(*lattice(2 * nxc, 2 * nyc, 2 * nzc))).max() > 1e-3
    # the coarse trilinear interpolant at each fine vertex, from the coarse
    # cell that contains it: a second construction of every row of P
    Xf, Yf, Zf = lattice(2 * nxc, 2 * nyc, 2 * nzc)
    h = np.array([1.0 / nxc, 2.0 / nyc, 0.5 / nzc])
    Mc = np.array([nxc + 1, nyc + 1, nzc + 1])
    for row, pt in enumerate(zip(Xf, Yf, Zf)):
        cell = np.minimum((np.array(pt) / h + 1e-12).astype(int), Mc - 2)
        t = np.array(pt) / h - cell
        ref = np.zeros(P.shape[1])
        for c in range(8):
            b = np.array([c & 1, (c >> 1) & 1, c >> 2])
            w = np.prod(np.where(b == 1, t, 1.0 - t))
            J = cell + b
            ref[J[0] + Mc[0] * (J[1] + Mc[1] * J[2])] += w
        assert np.abs(P[row] - ref).max() < 1e-13
