"""Python side of the FP64 CPU oracle (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline /
reference legs may import this module. It never touches the CUDA library and
shares no code with it; both sides read the same seeded inputs from
``paper_2408_12479_gb300.inputs`` (data recipes only) and nothing else.

Contents
--------
* 1D rules: Gauss-Lobatto-Legendre nodal points and Gauss-Legendre
  quadrature on [0, 1] (numpy's Legendre routines serve as library steps).
* Fibre dispersion constants H11, H22, H33 from (a, b) (Sec. 3, bivariate von
  Mises dispersion; scipy's Bessel and error functions as library steps).
* J^(-2/3) by the paper's fixed-count Newton iteration (Alg. 2), in FP64.
* Neumann (traction) load vectors on boundary faces, from the definition.
* ctypes wrappers of hx_oracle.c: residual, tangent apply, diagonal, dense
  element matrices, energy, node coordinates, pointwise material evaluation.
* Plain global algorithms built on those: Dirichlet-constrained operators,
  sparse assembly, the Chebyshev-Jacobi smoother (Chebyshev acceleration as
  in Saad, "Iterative Methods for Sparse Linear Systems", Sec. 12.3, applied
  to D^-1 K), and preconditioned CG (Saad, Alg. 9.1, with the Polak-Ribiere
  beta so an inexact preconditioner is tolerated) -- the paper's Sec. 6
  smoother and outer Krylov solver.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hx_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libhx_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hx_oracle.c with gcc (OpenMP) into oracle/_lib."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Material(C.Structure):
    _fields_ = [("law", C.c_int), ("mu", C.c_double), ("lam", C.c_double), ("kappa", C.c_double),
                ("k1", C.c_double), ("k2", C.c_double), ("Hd", C.c_double * 3), ("phi", C.c_double)]


class _Mesh(C.Structure):
    _fields_ = [("p", C.c_int), ("g", C.c_int), ("n_elem", C.c_int), ("n_nodes", C.c_int64),
                ("geo_nodes", C.c_void_p), ("geo_conn", C.c_void_p), ("dof_conn", C.c_void_p),
                ("frames", C.c_void_p), ("xi_node", C.c_void_p), ("xi_q", C.c_void_p),
                ("w_q", C.c_void_p), ("xi_geo", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            for name in ("orc_residual", "orc_apply", "orc_apply_spatial", "orc_diagonal", "orc_assemble"):
                f = getattr(L, name)
                f.restype = C.c_int
            L.orc_residual.argtypes = [P, P, P, P, P, C.c_int]
            L.orc_apply.argtypes = [P, P, P, P, P, P, C.c_int]
            L.orc_apply_spatial.argtypes = [P, P, P, P, P, P, C.c_int]
            L.orc_diagonal.argtypes = [P, P, P, P, P, C.c_int]
            L.orc_assemble.argtypes = [P, P, P, P, P, C.c_int]
            L.orc_body_force.restype = C.c_int
            L.orc_body_force.argtypes = [P, P, P]
            L.orc_energy.restype = C.c_double
            L.orc_energy.argtypes = [P, P, P]
            L.orc_node_coords.restype = C.c_int
            L.orc_node_coords.argtypes = [P, P]
            L.orc_qp_fields.restype = C.c_int
            L.orc_qp_fields.argtypes = [P, P, P, C.c_int, P, P, P]
            L.orc_material_point.restype = C.c_double
            L.orc_material_point.argtypes = [P, P, P, P, P, P, P, P, P]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# 1D rules and material constants
# ---------------------------------------------------------------------------

def gll_points(p: int) -> np.ndarray:
    """p+1 Gauss-Lobatto-Legendre points on [0, 1]: the end points and the
    roots of P_p'. The nodes of the Lagrange basis; the paper's deal.II
    elements (Sec. 2) do not name them, and these are the reading taken."""
    if p == 1:
        x = np.array([-1.0, 1.0])
    else:
        inner = np.polynomial.legendre.Legendre.basis(p).deriv().roots()
        x = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    return 0.5 * (x + 1.0)


def gauss_rule(nq: int):
    """nq-point Gauss-Legendre points and weights on [0, 1] (weights sum to 1);
    nq = p+1 per direction is the quadrature of the integrals of Sec. 2."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


def equispaced(g: int) -> np.ndarray:
    """Parameter points of a degree-g geometry map (trilinear or triquadratic
    elements with equispaced nodes; the paper's higher-order mapping of Sec. 6
    is the reading for the curved tube)."""
    return np.linspace(0.0, 1.0, g + 1)


def dispersion_H(a: float, b: float):
    """H11, H22, H33 of the generalized structure tensor from the in-plane and
    out-of-plane concentration parameters (a, b) (Sec. 3)."""
    from scipy.special import erf, i0, i1
    H33 = 1.0 / (4.0 * b) - math.exp(-2.0 * b) / (math.sqrt(2.0 * math.pi * b) * erf(math.sqrt(2.0 * b)))
    r = i1(a) / i0(a)
    H11 = 0.5 * (1.0 - H33) * (1.0 + r)
    H22 = 0.5 * (1.0 - H33) * (1.0 - r)
    return float(H11), float(H22), float(H33)


def jpow_newton(J: float, n_steps: int) -> float:
    """J^(-2/3) by the fixed-count Newton iteration of Sec. 4 ("stable and
    fast numerics", Alg. 2): x solves f(x) = x^-3 - J^2 = 0, f'(x) = -3 x^-4,
    starting from x_0 = 1 (the undeformed state) and taking n_steps updates
    x <- x - f(x)/f'(x). Plain FP64 evaluation of the definition; the error
    against the exact power is what the FP32 on-the-fly paths inherit."""
    x = 1.0
    J2 = J * J
    for _ in range(n_steps):
        f = x ** -3 - J2
        df = -3.0 * x ** -4
        x = x - f / df
    return x


@dataclass
class Material:
    law: int            # 0 cNH, 1 iNH, 2 fiber
    mu: float = 1.0
    lam: float = 0.0
    kappa: float = 0.0
    k1: float = 0.0
    k2: float = 0.0
    Hd: tuple = (0.0, 0.0, 0.0)
    phi: float = 0.0

    @classmethod
    def from_dict(cls, d: dict) -> "Material":
        Hd = (0.0, 0.0, 0.0)
        if d.get("law") == 2:
            Hd = dispersion_H(d["a"], d["b"])
        return cls(law=d["law"], mu=d.get("mu", 1.0), lam=d.get("lam", 0.0), kappa=d.get("kappa", 0.0),
                   k1=d.get("k1", 0.0), k2=d.get("k2", 0.0), Hd=Hd, phi=d.get("phi", 0.0))

    def c(self) -> _Material:
        return _Material(self.law, self.mu, self.lam, self.kappa, self.k1, self.k2,
                         (C.c_double * 3)(*self.Hd), self.phi)


def _ptr(a):
    return None if a is None else a.ctypes.data


class OracleMesh:
    """Holds the arrays of a mesh in the layout hx_oracle.c expects."""

    def __init__(self, mesh_input):
        m = mesh_input
        self.src = m
        self.p, self.g = m.p, m.geo_degree
        self.geo_nodes = np.ascontiguousarray(m.geo_nodes, dtype=np.float64)
        self.geo_conn = np.ascontiguousarray(m.geo_conn, dtype=np.int32)
        self.dof_conn = np.ascontiguousarray(m.dof_conn, dtype=np.int32)
        self.frames = None if m.frames is None else np.ascontiguousarray(m.frames, dtype=np.float64)
        self.xi_node = gll_points(m.p)
        self.xi_q, self.w_q = gauss_rule(m.p + 1)
        self.xi_geo = equispaced(m.geo_degree)
        self.n_nodes = int(m.n_nodes)
        self.n_elem = int(self.geo_conn.shape[0])
        self.dirichlet = np.asarray(m.dirichlet, dtype=bool)
        self._c = _Mesh(self.p, self.g, self.n_elem, self.n_nodes, _ptr(self.geo_nodes), _ptr(self.geo_conn),
                        _ptr(self.dof_conn), _ptr(self.frames), _ptr(self.xi_node), _ptr(self.xi_q),
                        _ptr(self.w_q), _ptr(self.xi_geo))

    @property
    def n_dofs(self):
        return 3 * self.n_nodes

    @property
    def nloc(self):
        return 3 * (self.p + 1) ** 3

    def cref(self):
        return C.byref(self._c)


def _vec(x, n):
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    assert x.shape[0] == n, (x.shape, n)
    return x


def _elems(elems):
    if elems is None:
        return None, 0
    e = np.ascontiguousarray(elems, dtype=np.int32)
    return e, int(e.shape[0])


class NonInvertible(RuntimeError):
    pass


def _check(nbad, what):
    if nbad < 0:
        raise MemoryError(what)
    if nbad > 0:
        raise NonInvertible(f"{what}: {nbad} element(s) with J <= 0 or det J0 <= 0")


# ---------------------------------------------------------------------------
# operators (pure operator, no constraints)
# ---------------------------------------------------------------------------

def node_coords(M: OracleMesh) -> np.ndarray:
    """Positions of the DoF nodes: the geometry map at the nodal points (the
    reference configuration of Sec. 2)."""
    X = np.zeros((M.n_nodes, 3))
    if lib().orc_node_coords(M.cref(), X.ctypes.data) != 0:
        raise MemoryError("node_coords")
    return X


def residual(M: OracleMesh, mat: Material, u, elems=None) -> np.ndarray:
    """R(u)_i = (Grad N_i, P(F)) by full quadrature (Sec. 2, Eq.
    mom_bal_nonlinear_material_residual, without loads); P from the laws of
    Sec. 3. elems restricts the sum to those elements."""
    u = _vec(u, M.n_dofs)
    r = np.zeros(M.n_dofs)
    e, ne = _elems(elems)
    mc = mat.c()
    _check(lib().orc_residual(M.cref(), C.byref(mc), u.ctypes.data, r.ctypes.data, _ptr(e), ne), "residual")
    return r


def apply(M: OracleMesh, mat: Material, u, du, elems=None) -> np.ndarray:
    """K(u) du = (Grad N_i, Grad du S + F D_uS[Grad du]) by full quadrature
    (Sec. 2, Eq. DDu_residual_material; D_uS of App. A, readings R3 and R4)."""
    u = _vec(u, M.n_dofs)
    du = _vec(du, M.n_dofs)
    out = np.zeros(M.n_dofs)
    e, ne = _elems(elems)
    mc = mat.c()
    _check(lib().orc_apply(M.cref(), C.byref(mc), u.ctypes.data, du.ctypes.data, out.ctypes.data, _ptr(e), ne),
           "apply")
    return out


def apply_spatial(M: OracleMesh, mat: Material, u, du, elems=None) -> np.ndarray:
    """K(u) du in the spatial form of Sec. 2, Eq. (stress_term_in_Ot_with_JC):
    (grad v, Jc:(grad du)^S + (grad du) tau) with the Sec. 5 spatial tau and
    Jc per law (iNH moduli pushed forward from App. A). Equal to apply() in
    exact arithmetic."""
    u = _vec(u, M.n_dofs)
    du = _vec(du, M.n_dofs)
    out = np.zeros(M.n_dofs)
    e, ne = _elems(elems)
    mc = mat.c()
    _check(lib().orc_apply_spatial(M.cref(), C.byref(mc), u.ctypes.data, du.ctypes.data, out.ctypes.data, _ptr(e),
                                   ne), "apply_spatial")
    return out


def body_force(M: OracleMesh, b) -> np.ndarray:
    """Load vector of a constant body force b (Sec. 2, the (v, B) term)."""
    bb = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(3))
    f = np.zeros(M.n_dofs)
    _check(lib().orc_body_force(M.cref(), bb.ctypes.data, f.ctypes.data), "body_force")
    return f


def lagrange(nodes, x):
    """Values and first derivatives of the Lagrange polynomials on `nodes` at
    the points x, each [len(x), len(nodes)], as plain products (derivative by
    the product rule): the tensor-product basis of Sec. 2 in one direction."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    V = np.ones((x.size, nodes.size))
    D = np.zeros((x.size, nodes.size))
    for a in range(nodes.size):
        for b in range(nodes.size):
            if b != a:
                den = nodes[a] - nodes[b]
                D[:, a] = D[:, a] * (x - nodes[b]) / den + V[:, a] / den
                V[:, a] = V[:, a] * (x - nodes[b]) / den
    return V, D


def traction_load(M: OracleMesh, faces, h):
    """Neumann load vector f_i = (N_i, h_N) over the boundary faces (Sec. 2,
    Eq. mom_bal_nonlinear_material_residual, the Gamma_N term; a dead load on
    the reference configuration).

    faces: [n, 2] pairs (element, local face); local face 2d + s is the face
    xi_d = s of the reference cube (d = 0, 1, 2; s = 0, 1). h(X, N) returns
    the nominal traction [k, 3] at points X [k, 3] with outward unit
    reference normals N [k, 3]. Each face is integrated with the
    (p+1) x (p+1) Gauss rule of the element's volume rule; the area element
    and the normal come from the cross product of the two in-face tangents of
    the geometry map."""
    faces = np.asarray(faces, dtype=np.int64).reshape(-1, 2)
    n = M.p + 1
    mg = M.g + 1
    f = np.zeros(M.n_dofs)
    xq, wq = M.xi_q, M.w_q
    for e, lf in faces:
        d, side = int(lf) // 2, int(lf) % 2
        a, b = [c for c in range(3) if c != d]
        # reference coordinates of the face points, [n*n, 3] (first in-face direction fastest)
        xi = np.zeros((n * n, 3))
        xi[:, d] = float(side)
        xi[:, a] = np.tile(xq, n)
        xi[:, b] = np.repeat(xq, n)
        w = np.tile(wq, n) * np.repeat(wq, n)
        # geometry map X(xi) and its three tangents dX/dxi_c
        Xg = M.geo_nodes[M.geo_conn[e]]              # [(g+1)^3, 3], xi1 fastest
        Vg = [lagrange(M.xi_geo, xi[:, c]) for c in range(3)]
        X = np.zeros((n * n, 3))
        T = np.zeros((3, n * n, 3))
        for k in range(mg):
            for j in range(mg):
                for i in range(mg):
                    node = Xg[i + mg * (j + mg * k)]
                    v = (Vg[0][0][:, i], Vg[1][0][:, j], Vg[2][0][:, k])
                    dv = (Vg[0][1][:, i], Vg[1][1][:, j], Vg[2][1][:, k])
                    X += np.outer(v[0] * v[1] * v[2], node)
                    T[0] += np.outer(dv[0] * v[1] * v[2], node)
                    T[1] += np.outer(v[0] * dv[1] * v[2], node)
                    T[2] += np.outer(v[0] * v[1] * dv[2], node)
        nv = np.cross(T[a], T[b])
        dA = np.linalg.norm(nv, axis=1)
        N = nv / dA[:, None]
        # outward: along +xi_d on the face xi_d = 1, along -xi_d on xi_d = 0
        sgn = np.sign(np.einsum("qi,qi->q", N, T[d])) * (1.0 if side == 1 else -1.0)
        N = N * sgn[:, None]
        hq = np.asarray(h(X, N), dtype=np.float64).reshape(n * n, 3) * (w * dA)[:, None]
        # nodal basis of the displacement space at the face points
        Vp = [lagrange(M.xi_node, xi[:, c])[0] for c in range(3)]
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    psi = Vp[0][:, i] * Vp[1][:, j] * Vp[2][:, k]
                    node = M.dof_conn[e, i + n * (j + n * k)]
                    f[3 * node:3 * node + 3] += psi @ hq
    return f


def diagonal(M: OracleMesh, mat: Material, u, elems=None) -> np.ndarray:
    """diag K(u), the Jacobi scaling of the smoother (Sec. 6), summed from the
    diagonals of the element matrices."""
    u = _vec(u, M.n_dofs)
    d = np.zeros(M.n_dofs)
    e, ne = _elems(elems)
    mc = mat.c()
    _check(lib().orc_diagonal(M.cref(), C.byref(mc), u.ctypes.data, d.ctypes.data, _ptr(e), ne), "diagonal")
    return d


def element_matrices(M: OracleMesh, mat: Material, u, elems=None) -> np.ndarray:
    """Dense element tangent matrices of Sec. 2, Eq. DDu_residual_material
    (one column per unit direction), [n_elem, 3 (p+1)^3, 3 (p+1)^3]."""
    u = _vec(u, M.n_dofs)
    e, ne = _elems(elems)
    n_list = ne if e is not None else M.n_elem
    Ke = np.zeros((n_list, M.nloc, M.nloc))
    mc = mat.c()
    _check(lib().orc_assemble(M.cref(), C.byref(mc), u.ctypes.data, Ke.ctypes.data, _ptr(e), ne), "assemble")
    return Ke


def energy(M: OracleMesh, mat: Material, u) -> float:
    """Stored energy Pi(u) = sum over points of JxW Psi(F) (Sec. 3 laws)."""
    u = _vec(u, M.n_dofs)
    mc = mat.c()
    return float(lib().orc_energy(M.cref(), C.byref(mc), u.ctypes.data))


def qp_fields(M: OracleMesh, u, elems):
    """Quadrature points of the given elements: their positions, weights JxW
    and deformation gradients F = I + Grad u (Sec. 2)."""
    u = _vec(u, M.n_dofs)
    e = np.ascontiguousarray(elems, dtype=np.int32)
    qq = (M.p + 1) ** 3
    JxW = np.zeros((len(e), qq))
    J0 = np.zeros((len(e), qq, 9))
    F = np.zeros((len(e), qq, 9))
    lib().orc_qp_fields(M.cref(), u.ctypes.data, e.ctypes.data, len(e), JxW.ctypes.data, J0.ctypes.data,
                        F.ctypes.data)
    return JxW, J0, F


def material_point(mat: Material, F, H=None, frame=None):
    """Psi, S, P, dP (and fibre auxiliaries) at one deformation gradient:
    the laws of Sec. 3 (Eq. NH_compressible, NH_nearly_incompressible,
    fiber_Psi) and their derivatives of App. A."""
    F = np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(9))
    Hh = None if H is None else np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(9))
    fr = None if frame is None else np.ascontiguousarray(np.asarray(frame, dtype=np.float64).reshape(9))
    psi = C.c_double(0.0)
    S = np.zeros(9)
    P = np.zeros(9)
    dP = np.zeros(9)
    aux = np.zeros(6)
    mc = mat.c()
    J = lib().orc_material_point(C.byref(mc), _ptr(fr), F.ctypes.data, _ptr(Hh), C.byref(psi), S.ctypes.data,
                                 P.ctypes.data, dP.ctypes.data if Hh is not None else None, aux.ctypes.data)
    return dict(J=J, psi=psi.value, S=S.reshape(3, 3), P=P.reshape(3, 3),
                dP=dP.reshape(3, 3) if Hh is not None else None, aux=aux)


def set_threads(n: int):
    lib().orc_set_num_threads(int(n))


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---------------------------------------------------------------------------
# global assembly and constrained operators
# ---------------------------------------------------------------------------

def assemble_sparse(M: OracleMesh, mat: Material, u):
    """Global sparse K(u) (pure operator, no constraints) from the dense
    element matrices (Sec. 2, Eq. DDu_residual_material)."""
    import scipy.sparse as sp
    Ke = element_matrices(M, mat, u)
    nn = (M.p + 1) ** 3
    dofs = (3 * M.dof_conn[:, :, None] + np.arange(3)[None, None, :]).reshape(M.n_elem, 3 * nn)
    rows = np.repeat(dofs, 3 * nn, axis=1).ravel()
    cols = np.tile(dofs, (1, 3 * nn)).ravel()
    return sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(M.n_dofs, M.n_dofs))


def constrain_matrix(K, mask):
    """Replace constrained rows/columns by identity rows (out_c = du_c): the
    Dirichlet part of the boundary conditions of Sec. 2."""
    import scipy.sparse as sp
    free = sp.diags((~mask).astype(np.float64))
    fix = sp.diags(mask.astype(np.float64))
    return (free @ K @ free + fix).tocsr()


def apply_constrained(M: OracleMesh, mat: Material, u, du):
    """K_c du: free rows of K applied to du with constrained entries zeroed;
    constrained rows return du itself (Sec. 2 tangent with Dirichlet rows)."""
    mask = M.dirichlet
    d = np.where(mask, 0.0, _vec(du, M.n_dofs))
    out = apply(M, mat, u, d)
    return np.where(mask, _vec(du, M.n_dofs), out)


def residual_constrained(M: OracleMesh, mat: Material, u):
    """R(u) with the Dirichlet rows set to zero (Sec. 2)."""
    r = residual(M, mat, u)
    r[M.dirichlet] = 0.0
    return r


def diagonal_constrained(M: OracleMesh, mat: Material, u):
    """diag K(u) with the Dirichlet rows set to one (Sec. 2, Sec. 6)."""
    d = diagonal(M, mat, u)
    d[M.dirichlet] = 1.0
    return d


# ---------------------------------------------------------------------------
# Chebyshev-Jacobi smoother and preconditioned CG (Sec. 6)
# ---------------------------------------------------------------------------

def chebyshev_smooth(Kop, rhs, x, inv_diag, degree, lambda_max, smoothing_range, zero_initial=False):
    """The Chebyshev-Jacobi smoother of Sec. 6: Chebyshev acceleration (Saad,
    Sec. 12.3) of the Jacobi iteration on D^-1 K x = D^-1 rhs with eigenvalue interval [lambda_max/smoothing_range, lambda_max]; degree
    steps, each using one residual rhs - K x (the first is rhs itself when x
    starts at zero). Written as the three-term recurrence
        d_0 = r_0 / theta,  rho_0 = delta/theta,
        rho_k = 1/(2 theta/delta - rho_{k-1}),
        d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k/delta) r_k,
        x_{k+1} = x_k + d_k,  r_k = D^-1 (rhs - K x_k)."""
    a = lambda_max / smoothing_range
    b = lambda_max
    theta = 0.5 * (b + a)
    delta = 0.5 * (b - a)
    x = np.array(x, dtype=np.float64, copy=True)
    if zero_initial:
        x[:] = 0.0
    d = None
    rho_prev = None
    for k in range(degree):
        if k == 0 and zero_initial:
            r = inv_diag * rhs
        else:
            r = inv_diag * (rhs - Kop(x))
        if k == 0:
            rho = delta / theta
            d = r / theta
        else:
            rho_new = 1.0 / (2.0 * theta / delta - rho_prev)
            d = rho_new * rho_prev * d + (2.0 * rho_new / delta) * r
            rho = rho_new
        x = x + d
        rho_prev = rho
    return x


def pcg(Kop, b, Mop, tol=1e-8, maxit=10000, x0=None):
    """Preconditioned CG with the Polak-Ribiere beta (the outer Krylov
    solver of Sec. 6; Saad, Alg. 9.1); stops when ||b - K x|| <= tol ||b||
    (recomputed residual checked at exit)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    r = b - Kop(x)
    bn = np.linalg.norm(b)
    z = Mop(r)
    p = z.copy()
    rz = r @ z
    it = 0
    hist = [np.linalg.norm(r) / bn]
    while it < maxit and hist[-1] > tol:
        Ap = Kop(p)
        alpha = rz / (p @ Ap)
        x += alpha * p
        r_new = r - alpha * Ap
        z_new = Mop(r_new)
        beta = (r_new @ (z_new - z)) / rz
        rz = r_new @ z_new
        p = z_new + beta * p
        r, z = r_new, z_new
        it += 1
        hist.append(np.linalg.norm(r) / bn)
    true_rel = np.linalg.norm(b - Kop(x)) / bn
    return x, it, true_rel, hist


def newton(M: OracleMesh, mat: Material, u0, f_ext=None, eps_abs=1e-10, eps_rel=1e-12, max_it=25):
    """Newton's method of Alg. 1 on R(u) - f_ext = 0 over the free DoFs, each
    update from a direct solve with the assembled constrained tangent. u0
    carries the Dirichlet values (Alg. 1: u_0 <- g_D on Gamma_D). Returns
    (u, residual norms per iterate)."""
    import scipy.sparse.linalg as spla
    mask = M.dirichlet
    u = _vec(u0, M.n_dofs).copy()
    f = np.zeros(M.n_dofs) if f_ext is None else _vec(f_ext, M.n_dofs)

    def res(v):
        r = residual(M, mat, v) - f
        r[mask] = 0.0
        return r
    r = res(u)
    norms = [float(np.linalg.norm(r))]
    k = 0
    while norms[-1] > eps_abs and norms[-1] > eps_rel * norms[0] and k < max_it:
        K = constrain_matrix(assemble_sparse(M, mat, u), mask)
        du = spla.spsolve(K.tocsc(), -r)
        du[mask] = 0.0
        u = u + du
        k += 1
        r = res(u)
        norms.append(float(np.linalg.norm(r)))
    return u, norms


def box_transfer_matrix(nx, ny, nz, pc, pf):
    """Dense prolongation of the degree-pc Lagrange space into the degree-pf
    space on a structured box of nx*ny*nz elements (per displacement
    component): P[I, J] = value of the coarse global basis function J at fine
    node I, evaluated in reference coordinates of an element containing the
    node (the element map is shared by both spaces). The p-transfer of the
    multigrid hierarchy of Sec. 6. Plain loops; small boxes."""
    xc, xf = gll_points(pc), gll_points(pf)

    def lag(xs, a, x):
        v = 1.0
        for b in range(len(xs)):
            if b != a:
                v *= (x - xs[b]) / (xs[a] - xs[b])
        return v
    Nf = [n * pf + 1 for n in (nx, ny, nz)]
    Nc = [n * pc + 1 for n in (nx, ny, nz)]
    P = np.zeros((Nf[0] * Nf[1] * Nf[2], Nc[0] * Nc[1] * Nc[2]))
    for K in range(Nf[2]):
        for J in range(Nf[1]):
            for I in range(Nf[0]):
                row = I + Nf[0] * (J + Nf[1] * K)
                loc = []
                for L, n in zip((I, J, K), (nx, ny, nz)):
                    e = min(L // pf, n - 1)
                    loc.append((e, L - e * pf))
                for c in range(pc + 1):
                    for b in range(pc + 1):
                        for a in range(pc + 1):
                            w = lag(xc, a, xf[loc[0][1]]) * lag(xc, b, xf[loc[1][1]]) * lag(xc, c, xf[loc[2][1]])
                            col = (loc[0][0] * pc + a) + Nc[0] * ((loc[1][0] * pc + b) + Nc[1] * (loc[2][0] * pc + c))
                            P[row, col] = w
    return P


def box_h_transfer_matrix(nxc, nyc, nzc):
    """Dense prolongation between the degree-1 spaces of a structured box of
    nxc*nyc*nzc elements (coarse) and the box with every direction split in
    two (fine), per displacement component: P[I, J] = value at fine lattice
    node I of the coarse lattice's piecewise-trilinear hat function J, both
    lattices in the coarse lattice's coordinates (fine node (i, j, k) sits at
    (i/2, j/2, k/2)). This is the h-step of the hp-multigrid hierarchy of
    Sec. 6 (Fehn et al.), the embedding of the coarse space in the fine one
    when the boxes are nested. Plain loops; small boxes."""
    def hat(t, c):
        return max(0.0, 1.0 - abs(t - c))
    Mc = [nxc + 1, nyc + 1, nzc + 1]
    Mf = [2 * nxc + 1, 2 * nyc + 1, 2 * nzc + 1]
    P = np.zeros((Mf[0] * Mf[1] * Mf[2], Mc[0] * Mc[1] * Mc[2]))
    for fk in range(Mf[2]):
        for fj in range(Mf[1]):
            for fi in range(Mf[0]):
                row = fi + Mf[0] * (fj + Mf[1] * fk)
                for ck in range(Mc[2]):
                    for cj in range(Mc[1]):
                        for ci in range(Mc[0]):
                            w = hat(fi / 2.0, ci) * hat(fj / 2.0, cj) * hat(fk / 2.0, ck)
                            if w != 0.0:
                                P[row, ci + Mc[0] * (cj + Mc[1] * ck)] = w
    return P
