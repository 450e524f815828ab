"""Seeded synthetic inputs: meshes, displacement states and directions.

This module is shared by the CUDA path's tests/benchmarks and by the CPU oracle's
tests. It holds only input recipes (vertex lattices, jitter, connectivity,
analytic displacement fields, random vectors) and none of the finite-element
method's arithmetic: no basis functions, no quadrature, no geometry map, no
material law. Whatever consumes these arrays interprets them with its own code.

Conventions shared by every consumer (they describe the data, not the method):

* Reference element axes (xi1, xi2, xi3); local node/vertex numbering inside an
  element is lexicographic with xi1 fastest: local index a + m*(b + m*c) for
  m nodes per direction.
* DoF vectors are node-major AoS: value of component c at node I sits at
  3*I + c.
* Box meshes: element (ex, ey, ez) has index ex + nx*(ey + ny*ez); the degree-p
  node lattice has (nx*p+1) x (ny*p+1) x (nz*p+1) nodes numbered
  I + Nx*(J + Ny*K).
* Tube meshes: reference axes are (radial, circumferential, axial); the
  circumferential direction is periodic (no duplicated seam nodes).

Workload shapes follow the paper's synthetic cubes (Sec. 7.2, Table 3) and the
five workload descriptions of this project (small affine cube, jittered 32^3
cube, 48^3 compressed cube, fibre-reinforced tube, batch of cubes).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2408_12479


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class MeshInput:
    """Host-side description of a hexahedral mesh (geometry + DoF topology)."""

    p: int                      # FE degree of the displacement space
    geo_degree: int             # 1 = trilinear vertices, 2 = triquadratic nodes
    geo_nodes: np.ndarray       # (n_geo, 3) float64
    geo_conn: np.ndarray        # (n_elem, (g+1)^3) int32, lexicographic
    dof_conn: np.ndarray        # (n_elem, (p+1)^3) int32, lexicographic
    n_nodes: int                # number of DoF nodes (3 DoFs each)
    dirichlet: np.ndarray       # (3*n_nodes,) uint8, 1 = constrained
    box: tuple | None = None    # (nx, ny, nz) for structured boxes, else None
    frames: np.ndarray | None = None  # (n_elem, 9) fibre frames E1,E2,E3 or None
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return int(self.geo_conn.shape[0])

    @property
    def n_dofs(self) -> int:
        return 3 * self.n_nodes


# --------------------------------------------------------------------------
# box meshes
# --------------------------------------------------------------------------

def box_vertices(nx, ny, nz, lengths=(1.0, 1.0, 1.0), jitter=0.0, seed=0):
    """Vertex lattice of an nx*ny*nz box; interior vertices jittered by
    U[-jitter*h, jitter*h] per coordinate (boundary vertices stay on the
    planar faces)."""
    Lx, Ly, Lz = lengths
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    zs = np.linspace(0.0, Lz, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if jitter > 0.0:
        g = rng(seed)
        h = np.array([Lx / nx, Ly / ny, Lz / nz])
        K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1),
                              np.arange(nx + 1), indexing="ij")
        interior = ((I > 0) & (I < nx) & (J > 0) & (J < ny) & (K > 0) & (K < nz)).ravel()
        d = g.uniform(-1.0, 1.0, size=V.shape) * (jitter * h)[None, :]
        V[interior] += d[interior]
    return V


def box_geo_conn(nx, ny, nz):
    ex, ey, ez = _elem_grid(nx, ny, nz)
    conn = np.empty((nx * ny * nz, 8), dtype=np.int64)
    for c in range(2):
        for b in range(2):
            for a in range(2):
                conn[:, a + 2 * (b + 2 * c)] = (ex + a) + (nx + 1) * ((ey + b) + (ny + 1) * (ez + c))
    return conn.astype(np.int32)


def box_dof_conn(nx, ny, nz, p):
    n = p + 1
    Nx, Ny = nx * p + 1, ny * p + 1
    ex, ey, ez = _elem_grid(nx, ny, nz)
    conn = np.empty((nx * ny * nz, n ** 3), dtype=np.int64)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                conn[:, i + n * (j + n * k)] = (ex * p + i) + Nx * ((ey * p + j) + Ny * (ez * p + k))
    return conn.astype(np.int32)


def _elem_grid(nx, ny, nz):
    e = np.arange(nx * ny * nz)
    return e % nx, (e // nx) % ny, e // (nx * ny)


def box_dirichlet_x0(nx, ny, nz, p):
    """Mask clamping every DoF on the face x = 0 (lattice index I = 0)."""
    Nx, Ny, Nz = nx * p + 1, ny * p + 1, nz * p + 1
    I = np.arange(Nx * Ny * Nz) % Nx
    m = (I == 0).astype(np.uint8)
    return np.repeat(m, 3)


def box_dirichlet_triaxial(nx, ny, nz, p):
    """Symmetry clamps (component d on the face x_d = 0) plus component d on
    the far face x_d = L_d, for d = x, y, z: with the far faces' normal
    displacements prescribed this is triaxial compression (or extension),
    whose solution is the homogeneous state."""
    Nx, Ny, Nz = nx * p + 1, ny * p + 1, nz * p + 1
    idx = np.arange(Nx * Ny * Nz)
    I_, J_, K_ = idx % Nx, (idx // Nx) % Ny, idx // (Nx * Ny)
    m = np.zeros((idx.size, 3), np.uint8)
    m[:, 0] = (I_ == 0) | (I_ == Nx - 1)
    m[:, 1] = (J_ == 0) | (J_ == Ny - 1)
    m[:, 2] = (K_ == 0) | (K_ == Nz - 1)
    return m.ravel()


def box_boundary_faces(nx, ny, nz, side):
    """(element, local face) pairs of one side of a box: side 2d + s is the
    plane x_d = 0 (s = 0) or x_d = L_d (s = 1); the elements' local face has
    the same number (reference axes along x, y, z)."""
    ex, ey, ez = _elem_grid(nx, ny, nz)
    d, s = divmod(int(side), 2)
    idx = (ex, ey, ez)[d]
    last = (nx, ny, nz)[d] - 1
    e = np.nonzero(idx == (last if s else 0))[0]
    return np.stack([e, np.full(e.size, side)], axis=1).astype(np.int32)


def box_mesh(n, p, jitter=0.0, seed=0, lengths=(1.0, 1.0, 1.0), clamp=False, name=""):
    nx = ny = nz = int(n)
    V = box_vertices(nx, ny, nz, lengths, jitter, seed)
    n_nodes = (nx * p + 1) * (ny * p + 1) * (nz * p + 1)
    dmask = box_dirichlet_x0(nx, ny, nz, p) if clamp else np.zeros(3 * n_nodes, np.uint8)
    return MeshInput(p=p, geo_degree=1, geo_nodes=V, geo_conn=box_geo_conn(nx, ny, nz),
                     dof_conn=box_dof_conn(nx, ny, nz, p), n_nodes=n_nodes,
                     dirichlet=dmask, box=(nx, ny, nz), name=name or f"cube{n}_p{p}")


# --------------------------------------------------------------------------
# thick-walled tube with a triquadratic geometry description
# --------------------------------------------------------------------------

def tube_mesh(p, n_r=8, n_theta=16, n_z=64, r_in=1.0, r_out=1.3, length=10.0,
              clamp=False, name=""):
    """Tube of n_theta (circumferential, periodic) x n_r (radial) x n_z (axial)
    elements. Geometry nodes of every element form a 3x3x3 lattice placed
    exactly on (r, theta, z) at parameter values {0, 1/2, 1}; reference axes are
    (r, theta, z), which is right-handed. Per-element fibre frames are
    E1 = circumferential, E2 = axial, E3 = radial at the element's mid-angle."""
    Gr, Gt, Gz = 2 * n_r + 1, 2 * n_theta, 2 * n_z + 1
    a = np.arange(Gr)
    b = np.arange(Gt)
    c = np.arange(Gz)
    C, B, A = np.meshgrid(c, b, a, indexing="ij")
    r = r_in + (r_out - r_in) * A.ravel() / (2 * n_r)
    th = 2.0 * math.pi * B.ravel() / (2 * n_theta)
    z = length * C.ravel() / (2 * n_z)
    geo = np.stack([r * np.cos(th), r * np.sin(th), z], axis=1)

    ne = n_r * n_theta * n_z
    e = np.arange(ne)
    ir, it, iz = e % n_r, (e // n_r) % n_theta, e // (n_r * n_theta)
    gconn = np.empty((ne, 27), dtype=np.int64)
    for kc in range(3):
        for kb in range(3):
            for ka in range(3):
                gconn[:, ka + 3 * (kb + 3 * kc)] = (2 * ir + ka) + Gr * (((2 * it + kb) % Gt) + Gt * (2 * iz + kc))

    n = p + 1
    Nr, Nt, Nz = n_r * p + 1, n_theta * p, n_z * p + 1
    dconn = np.empty((ne, n ** 3), dtype=np.int64)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                dconn[:, i + n * (j + n * k)] = (ir * p + i) + Nr * (((it * p + j) % Nt) + Nt * (iz * p + k))
    n_nodes = Nr * Nt * Nz

    thc = 2.0 * math.pi * (it + 0.5) / n_theta
    frames = np.zeros((ne, 9))
    frames[:, 0], frames[:, 1] = -np.sin(thc), np.cos(thc)        # E1 circumferential
    frames[:, 5] = 1.0                                             # E2 axial
    frames[:, 6], frames[:, 7] = np.cos(thc), np.sin(thc)          # E3 radial

    if clamp:
        K = np.arange(n_nodes) // (Nr * Nt)
        dmask = np.repeat((K == 0).astype(np.uint8), 3)
    else:
        dmask = np.zeros(3 * n_nodes, np.uint8)
    return MeshInput(p=p, geo_degree=2, geo_nodes=geo, geo_conn=gconn.astype(np.int32),
                     dof_conn=dconn.astype(np.int32), n_nodes=n_nodes, dirichlet=dmask,
                     box=None, frames=frames, name=name or f"tube_p{p}",
                     extra=dict(n_r=n_r, n_theta=n_theta, n_z=n_z, r_in=r_in, r_out=r_out,
                                length=length))


def tube_dirichlet_symmetry(p, n_r=8, n_theta=16, n_z=64):
    """Constraints of a tube that leave its axisymmetric deformations free:
    u_z = 0 on the bottom (z = 0), u_y = 0 on the nodes at theta = 0 and pi,
    u_x = 0 on those at theta = pi/2 and 3 pi/2 (the mesh's mirror planes;
    together they remove the rigid motions). Needs n_theta p divisible by 4."""
    Nr, Nt, Nz = n_r * p + 1, n_theta * p, n_z * p + 1
    if Nt % 4:
        raise ValueError("n_theta * p must be divisible by 4")
    idx = np.arange(Nr * Nt * Nz)
    jt, kz = (idx // Nr) % Nt, idx // (Nr * Nt)
    m = np.zeros((idx.size, 3), np.uint8)
    m[:, 0] = (jt == Nt // 4) | (jt == 3 * Nt // 4)
    m[:, 1] = (jt == 0) | (jt == Nt // 2)
    m[:, 2] = kz == 0
    return m.ravel()


def tube_boundary_faces(n_r, n_theta, n_z, which):
    """(element, local face) pairs of a tube surface: "inner" (r = r_in,
    local face 0), "outer" (r = r_out, face 1), "bottom" (z = 0, face 4) or
    "top" (z = length, face 5); elements are ir + n_r*(it + n_theta*iz)."""
    e = np.arange(n_r * n_theta * n_z)
    ir, iz = e % n_r, e // (n_r * n_theta)
    sel, lf = {"inner": (ir == 0, 0), "outer": (ir == n_r - 1, 1),
               "bottom": (iz == 0, 4), "top": (iz == n_z - 1, 5)}[which]
    e = e[sel]
    return np.stack([e, np.full(e.size, lf)], axis=1).astype(np.int32)


def constant_frames(n_elem):
    """Per-element fibre frames equal to the Cartesian axes."""
    f = np.zeros((n_elem, 9))
    f[:, 0] = f[:, 4] = f[:, 8] = 1.0
    return f


# --------------------------------------------------------------------------
# displacement states and directions
# --------------------------------------------------------------------------

@dataclass
class SineField:
    """u_c(X) = amp * sum_j sin(pi * sum_d k_cjd X_d / L_d + phi_cj), with k in
    {0,1,2}^3 minus the zero vector, plus an optional affine part
    A (X - X0)."""

    k: np.ndarray         # (3, nterms, 3)
    phi: np.ndarray       # (3, nterms)
    amp: float
    L: np.ndarray         # (3,)
    affine: np.ndarray | None = None
    x0: np.ndarray | None = None

    def __call__(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        u = np.zeros_like(X)
        arg_scale = math.pi / self.L
        for c in range(3):
            for j in range(self.k.shape[1]):
                u[:, c] += np.sin((X * (self.k[c, j] * arg_scale)).sum(axis=1) + self.phi[c, j])
        u *= self.amp
        if self.affine is not None:
            u += (X - self.x0) @ self.affine.T
        return u

    def grad_bound(self) -> float:
        """Upper bound of |du_c/dX_d| of the sine part."""
        s = np.abs(self.k) * (math.pi / self.L)[None, None, :]
        return float(self.amp * s.sum(axis=1).max())


def sine_field(seed, strain=None, amp=None, nterms=3, L=(1.0, 1.0, 1.0)):
    """Seeded low-frequency sine field. Give either the amplitude directly or a
    target strain (the amplitude is then chosen so that the gradient bound
    equals it)."""
    g = rng(seed)
    L = np.asarray(L, dtype=np.float64)
    k = np.zeros((3, nterms, 3), dtype=np.int64)
    for c in range(3):
        for j in range(nterms):
            while True:
                kk = g.integers(0, 3, size=3)
                if kk.any():
                    break
            k[c, j] = kk
    phi = g.uniform(0.0, 2.0 * math.pi, size=(3, nterms))
    f = SineField(k=k, phi=phi, amp=1.0, L=L)
    if amp is not None:
        f.amp = float(amp)
    else:
        f.amp = float(strain) / f.grad_bound()
    return f


def compression_field(seed, J_target=0.9, sine_amp=0.005, center=(0.5, 0.5, 0.5)):
    """Uniform volumetric compression to J ~ J_target about `center` plus a
    small sine perturbation."""
    f = sine_field(seed, amp=sine_amp)
    s = J_target ** (1.0 / 3.0) - 1.0
    f.affine = s * np.eye(3)
    f.x0 = np.asarray(center, dtype=np.float64)
    return f


def inflation_field(seed, radial=0.02, sine_strain=0.01, L=(1.3, 1.3, 10.0)):
    """Radial inflation u = radial * (X, Y, 0) plus sines at the given strain."""
    f = sine_field(seed, strain=sine_strain, L=L)
    f.affine = np.diag([radial, radial, 0.0])
    f.x0 = np.zeros(3)
    return f


def random_direction(n_dofs, seed):
    """Uniform[-1, 1] per DoF."""
    return rng(seed).uniform(-1.0, 1.0, size=n_dofs)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

MAT_CNH = dict(law=0, mu=1.0, lam=10.0)
MAT_INH = dict(law=1, mu=1.0, kappa=1.0e3)
# fibre-reinforced tube: k1 = 1, k2 = 10, +-40 degrees, bulk modulus from the
# aortic-media ratio kappa/mu = 3084.3/62.1, dispersion (a, b) = (3.62, 34.3)
MAT_FIBER = dict(law=2, mu=1.0, kappa=3084.3 / 62.1, k1=1.0, k2=10.0,
                 a=3.62, b=34.3, phi=math.radians(40.0))


def workload_small_cube(seed=SEED_BASE + 1):
    """4^3 affine unit cube, p = 2, u = 0.01 * 3 sines per component, delta-u
    uniform[-1, 1] (about 1.9k free DoFs with the x = 0 face clamped)."""
    m = box_mesh(4, 2, jitter=0.0, seed=seed, clamp=True, name="cube4_p2")
    return m, sine_field(seed, amp=0.01), seed


def workload_jittered_cube(p, n=32, seed=SEED_BASE + 2):
    """n^3 cube with interior vertices jittered by +-10% of h, sines at 5% strain."""
    m = box_mesh(n, p, jitter=0.1, seed=seed, name=f"cube{n}_p{p}_jitter")
    return m, sine_field(seed + 17, strain=0.05), seed


def workload_batch(n_meshes=64, seed=SEED_BASE + 5):
    """Batch of independent cNH cubes: n^3 elements with n ~ U{8..24}, degree
    p ~ U{2,3,4,5}, interior vertices jittered by +-10% of h, each with its own
    seeded 5% sine state (about 30 M DoFs in total)."""
    g = rng(seed)
    out = []
    for k in range(n_meshes):
        n = int(g.integers(8, 25))
        p = int(g.integers(2, 6))
        m = box_mesh(n, p, jitter=0.1, seed=seed + 100 + k, name=f"batch{k}_cube{n}_p{p}")
        out.append((m, sine_field(seed + 1000 + k, strain=0.05), seed + 2000 + k))
    return out


def box_dirichlet_symmetry(nx, ny, nz, p):
    """Symmetry clamps: component x on the face x = 0, y on y = 0, z on z = 0
    (removes the rigid motions; a compression towards the origin satisfies
    them)."""
    Nx, Ny, Nz = nx * p + 1, ny * p + 1, nz * p + 1
    idx = np.arange(Nx * Ny * Nz)
    I_, J_, K_ = idx % Nx, (idx // Nx) % Ny, idx // (Nx * Ny)
    m = np.zeros((idx.size, 3), np.uint8)
    m[:, 0] = I_ == 0
    m[:, 1] = J_ == 0
    m[:, 2] = K_ == 0
    return m.ravel()


def workload_uniaxial(n, p, stretch, lengths=(1.0, 1.0, 1.0)):
    """Unit box (no jitter) under uniaxial stretch: symmetry clamps on x = 0,
    y = 0, z = 0 and the prescribed u_x = (stretch - 1) L_x on the face
    x = L_x; the lateral faces are free. Returns the mesh and the initial
    iterate u_0 = ((stretch - 1) x, 0, 0), which carries the prescribed values
    on the clamped faces."""
    m = box_mesh(n, p, lengths=lengths, name=f"uniaxial{n}_p{p}")
    Nx, Ny, Nz = n * p + 1, n * p + 1, n * p + 1
    mask = box_dirichlet_symmetry(n, n, n, p).reshape(-1, 3).copy()
    I_ = np.arange(Nx * Ny * Nz) % Nx
    mask[I_ == Nx - 1, 0] = 1
    m.dirichlet = mask.ravel().astype(np.uint8)
    u0 = np.zeros((Nx * Ny * Nz, 3))
    u0[:, 0] = (stretch - 1.0) * lengths[0] * I_ / (Nx - 1)
    return m, u0.ravel()


@dataclass
class CompressionField:
    """u_c = s X_c + a X_c sum_j sin(pi k_cj . X + phi_cj): uniform compression
    towards the origin (J = (1+s)^3) plus sines that vanish on the symmetry
    faces X_c = 0."""

    s: float
    sines: SineField

    def __call__(self, X):
        X = np.asarray(X, dtype=np.float64)
        return self.s * X + X * self.sines(X)


def workload_triaxial_compression(n=48, p=4, J_target=0.9999, seed=SEED_BASE + 3):
    """The compressed cube as a boundary-value problem (iNH, kappa = 1e3 mu):
    the n^3 jittered cube with symmetry clamps and the far faces' normal
    displacements prescribed to (J_target^(1/3) - 1) L; returns the mesh,
    u_0 (zero except the prescribed values) and the exact solution, the
    homogeneous compression u = (J_target^(1/3) - 1) X, which the
    discretisation contains (trilinear geometry)."""
    m = box_mesh(n, p, jitter=0.1, seed=seed, name=f"cube{n}_p{p}_triaxial")
    m.dirichlet = box_dirichlet_triaxial(n, n, n, p)
    return m, J_target ** (1.0 / 3.0) - 1.0


def workload_tube_inflation(p=3, n_r=8, n_theta=16, n_z=64, pressure=0.02):
    """The fibre tube (16 x 8 x 64 elements, Q2 geometry) inflated by a dead
    pressure on its inner surface, with the symmetry constraints of
    tube_dirichlet_symmetry; returns the mesh, the inner faces and the
    pressure."""
    m = tube_mesh(p, n_r=n_r, n_theta=n_theta, n_z=n_z, name=f"tube_p{p}_inflation")
    m.dirichlet = tube_dirichlet_symmetry(p, n_r, n_theta, n_z)
    return m, tube_boundary_faces(n_r, n_theta, n_z, "inner"), pressure


def workload_compressed_cube(n=48, p=4, J_target=0.9, sine_amp=0.005, seed=SEED_BASE + 3):
    """n^3 jittered cube (iNH, kappa = 1e3 mu): compression to J ~ J_target plus a
    small sine perturbation; symmetry clamps on the three faces through the
    origin."""
    m = box_mesh(n, p, jitter=0.1, seed=seed, name=f"cube{n}_p{p}_compressed")
    m.dirichlet = box_dirichlet_symmetry(n, n, n, p)
    f = CompressionField(J_target ** (1.0 / 3.0) - 1.0, sine_field(seed + 11, amp=sine_amp))
    return m, f, seed
