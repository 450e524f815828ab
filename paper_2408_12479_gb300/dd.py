"""Element-partitioned (domain-decomposed) operator application over ranks.

The tangent apply is a sum of element contributions (Sec. 2 weak form), so a
partition of the elements over ranks gives, on each rank, the partial
vector of its own elements; the full result on the nodes a rank touches is
the sum of the partial vectors of every rank touching them. The exchange is
therefore one sum over the interface nodes after each apply, plus the scalar
reductions of the Krylov solver (dot products). This module holds:

* the slab partition of a structured box, each slab's sub-mesh and its node
  range, and the interface sum over torch.distributed (any backend);
* SlabSystem: the Dirichlet-constrained tangent on rank-local vectors, its
  owner-rule dot product, the Chebyshev-Jacobi smoother, CG (Sec. 6) and
  Newton's method (Alg. 1) over the slabs.

The local work (apply, residual, diagonal, state refresh of the rank's
sub-mesh) is supplied by the caller as callables: the device kernels of the
library on GPU ranks, the oracle in the CPU tests.
"""
from __future__ import annotations

import numpy as np


def slab_partition(nz: int, world: int) -> list[tuple[int, int]]:
    """Split nz element layers into `world` contiguous slabs [z0, z1)."""
    if world < 1 or world > nz:
        raise ValueError("need 1 <= world <= nz")
    cuts = np.linspace(0, nz, world + 1).round().astype(int)
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def slab_elements(nx: int, ny: int, z0: int, z1: int) -> np.ndarray:
    """Element ids (lexicographic, x fastest) of the layers z0 <= ez < z1."""
    return np.arange(z0 * nx * ny, z1 * nx * ny, dtype=np.int32)


def slab_node_range(nx: int, ny: int, p: int, z0: int, z1: int) -> tuple[int, int]:
    """Node ids [n0, n1) touched by the slab (node lattice x fastest)."""
    Nx, Ny = nx * p + 1, ny * p + 1
    return z0 * p * Nx * Ny, (z1 * p + 1) * Nx * Ny


def interface_sum(partial, nx: int, ny: int, p: int, slabs, rank: int, group=None):
    """Sum the partial vectors of neighbouring slabs on their shared node
    planes, in place. partial: this rank's vector over ALL nodes ([n_nodes, 3]
    flattened, zero outside its slab). Each interior interface (one node plane
    of (Nx*Ny) nodes between slabs r and r+1) is exchanged with the neighbour
    by point-to-point send/recv of that plane only."""
    plane = 3 * (nx * p + 1) * (ny * p + 1)
    z0, z1 = slabs[rank]
    return _add_neighbour_planes(partial, plane, [(rank - 1, z0 * p * plane), (rank + 1, z1 * p * plane)],
                                 len(slabs), group)


def _add_neighbour_planes(v, plane, pairs, world, group):
    """For each (neighbour rank, offset) with a valid neighbour: send this
    rank's `plane` values at the offset, receive the neighbour's, and add them
    in place once every exchange has completed."""
    import torch
    import torch.distributed as dist
    reqs, bufs = [], []
    for nb, off in pairs:
        if 0 <= nb < world:
            mine = v[off:off + plane].clone()
            other = torch.empty_like(mine)
            reqs.append(dist.isend(mine, nb, group=group))
            reqs.append(dist.irecv(other, nb, group=group))
            bufs.append((off, other))
    for r in reqs:
        r.wait()
    for off, other in bufs:
        v[off:off + plane] += other
    return v


# --------------------------------------------------------------------------
# rank-local vectors and the Krylov solve over slabs
# --------------------------------------------------------------------------
#
# Each rank holds only the nodes its slab touches: the node range
# slab_node_range(...) of the global lattice, in the same order, so a
# rank-local DoF vector is the slice [3 n0, 3 n1) of the global one. The node
# plane between slabs r and r+1 lives on both ranks. Vectors handed to and
# returned by the functions below are "consistent": both copies of a shared
# plane hold the full (summed) value. A partial vector -- the sum over this
# rank's elements only, as a local apply, residual or diagonal returns it --
# becomes consistent by interface_sum_local.

def slab_mesh(m, slab):
    """The sub-box of a structured, trilinear box mesh that slab (z0, z1)
    covers, numbered locally (x fastest, as the global lattice), with no
    constraints: the local operator is the pure sum over the slab's elements.
    Its node order is the global node range of the slab."""
    from . import inputs as _inputs
    if m.box is None or m.geo_degree != 1:
        raise ValueError("slab_mesh needs a structured box with trilinear geometry")
    nx, ny, nz = m.box
    z0, z1 = slab
    if not 0 <= z0 < z1 <= nz:
        raise ValueError("slab outside the box")
    nv = (nx + 1) * (ny + 1)
    nzl = z1 - z0
    n_nodes = (nx * m.p + 1) * (ny * m.p + 1) * (nzl * m.p + 1)
    frames = None
    if m.frames is not None:
        frames = m.frames[z0 * nx * ny:z1 * nx * ny]
    return _inputs.MeshInput(p=m.p, geo_degree=1, geo_nodes=np.ascontiguousarray(m.geo_nodes[z0 * nv:(z1 + 1) * nv]),
                             geo_conn=_inputs.box_geo_conn(nx, ny, nzl),
                             dof_conn=_inputs.box_dof_conn(nx, ny, nzl, m.p), n_nodes=n_nodes,
                             dirichlet=np.zeros(3 * n_nodes, np.uint8), box=(nx, ny, nzl), frames=frames,
                             name=f"{m.name}_z{z0}-{z1}")


def local_slice(nx, ny, p, slab):
    """The DoF slice [3 n0, 3 n1) of a global vector that a slab's rank holds."""
    n0, n1 = slab_node_range(nx, ny, p, slab[0], slab[1])
    return slice(3 * n0, 3 * n1)


def owned_mask(nx, ny, p, slabs, rank):
    """Local DoFs this rank counts in global reductions: all of its nodes but
    the lowest node plane when a slab lies below (that plane belongs to the
    rank below), so every global DoF is counted exactly once."""
    z0, z1 = slabs[rank]
    plane = 3 * (nx * p + 1) * (ny * p + 1)
    n = plane * ((z1 - z0) * p + 1)
    own = np.ones(n, dtype=bool)
    if rank > 0:
        own[:plane] = False
    return own


def interface_sum_local(v, nx, ny, p, slabs, rank, group=None):
    """In place: add the neighbours' partial values on the shared node planes
    of a rank-local vector (lowest local plane with rank-1, highest with
    rank+1), one plane exchanged per neighbour by isend/irecv."""
    z0, z1 = slabs[rank]
    plane = 3 * (nx * p + 1) * (ny * p + 1)
    return _add_neighbour_planes(v, plane, [(rank - 1, 0), (rank + 1, (z1 - z0) * p * plane)], len(slabs), group)


class SlabSystem:
    """The Dirichlet-constrained tangent K_c over an element-slab partition of
    a structured box, on rank-local consistent vectors.

    apply_local(v) -> the partial vector sum_{e in slab} K_e v_e of the
    rank's sub-mesh (e.g. the device tangent apply of slab_mesh(...) with its
    own quadrature-point cache); constrained: this rank's slice of the global
    Dirichlet mask. K_c v = K v on free rows with constrained entries of v
    zeroed first, and v itself on constrained rows (the single-mesh
    convention). Global reductions sum owned DoFs and all-reduce the scalar,
    the one collective besides the interface exchange. With one slab (world
    1) no collective is issued."""

    def __init__(self, nx, ny, p, slabs, rank, apply_local, constrained, group=None):
        import torch
        self.nx, self.ny, self.p = nx, ny, p
        self.slabs, self.rank, self.group = slabs, rank, group
        self.apply_local = apply_local
        self.world = len(slabs)
        self.cmask = torch.as_tensor(np.asarray(constrained, dtype=bool))
        self.own = torch.as_tensor(owned_mask(nx, ny, p, slabs, rank))
        if self.cmask.numel() != self.own.numel():
            raise ValueError("constraint mask does not match the slab's DoFs")

    def _to(self, v):
        if self.cmask.device != v.device:
            self.cmask = self.cmask.to(v.device)
            self.own = self.own.to(v.device)

    def assemble(self, partial):
        """Make a partial vector consistent (interface sum), in place."""
        if self.world > 1:
            interface_sum_local(partial, self.nx, self.ny, self.p, self.slabs, self.rank, self.group)
        return partial

    def dot(self, a, b):
        """Global a.b over the owned DoFs of every rank."""
        import torch
        import torch.distributed as dist
        self._to(a)
        s = torch.sum(torch.where(self.own, a * b, torch.zeros((), dtype=a.dtype, device=a.device)))
        s = s.reshape(1).to(torch.float64)
        if self.world > 1:
            dist.all_reduce(s, group=self.group)
        return float(s.item())

    def apply(self, v):
        """K_c v (consistent in, consistent out)."""
        import torch
        self._to(v)
        vv = torch.where(self.cmask, torch.zeros((), dtype=v.dtype, device=v.device), v)
        w = self.assemble(self.apply_local(vv))
        return torch.where(self.cmask, v, w)

    def diagonal(self, partial_diag):
        """Consistent diag(K_c) from this rank's partial diagonal of the pure
        operator: interface sum, then 1 on constrained rows."""
        import torch
        self._to(partial_diag)
        d = self.assemble(partial_diag.clone())
        return torch.where(self.cmask, torch.ones((), dtype=d.dtype, device=d.device), d)

    def lambda_max(self, inv_diag, iters=30, seed=1):
        """Largest eigenvalue of D^-1 K_c by power iteration, scaled up by
        1.1 as a safe upper bound for Chebyshev. The start vector is a hash
        of the global DoF index (Knuth's multiplicative hash), so both copies
        of a shared plane start equal and the result does not depend on the
        partition."""
        import torch
        sl = local_slice(self.nx, self.ny, self.p, self.slabs[self.rank])
        i = torch.arange(sl.start, sl.stop, dtype=torch.int64)
        h = ((i + seed) * 2654435761) % 4294967296
        x = (0.5 + h.to(torch.float64) / 4294967296.0).to(inv_diag.device, inv_diag.dtype)
        lam = 0.0
        for _ in range(iters):
            x = x / (self.dot(x, x) ** 0.5)
            y = inv_diag * self.apply(x)
            lam = self.dot(x, y) / self.dot(x, x)
            x = y
        return 1.1 * lam

    def chebyshev(self, rhs, x, inv_diag, degree, lambda_max, smoothing_range, zero_initial=False):
        """degree steps of Chebyshev-accelerated Jacobi on K_c x = rhs
        (Sec. 6 smoother; the same three-term recurrence as the single-mesh
        smoother over the interval [lambda_max/smoothing_range, lambda_max]
        of D^-1 K_c). Returns the new x."""
        a = lambda_max / smoothing_range
        theta, delta = 0.5 * (lambda_max + a), 0.5 * (lambda_max - a)
        x = x.clone()
        if zero_initial:
            x.zero_()
        d, rho = None, None
        for k in range(degree):
            r = inv_diag * (rhs if (k == 0 and zero_initial) else rhs - self.apply(x))
            if k == 0:
                rho_k = delta / theta
                d = r / theta
            else:
                rho_k = 1.0 / (2.0 * theta / delta - rho)
                d = (rho_k * rho) * d + (2.0 * rho_k / delta) * r
            x = x + d
            rho = rho_k
        return x

    def cg(self, b, x0=None, precond=None, tol=1e-10, max_iter=1000):
        """Preconditioned CG on K_c x = b (Polak-Ribiere beta, so a
        preconditioner that varies slightly between calls is tolerated);
        stops when ||b - K_c x|| <= tol ||b|| on the recursive residual and
        returns (x, iterations, true relative residual). A non-positive
        curvature p.K_c p raises (K_c must be SPD). precond(r) -> z, default
        the identity."""
        import torch
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        M = precond if precond is not None else (lambda r: r)
        r = b - self.apply(x)
        bn = self.dot(b, b) ** 0.5
        if bn == 0.0:
            return x, 0, 0.0
        z = M(r)
        p = z.clone()
        rz = self.dot(r, z)
        it = 0
        rn = self.dot(r, r) ** 0.5
        while it < max_iter and rn > tol * bn:
            Ap = self.apply(p)
            pAp = self.dot(p, Ap)
            if not pAp > 0.0:
                raise RuntimeError(f"SlabSystem.cg: non-positive curvature {pAp:.3e} at iteration {it}")
            alpha = rz / pAp
            x = x + alpha * p
            r_new = r - alpha * Ap
            z_new = M(r_new)
            beta = self.dot(r_new, z_new - z) / rz
            rz = self.dot(r_new, z_new)
            p = z_new + beta * p
            r, z = r_new, z_new
            rn = self.dot(r, r) ** 0.5
            it += 1
        r_true = b - self.apply(x)
        true_rel = self.dot(r_true, r_true) ** 0.5 / bn
        return x, it, true_rel

    def newton(self, u, residual_local, set_state, diagonal_local, f_ext=None, eps_abs=1e-10, eps_rel=1e-8,
               max_newton=20, cg_tol=1e-8, cg_max_iter=5000, cheb_degree=0, smoothing_range=15.0):
        """Newton's method (Alg. 1) on R(u) - f_ext = 0 over the free DoFs,
        partitioned by slabs. u: this rank's consistent state, with the
        Dirichlet values already in its constrained entries (left unchanged);
        residual_local(u) -> the partial residual of the rank's elements (pure
        operator); set_state(u) refreshes the linearization point that
        apply_local and diagonal_local use (Alg. 1's quadrature-point update);
        diagonal_local() -> the partial diagonal of the pure operator; f_ext:
        consistent external load (or None). Each update solves K_c du = -r by
        CG with Jacobi (cheb_degree 0) or Chebyshev(cheb_degree)-Jacobi
        preconditioning. Returns (u, report) with the iteration counts and
        the first and last residual norms."""
        import torch
        self._to(u)
        u = u.clone()
        rep = {"newton_iters": 0, "cg_iters": 0, "res0": None, "res": None, "converged": False}
        for k in range(max_newton + 1):
            r = self.assemble(residual_local(u))
            if f_ext is not None:
                r = r - f_ext
            r = torch.where(self.cmask, torch.zeros((), dtype=r.dtype, device=r.device), r)
            nrm = self.dot(r, r) ** 0.5
            if k == 0:
                rep["res0"] = nrm
            rep["res"] = nrm
            if nrm <= eps_abs or nrm <= eps_rel * rep["res0"]:
                rep["converged"] = True
                break
            if k == max_newton:
                break
            set_state(u)
            inv_d = 1.0 / self.diagonal(diagonal_local())
            if cheb_degree > 0:
                lam = self.lambda_max(inv_d)

                def precond(v):
                    return self.chebyshev(v, torch.zeros_like(v), inv_d, cheb_degree, lam, smoothing_range,
                                          zero_initial=True)
            else:
                def precond(v):
                    return inv_d * v
            du, its, _ = self.cg(-r, precond=precond, tol=cg_tol, max_iter=cg_max_iter)
            u = u + du
            rep["newton_iters"] += 1
            rep["cg_iters"] += its
        return u, rep
