"""Element-partitioned (domain-decomposed) operator application over ranks.

The tangent apply is a sum of element contributions (Sec. 2 weak form), so a
partition of the elements over ranks gives, on each rank, the partial
vector of its own elements; the full result on the nodes a rank touches is
the sum of the partial vectors of every rank touching them. The exchange is
therefore one sum over the interface nodes after each apply, plus the scalar
reductions of the Krylov solver (dot products). This module holds that
exchange: a slab partition of a structured box, the interface node sets, and
the interface sum over torch.distributed (any backend). The local apply is a
callable supplied by the caller (the device apply of the rank's sub-mesh).
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
    import torch
    import torch.distributed as dist
    Nx, Ny = nx * p + 1, ny * p + 1
    plane = 3 * Nx * Ny
    v = partial
    z0, z1 = slabs[rank]
    reqs, bufs = [], []
    for nb, zplane in ((rank - 1, z0), (rank + 1, z1)):
        if 0 <= nb < len(slabs):
            off = zplane * p * plane
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
