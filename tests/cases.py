"""Shared test cases: materials and seeded states used by the oracle and the
GPU path (input recipes only; all arithmetic of the method lives on either
side)."""
import math

import numpy as np

from oracle import oracle as O
from paper_2408_12479_gb300 import inputs as I

FRAME = np.array([0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 1.0, 0.0, 0.0])  # E1 = y, E2 = z, E3 = x

MATS = {
    "cNH": dict(law=0, mu=1.0, lam=10.0),
    "iNH": dict(law=1, mu=1.0, kappa=50.0),
    "fiber": dict(law=2, mu=1.0, kappa=3084.3 / 62.1, k1=1.0, k2=10.0, a=3.62, b=34.3, phi=math.radians(40.0)),
}
LAWS = list(MATS)


def oracle_material(name_or_dict):
    d = MATS[name_or_dict] if isinstance(name_or_dict, str) else name_or_dict
    return O.Material.from_dict(d)


def small_cube(n, p, law, jitter=0.1, seed=7, clamp=False):
    m = I.box_mesh(n, p, jitter=jitter, seed=seed, clamp=clamp)
    if law == "fiber":
        m.frames = np.tile(FRAME, (m.n_elem, 1))
    return m


def state_for(mesh_input, law, seed, strain=0.05):
    """Seeded displacement state at the oracle's node positions. For the fibre
    law both families are stretched (y and z by 8%) so that every point has
    I* - 1 well away from the switch."""
    M = O.OracleMesh(mesh_input)
    X = O.node_coords(M)
    f = I.sine_field(seed, strain=strain)
    u = f(X)
    if law == "fiber":
        u += X @ np.diag([0.0, 0.08, 0.08])
    return M, X, u.ravel()


def fibre_switch_margin(M, mat, u):
    """Smallest |I* - 1| over all quadrature points of the mesh (oracle)."""
    _, _, F = O.qp_fields(M, u, np.arange(M.n_elem))
    mats = []
    E1, E2 = FRAME[:3], FRAME[3:6]
    for ph in (mat.phi, -mat.phi):
        M1 = math.cos(ph) * E1 + math.sin(ph) * E2
        C = np.einsum("qki,qkj->qij", F.reshape(-1, 3, 3), F.reshape(-1, 3, 3))
        mats.append(np.abs(np.einsum("i,qij,j->q", M1, C, M1) - 1.0).min())
    return min(mats)
