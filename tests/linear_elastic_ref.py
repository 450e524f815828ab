"""Independent linear-elastic stiffness on affine box meshes (test pin only).

Written in the textbook B-matrix (Voigt) form, K = sum_q w_q det(J) B^T D B,
with 1D Lagrange polynomials built from numpy Polynomial objects on the
closed-form Gauss-Lobatto points of p = 1, 2, 3. It shares nothing with the
oracle's tensor code; the hyperelastic tangent at u = 0 must reduce to it
(Sec. 3: at F = I every law linearises to isotropic linear elasticity).
"""
import math

import numpy as np
import scipy.sparse as sp

GLL_CLOSED_FORM = {
    1: [0.0, 1.0],
    2: [0.0, 0.5, 1.0],
    3: [0.0, 0.5 * (1 - 1 / math.sqrt(5)), 0.5 * (1 + 1 / math.sqrt(5)), 1.0],
}


def _lagrange_1d(p):
    xs = GLL_CLOSED_FORM[p]
    polys = []
    for a in range(p + 1):
        others = [xs[b] for b in range(p + 1) if b != a]
        P = np.polynomial.Polynomial.fromroots(others)
        polys.append(P / P(xs[a]))
    return polys


def lame_D(mu, lam):
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    for i in range(3):
        D[i, i] += 2 * mu
    for i in range(3, 6):
        D[i, i] = mu
    return D


def element_stiffness(p, h, mu, lam):
    """Stiffness of one axis-aligned box element with edge lengths h=(hx,hy,hz).
    Rows/columns ordered node-major (node a, component c) -> 3a + c, nodes
    lexicographic with x fastest."""
    polys = _lagrange_1d(p)
    dpolys = [P.deriv() for P in polys]
    xq, wq = np.polynomial.legendre.leggauss(p + 1)
    xq = 0.5 * (xq + 1)
    wq = 0.5 * wq
    n = p + 1
    nn = n ** 3
    D = lame_D(mu, lam)
    K = np.zeros((3 * nn, 3 * nn))
    detJ = h[0] * h[1] * h[2]
    for qz in range(n):
        for qy in range(n):
            for qx in range(n):
                B = np.zeros((6, 3 * nn))
                for k in range(n):
                    for j in range(n):
                        for i in range(n):
                            a = i + n * (j + n * k)
                            gx = dpolys[i](xq[qx]) * polys[j](xq[qy]) * polys[k](xq[qz]) / h[0]
                            gy = polys[i](xq[qx]) * dpolys[j](xq[qy]) * polys[k](xq[qz]) / h[1]
                            gz = polys[i](xq[qx]) * polys[j](xq[qy]) * dpolys[k](xq[qz]) / h[2]
                            c = 3 * a
                            B[0, c] = gx
                            B[1, c + 1] = gy
                            B[2, c + 2] = gz
                            B[3, c + 1] = gz
                            B[3, c + 2] = gy
                            B[4, c] = gz
                            B[4, c + 2] = gx
                            B[5, c] = gy
                            B[5, c + 1] = gx
                K += wq[qx] * wq[qy] * wq[qz] * detJ * B.T @ D @ B
    return K


def global_stiffness(mesh_input, lengths, mu, lam):
    nx, ny, nz = mesh_input.box
    h = (lengths[0] / nx, lengths[1] / ny, lengths[2] / nz)
    Ke = element_stiffness(mesh_input.p, h, mu, lam)
    conn = mesh_input.dof_conn
    nloc = Ke.shape[0]
    dofs = (3 * conn[:, :, None] + np.arange(3)[None, None, :]).reshape(conn.shape[0], nloc)
    rows = np.repeat(dofs, nloc, axis=1).ravel()
    cols = np.tile(dofs, (1, nloc)).ravel()
    vals = np.tile(Ke.ravel(), conn.shape[0])
    n = 3 * mesh_input.n_nodes
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
