/*
 * hx_loads.h -- external load vectors of the hyperelastic problem, computed on
 * the host from a mesh description (no device, no context).
 *
 * They enter Newton's method (hx_newton_solve) as f_ext; they are constant
 * within a load step and are computed once per load, so they run on the host.
 */
#ifndef HX_LOADS_H
#define HX_LOADS_H

#include "hx.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Neumann load vector of a dead load on boundary faces: the Gamma_N term of
 * the residual, f_i = (N_i, h_N)_{Gamma_N} (Sec. 2, Eq.
 * mom_bal_nonlinear_material_residual), with h_N the nominal traction on the
 * reference configuration (P N = h_N).
 *
 *  desc     mesh description as for hx_setup_mesh (geometry nodes and
 *           connectivity; dof_conn may be NULL for a structured box). Only
 *           p, geo_degree, n_nodes, geo_nodes, n_geo_nodes, geo_conn,
 *           dof_conn, nx, ny, nz and n_elem are read.
 *  faces    [n_faces][2] int32 pairs (element, local face); local face 2d+s
 *           is the face xi_d = s of the reference cube (d = 0, 1, 2 along
 *           the element's lexicographic axes; s = 0, 1). n_faces may be 0.
 *  mode     0: value[0..2] is a constant traction vector h_N;
 *           1: value[0] is a pressure p acting against the outward unit
 *              normal of the reference surface, h_N = -p N.
 *  f_host   [n_nodes][3] FP64 host array; the load is ADDED to its contents,
 *           so several faces or loads accumulate. Constrained rows get their
 *           share like any other (Newton ignores constrained rows).
 *
 * Each face is integrated with the (p+1) x (p+1) Gauss-Legendre rule; the
 * area element and the normal come from the two in-face tangents of the
 * geometry map. Returns HX_ERR_ARG for a bad argument (null pointer, element
 * or face out of range, unknown mode) and HX_ERR_NONINVERTIBLE for a face
 * with a zero area element at a quadrature point; f_host is then partly
 * updated. Host memory only; thread-safe. */
hx_status hx_traction_load(const hx_mesh_desc *desc, int32_t n_faces, const int32_t *faces, int32_t mode,
                           const double *value, double *f_host);

#ifdef __cplusplus
}
#endif
#endif /* HX_LOADS_H */
