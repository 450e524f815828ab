// hx_loads.cpp -- external load vectors on the host (include/hx_loads.h).
//
// The Neumann load f_i = (N_i, h_N) over boundary faces (Sec. 2, the Gamma_N
// term of Eq. mom_bal_nonlinear_material_residual) for a dead load on the
// reference configuration. It is computed once per load step from the mesh
// description, so it runs on the host; nothing here touches the device.

#include <stdint.h>

#include <cmath>
#include <vector>

#include "hx_loads.h"

namespace {

const double kPi = 3.14159265358979323846;

// Legendre polynomial P_n and its derivative at x in (-1, 1), by the
// three-term recurrence (k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2}).
void legendre(int n, double x, double &P, double &dP) {
    double p0 = 1.0, p1 = x;
    if (n == 0) {
        P = 1.0;
        dP = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    P = p1;
    dP = n * (x * p1 - p0) / (x * x - 1.0);
}

// n-point Gauss-Legendre rule on [0, 1]: the roots of P_n by Newton's method
// from the Chebyshev-like guesses cos(pi (i + 3/4) / (n + 1/2)); weights
// 2 / ((1 - x^2) P_n'(x)^2), halved for the unit interval.
void gauss_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), P = 0.0, dP = 0.0;
        for (int it = 0; it < 100; ++it) {
            legendre(n, z, P, dP);
            const double dz = P / dP;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        legendre(n, z, P, dP);
        // roots come out in decreasing order; store them increasing on [0, 1]
        x[n - 1 - i] = 0.5 * (1.0 + z);
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dP * dP);
    }
}

// The p+1 Gauss-Lobatto-Legendre points on [0, 1]: the end points and the
// roots of P_p', found by Newton's method on P_p' with
// P_p'' = (2 x P_p' - p (p+1) P_p) / (1 - x^2), from -cos(pi i / p).
void gll_points(int p, std::vector<double> &x) {
    x.assign(p + 1, 0.0);
    x[0] = 0.0;
    x[p] = 1.0;
    for (int i = 1; i < p; ++i) {
        double z = -std::cos(kPi * i / p), P = 0.0, dP = 0.0;
        for (int it = 0; it < 100; ++it) {
            legendre(p, z, P, dP);
            const double d2P = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
            const double dz = dP / d2P;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 + z);
    }
}

// Lagrange polynomials on nodes z (m of them) at t: values V[a] and first
// derivatives D[a] (sum over the left-out factor of the product rule).
void lagrange(const std::vector<double> &z, double t, double *V, double *D) {
    const int m = (int)z.size();
    for (int a = 0; a < m; ++a) {
        double v = 1.0, d = 0.0;
        for (int b = 0; b < m; ++b) {
            if (b == a) continue;
            double prod = 1.0 / (z[a] - z[b]);
            for (int c = 0; c < m; ++c)
                if (c != a && c != b) prod *= (t - z[c]) / (z[a] - z[c]);
            d += prod;
            v *= (t - z[b]) / (z[a] - z[b]);
        }
        V[a] = v;
        D[a] = d;
    }
}

}  // namespace

extern "C" hx_status hx_traction_load(const hx_mesh_desc *desc, int32_t n_faces, const int32_t *faces, int32_t mode,
                                      const double *value, double *f_host) {
    if (!desc || !value || !f_host || n_faces < 0 || (n_faces > 0 && !faces) || (mode != 0 && mode != 1))
        return HX_ERR_ARG;
    const int p = desc->p, g = desc->geo_degree;
    if (p < 1 || p > 8 || (g != 1 && g != 2) || desc->n_elem < 0 || desc->n_nodes < 1 || !desc->geo_nodes ||
        !desc->geo_conn || desc->n_geo_nodes < 1)
        return HX_ERR_ARG;
    const bool structured = desc->dof_conn == nullptr;
    if (structured && (desc->nx < 1 || desc->ny < 1 || desc->nz < 1 ||
                       (int64_t)desc->nx * desc->ny * desc->nz != desc->n_elem))
        return HX_ERR_ARG;
    const int n = p + 1, mg = g + 1, ng3 = mg * mg * mg, nn3 = n * n * n;
    std::vector<double> xq, wq, xn, xg(mg);
    gauss_rule(n, xq, wq);
    gll_points(p, xn);
    for (int i = 0; i < mg; ++i) xg[i] = (double)i / g;
    const int64_t Nx = (int64_t)desc->nx * p + 1, Ny = (int64_t)desc->ny * p + 1;

    std::vector<double> gV(3 * mg), gD(3 * mg), pV(3 * n), pD(3 * n);
    for (int32_t fi = 0; fi < n_faces; ++fi) {
        const int32_t e = faces[2 * fi], lf = faces[2 * fi + 1];
        if (e < 0 || e >= desc->n_elem || lf < 0 || lf > 5) return HX_ERR_ARG;
        const int d = lf / 2, side = lf % 2;
        const int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;  // the two in-face axes, increasing
        const int32_t *gc = desc->geo_conn + (int64_t)e * ng3;
        for (int i = 0; i < ng3; ++i)
            if (gc[i] < 0 || gc[i] >= desc->n_geo_nodes) return HX_ERR_ARG;
        int64_t base = 0;
        if (structured) {
            const int64_t ex = e % desc->nx, ey = (e / desc->nx) % desc->ny, ez = e / ((int64_t)desc->nx * desc->ny);
            base = ex * p + Nx * (ey * p + Ny * (ez * p));
        }
        for (int qb = 0; qb < n; ++qb) {
            for (int qa = 0; qa < n; ++qa) {
                double xi[3];
                xi[d] = (double)side;
                xi[a] = xq[qa];
                xi[b] = xq[qb];
                for (int c = 0; c < 3; ++c) {
                    lagrange(xg, xi[c], &gV[c * mg], &gD[c * mg]);
                    lagrange(xn, xi[c], &pV[c * n], &pD[c * n]);
                }
                // tangents dX/dxi_c of the geometry map at the point
                double T[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                for (int k = 0; k < mg; ++k)
                    for (int j = 0; j < mg; ++j)
                        for (int i = 0; i < mg; ++i) {
                            const double *X = desc->geo_nodes + 3 * (int64_t)gc[i + mg * (j + mg * k)];
                            const double w0 = gD[i] * gV[mg + j] * gV[2 * mg + k];
                            const double w1 = gV[i] * gD[mg + j] * gV[2 * mg + k];
                            const double w2 = gV[i] * gV[mg + j] * gD[2 * mg + k];
                            for (int r = 0; r < 3; ++r) {
                                T[0][r] += w0 * X[r];
                                T[1][r] += w1 * X[r];
                                T[2][r] += w2 * X[r];
                            }
                        }
                const double nv[3] = {T[a][1] * T[b][2] - T[a][2] * T[b][1], T[a][2] * T[b][0] - T[a][0] * T[b][2],
                                      T[a][0] * T[b][1] - T[a][1] * T[b][0]};
                const double dA = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
                if (!(dA > 0.0)) return HX_ERR_NONINVERTIBLE;
                // outward: along +xi_d on the face xi_d = 1, along -xi_d on xi_d = 0
                const double along = nv[0] * T[d][0] + nv[1] * T[d][1] + nv[2] * T[d][2];
                if (!(along != 0.0)) return HX_ERR_NONINVERTIBLE;
                const double sgn = ((along > 0.0) == (side == 1)) ? 1.0 : -1.0;
                double h[3];
                for (int r = 0; r < 3; ++r) h[r] = mode == 0 ? value[r] : -value[0] * sgn * nv[r] / dA;
                const double s = wq[qa] * wq[qb] * dA;
                for (int k = 0; k < n; ++k)
                    for (int j = 0; j < n; ++j)
                        for (int i = 0; i < n; ++i) {
                            const double psi = pV[i] * pV[n + j] * pV[2 * n + k] * s;
                            if (psi == 0.0) continue;
                            int64_t node;
                            if (structured)
                                node = base + i + Nx * (j + Ny * (int64_t)k);
                            else
                                node = desc->dof_conn[(int64_t)e * nn3 + i + n * (j + n * k)];
                            if (node < 0 || node >= desc->n_nodes) return HX_ERR_ARG;
                            for (int r = 0; r < 3; ++r) f_host[3 * node + r] += psi * h[r];
                        }
            }
        }
    }
    return HX_OK;
}
