/*
 * hx_oracle.c -- FP64 CPU oracle for the matrix-free hyperelastic operators of
 * "Matrix-Free Higher-Order Finite Element Methods for Hyperelasticity"
 * (arXiv 2408.12479).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this code;
 * it is used by the tests, by the package's smoke check and by the timed CPU
 * baseline of the benchmark. It shares no source with the CUDA library.
 *
 * What it computes is the plain Galerkin definition, element by element, with
 * full three-dimensional basis evaluation at every quadrature point (no sum
 * factorization, no caching of material data):
 *
 *   residual  R_{j,a} = sum_e sum_q JxW_q  dN_j/dX_b (q)  P_ab(F_q)        Sec. 2, Eq. (mom_bal_nonlinear_material_residual)
 *   tangent   (K du)_{j,a} = sum_e sum_q JxW_q dN_j/dX_b [H S + F D_uS[H]]_ab
 *             with H = Grad du                                             Sec. 2, Eq. (DDu_residual_material)
 *   energy    Pi(u) = sum_e sum_q JxW_q Psi(F_q)                           Sec. 3
 *   load      f_{j,a} = sum_e sum_q JxW_q N_j(q) b_a, constant body force b  Sec. 2, (v, B)
 *   tangent, spatial form (integration over Omega_t, pulled to Omega_0):
 *             (K du)_{j,a} = sum_e sum_q JxW_q dN_j/dx_b [Jc:(grad du)^S + (grad du) tau]_ab
 *             with grad = Grad F^-1                                        Sec. 2, Eq. (stress_term_in_Ot_with_JC)
 *
 * Material laws (Sec. 3; derivatives from Appendix A) in their textbook form:
 *   cNH   Psi = mu/2 (I1 - 3 - 2 ln J) + lambda ln^2 J                     Eq. (NH_compressible)
 *         S = mu I - (mu - 2 lambda ln J) C^-1
 *         D_uS = -(mu - 2 lambda ln J) D_uC^-1 + 2 lambda tr(F^-1 H) C^-1  App. A
 *   iNH   Psi = mu/2 (J^-2/3 I1 - 3) + kappa/4 (J^2 - 1 - 2 ln J)          Eq. (NH_nearly_incompressible)
 *         S = mu J^-2/3 I + [kappa/2 (J^2-1) - mu/3 J^-2/3 I1] C^-1
 *         D_uS as Eq. (NH_DDuS) of App. A, whose D_uC^-1 term carries the sign
 *         that follows from differentiating S (the Sec. 5 restatement prints
 *         the opposite sign in front of 2 c1 [F^-1 H C^-1]^S; it is not used)
 *   fiber Psi = Psi_iNH + sum_{i=4,6} k1/(2 k2) [exp(k2 E_i^2) - 1] if I_i* > 1  Eq. (fiber_Psi)
 *         E_i = H_i : C - 1,  I_i* = M1.C M1,  H_i = sum_k H_kk M_k (x) M_k      Eq. (fiber_Ei)
 *         S += 2 k1 exp(k2 E_i^2) E_i H_i,
 *         D_uS += 2 k1 exp(k2 E_i^2)(2 k2 E_i^2 + 1)(H_i : D_uC) H_i             Eq. (DduS_fiber)
 *   with D_uC^-1 = -(F^-1 H C^-1 + (F^-1 H C^-1)^T), D_uC = F^T H + H^T F,
 *   (1/J) D_uJ = tr(F^-1 H), D_uI1 = 2 tr(F^T H)                           App. A
 *
 * Fibre families (reading of the garbled basis in Sec. 3): with the
 * per-element frame (E1 circumferential, E2 longitudinal, E3 radial) and angle
 * Phi, family 4 uses M1 = cos Phi E1 + sin Phi E2, M2 = -sin Phi E1 + cos Phi E2,
 * M3 = E3; family 6 the same with -Phi. The tension switch I_i* > 1 is strict.
 *
 * Discretisation (the paper builds on deal.II FE_Q): Lagrange polynomials on
 * the p+1 nodal points passed in (Gauss-Lobatto-Legendre on [0,1]); tensor
 * product quadrature with the 1D points and weights passed in (Gauss-Legendre,
 * p+1 points); geometry: Lagrange polynomials of degree g on equispaced
 * points, vertex/node coordinates from geo_nodes.
 *
 * Conventions: 3x3 tensors are row-major double[9], A[r*3+c]; DoF vectors are
 * node-major [node][3]; local node numbering is lexicographic, xi1 fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int law; /* 0 cNH, 1 iNH, 2 fiber */
    double mu, lambda, kappa, k1, k2;
    double Hd[3]; /* H11, H22, H33 of the generalized structure tensor */
    double phi;   /* mean in-plane fibre angle (rad) */
} orc_material;

typedef struct {
    int p, g;                 /* FE degree, geometry degree */
    int n_elem;
    int64_t n_nodes;
    const double *geo_nodes;  /* [n_geo][3] */
    const int32_t *geo_conn;  /* [n_elem][(g+1)^3] */
    const int32_t *dof_conn;  /* [n_elem][(p+1)^3] */
    const double *frames;     /* [n_elem][9] E1,E2,E3 (fiber law) or NULL */
    const double *xi_node;    /* [p+1] nodal points on [0,1] */
    const double *xi_q;       /* [p+1] quadrature points on [0,1] */
    const double *w_q;        /* [p+1] quadrature weights (sum 1) */
    const double *xi_geo;     /* [g+1] geometry points on [0,1] */
} orc_mesh;

/* ------------------------------------------------------------------ */
/* small dense 3x3 algebra                                              */
/* ------------------------------------------------------------------ */
static void m_mul(const double *A, const double *B, double *C) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[r * 3 + k] * B[k * 3 + c];
            C[r * 3 + c] = s;
        }
}
static void m_tmul(const double *A, const double *B, double *C) { /* A^T B */
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[k * 3 + r] * B[k * 3 + c];
            C[r * 3 + c] = s;
        }
}
static void m_transpose(const double *A, double *T) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) T[c * 3 + r] = A[r * 3 + c];
}
static double m_det(const double *A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}
/* inverse via the adjugate; returns the determinant */
static double m_inv(const double *A, double *Ai) {
    double d = m_det(A);
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) / d;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) / d;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) / d;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) / d;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) / d;
    return d;
}
static double m_trace(const double *A) { return A[0] + A[4] + A[8]; }
static double m_ddot(const double *A, const double *B) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += A[i] * B[i];
    return s;
}

/* ------------------------------------------------------------------ */
/* material laws                                                        */
/* ------------------------------------------------------------------ */
typedef struct {
    double M1[2][3]; /* mean fibre direction of families 4 and 6 */
    double Hs[2][9]; /* structure tensors H_4, H_6 */
} orc_fibres;

static void fibres_from_frame(const orc_material *m, const double *frame, orc_fibres *fb) {
    const double *E1 = frame, *E2 = frame + 3, *E3 = frame + 6;
    for (int f = 0; f < 2; ++f) {
        double ph = (f == 0) ? m->phi : -m->phi;
        double c = cos(ph), s = sin(ph);
        double M[3][3];
        for (int d = 0; d < 3; ++d) {
            M[0][d] = c * E1[d] + s * E2[d];
            M[1][d] = -s * E1[d] + c * E2[d];
            M[2][d] = E3[d];
        }
        for (int d = 0; d < 3; ++d) fb->M1[f][d] = M[0][d];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc)
                fb->Hs[f][r * 3 + cc] = m->Hd[0] * M[0][r] * M[0][cc] + m->Hd[1] * M[1][r] * M[1][cc] +
                                        m->Hd[2] * M[2][r] * M[2][cc];
    }
}

/* Everything a law needs at one point, computed from F by the definitions. */
typedef struct {
    double F[9], Finv[9], C[9], Cinv[9];
    double J, lnJ, j23, I1;
    double Ei[2], Istar[2];
    int active[2];
} orc_state;

static void state_from_F(const orc_material *m, const orc_fibres *fb, const double *F, orc_state *s) {
    memcpy(s->F, F, sizeof(double) * 9);
    s->J = m_inv(F, s->Finv);
    m_tmul(F, F, s->C);
    m_inv(s->C, s->Cinv);
    s->lnJ = log(s->J);
    s->j23 = pow(s->J, -2.0 / 3.0);
    s->I1 = m_trace(s->C);
    for (int f = 0; f < 2; ++f) {
        s->Ei[f] = 0.0;
        s->Istar[f] = 0.0;
        s->active[f] = 0;
    }
    if (m->law == 2) {
        for (int f = 0; f < 2; ++f) {
            s->Ei[f] = m_ddot(fb->Hs[f], s->C) - 1.0;
            double st = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) st += fb->M1[f][r] * s->C[r * 3 + c] * fb->M1[f][c];
            s->Istar[f] = st;
            s->active[f] = st > 1.0;
        }
    }
}

static double law_psi(const orc_material *m, const orc_state *s) {
    if (m->law == 0)
        return 0.5 * m->mu * (s->I1 - 3.0 - 2.0 * s->lnJ) + m->lambda * s->lnJ * s->lnJ;
    double psi = 0.5 * m->mu * (s->j23 * s->I1 - 3.0) + 0.25 * m->kappa * (s->J * s->J - 1.0 - 2.0 * s->lnJ);
    if (m->law == 2)
        for (int f = 0; f < 2; ++f)
            if (s->active[f]) psi += m->k1 / (2.0 * m->k2) * (exp(m->k2 * s->Ei[f] * s->Ei[f]) - 1.0);
    return psi;
}

static void law_S(const orc_material *m, const orc_fibres *fb, const orc_state *s, double *S) {
    if (m->law == 0) {
        double a = m->mu - 2.0 * m->lambda * s->lnJ;
        for (int i = 0; i < 9; ++i) S[i] = -a * s->Cinv[i];
        S[0] += m->mu;
        S[4] += m->mu;
        S[8] += m->mu;
        return;
    }
    double c1 = 0.5 * m->kappa * (s->J * s->J - 1.0) - m->mu / 3.0 * s->j23 * s->I1;
    for (int i = 0; i < 9; ++i) S[i] = c1 * s->Cinv[i];
    S[0] += m->mu * s->j23;
    S[4] += m->mu * s->j23;
    S[8] += m->mu * s->j23;
    if (m->law == 2)
        for (int f = 0; f < 2; ++f)
            if (s->active[f]) {
                double E = s->Ei[f];
                double c = 2.0 * m->k1 * exp(m->k2 * E * E) * E;
                for (int i = 0; i < 9; ++i) S[i] += c * fb->Hs[f][i];
            }
}

/* directional derivative D_uS[H] at the state s (Appendix A) */
static void law_dS(const orc_material *m, const orc_fibres *fb, const orc_state *s, const double *H, double *dS) {
    double A[9], B[9], dCinv[9], dC[9];
    m_mul(s->Finv, H, A);       /* F^-1 H */
    m_mul(A, s->Cinv, B);       /* F^-1 H C^-1 */
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) dCinv[r * 3 + c] = -(B[r * 3 + c] + B[c * 3 + r]);
    double t = m_trace(A);      /* (1/J) D_uJ */
    if (m->law == 0) {
        double a = m->mu - 2.0 * m->lambda * s->lnJ;
        for (int i = 0; i < 9; ++i) dS[i] = -a * dCinv[i] + 2.0 * m->lambda * t * s->Cinv[i];
        return;
    }
    double FtH[9];
    m_tmul(s->F, H, FtH);
    double dI1 = 2.0 * m_trace(FtH);
    double c1 = 0.5 * m->kappa * (s->J * s->J - 1.0) - m->mu / 3.0 * s->j23 * s->I1;
    double c2 = 2.0 * m->mu / 9.0 * s->j23 * s->I1 + m->kappa * s->J * s->J;
    double cC = t * c2 - m->mu / 3.0 * s->j23 * dI1;
    for (int i = 0; i < 9; ++i) dS[i] = c1 * dCinv[i] + cC * s->Cinv[i];
    double cI = -2.0 * m->mu / 3.0 * s->j23 * t;
    dS[0] += cI;
    dS[4] += cI;
    dS[8] += cI;
    if (m->law == 2) {
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) dC[r * 3 + c] = FtH[r * 3 + c] + FtH[c * 3 + r];
        for (int f = 0; f < 2; ++f)
            if (s->active[f]) {
                double E = s->Ei[f];
                double c3 = 2.0 * m->k1 * exp(m->k2 * E * E);
                double cf = c3 * (2.0 * m->k2 * E * E + 1.0) * m_ddot(fb->Hs[f], dC);
                for (int i = 0; i < 9; ++i) dS[i] += cf * fb->Hs[f][i];
            }
    }
}

/* P = F S and dP = H S + F D_uS[H] */
static void law_P(const orc_material *m, const orc_fibres *fb, const orc_state *s, double *P) {
    double S[9];
    law_S(m, fb, s, S);
    m_mul(s->F, S, P);
}
static void law_dP(const orc_material *m, const orc_fibres *fb, const orc_state *s, const double *H, double *dP) {
    double S[9], dS[9], T1[9], T2[9];
    law_S(m, fb, s, S);
    law_dS(m, fb, s, H, dS);
    m_mul(H, S, T1);
    m_mul(s->F, dS, T2);
    for (int i = 0; i < 9; ++i) dP[i] = T1[i] + T2[i];
}

/* Spatial quantities of Sec. 5 ("spatial integration" paragraphs), from the
 * definitions: b = F F^T, the Kirchhoff stress tau = F S F^T written per law,
 * and the action of the pushed-forward moduli J c on a symmetric tensor e:
 *   cNH   tau = mu b - (mu - 2 lambda ln J) I
 *         Jc:e = 2 (mu - 2 lambda ln J) e + 2 lambda tr(e) I
 *   iNH   tau = mu J^-2/3 b + c1 I
 *         Jc:e = -2 c1 e + c2 tr(e) I - 2 mu/3 J^-2/3 [tr(e) b + (b:e) I]
 *   fiber tau += sum_i c3 E_i F H_i F^T
 *         Jc:e += sum_i 2 c3 (2 k2 E_i^2 + 1) [(F H_i F^T) : e] F H_i F^T
 * with c1, c2 of Sec. 5 and c3 = 2 k1 exp(k2 E_i^2) for an active family.
 * The iNH moduli are the push-forward of the material D_uS of App. A: its
 * I (x) C^-1 part maps to tr(e) b + (b:e) I (the Sec. 5 restatement prints
 * -4 mu/3 J^-2/3 tr(e) C instead; that form is not used). */
static void law_tau(const orc_material *m, const orc_fibres *fb, const orc_state *s, double *b, double *tau) {
    double Ft[9];
    m_transpose(s->F, Ft);
    m_mul(s->F, Ft, b);
    if (m->law == 0) {
        for (int i = 0; i < 9; ++i) tau[i] = m->mu * b[i];
        double a = m->mu - 2.0 * m->lambda * s->lnJ;
        tau[0] -= a;
        tau[4] -= a;
        tau[8] -= a;
        return;
    }
    double c1 = 0.5 * m->kappa * (s->J * s->J - 1.0) - m->mu / 3.0 * s->j23 * s->I1;
    for (int i = 0; i < 9; ++i) tau[i] = m->mu * s->j23 * b[i];
    tau[0] += c1;
    tau[4] += c1;
    tau[8] += c1;
    if (m->law == 2)
        for (int f = 0; f < 2; ++f)
            if (s->active[f]) {
                double E = s->Ei[f], FH[9], h[9];
                double c3 = 2.0 * m->k1 * exp(m->k2 * E * E);
                m_mul(s->F, fb->Hs[f], FH);
                m_mul(FH, Ft, h);
                for (int i = 0; i < 9; ++i) tau[i] += c3 * E * h[i];
            }
}

static void law_Jc(const orc_material *m, const orc_fibres *fb, const orc_state *s, const double *b,
                   const double *e, double *out) {
    double tr = m_trace(e);
    if (m->law == 0) {
        double a = m->mu - 2.0 * m->lambda * s->lnJ;
        for (int i = 0; i < 9; ++i) out[i] = 2.0 * a * e[i];
        out[0] += 2.0 * m->lambda * tr;
        out[4] += 2.0 * m->lambda * tr;
        out[8] += 2.0 * m->lambda * tr;
        return;
    }
    double c1 = 0.5 * m->kappa * (s->J * s->J - 1.0) - m->mu / 3.0 * s->j23 * s->I1;
    double c2 = 2.0 * m->mu / 9.0 * s->j23 * s->I1 + m->kappa * s->J * s->J;
    double g = 2.0 * m->mu / 3.0 * s->j23;
    double be = m_ddot(b, e);
    for (int i = 0; i < 9; ++i) out[i] = -2.0 * c1 * e[i] - g * tr * b[i];
    for (int d = 0; d < 3; ++d) out[d * 4] += c2 * tr - g * be;
    if (m->law == 2) {
        double Ft[9];
        m_transpose(s->F, Ft);
        for (int f = 0; f < 2; ++f)
            if (s->active[f]) {
                double E = s->Ei[f], FH[9], h[9];
                double c3 = 2.0 * m->k1 * exp(m->k2 * E * E);
                m_mul(s->F, fb->Hs[f], FH);
                m_mul(FH, Ft, h);
                double cf = 2.0 * c3 * (2.0 * m->k2 * E * E + 1.0) * m_ddot(h, e);
                for (int i = 0; i < 9; ++i) out[i] += cf * h[i];
            }
    }
}

/* spatial tangent integrand sigma = Jc:(g)^S + g tau for g = grad du */
static void law_spatial(const orc_material *m, const orc_fibres *fb, const orc_state *s, const double *g,
                        double *sigma) {
    double b[9], tau[9], e[9], gt[9];
    law_tau(m, fb, s, b, tau);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) e[r * 3 + c] = 0.5 * (g[r * 3 + c] + g[c * 3 + r]);
    law_Jc(m, fb, s, b, e, sigma);
    m_mul(g, tau, gt);
    for (int i = 0; i < 9; ++i) sigma[i] += gt[i];
}

/* Pointwise evaluation for the material pins: given F (and H), return
 * Psi, S, P and dP. frame may be NULL for the isotropic laws. Returns J. */
double orc_material_point(const orc_material *m, const double *frame, const double *F, const double *H,
                          double *psi, double *S, double *P, double *dP, double *aux) {
    orc_fibres fb;
    memset(&fb, 0, sizeof fb);
    if (m->law == 2 && frame) fibres_from_frame(m, frame, &fb);
    orc_state s;
    state_from_F(m, &fb, F, &s);
    if (psi) *psi = law_psi(m, &s);
    if (S) law_S(m, &fb, &s, S);
    if (P) law_P(m, &fb, &s, P);
    if (dP && H) law_dP(m, &fb, &s, H, dP);
    if (aux) { /* E_4, E_6, I*_4, I*_6, active flags */
        aux[0] = s.Ei[0];
        aux[1] = s.Ei[1];
        aux[2] = s.Istar[0];
        aux[3] = s.Istar[1];
        aux[4] = s.active[0];
        aux[5] = s.active[1];
    }
    return s.J;
}

/* ------------------------------------------------------------------ */
/* 1D Lagrange polynomials (product formula) and the 3D tables           */
/* ------------------------------------------------------------------ */
static double lag(const double *xs, int n, int a, double x) {
    double v = 1.0;
    for (int b = 0; b < n; ++b)
        if (b != a) v *= (x - xs[b]) / (xs[a] - xs[b]);
    return v;
}
static double lag_d(const double *xs, int n, int a, double x) {
    double s = 0.0;
    for (int m = 0; m < n; ++m) {
        if (m == a) continue;
        double v = 1.0 / (xs[a] - xs[m]);
        for (int b = 0; b < n; ++b)
            if (b != a && b != m) v *= (x - xs[b]) / (xs[a] - xs[b]);
        s += v;
    }
    return s;
}

/* Full 3D tables at the quadrature points: value N[q][a] and reference
 * gradient dN[q][a][3] of every tensor-product basis function a (nodes xs, n
 * per direction), evaluated at every tensor-product point q (points xq, nq per
 * direction). */
static void tabulate(const double *xs, int n, const double *xq, int nq, double *N, double *dN) {
    int nn = n * n * n, qq = nq * nq * nq;
    for (int qz = 0; qz < nq; ++qz)
        for (int qy = 0; qy < nq; ++qy)
            for (int qx = 0; qx < nq; ++qx) {
                int q = qx + nq * (qy + nq * qz);
                double X = xq[qx], Y = xq[qy], Z = xq[qz];
                for (int k = 0; k < n; ++k)
                    for (int j = 0; j < n; ++j)
                        for (int i = 0; i < n; ++i) {
                            int a = i + n * (j + n * k);
                            double li = lag(xs, n, i, X), lj = lag(xs, n, j, Y), lk = lag(xs, n, k, Z);
                            if (N) N[(size_t)q * nn + a] = li * lj * lk;
                            if (dN) {
                                double *d = dN + ((size_t)q * nn + a) * 3;
                                d[0] = lag_d(xs, n, i, X) * lj * lk;
                                d[1] = li * lag_d(xs, n, j, Y) * lk;
                                d[2] = li * lj * lag_d(xs, n, k, Z);
                            }
                        }
            }
    (void)qq;
}

typedef struct {
    int n, nn, nq, qq, ng, ngg;
    double *dN;   /* [qq][nn][3] FE basis reference gradients */
    double *dNg;  /* [qq][ngg][3] geometry basis reference gradients */
    double *W;    /* [qq] tensor weights */
    double *Nv;   /* [qq][nn] FE basis values */
} orc_tables;

static int tables_init(const orc_mesh *M, orc_tables *T) {
    T->n = M->p + 1;
    T->nn = T->n * T->n * T->n;
    T->nq = M->p + 1;
    T->qq = T->nq * T->nq * T->nq;
    T->ng = M->g + 1;
    T->ngg = T->ng * T->ng * T->ng;
    T->dN = (double *)malloc(sizeof(double) * (size_t)T->qq * T->nn * 3);
    T->dNg = (double *)malloc(sizeof(double) * (size_t)T->qq * T->ngg * 3);
    T->W = (double *)malloc(sizeof(double) * (size_t)T->qq);
    T->Nv = (double *)malloc(sizeof(double) * (size_t)T->qq * T->nn);
    if (!T->dN || !T->dNg || !T->W || !T->Nv) return -1;
    tabulate(M->xi_node, T->n, M->xi_q, T->nq, T->Nv, T->dN);
    tabulate(M->xi_geo, T->ng, M->xi_q, T->nq, NULL, T->dNg);
    for (int qz = 0; qz < T->nq; ++qz)
        for (int qy = 0; qy < T->nq; ++qy)
            for (int qx = 0; qx < T->nq; ++qx)
                T->W[qx + T->nq * (qy + T->nq * qz)] = M->w_q[qx] * M->w_q[qy] * M->w_q[qz];
    return 0;
}
static void tables_free(orc_tables *T) {
    free(T->dN);
    free(T->dNg);
    free(T->W);
    free(T->Nv);
}

/* Geometry at quadrature point q of element e: J0 = dX/dxi, returns
 * JxW and the physical gradients gX[a][3] of all FE basis functions. */
static double geometry_qp(const orc_mesh *M, const orc_tables *T, int e, int q, double *gX, double *J0out) {
    double J0[9] = {0}, J0i[9];
    const int32_t *gc = M->geo_conn + (size_t)e * T->ngg;
    for (int a = 0; a < T->ngg; ++a) {
        const double *X = M->geo_nodes + (size_t)gc[a] * 3;
        const double *d = T->dNg + ((size_t)q * T->ngg + a) * 3;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) J0[r * 3 + c] += X[r] * d[c];
    }
    double det = m_inv(J0, J0i);
    if (J0out) memcpy(J0out, J0, sizeof J0);
    if (gX) {
        for (int a = 0; a < T->nn; ++a) {
            const double *d = T->dN + ((size_t)q * T->nn + a) * 3;
            for (int b = 0; b < 3; ++b) /* dN/dX_b = sum_c dN/dxi_c (J0^-1)_{cb} */
                gX[a * 3 + b] = d[0] * J0i[0 * 3 + b] + d[1] * J0i[1 * 3 + b] + d[2] * J0i[2 * 3 + b];
        }
    }
    return det * T->W[q];
}

/* Grad v = sum_a v_a (x) dN_a/dX  for element-local values v[a][3] */
static void grad_local(const orc_tables *T, const double *gX, const double *v, double *G) {
    for (int i = 0; i < 9; ++i) G[i] = 0.0;
    for (int a = 0; a < T->nn; ++a)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) G[r * 3 + c] += v[a * 3 + r] * gX[a * 3 + c];
}

static void gather(const orc_mesh *M, const orc_tables *T, int e, const double *u, double *ue) {
    const int32_t *dc = M->dof_conn + (size_t)e * T->nn;
    for (int a = 0; a < T->nn; ++a)
        for (int c = 0; c < 3; ++c) ue[a * 3 + c] = u ? u[(size_t)dc[a] * 3 + c] : 0.0;
}

static void elem_fibres(const orc_mesh *M, const orc_material *m, int e, orc_fibres *fb) {
    memset(fb, 0, sizeof *fb);
    if (m->law == 2 && M->frames) fibres_from_frame(m, M->frames + (size_t)e * 9, fb);
}

/* ------------------------------------------------------------------ */
/* element kernels                                                      */
/* ------------------------------------------------------------------ */
enum { OP_RESIDUAL = 0, OP_APPLY = 1, OP_DIAG = 2, OP_APPLY_SPATIAL = 3 };

/* Element vector of the chosen operator; returns 0, or 1 if J <= 0 or
 * det J0 <= 0 was met at some quadrature point. */
static int element_vector(const orc_mesh *M, const orc_material *m, const orc_tables *T, int e, int op,
                          const double *u, const double *du, double *ve, double *work) {
    double *gX = work;                       /* nn*3 */
    double *ue = work + T->nn * 3;           /* nn*3 */
    double *due = work + T->nn * 6;          /* nn*3 */
    int bad = 0;
    orc_fibres fb;
    elem_fibres(M, m, e, &fb);
    gather(M, T, e, u, ue);
    if (op == OP_APPLY || op == OP_APPLY_SPATIAL) gather(M, T, e, du, due);
    for (int i = 0; i < T->nn * 3; ++i) ve[i] = 0.0;
    for (int q = 0; q < T->qq; ++q) {
        double J0[9];
        double JxW = geometry_qp(M, T, e, q, gX, J0);
        if (m_det(J0) <= 0.0) bad = 1;
        double Gu[9], F[9];
        grad_local(T, gX, ue, Gu);
        for (int i = 0; i < 9; ++i) F[i] = Gu[i];
        F[0] += 1.0;
        F[4] += 1.0;
        F[8] += 1.0;
        orc_state s;
        state_from_F(m, &fb, F, &s);
        if (!(s.J > 0.0)) bad = 1;
        if (op == OP_RESIDUAL || op == OP_APPLY) {
            double P[9];
            if (op == OP_RESIDUAL) {
                law_P(m, &fb, &s, P);
            } else {
                double H[9];
                grad_local(T, gX, due, H);
                law_dP(m, &fb, &s, H, P);
            }
            for (int a = 0; a < T->nn; ++a)
                for (int r = 0; r < 3; ++r)
                    ve[a * 3 + r] += JxW * (P[r * 3 + 0] * gX[a * 3 + 0] + P[r * 3 + 1] * gX[a * 3 + 1] +
                                            P[r * 3 + 2] * gX[a * 3 + 2]);
        } else if (op == OP_APPLY_SPATIAL) {
            /* g = grad du = (Grad du) F^-1; test gradients dN_j/dx = F^-T dN_j/dX */
            double H[9], g[9], sig[9];
            grad_local(T, gX, due, H);
            m_mul(H, s.Finv, g);
            law_spatial(m, &fb, &s, g, sig);
            for (int a = 0; a < T->nn; ++a) {
                double gx[3];
                for (int d = 0; d < 3; ++d)
                    gx[d] = gX[a * 3 + 0] * s.Finv[0 * 3 + d] + gX[a * 3 + 1] * s.Finv[1 * 3 + d] +
                            gX[a * 3 + 2] * s.Finv[2 * 3 + d];
                for (int r = 0; r < 3; ++r)
                    ve[a * 3 + r] += JxW * (sig[r * 3 + 0] * gx[0] + sig[r * 3 + 1] * gx[1] + sig[r * 3 + 2] * gx[2]);
            }
        } else { /* OP_DIAG: K_e[(a,r),(a,r)] with H = e_r (x) dN_a/dX */
            for (int a = 0; a < T->nn; ++a)
                for (int r = 0; r < 3; ++r) {
                    double H[9] = {0}, dP[9];
                    for (int c = 0; c < 3; ++c) H[r * 3 + c] = gX[a * 3 + c];
                    law_dP(m, &fb, &s, H, dP);
                    ve[a * 3 + r] += JxW * (dP[r * 3 + 0] * gX[a * 3 + 0] + dP[r * 3 + 1] * gX[a * 3 + 1] +
                                            dP[r * 3 + 2] * gX[a * 3 + 2]);
                }
        }
    }
    return bad;
}

static int64_t list_len(const orc_mesh *M, const int32_t *elems, int n_list) {
    return elems ? n_list : M->n_elem;
}

/* Run an element operator over all elements (elems == NULL) or over the
 * listed ones, and sum the element vectors into out[n_nodes*3] in list
 * order. Returns the number of elements with a non-invertible point. */
static int run_vector_op(const orc_mesh *M, const orc_material *m, int op, const double *u, const double *du,
                         double *out, const int32_t *elems, int n_list) {
    orc_tables T;
    if (tables_init(M, &T)) return -1;
    int64_t ne = list_len(M, elems, n_list);
    size_t vl = (size_t)T.nn * 3;
    double *V = (double *)malloc(sizeof(double) * vl * (size_t)(ne > 0 ? ne : 1));
    int nbad = 0;
#pragma omp parallel reduction(+ : nbad)
    {
        double *work = (double *)malloc(sizeof(double) * (size_t)T.nn * 9);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < ne; ++i) {
            int e = elems ? elems[i] : (int)i;
            nbad += element_vector(M, m, &T, e, op, u, du, V + vl * (size_t)i, work);
        }
        free(work);
    }
    memset(out, 0, sizeof(double) * (size_t)M->n_nodes * 3);
    for (int64_t i = 0; i < ne; ++i) {
        int e = elems ? elems[i] : (int)i;
        const int32_t *dc = M->dof_conn + (size_t)e * T.nn;
        for (int a = 0; a < T.nn; ++a)
            for (int c = 0; c < 3; ++c) out[(size_t)dc[a] * 3 + c] += V[vl * (size_t)i + a * 3 + c];
    }
    free(V);
    tables_free(&T);
    return nbad;
}

int orc_residual(const orc_mesh *M, const orc_material *m, const double *u, double *r, const int32_t *elems,
                 int n_list) {
    return run_vector_op(M, m, OP_RESIDUAL, u, NULL, r, elems, n_list);
}

int orc_apply(const orc_mesh *M, const orc_material *m, const double *u, const double *du, double *out,
              const int32_t *elems, int n_list) {
    return run_vector_op(M, m, OP_APPLY, u, du, out, elems, n_list);
}

int orc_apply_spatial(const orc_mesh *M, const orc_material *m, const double *u, const double *du, double *out,
                      const int32_t *elems, int n_list) {
    return run_vector_op(M, m, OP_APPLY_SPATIAL, u, du, out, elems, n_list);
}

int orc_diagonal(const orc_mesh *M, const orc_material *m, const double *u, double *diag, const int32_t *elems,
                 int n_list) {
    return run_vector_op(M, m, OP_DIAG, u, NULL, diag, elems, n_list);
}

/* Dense element matrices K_e[(a,r),(b,c)] (row = test function a, component
 * r; column = trial function b, component c), one per listed element,
 * written to Ke[n_list][3nn][3nn]. */
int orc_assemble(const orc_mesh *M, const orc_material *m, const double *u, double *Ke, const int32_t *elems,
                 int n_list) {
    orc_tables T;
    if (tables_init(M, &T)) return -1;
    int64_t ne = list_len(M, elems, n_list);
    size_t nd = (size_t)T.nn * 3;
    int nbad = 0;
#pragma omp parallel reduction(+ : nbad)
    {
        double *gX = (double *)malloc(sizeof(double) * nd);
        double *ue = (double *)malloc(sizeof(double) * nd);
        double *A = (double *)malloc(sizeof(double) * 81);
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < ne; ++i) {
            int e = elems ? elems[i] : (int)i;
            double *K = Ke + nd * nd * (size_t)i;
            memset(K, 0, sizeof(double) * nd * nd);
            orc_fibres fb;
            elem_fibres(M, m, e, &fb);
            gather(M, &T, e, u, ue);
            for (int q = 0; q < T.qq; ++q) {
                double J0[9];
                double JxW = geometry_qp(M, &T, e, q, gX, J0);
                double Gu[9], F[9];
                grad_local(&T, gX, ue, Gu);
                for (int k = 0; k < 9; ++k) F[k] = Gu[k];
                F[0] += 1.0;
                F[4] += 1.0;
                F[8] += 1.0;
                orc_state s;
                state_from_F(m, &fb, F, &s);
                if (!(s.J > 0.0) || m_det(J0) <= 0.0) nbad++;
                /* fourth-order tangent A[(r,d),(c,f)] = dP_rd / dF_cf */
                for (int c = 0; c < 3; ++c)
                    for (int f = 0; f < 3; ++f) {
                        double H[9] = {0}, dP[9];
                        H[c * 3 + f] = 1.0;
                        law_dP(m, &fb, &s, H, dP);
                        for (int k = 0; k < 9; ++k) A[k * 9 + c * 3 + f] = dP[k];
                    }
                for (int a = 0; a < T.nn; ++a)
                    for (int r = 0; r < 3; ++r) {
                        size_t row = (size_t)a * 3 + r;
                        for (int b = 0; b < T.nn; ++b)
                            for (int c = 0; c < 3; ++c) {
                                double s2 = 0.0;
                                for (int d = 0; d < 3; ++d)
                                    for (int f = 0; f < 3; ++f)
                                        s2 += gX[a * 3 + d] * A[(r * 3 + d) * 9 + c * 3 + f] * gX[b * 3 + f];
                                K[row * nd + (size_t)b * 3 + c] += JxW * s2;
                            }
                    }
            }
        }
        free(gX);
        free(ue);
        free(A);
    }
    tables_free(&T);
    return nbad;
}

/* Total strain energy Pi(u) = sum_e sum_q JxW Psi(F) (summed in element order). */
double orc_energy(const orc_mesh *M, const orc_material *m, const double *u) {
    orc_tables T;
    if (tables_init(M, &T)) return NAN;
    double *Pe = (double *)malloc(sizeof(double) * (size_t)(M->n_elem > 0 ? M->n_elem : 1));
#pragma omp parallel
    {
        double *gX = (double *)malloc(sizeof(double) * (size_t)T.nn * 3);
        double *ue = (double *)malloc(sizeof(double) * (size_t)T.nn * 3);
#pragma omp for schedule(dynamic, 4)
        for (int e = 0; e < M->n_elem; ++e) {
            orc_fibres fb;
            elem_fibres(M, m, e, &fb);
            gather(M, &T, e, u, ue);
            double acc = 0.0;
            for (int q = 0; q < T.qq; ++q) {
                double JxW = geometry_qp(M, &T, e, q, gX, NULL);
                double Gu[9], F[9];
                grad_local(&T, gX, ue, Gu);
                for (int k = 0; k < 9; ++k) F[k] = Gu[k];
                F[0] += 1.0;
                F[4] += 1.0;
                F[8] += 1.0;
                orc_state s;
                state_from_F(m, &fb, F, &s);
                acc += JxW * law_psi(m, &s);
            }
            Pe[e] = acc;
        }
        free(gX);
        free(ue);
    }
    double tot = 0.0;
    for (int e = 0; e < M->n_elem; ++e) tot += Pe[e];
    free(Pe);
    tables_free(&T);
    return tot;
}

/* Physical coordinates of every DoF node (the geometry map evaluated at the
 * nodal points), X[n_nodes][3]; nodes shared by elements are written by each
 * owner (identical for a conforming geometry). */
int orc_node_coords(const orc_mesh *M, double *X) {
    int n = M->p + 1, nn = n * n * n, ng = M->g + 1, ngg = ng * ng * ng;
    double *Ng = (double *)malloc(sizeof(double) * (size_t)nn * ngg);
    if (!Ng) return -1;
    /* geometry basis values at the FE nodal points */
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < ng; ++c)
                    for (int b = 0; b < ng; ++b)
                        for (int a = 0; a < ng; ++a)
                            Ng[(size_t)(i + n * (j + n * k)) * ngg + a + ng * (b + ng * c)] =
                                lag(M->xi_geo, ng, a, M->xi_node[i]) * lag(M->xi_geo, ng, b, M->xi_node[j]) *
                                lag(M->xi_geo, ng, c, M->xi_node[k]);
#pragma omp parallel for schedule(static)
    for (int e = 0; e < M->n_elem; ++e) {
        const int32_t *gc = M->geo_conn + (size_t)e * ngg;
        const int32_t *dc = M->dof_conn + (size_t)e * nn;
        for (int a = 0; a < nn; ++a) {
            double x[3] = {0, 0, 0};
            for (int b = 0; b < ngg; ++b)
                for (int d = 0; d < 3; ++d) x[d] += Ng[(size_t)a * ngg + b] * M->geo_nodes[(size_t)gc[b] * 3 + d];
            for (int d = 0; d < 3; ++d) X[(size_t)dc[a] * 3 + d] = x[d];
        }
    }
    free(Ng);
    return 0;
}

/* Per-quadrature-point geometry and deformation for the listed elements:
 * JxW[i][qq], J0[i][qq][9], F[i][qq][9]. */
int orc_qp_fields(const orc_mesh *M, const double *u, const int32_t *elems, int n_list, double *JxW_out,
                  double *J0_out, double *F_out) {
    orc_tables T;
    if (tables_init(M, &T)) return -1;
    double *gX = (double *)malloc(sizeof(double) * (size_t)T.nn * 3);
    double *ue = (double *)malloc(sizeof(double) * (size_t)T.nn * 3);
    for (int i = 0; i < n_list; ++i) {
        int e = elems[i];
        gather(M, &T, e, u, ue);
        for (int q = 0; q < T.qq; ++q) {
            double J0[9], Gu[9];
            double jw = geometry_qp(M, &T, e, q, gX, J0);
            grad_local(&T, gX, ue, Gu);
            size_t o = (size_t)i * T.qq + q;
            if (JxW_out) JxW_out[o] = jw;
            if (J0_out) memcpy(J0_out + o * 9, J0, sizeof J0);
            if (F_out) {
                for (int k = 0; k < 9; ++k) F_out[o * 9 + k] = Gu[k];
                F_out[o * 9 + 0] += 1.0;
                F_out[o * 9 + 4] += 1.0;
                F_out[o * 9 + 8] += 1.0;
            }
        }
    }
    free(gX);
    free(ue);
    tables_free(&T);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Load vector of a constant body force b: f_{j,a} = sum_e sum_q JxW_q N_j(q) b_a
 * (the (v, B) term of the residual, Sec. 2), summed in element order. */
int orc_body_force(const orc_mesh *M, const double *b, double *f) {
    orc_tables T;
    if (tables_init(M, &T)) return -1;
    memset(f, 0, sizeof(double) * (size_t)M->n_nodes * 3);
    int nbad = 0;
    for (int e = 0; e < M->n_elem; ++e) {
        const int32_t *dc = M->dof_conn + (size_t)e * T.nn;
        for (int q = 0; q < T.qq; ++q) {
            double J0[9];
            double JxW = geometry_qp(M, &T, e, q, NULL, J0);
            if (m_det(J0) <= 0.0) nbad = 1;
            for (int a = 0; a < T.nn; ++a) {
                double w = JxW * T.Nv[(size_t)q * T.nn + a];
                for (int c = 0; c < 3; ++c) f[(size_t)dc[a] * 3 + c] += w * b[c];
            }
        }
    }
    tables_free(&T);
    return nbad;
}
