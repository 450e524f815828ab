// Vector kernels of the solver layer (hx_vec.cu); asynchronous on stream s.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hx.h"

namespace hx {

constexpr int RED_BLOCKS = 512;  // fixed reduction grid (deterministic sums)

struct CgScalars {
    double rz, pAp, alpha, beta, rr;
    int bad;
};

cudaError_t copy_idx(const int64_t *idx, int64_t n, const void *src, void *dst, int prec, cudaStream_t s);
cudaError_t set_idx(const int64_t *idx, int64_t n, double val, void *dst, int prec, cudaStream_t s);
cudaError_t cheb_update(int64_t n, const void *rhs, const void *Kx, const void *dinv, void *d, void *x, double cd,
                        double cr, int first, int prec, cudaStream_t s);
// out[j] = a_j . b_j for j < k (k <= 3); partial holds 3*RED_BLOCKS doubles
cudaError_t dots(int64_t n, int k, const double *a0, const double *b0, const double *a1, const double *b1,
                 const double *a2, const double *b2, double *partial, double *out, cudaStream_t s);
cudaError_t cg_alpha(CgScalars *sc, cudaStream_t s);
cudaError_t cg_xr(int64_t n, const CgScalars *sc, const double *p, const double *Ap, double *x, double *r, float *r32,
                  cudaStream_t s);
cudaError_t cg_beta(CgScalars *sc, const double *dots3, cudaStream_t s);
cudaError_t cg_p(int64_t n, const CgScalars *sc, const double *z, double *p, double *zold, cudaStream_t s);
cudaError_t to_f32(int64_t n, const double *a, float *b, cudaStream_t s);
cudaError_t to_f64(int64_t n, const float *a, double *b, cudaStream_t s);
cudaError_t sub(int64_t n, const double *a, const double *b, double *y, cudaStream_t s);
// y = a x + b y (b == 0: y = a x)
cudaError_t axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t s);
cudaError_t normalize(int64_t n, const double *nrm2, const double *x, double *y, cudaStream_t s);
cudaError_t scale(int64_t n, const double *dinv, const double *x, double *y, cudaStream_t s);
cudaError_t invert(int64_t n, const void *x, void *y, int prec, cudaStream_t s);
cudaError_t random_vec(int64_t n, uint64_t seed, double *y, cudaStream_t s);
// y = a x + b y in precision prec (b == 0: y = a x)
cudaError_t axpby_p(int64_t n, double a, const void *x, double b, void *y, int prec, cudaStream_t s);

// Transfer between two Lagrange spaces on the same structured box of
// nx*ny*nz elements (degrees ps and pd). M[a_d][a_s] = l^s_{a_s}(xi^d_{a_d}),
// the source's 1D basis at the destination's 1D nodes. interp: every
// destination node takes the source function's value there, evaluated in its
// lowest-index element (exact for a continuous source; add != 0 adds it).
// interp_t: the transpose, dst_src += M^T src_dst, through atomic adds (dst
// zeroed by the caller).
struct InterpTab {
    int ps, pd;
    double M[7][7];
};
cudaError_t interp(const InterpTab &t, int nx, int ny, int nz, const void *src, void *dst, int add, int prec,
                   cudaStream_t s);
cudaError_t interp_t(const InterpTab &t, int nx, int ny, int nz, const void *src_fine, void *dst_coarse, int prec,
                     cudaStream_t s);
cudaError_t fma_probe(int prec, int sm_count, double *flops);

// h-transfers between degree-1 spaces on a structured box of nxc*nyc*nzc
// elements (coarse) and its 2x refinement in index space (fine: 2nxc*2nyc*2nzc
// elements; node lattices x fastest). A coarse lattice node (i, j, k) sits at
// fine lattice node (2i, 2j, 2k), and a coarse function is carried to the
// fine nodes by trilinear interpolation in lattice coordinates (weights 1 and
// 1/2 per direction).
// h_prolong: xf (+)= P xc (add != 0 adds); h_restrict: bc = P^T rf (a 27-point
// gather per coarse node, no atomics); h_inject: uc = uf at the shared nodes.
cudaError_t h_prolong(int nxc, int nyc, int nzc, const void *xc, void *xf, int add, int prec, cudaStream_t s);
cudaError_t h_restrict(int nxc, int nyc, int nzc, const void *rf, void *bc, int prec, cudaStream_t s);
cudaError_t h_inject(int nxc, int nyc, int nzc, const double *uf, double *uc, cudaStream_t s);
// Coarse solve: x = the Jacobi-preconditioned CG iterate (FP64, one CTA) for
// A x = b from x = 0, with A the dense column-major n x n matrix (n <=
// COARSE_MAX), dinv its inverse diagonal; stops after max_iter iterations or
// once ||r|| <= tol ||b|| or at non-positive curvature; b and x in `prec`.
// iters (device int, may be null) receives the iterations taken.
constexpr int COARSE_MAX = 1024;
cudaError_t coarse_pcg(int n, const double *A, const double *dinv, const void *b, void *x, int max_iter, double tol,
                       int *iters, int prec, cudaStream_t s);

// ---- batched CG: the meshes of a batch iterate in lockstep -----------------
// Every batched vector is the concatenation of per-mesh segments; mesh i owns
// [off, off + n) (off a multiple of 4). Kernels run on a (blocks, meshes)
// grid; per-mesh scalars stay on the device.
struct BSeg {
    int64_t off, n;
    double *x;            // the caller's solution vector of mesh i
    const double *rhs;    // the caller's right-hand side of mesh i
    const int64_t *cidx;  // constrained DoFs of mesh i (local indices)
    int64_t ncon;
};
struct BScal {
    double rz, pAp, alpha, beta, rr, bb, tol2;
    int active, bad, iters;
};
constexpr int BRB = 64;  // reduction blocks per mesh (fixed: repeatable sums)
// dots[3 i + j] = a_j . b_j over mesh i's segment, j < k (k <= 3)
// (sc non-null: meshes that are no longer active are skipped, here and below)
cudaError_t bdots(int nm, const BSeg *seg, int k, const double *a0, const double *b0, const double *a1,
                  const double *b1, const double *a2, const double *b2, double *partial, double *dots,
                  const BScal *sc, cudaStream_t s);
// y = x_i (gather, dir 0) or x_i = y (scatter, dir 1) / y = rhs_i (dir 2)
cudaError_t bcopy(int nm, int64_t max_n, const BSeg *seg, double *y, int dir, cudaStream_t s);
// out[cidx] = du[cidx] on every mesh's constrained DoFs (identity rows)
cudaError_t bcopy_idx(int nm, const BSeg *seg, const void *du, void *out, int prec, const BScal *sc, cudaStream_t s);
// y = a - b over the concatenation
cudaError_t bsub(int64_t n, const double *a, const double *b, double *y, cudaStream_t s);
// scalars after the initial residual: rz = dots[0], rr = dots[1], bb = dots[2]
cudaError_t bscal_init(int nm, BScal *sc, const double *dots, double tol, cudaStream_t s);
cudaError_t bscal_alpha(int nm, BScal *sc, const double *dots, cudaStream_t s);
// x += alpha p, r -= alpha Ap per mesh; r32 = (float) r if non-null
cudaError_t bxr(int nm, int64_t max_n, const BSeg *seg, const BScal *sc, const double *p, const double *Ap, double *x,
                double *r, float *r32, cudaStream_t s);
cudaError_t bscal_beta(int nm, BScal *sc, const double *dots, cudaStream_t s);
// p = z + beta p, zold = z per mesh
cudaError_t bp(int nm, int64_t max_n, const BSeg *seg, const BScal *sc, const double *z, double *p, double *zold,
               cudaStream_t s);
// Chebyshev step `step` of the per-mesh coefficients coef[(i * degree + step) * 2 + {cd, cr}]:
// r = dinv (rhs - Kx) (Kx null: dinv rhs), d = cd d + cr r (step 0: cr r), x += d (step 0 with Kx null: x = d)
cudaError_t bcheb(int nm, int64_t max_n, const BSeg *seg, const double *coef, int degree, int step, const void *rhs,
                  const void *Kx, const void *dinv, void *d, void *x, int prec, const BScal *sc, cudaStream_t s);

// Ordered assembly (deterministic scatter): E holds every element's local
// vector, E[3 (e NQ + a) + c] for local node a = i + n (j + n k), n = p + 1.
// out[3 I + c] = the sum over the elements containing node I, taken in
// ascending element order, of their entries at I; constrained DoFs (dmask)
// get 0. gather_box: structured box of nx*ny*nz elements (node lattice x
// fastest); gather_csr: any mesh, with ptr[I]..ptr[I+1] indexing slot[] =
// e*NQ + a in ascending order.
cudaError_t gather_box(int64_t n_nodes, int p, int nx, int ny, int nz, const void *E, const uint8_t *dmask, void *out,
                       int prec, cudaStream_t s);
cudaError_t gather_csr(int64_t n_nodes, const int64_t *ptr, const int64_t *slot, const void *E, const uint8_t *dmask,
                       void *out, int prec, cudaStream_t s);

}  // namespace hx
