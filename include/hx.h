/*
 * hx.h -- C ABI of the GB300 library for matrix-free hyperelastic operators
 * on hexahedral Q_p elements (arXiv 2408.12479, "Matrix-Free Higher-Order
 * Finite Element Methods for Hyperelasticity").
 *
 * The library evaluates, matrix-free and with sum factorization,
 *   the nonlinear residual  R(u)_i = (Grad N_i, P(F))_Omega0        Sec. 2, Eq. (mom_bal_nonlinear_material_residual)
 *   the tangent action      K(u_k) du = (Grad N_i, Grad du S + F D_uS[Grad du])   Sec. 2, Eq. (DDu_residual_material)
 * for three laws (Sec. 3): compressible neo-Hookean (cNH, Eq. NH_compressible),
 * nearly incompressible neo-Hookean (iNH, Eq. NH_nearly_incompressible) and the
 * two-family dispersed fibre model (fiber, Eq. fiber_Psi), in FP64 or FP32,
 * with the quadrature-point storage strategies of Sec. 5 / Table 2.
 *
 * Discretisation: Lagrange polynomials of degree p on the p+1
 * Gauss-Lobatto-Legendre points per direction, (p+1)^3 Gauss-Legendre
 * quadrature points per element, geometry given by trilinear (8 vertices) or
 * triquadratic (27 nodes, equispaced parameter points) element maps.
 *
 * Conventions for every call:
 *  - Pointers named *_dev are device pointers owned by the caller; *_host are
 *    host pointers owned by the caller. The library copies what it keeps.
 *  - A DoF vector holds 3*n_nodes values, node-major: component c of node I
 *    at index 3*I+c. Its scalar type follows the call's hx_prec (double for
 *    HX_FP64, float for HX_FP32). Vectors must be 16-byte aligned.
 *  - Calls are asynchronous on the context's CUDA stream. Argument errors are
 *    returned synchronously. Device-side errors (a quadrature point with
 *    J <= 0 or det J0 <= 0, a NaN state) set a device flag that hx_sync()
 *    and hx_precompute_qp() (on its next call) turn into a status.
 *  - The library never traps or aborts: every failure is a status, and
 *    hx_last_error() gives a one-line message.
 *  - Constrained DoFs (Dirichlet mask): residual rows are zero; tangent and
 *    diagonal rows are the identity (out_i = du_i, diag_i = 1); the operator
 *    sees constrained entries of du as zero.
 *  - Calls that work on a mesh or context expect its device to be current on
 *    the calling thread. Calls that select a device themselves (hx_create,
 *    hx_setup_mesh, hx_measure_fma_peak, the first
 *    hx_chebyshev_smooth_noalloc call on a device) make it current only while
 *    they run and restore the caller's current device before returning.
 */
#ifndef HX_H
#define HX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hx_ctx hx_ctx;   /* device, stream, error string */
typedef struct hx_mesh hx_mesh; /* device mesh, geometry, qp cache, workspace */
typedef struct hx_batch hx_batch;

typedef enum {
    HX_OK = 0,
    HX_ERR_ARG = 1,            /* invalid argument (null pointer, size, enum) */
    HX_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    HX_ERR_NONINVERTIBLE = 3,  /* J <= 0 or det J0 <= 0 at some quadrature point */
    HX_ERR_NOT_READY = 4,      /* tangent/diagonal needs hx_precompute_qp first */
    HX_ERR_TIMEOUT = 5,        /* hx_sync waited longer than its limit */
    HX_ERR_NOT_CONVERGED = 6,  /* iterative solver hit its iteration limit */
    HX_ERR_NAN = 7,            /* a NaN/Inf met in the state or in a solver scalar */
    HX_ERR_UNSUPPORTED = 8     /* degree/law/storage combination not built */
} hx_status;

typedef enum { HX_CNH = 0, HX_INH = 1, HX_FIBER = 2 } hx_law;
typedef enum { HX_FP64 = 0, HX_FP32 = 1 } hx_prec;

/* Storage strategies of Sec. 5 (material configuration), refreshed by
 * hx_precompute_qp once per Newton state (Alg. 1, "update quadrature point
 * data"):
 *   HX_RECOMPUTE      nothing per qp but the geometry; the tangent re-reads
 *                     u_k and rebuilds F, F^-1, C^-1, J-1, ln J, J^-2/3 and S
 *                     at every quadrature point ("on-the-fly", stage i);
 *   HX_CACHE_F        Grad u_k (= F - I) and the law's scalars (1/J and ln J
 *                     for cNH; 1/J, J^-2/3, c1, c2 and the stress scalar for
 *                     iNH; plus the fibre factors for fiber) -- stage ii;
 *   HX_CACHE_TENSORS  F - I, F^-1, C^-1, S and the tangent scalars -- the
 *                     paper's stage iii "scalars and tensors".
 * Geometry (J0^-1 and JxW per qp) is stored once at mesh setup for all three.
 *   HX_SPATIAL_TENSORS integration over the spatial configuration (Sec. 2,
 *                     Eq. stress_term_in_Ot_with_JC; Sec. 5 "spatial
 *                     integration" paragraphs; Table 2, Omega_t, tensors):
 *                     the tangent is (grad v, Jc:(grad du)^S + (grad du) tau)
 *                     over Omega_0 with grad = Grad F^-1. Stored per qp: the
 *                     inverse deformed mapping J_t^-1 = J0^-1 F^-1 and the
 *                     symmetric tensors and scalars of tau and Jc, scaled by
 *                     JxW (17 fields for cNH, 23 iNH, 35 fiber); the stored
 *                     geometry is not read. */
typedef enum { HX_RECOMPUTE = 0, HX_CACHE_F = 1, HX_CACHE_TENSORS = 2, HX_SPATIAL_TENSORS = 3 } hx_storage;

/* Material parameters (Sec. 3, Table 1). lambda is used by cNH only (note
 * Psi_cNH = mu/2(I1 - 3 - 2 ln J) + lambda ln^2 J, so the small-strain Lame
 * constant is 2 lambda). kappa is the bulk modulus of iNH/fiber. For fiber:
 * k1, k2 of the exponential fibre energy, dispersion (a, b) from which H11,
 * H22, H33 are computed (see hx_fibre_dispersion), and phi the mean in-plane
 * fibre angle in radians (family 4 at +phi, family 6 at -phi). */
typedef struct {
    int32_t law; /* hx_law */
    double mu, lambda, kappa;
    double k1, k2, a, b, phi;
} hx_material;

/* Mesh description (host arrays, copied by hx_setup_mesh).
 *  geo_nodes   [n_geo_nodes][3] vertex (g = 1) or node (g = 2) coordinates
 *  geo_conn    [n_elem][(g+1)^3] geometry node ids, lexicographic xi1 fastest
 *  dof_conn    [n_elem][(p+1)^3] DoF node ids, lexicographic xi1 fastest;
 *              may be NULL for a structured box (nx, ny, nz > 0), in which
 *              case element (ex,ey,ez) = ex + nx*(ey + ny*ez) owns nodes
 *              (ex*p+i) + (nx*p+1)*((ey*p+j) + (ny*p+1)*(ez*p+k))
 *  dirichlet   [3*n_nodes] 1 = constrained DoF, or NULL for none
 *  fibre_frames[n_elem][9] (E1 circumferential, E2 longitudinal, E3 radial)
 *              per element, required for HX_FIBER, ignored otherwise. */
typedef struct {
    int32_t n_elem;
    int32_t p;          /* 1..6 */
    int32_t geo_degree; /* 1 or 2 */
    int64_t n_nodes;
    const double *geo_nodes;
    int64_t n_geo_nodes;
    const int32_t *geo_conn;
    const int32_t *dof_conn;
    int32_t nx, ny, nz;
    const uint8_t *dirichlet;
    const double *fibre_frames;
} hx_mesh_desc;

/* ---- context ------------------------------------------------------------ */
/* Create a context on `device`, issuing all work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). */
hx_status hx_create(hx_ctx **ctx, int device, void *cuda_stream);
void hx_destroy(hx_ctx *ctx);
/* Rebind the context to another stream (subsequent calls only). */
hx_status hx_set_stream(hx_ctx *ctx, void *cuda_stream);
/* Message of the last failing call on this context ("" if none). */
const char *hx_last_error(hx_ctx *ctx);
/* Wait (polling, at most timeout_ms; <0 = no limit) for the context's stream,
 * then report device-side errors: HX_ERR_NONINVERTIBLE / HX_ERR_NAN, else
 * HX_OK. The device flag is cleared once reported. HX_ERR_TIMEOUT leaves the
 * work running. */
hx_status hx_sync(hx_ctx *ctx, int timeout_ms);

/* ---- mesh --------------------------------------------------------------- */
/* Upload a mesh and compute the geometry at every quadrature point (J0^-1 and
 * JxW, FP64 and FP32 copies). Fails with HX_ERR_NONINVERTIBLE if some
 * quadrature point has det J0 <= 0 (mapping check, Sec. 6). Synchronous. */
hx_status hx_setup_mesh(hx_ctx *ctx, const hx_mesh_desc *desc, const hx_material *mat, hx_mesh **mesh);
void hx_destroy_mesh(hx_mesh *mesh);
/* Number of DoF nodes, elements and quadrature points of a mesh. */
hx_status hx_mesh_info(const hx_mesh *mesh, int64_t *n_nodes, int64_t *n_elem, int64_t *n_qp);
/* Physical coordinates of the DoF nodes (the geometry map at the GLL points),
 * X_dev[n_nodes][3] FP64 on the device. */
hx_status hx_node_coords(hx_mesh *mesh, double *X_dev);
/* Bytes the tangent apply streams per call for (storage, prec), counting the
 * two DoF vectors once each, the qp cache and the per-qp geometry; this is the
 * figure behind the HBM-roofline fraction. */
hx_status hx_apply_bytes(const hx_mesh *mesh, int32_t storage, int32_t prec, double *bytes);

/* ---- hot path ----------------------------------------------------------- */
/* Update the quadrature-point data at the Newton state u_dev (FP64 vector):
 * interpolate Grad u_k with sum factorization and store what the strategy
 * keeps, computed in FP64 (J-1 from the components of Grad u, ln J as
 * ln_{+1}(J-1), J^-2/3 exactly) and stored in store_prec. This is Alg. 1's
 * "update quadrature point data" (Sec. 5). The first call per mesh allocates
 * the cache (call it before any stream capture). Returns HX_ERR_ARG for a bad
 * argument, HX_ERR_CUDA if an allocation or launch fails, else HX_OK without
 * waiting: a J <= 0 or non-finite value met at a quadrature point sets the
 * mesh's device flag, which hx_sync reports. */
hx_status hx_precompute_qp(hx_mesh *mesh, const double *u_dev, int32_t store_prec, int32_t storage);

/* r = R(u) (Sec. 2), constrained rows zero. u_dev, r_dev in `prec`. The state
 * is recomputed from u at every quadrature point (no cache needed). */
hx_status hx_residual(hx_mesh *mesh, const void *u_dev, void *r_dev, int32_t prec);

/* out = K(u_k) du (Sec. 2, Eq. DDu_residual_material; Sec. 5 storage forms),
 * using the cache of the last hx_precompute_qp; `prec` must equal its
 * store_prec. du_dev and out_dev must not overlap. */
hx_status hx_tangent_apply(hx_mesh *mesh, const void *du_dev, void *out_dev, int32_t prec);

/* Same operator with host vectors; returns after the result is on the host.
 * Uses device staging buffers owned by the mesh. On a structured box (not
 * the fibre law, atomic assembly, at least four element layers) the work runs
 * in z-slabs of element layers on the context stream and two copy streams
 * owned by the mesh (created on the first call): the copy of a slab's node
 * layers to the device overlaps the apply of the slab before it, and node
 * layers that no later slab touches are copied back while the next slabs
 * run. Other meshes copy the whole vectors, apply and copy back, on the
 * context stream. du_host and out_host should be page-locked for the copies
 * to overlap. */
hx_status hx_tangent_apply_host(hx_mesh *mesh, const void *du_host, void *out_host, int32_t prec);
/* slabs = 0: hx_tangent_apply_host copies whole vectors on every mesh; 1
 * (default): slabs where they apply, at most the library's default count;
 * 2..8: at most that many slabs (fewer where the element layers or the
 * 16-byte alignment of the slab starts require). HX_ERR_ARG otherwise. */
hx_status hx_set_host_apply_slabs(hx_mesh *mesh, int32_t slabs);

/* Autotuner: time every compiled variant of the tangent apply for the mesh's
 * current cache at `prec` and keep the fastest for later hx_tangent_apply
 * calls. The variants differ in how the quadrature-point data arrives and in
 * the tile (elements per CTA):
 *   0, 1: per-thread loads one point ahead plus an L2 prefetch of the next
 *         tile (default tile, half tile);
 *   3, 4: bulk copies into shared memory one tile ahead, quadrature points
 *         taken in column order (default tile, half tile);
 *   2, 5: as 3/4 with a stage and an mbarrier per warp, where one warp
 *         holds whole elements (FP32, p <= 4: 32 / (p+1)^2 elements per
 *         warp below p = 4, one at p = 4; caching strategies): no phase
 *         waits for more than its own warp (small and large CTAs).
 * Returns the fastest index and the six mean times in ms (a variant that
 * cannot launch, e.g. a staged tile whose chunks would not be 16-byte aligned
 * or would not fit in shared memory, reports a negative time). Uses
 * du_dev/out_dev as scratch vectors of the mesh's size; synchronous. */
hx_status hx_autotune(hx_mesh *mesh, int32_t prec, const void *du_dev, void *out_dev, int32_t reps,
                      int32_t *best_variant, double times_ms[6]);
/* Pin the tangent-apply variant (0-5, as numbered by hx_autotune) used for the
 * mesh's `storage` cache at `prec`. HX_ERR_ARG for an unknown variant; a
 * variant that cannot launch on this mesh makes hx_tangent_apply return
 * HX_ERR_CUDA. */
hx_status hx_set_apply_variant(hx_mesh *mesh, int32_t prec, int32_t storage, int32_t variant);

/* How the operator kernels (tangent apply, residual, diagonal) of one mesh
 * assemble element contributions into the output vector.
 * HX_SCATTER_ATOMIC (default): atomic adds into the zeroed output. The order
 *   of the additions at a shared node varies between runs, so results agree
 *   only to rounding (each node sums at most 8 contributions on a box).
 * HX_SCATTER_ORDERED: each element stores its local vector into a
 *   mesh-owned element buffer (n_elem (p+1)^3 * 3 values, allocated on first
 *   use), and a second kernel sums every node's contributions in ascending
 *   element order: bitwise repeatable results, for one more pass over that
 *   buffer. On a connectivity mesh the first switch to ordered mode builds a
 *   node -> element list on the host (synchronous).
 * The batch apply and the multigrid levels keep atomic adds. The paper's
 * element loops are serial per MPI rank; this mode is the GPU's way to the
 * same fixed summation order (a conflict-free scatter without colouring).
 * HX_ERR_ARG for an unknown mode. */
typedef enum { HX_SCATTER_ATOMIC = 0, HX_SCATTER_ORDERED = 1 } hx_scatter;
hx_status hx_set_scatter_mode(hx_mesh *mesh, int32_t mode);

/* Test hook for the device-side wait limits (no counterpart in the paper):
 * with skip_stage_copies != 0 the staged apply variants (2-5) issue no bulk
 * copy, so their stage never fills and each CTA's bounded wait gives up after
 * wait_limit_cycles clock cycles (0 = the default, 2^32); the CTA then sets
 * the device timeout flag and returns, and the next hx_sync reports
 * HX_ERR_TIMEOUT. No fault or trap is raised and the context stays usable;
 * the output of such an apply is incomplete. Call again with 0, 0 to restore
 * normal operation. HX_ERR_ARG for a negative limit. */
hx_status hx_set_wait_test(hx_mesh *mesh, int32_t skip_stage_copies, int64_t wait_limit_cycles);

/* diag(K(u_k)), constrained entries 1 (needed by the Jacobi smoother,
 * Sec. 6); sum-factorized from the per-qp tangent blocks. */
hx_status hx_diagonal(hx_mesh *mesh, void *diag_dev, int32_t prec);

/* `degree` steps of Chebyshev-accelerated Jacobi on K x = rhs (Sec. 6,
 * smoother), in place on x, eigenvalue interval
 * [lambda_max/smoothing_range, lambda_max] of D^-1 K, inv_diag = D^-1.
 * zero_initial != 0 treats x as zero on entry (saves one operator apply).
 * Every step applies the tangent of the last hx_precompute_qp in `prec`. */
hx_status hx_chebyshev_smooth(hx_mesh *mesh, const void *rhs_dev, void *x_dev, const void *inv_diag_dev,
                              int32_t degree, double lambda_max, double smoothing_range, int32_t zero_initial,
                              int32_t prec);

/* hx_chebyshev_smooth without any device allocation. This entry point has no
 * counterpart in the paper; it exists for callers that cannot allocate device
 * memory while they run -- an application whose memory is fully reserved by
 * another framework's caching allocator, or a latency-critical loop where
 * cudaMalloc/cudaFree would synchronise the device. Same arguments and result
 * as hx_chebyshev_smooth; its two scratch vectors (the Chebyshev update and
 * K x) live in a file-scope device array of 2 * 1,048,576 doubles (16 MiB)
 * that every GPU loading the library holds until the process exits. Meshes
 * with more than 1,048,576 DoFs are rejected with HX_ERR_ARG. The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture. All calls share the array and it
 * keeps the last call's contents (every call overwrites what it reads), so
 * calls that overlap on the GPU -- on different streams or contexts of one
 * device -- race. No cudaMalloc, cudaFree or allocating library routine is
 * called. */
hx_status hx_chebyshev_smooth_noalloc(hx_mesh *mesh, const void *rhs_dev, void *x_dev, const void *inv_diag_dev,
                                      int32_t degree, double lambda_max, double smoothing_range,
                                      int32_t zero_initial, int32_t prec);

/* Largest eigenvalue of D^-1 K by `iters` power iterations from a seeded
 * random start (FP64, on the device); *out receives the Rayleigh quotient. */
hx_status hx_estimate_lambda_max(hx_mesh *mesh, const double *inv_diag_dev, int32_t iters, uint64_t seed,
                                 double *out);

/* FP64 preconditioned CG on K(u_k) x = rhs (constrained operator), with a
 * Chebyshev(degree)-Jacobi preconditioner applied in precond_prec (Sec. 6:
 * FP64 outer Krylov, FP32 preconditioner). x_dev holds the start and
 * receives the solution; stops when ||rhs - K x|| <= tol ||rhs|| (true
 * residual rechecked at exit) or after max_iter iterations
 * (HX_ERR_NOT_CONVERGED). One iteration runs as a captured CUDA graph.
 * Requires hx_precompute_qp at FP64 and, for an FP32 preconditioner, at FP32
 * as well (both caches are kept). */
typedef struct {
    int32_t degree;            /* Chebyshev degree (0 = plain Jacobi) */
    double lambda_max;         /* upper eigenvalue bound of D^-1 K */
    double smoothing_range;    /* lambda_min = lambda_max / range */
    int32_t precond_prec;      /* hx_prec */
    int32_t use_graph;         /* capture one iteration in a CUDA graph */
} hx_cg_options;
hx_status hx_cg_solve(hx_mesh *mesh, const double *rhs_dev, double *x_dev, double tol, int32_t max_iter,
                      const hx_cg_options *opt, int32_t *iters, double *rel_residual);

/* Pointwise evaluation of the mesh's law for the forward-stability study
 * (Sec. 7.1): at n displacement gradients G (Grad u) and directions H, all
 * FP64 device arrays [n][9] row-major, compute S, P = F S and dP = H S +
 * F D_uS[H] ([n][9], FP64 device) in precision `prec` (inputs rounded to it
 * first). form 0: the stable forms of Sec. 4 (J-1 from the components of G,
 * ln J = ln_{+1}(J-1), C^-1 = F^-1 F^-T, E = (G + G^T + G^T G)/2,
 * J^-2/3 = exp(-2/3 ln J)); 1: the same with J^-2/3 by Alg. 2; 2: the
 * standard forms of Sec. 3 / App. A (F = I + G, C = F^T F inverted directly,
 * det F, log, pow). Fibre structure tensors are those of element `elem`. */
hx_status hx_material_eval(hx_mesh *mesh, int32_t elem, int32_t form, int32_t prec, int64_t n, const double *G_dev,
                           const double *H_dev, double *S_dev, double *P_dev, double *dP_dev);

/* Load vector of a constant body force b[3] (Sec. 2, the (v, B) term of the
 * residual): f_i = sum_e sum_q JxW_q N_i(x_q) b, FP64, f_dev[n_nodes][3]
 * overwritten; constrained rows are zero. */
hx_status hx_body_force(hx_mesh *mesh, const double b[3], double *f_dev);

/* Newton's method of Alg. 1 on R(u) - f_ext = 0 over the free DoFs: while
 * ||r|| > eps_abs and ||r|| > eps_rel ||r_0|| and k < max_newton, update the
 * quadrature-point data at u_k (strategy `storage`, FP64 and the
 * preconditioner's precision), solve K du = -r with hx_cg_solve (Chebyshev
 * (cg_degree)-Jacobi, lambda_max = 1.2 x a power-iteration estimate with
 * lambda_iters steps) and set u_k += du. u_dev (FP64, [n_nodes][3]) holds u_0
 * with the Dirichlet values already in its constrained entries (Alg. 1's
 * u_0 <- g_D), which the updates leave unchanged; it receives the last
 * iterate. f_ext_dev (FP64, may be NULL) is the external load vector, e.g.
 * from hx_body_force. A linear solve that stops at cg_max_iter still updates
 * u (inexact Newton); a CG breakdown returns its status. Returns
 * HX_ERR_NOT_CONVERGED if the tolerances are not met within max_newton steps.
 * Synchronous. */
typedef struct hx_mg hx_mg;
typedef struct {
    double eps_abs, eps_rel;
    int32_t max_newton;
    int32_t storage;         /* hx_storage refreshed at every Newton step */
    int32_t cg_degree;       /* Chebyshev degree of the preconditioner */
    double smoothing_range;  /* lambda_min = lambda_max / range */
    int32_t precond_prec;    /* hx_prec of the preconditioner */
    double cg_tol;           /* relative tolerance of each linear solve */
    int32_t cg_max_iter;
    int32_t lambda_iters;
    hx_mg *mg;               /* non-NULL: the linear solves use hx_mg_cg_solve with this
                                p-multigrid (built on the same mesh), refreshed by
                                hx_mg_setup at every Newton step; cg_degree,
                                smoothing_range, precond_prec and lambda_iters are then
                                taken from the multigrid's own options */
} hx_newton_options;
typedef struct {
    int32_t newton_iters;    /* Newton updates performed */
    int32_t cg_iters;        /* CG iterations over all steps */
    double res0, res;        /* ||r(u_0)||_2 and ||r(u_k)||_2 */
    int32_t converged;
} hx_newton_report;
hx_status hx_newton_solve(hx_mesh *mesh, double *u_dev, const double *f_ext_dev, const hx_newton_options *opt,
                          hx_newton_report *report);

/* ---- hp-multigrid preconditioner (Sec. 6) ------------------------------- */
/* p-levels of degree p, floor(p/2), ... down to min_degree on the mesh's
 * structured box (same elements and geometry), then, once the degree is 1,
 * up to h_levels h-levels: the degree-1 box halved in every direction while
 * all three element counts are even (trilinear geometry only). A coarse
 * vertex is the finer box's vertex at twice its lattice index, so jittered
 * boxes coarsen too; the hierarchy is then not nested and the h-transfers
 * act in lattice coordinates (prolongation = trilinear interpolation of the
 * coarser lattice function at the finer lattice nodes, which is the exact
 * embedding when the boxes are nested). The Dirichlet constraints must be
 * whole faces, component by component, and are carried to every level;
 * other meshes give HX_ERR_UNSUPPORTED. At most 16 levels.
 * The V-cycle smooths with smoother_degree steps of Chebyshev-Jacobi on
 * [lambda_max/smoothing_range, lambda_max] of D^-1 K per level (before and
 * after the coarse correction). On the coarsest level it runs, if
 * coarse_cg_iters > 0, FP64 Jacobi-preconditioned CG on that level's tangent
 * (assembled once per hx_mg_setup from the matrix-free operator; at most
 * 1024 DoFs, else HX_ERR_UNSUPPORTED) for at most coarse_cg_iters
 * iterations or down to a relative residual of coarse_cg_tol -- the paper's
 * coarse solver is AMG or a direct solve; this is its stand-in -- and else
 * coarse_degree steps of Chebyshev-Jacobi on [lambda_max/coarse_range,
 * lambda_max]. p-transfers: prolongation = interpolation of the coarser
 * Lagrange function at the finer nodes, restriction = its transpose; the
 * linearization point of a coarser level is the finer state evaluated at its
 * nodes (for an h-level: at the shared lattice nodes). All level operators
 * are the matrix-free tangent in precond_prec with the `storage` strategy.
 * The mesh must outlive the multigrid object. */
typedef struct {
    int32_t smoother_degree;
    double smoothing_range;
    int32_t coarse_degree;
    double coarse_range;
    int32_t precond_prec;
    int32_t storage;
    int32_t lambda_iters;     /* power iterations per level (x1.2 safety) */
    int32_t min_degree;       /* coarsest degree (>= 1): levels stop once p/2 would fall below it */
    double coarse_weight;     /* coarse corrections are added scaled by this weight (0 < w <= 1) */
    int32_t h_levels;         /* at most this many h-coarsenings after the p-levels (0: none) */
    int32_t coarse_cg_iters;  /* > 0: coarse FP64 Jacobi-CG with this iteration limit; 0: Chebyshev */
    double coarse_cg_tol;     /* relative residual at which the coarse CG stops (> 0 if used) */
} hx_mg_options;
hx_status hx_mg_create(hx_mesh *mesh, const hx_mg_options *opt, hx_mg **mg);
void hx_mg_destroy(hx_mg *mg);
/* Number of levels and their degrees (degrees may be NULL; at most 16). */
hx_status hx_mg_info(const hx_mg *mg, int32_t *n_levels, int32_t *degrees);
/* Degree and element counts of one level. */
hx_status hx_mg_level(const hx_mg *mg, int32_t level, int32_t *p, int32_t *nx, int32_t *ny, int32_t *nz);
/* Iterations the coarse CG took in the last V-cycle (synchronous; -1 if the
 * coarsest level runs Chebyshev or no V-cycle ran yet). */
hx_status hx_mg_coarse_iters(const hx_mg *mg, int32_t *iters);
/* Per Newton state (Alg. 1): transfer u_dev (FP64) to every level, refresh the
 * quadrature-point data (FP64 and precond_prec), the inverse diagonals and the
 * eigenvalue bounds. Synchronous; reports J <= 0 as HX_ERR_NONINVERTIBLE. */
hx_status hx_mg_setup(hx_mg *mg, const double *u_dev);
/* x = one V-cycle applied to b (finest level, precond_prec vectors). */
hx_status hx_mg_vcycle(hx_mg *mg, const void *b_dev, void *x_dev);
/* Transfer between level `level` and level+1 in `prec`: dir 0 prolongation
 * (src on level+1, dst on level), 1 restriction (src on level, dst on
 * level+1, overwritten), 2 state transfer (src on level, dst on level+1;
 * FP64 only between h-levels). */
hx_status hx_mg_transfer(hx_mg *mg, int32_t level, int32_t dir, const void *src_dev, void *dst_dev, int32_t prec);
/* FP64 flexible CG on the finest tangent with one V-cycle as preconditioner
 * (same stopping rule and statuses as hx_cg_solve); needs hx_mg_setup at the
 * current state. */
hx_status hx_mg_cg_solve(hx_mg *mg, const double *rhs_dev, double *x_dev, double tol, int32_t max_iter,
                         int32_t use_graph, int32_t *iters, double *rel_residual);

/* Fibre dispersion constants H11, H22, H33 from (a, b) (Sec. 3). Host only. */
hx_status hx_fibre_dispersion(double a, double b, double H[3]);

/* ---- batches of meshes (many uneven problems in one launch) -------------- */
/* Group meshes of one context and one law (possibly of different degrees,
 * sizes and Newton states) so that one persistent launch applies every mesh's
 * tangent: the kernel walks a device work list of (mesh, element tile) items
 * sorted by degree and dispatches each to the code of its degree. The meshes
 * stay owned by the caller and must outlive the batch. */
hx_status hx_batch_create(hx_ctx *ctx, hx_mesh *const *meshes, int32_t n_meshes, hx_batch **batch);
void hx_batch_destroy(hx_batch *batch);
/* out_i = K_i du_i for every mesh i in one launch (plus one launch that zeroes
 * the outputs); du/out are host arrays of n_meshes device pointers. Every mesh
 * needs a cache at `prec` from hx_precompute_qp, all with the same caching
 * strategy (HX_CACHE_F, HX_CACHE_TENSORS or HX_SPATIAL_TENSORS; HX_RECOMPUTE
 * gives HX_ERR_UNSUPPORTED). */
hx_status hx_batch_tangent_apply(hx_batch *batch, const void *const *du_dev, void *const *out_dev, int32_t prec);
/* Batched FP64 CG (Sec. 6 outer Krylov solver, over many independent
 * problems): solves K_i x_i = rhs_i for every mesh i of the batch (the
 * constrained tangent of its last hx_precompute_qp), preconditioned by
 * `degree` steps of Chebyshev-Jacobi on [lambda_i/smoothing_range, lambda_i]
 * of D_i^-1 K_i in precond_prec (lambda_i: 1.2 x a 20-step power estimate,
 * per mesh). The meshes iterate in lockstep: every operator application of
 * an iteration is one persistent launch over all meshes, the dot products
 * and the CG scalars are kept per mesh on the device, and a mesh whose
 * residual reached ||r_i|| <= tol ||rhs_i|| stops changing. With use_graph,
 * one whole iteration (FP64 operator, dot products, updates and the
 * preconditioner's applies) is captured once as a CUDA graph and replayed.
 * rhs_dev/x_dev: host arrays of n_meshes device pointers (x holds the start
 * and receives the solution); iters / rel_residual: host arrays of n_meshes
 * receiving each mesh's iterations and true relative residual (may be
 * NULL). Every mesh needs caches in FP64 and in precond_prec with one
 * caching strategy. Statuses: HX_ERR_NOT_CONVERGED if some mesh missed tol
 * within max_iter iterations, HX_ERR_NAN on a breakdown (non-positive
 * curvature or NaN) of some mesh, whose rel_residual entry is then NaN (the
 * other meshes' results stay valid). Synchronous; workspace (about 10 FP64 and
 * 5 FP32 vectors of the batch's total size) is allocated by the first call
 * and kept by the batch. */
hx_status hx_batch_cg_solve(hx_batch *batch, const double *const *rhs_dev, double *const *x_dev, double tol,
                            int32_t max_iter, int32_t degree, double smoothing_range, int32_t precond_prec,
                            int32_t use_graph, int32_t *iters, double *rel_residual);

/* ---- measurement support ------------------------------------------------- */
/* Peak FMA throughput of this device for `prec`, measured by a dependent-FMA
 * kernel over all SMs (flop/s, 2 flops per FMA). Synchronous. */
hx_status hx_measure_fma_peak(hx_ctx *ctx, int32_t prec, double *flops);
/* Number of this library's kernel launches since the counter was reset. */
uint64_t hx_launch_count(hx_ctx *ctx, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* HX_H */
