// Internal definitions shared by the host API (hx_api.cu) and the per-degree
// kernel translation units (hx_ops.cu compiled once per polynomial degree).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hx.h"

#define HX_PMIN 1
#define HX_PMAX 6
#define HX_NMAX (HX_PMAX + 1)
// bytes allocated past the end of every point array: the staged applies copy
// whole 16-byte aligned windows, which may reach past the last point
#define HX_ARRAY_SLACK 512

namespace hx {

enum Op { OP_APPLY = 0, OP_RESIDUAL = 1, OP_PRECOMPUTE = 2, OP_DIAG = 3 };

// Number of stored quadrature-point fields per (law, storage); the layout of
// each field set is documented in hx_kernels.cuh next to the code that
// writes it.
__host__ __device__ constexpr int qp_fields(int law, int storage) {
    if (storage == HX_RECOMPUTE) return 0;
    if (storage == HX_CACHE_F) return law == HX_CNH ? 11 : (law == HX_INH ? 14 : 18);
    if (storage == HX_SPATIAL_TENSORS) return law == HX_CNH ? 17 : (law == HX_INH ? 23 : 35);
    return law == HX_CNH ? 31 : (law == HX_INH ? 33 : 35);
}

struct MatParams {
    double mu, lambda, kappa, k1, k2;
};
struct MatParamsF {
    float mu, lambda, kappa, k1, k2;
};

// Division of 0 <= n < 2^31 by a divisor fixed per mesh, with a multiply-high
// and two shifts instead of an integer division (Granlund and Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, the
// unsigned case): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// t = mulhi(m, n) and n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct FastDiv {
    uint32_t m, s1, s2;
};

// Plain-old-data view of a device mesh, passed by value to every kernel.
struct MeshView {
    int p, n_elem;
    int64_t n_nodes, n_qp;
    int64_t qs;                  // field stride of the SoA point arrays: n_qp rounded up to 32
    int structured, nx, ny, nz;
    FastDiv fnx, fny;            // division by nx and by ny (structured boxes)
    int64_t Nx, Ny;              // node lattice extents of a structured box
    const int32_t *dof_conn;     // [n_elem][(p+1)^3] or null (structured)
    const void *geo;             // [10][qs] of T: (J0^-1)_{ed} at field 3e+d, JxW at field 9
    const double *geo64;         // the same in FP64 (precompute)
    const void *qp;              // [nf][qs] of T (strategy cache)
    const void *uk;              // u_k in T (recompute strategy)
    int nf;
    const uint8_t *dmask;        // [3 n_nodes] or null
    const void *fibH;            // [12][n_elem] of T: H_4 (sym 6), H_6 (sym 6)
    const double *fibH64;        // the same in FP64
    const double *fibM;          // [6][n_elem] mean fibre directions M1 of families 4, 6
    int *err;                    // device error flags: [0] non-invertible, [1] NaN, [2] wait gave up
    MatParams mat;
    MatParamsF matf;  // the same constants rounded once to FP32
    int law;
    int l2pf;         // apply kernel (register-prefetch variants): prefetch the next tile's qp data into L2
    // test hook (hx_set_wait_test): 1 = the staged apply issues no bulk copy,
    // so its bounded wait runs out; wait_limit = cycles a bounded wait polls
    // before it gives up
    int skip_stage_copies;
    long long wait_limit;
    // ordered assembly: element-local results go to elem_out[3 (e NQ + a) + c]
    // with plain stores instead of atomic adds into the output (null: atomic)
    void *elem_out;
};

// Kernel entry points provided by each (degree, precision) translation unit
// (hx_ops.cu compiled with HX_P and HX_UNIT_F32). All launchers are asynchronous
// on the given stream and return the launch error, if any.
struct PrecOps {
    int p, prec;
    // upload the 1D tables of this degree into the unit's constant memory:
    // B[q][a] nodal basis at Gauss points, D[q][r] collocation derivative on the
    // Gauss points, Gd[q][a] nodal-basis derivative at Gauss points, weights
    // w[q]; geometry bases (degree 1 and 2, equispaced) at the Gauss points
    // (value, derivative) and at the nodal points (value), [g-1][a][q].
    cudaError_t (*upload_tables)(const double *B, const double *D, const double *Gd, const double *w,
                                 const double *geoV, const double *geoD, const double *geoVn);
    // geometry at every quadrature point (FP64 unit only; writes both copies)
    cudaError_t (*geometry)(const MeshView &m, const double *geo_nodes, const int32_t *geo_conn, int g,
                            double *geo64, float *geo32, cudaStream_t s);
    cudaError_t (*node_coords)(const MeshView &m, const double *geo_nodes, const int32_t *geo_conn, int g,
                               double *X, cudaStream_t s);
    // qp cache at state u (FP64 in), stored in this unit's precision
    cudaError_t (*precompute)(const MeshView &m, int storage, const double *u, void *qp, cudaStream_t s);
    cudaError_t (*apply)(const MeshView &m, int storage, const void *du, void *out, cudaStream_t s, int variant);
    cudaError_t (*residual)(const MeshView &m, const void *u, void *r, cudaStream_t s);
    cudaError_t (*diagonal)(const MeshView &m, int storage, void *diag, cudaStream_t s);
    // pointwise law evaluation at n gradients (form: 0 stable, 1 stable with
    // Alg. 2 for J^-2/3, 2 standard), fibre data of element e
    cudaError_t (*material_eval)(const MeshView &m, int e, int form, int64_t n, const double *G, const double *H,
                                 double *S, double *P, double *dP, cudaStream_t s);
    // f += load vector of a constant body force (FP64 unit only)
    cudaError_t (*body_force)(const MeshView &m, const double *b, double *f, cudaStream_t s);
    int n_variants;  // tile variants of apply available to the autotuner
};

const PrecOps *prec_ops(int p, int prec);

// One mesh of a batch as the batch kernel sees it.
struct BatchMesh {
    MeshView m;
    const void *du;
    void *out;
    int64_t n_dofs;
    const int *active;  // non-null: the mesh is skipped while *active == 0 (batched CG)
};

// Entry points of the batch unit of one precision (hx_batch.cu).
struct BatchOps {
    int prec;
    cudaError_t (*upload_tables)(int p, const double *B, const double *D, const double *Gd, const double *w,
                                 const double *geoV, const double *geoD, const double *geoVn);
    int (*epb)(int p, int law, int storage);  // elements per work item of degree p
    cudaError_t (*apply)(int law, int storage, const BatchMesh *meshes, const int2 *items, int nitems,
                         cudaStream_t s);
    cudaError_t (*zero)(const BatchMesh *meshes, int nmesh, cudaStream_t s);
};
const BatchOps *batch_ops(int prec);

}  // namespace hx

struct hx_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int *d_flags = nullptr;  // [3] device error flags
    int sm_count = 0;
    uint64_t launches = 0;
};
