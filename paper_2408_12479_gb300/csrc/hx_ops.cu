// hx_ops.cu -- fused matrix-free operator kernels for one polynomial degree
// and one precision. Compiled once per (HX_P, HX_UNIT_F32) pair; every unit
// keeps its own 1D tables in constant memory and exports one PrecOps table.
// The kernel bodies are in hx_core.cuh.
#include <cuda_runtime.h>
#include <algorithm>
#include <stdint.h>

#include <type_traits>

#include "hx_internal.h"

#ifndef HX_P
#error "HX_P must be defined"
#endif
#ifndef HX_UNIT_F32
#define HX_UNIT_F32 0
#endif

#define HX_CAT2(a, b) a##b
#define HX_CAT(a, b) HX_CAT2(a, b)
#if HX_UNIT_F32
#define HX_OPS_NAME HX_CAT(HX_CAT(hx_prec_ops_p, HX_P), _f32)
#else
#define HX_OPS_NAME HX_CAT(HX_CAT(hx_prec_ops_p, HX_P), _f64)
#endif

namespace hx_unit {
#if HX_UNIT_F32
typedef float Real;
#else
typedef double Real;
#endif
namespace {
#include "hx_core.cuh"

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// elements per CTA of the apply/residual/precompute kernels: shared memory per
// CTA stays near 64 KB (FP64) so that several CTAs fit on one SM
constexpr int epb_default() {
    return N <= 3 ? 16 : (N == 4 ? 8 : (N == 5 ? 4 : 2));
}
// elements per CTA of the column-layout apply (n^2 threads each)
constexpr int EPB_A = sizeof(Real) == 4 ? (N <= 2 ? 32 : (N == 3 ? 16 : (N <= 5 ? 8 : 4)))
                                         : (N <= 2 ? 16 : (N == 3 ? 8 : (N <= 5 ? 4 : 2)));

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

int sm_count() {
    static int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

template <int EPB, int LAW, int STORAGE, bool STAGED>
cudaError_t launch_apply_t(const hx::MeshView &m, const void *du, void *out, cudaStream_t s) {
    using SM = ApplySmem<EPB, LAW, STORAGE, STAGED>;
    auto kern = k_apply<EPB, LAW, STORAGE, STAGED>;
    constexpr size_t smem = SM::bytes;
    constexpr int NTH = apply_threads<STAGED && ROWSW>(EPB);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    static int per_sm = [&] {
        if (set_smem(kern, smem) != cudaSuccess) return 0;
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, NTH, smem) != cudaSuccess) return 0;
        return b;
    }();
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const int ntiles = (m.n_elem + EPB - 1) / EPB;
    if (ntiles == 0) return cudaSuccess;
    const int grid = ntiles < per_sm * sm_count() ? ntiles : per_sm * sm_count();
    kern<<<grid, NTH, smem, s>>>(m, (const Real *)du, (Real *)out, ntiles);
    return cudaGetLastError();
}

// Elements per CTA of the half-tile staged variant at n >= 6, where a
// staged element takes 24-38 KB of shared memory: the tile size, up to the
// default, that keeps the most elements resident per SM.
template <int LAW, int STORAGE>
constexpr int epb_resident() {
    int best = 1, most = 0;
    for (int e = 1; e <= EPB_A; ++e) {
        const int vw = 16 / (int)sizeof(Real);
        const int fe = (e * NQ) % vw == 0 ? e * NQ : (e * NQ + 2 * vw - 2) / vw * vw;
        const size_t b = ((size_t)(STORAGE == HX_RECOMPUTE ? 6 : 3) * e * CES * sizeof(Real) + 15) / 16 * 16 +
                         (size_t)QpFields<LAW, STORAGE>::n * fe * sizeof(Real);
        const int ctas = (int)((size_t)227 * 1024 / b);
        if (e * ctas >= most) {
            most = e * ctas;
            best = e;
        }
    }
    return best;
}

// Warp-decoupled staged apply (k_apply_wd): W warps per CTA, each with a
// group of whole elements and its own stage; FP32 up to n = 5 and the caching
// strategies only.
// warps per CTA of variant 2: at n = 4 a warp's cubes and stage take 14.5 KB,
// and two-warp CTAs pack the SM's shared memory best
constexpr int WD_LO = N == 4 ? 2 : 4;
template <int W, int LAW, int STORAGE>
cudaError_t launch_apply_wd_t(const hx::MeshView &m, const void *du, void *out, cudaStream_t s) {
    if constexpr (!WD_OK || STORAGE == HX_RECOMPUTE) {
        return cudaErrorInvalidConfiguration;
    } else {
        auto kern = k_apply_wd<W, LAW, STORAGE>;
        constexpr size_t smem = wd_smem_bytes<W, LAW, STORAGE>();
        constexpr int NTH = W * 32;
        if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
        static int per_sm = [&] {
            if (set_smem(kern, smem) != cudaSuccess) return 0;
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            int b = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, NTH, smem) != cudaSuccess) return 0;
            return b;
        }();
        if (per_sm <= 0) return cudaErrorInvalidConfiguration;
        const int ngroups = (m.n_elem + WEPW - 1) / WEPW;
        const int ntiles = (ngroups + W - 1) / W;
        if (ntiles == 0) return cudaSuccess;
        const int grid = ntiles < per_sm * sm_count() ? ntiles : per_sm * sm_count();
        kern<<<grid, NTH, smem, s>>>(m, (const Real *)du, (Real *)out, ntiles);
        return cudaGetLastError();
    }
}

// variants: how the quadrature-point fields arrive and the tile shape:
// register prefetch one point ahead with an L2 bulk prefetch of the next tile
// (0: default, 1: half elements per CTA), bulk copies into a shared stage one
// tile ahead (3: default, 4: half; from n = 6 on, the tile that keeps the most
// elements resident; chunks that do not start on 16-byte boundaries are
// copied as aligned windows), and the warp-decoupled staged apply with a
// stage per warp (2: WD_LO warps per CTA, 5: twice as many), built only where
// whole elements fit one warp (FP32, p <= 4) and not for the recompute
// strategy.
template <int LAW, int STORAGE>
cudaError_t apply_variant(const hx::MeshView &m0, const void *du, void *out, cudaStream_t s, int variant) {
    hx::MeshView m = m0;
    m.l2pf = 1;
    constexpr int EH = EPB_A > 1 ? EPB_A / 2 : 1;
    switch (variant) {
        case 1: return launch_apply_t<EH, LAW, STORAGE, false>(m, du, out, s);
        case 2: return launch_apply_wd_t<WD_LO, LAW, STORAGE>(m, du, out, s);
        case 3: return launch_apply_t<EPB_A, LAW, STORAGE, true>(m, du, out, s);
        case 4: return launch_apply_t<(N >= 6 ? epb_resident<LAW, STORAGE>() : EH), LAW, STORAGE, true>(m, du, out, s);
        case 5: return launch_apply_wd_t<2 * WD_LO, LAW, STORAGE>(m, du, out, s);
        default: return launch_apply_t<EPB_A, LAW, STORAGE, false>(m, du, out, s);
    }
}

cudaError_t op_apply(const hx::MeshView &m, int storage, const void *du, void *out, cudaStream_t s, int variant) {
#define HX_APPLY_CASE(L, S) \
    if (m.law == L && storage == S) return apply_variant<L, S>(m, du, out, s, variant);
    HX_APPLY_CASE(HX_CNH, HX_RECOMPUTE)
    HX_APPLY_CASE(HX_CNH, HX_CACHE_F)
    HX_APPLY_CASE(HX_CNH, HX_CACHE_TENSORS)
    HX_APPLY_CASE(HX_CNH, HX_SPATIAL_TENSORS)
    HX_APPLY_CASE(HX_INH, HX_RECOMPUTE)
    HX_APPLY_CASE(HX_INH, HX_CACHE_F)
    HX_APPLY_CASE(HX_INH, HX_CACHE_TENSORS)
    HX_APPLY_CASE(HX_INH, HX_SPATIAL_TENSORS)
    HX_APPLY_CASE(HX_FIBER, HX_RECOMPUTE)
    HX_APPLY_CASE(HX_FIBER, HX_CACHE_F)
    HX_APPLY_CASE(HX_FIBER, HX_CACHE_TENSORS)
    HX_APPLY_CASE(HX_FIBER, HX_SPATIAL_TENSORS)
#undef HX_APPLY_CASE
    return cudaErrorInvalidValue;
}

template <int LAW>
cudaError_t launch_residual_t(const hx::MeshView &m, const void *u, void *r, cudaStream_t s) {
    constexpr int EPB = EPB_A;
    auto kern = k_residual_col<EPB, LAW>;
    constexpr size_t smem = (size_t)3 * EPB * CES * sizeof(Real);
    static int per_sm = [&] {
        if (set_smem(kern, smem) != cudaSuccess) return 0;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, col_threads(EPB), smem) != cudaSuccess) return 0;
        return b;
    }();
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const int ntiles = (m.n_elem + EPB - 1) / EPB;
    if (ntiles == 0) return cudaSuccess;
    const int grid = ntiles < per_sm * sm_count() ? ntiles : per_sm * sm_count();
    kern<<<grid, col_threads(EPB), smem, s>>>(m, (const Real *)u, (Real *)r, ntiles);
    return cudaGetLastError();
}

cudaError_t op_residual(const hx::MeshView &m, const void *u, void *r, cudaStream_t s) {
    if (m.law == HX_CNH) return launch_residual_t<HX_CNH>(m, u, r, s);
    if (m.law == HX_INH) return launch_residual_t<HX_INH>(m, u, r, s);
    if (m.law == HX_FIBER) return launch_residual_t<HX_FIBER>(m, u, r, s);
    return cudaErrorInvalidValue;
}

template <int LAW, int STORAGE>
cudaError_t launch_precompute_t(const hx::MeshView &m, const double *u, void *qp, cudaStream_t s) {
    constexpr int EPB = epb_default();
    auto kern = k_precompute<EPB, LAW, STORAGE>;
    const size_t smem = (size_t)15 * EPB * SZ * sizeof(double);
    static cudaError_t attr = set_smem(kern, smem);
    if (attr != cudaSuccess) return attr;
    const int grid = (m.n_elem + EPB - 1) / EPB;
    if (grid == 0) return cudaSuccess;
    kern<<<grid, threads_for(EPB), smem, s>>>(m, u, (Real *)qp);
    return cudaGetLastError();
}

cudaError_t op_precompute(const hx::MeshView &m, int storage, const double *u, void *qp, cudaStream_t s) {
    if (storage == HX_RECOMPUTE) {
        // the recompute strategy keeps u_k itself (in Real) and only checks J
        k_convert_uk<<<1024, 256, 0, s>>>(u, (Real *)qp, 3 * m.n_nodes);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
#define HX_PRE_CASE(L, S) \
    if (m.law == L && storage == S) return launch_precompute_t<L, S>(m, u, qp, s);
    HX_PRE_CASE(HX_CNH, HX_RECOMPUTE)
    HX_PRE_CASE(HX_CNH, HX_CACHE_F)
    HX_PRE_CASE(HX_CNH, HX_CACHE_TENSORS)
    HX_PRE_CASE(HX_CNH, HX_SPATIAL_TENSORS)
    HX_PRE_CASE(HX_INH, HX_RECOMPUTE)
    HX_PRE_CASE(HX_INH, HX_CACHE_F)
    HX_PRE_CASE(HX_INH, HX_CACHE_TENSORS)
    HX_PRE_CASE(HX_INH, HX_SPATIAL_TENSORS)
    HX_PRE_CASE(HX_FIBER, HX_RECOMPUTE)
    HX_PRE_CASE(HX_FIBER, HX_CACHE_F)
    HX_PRE_CASE(HX_FIBER, HX_CACHE_TENSORS)
    HX_PRE_CASE(HX_FIBER, HX_SPATIAL_TENSORS)
#undef HX_PRE_CASE
    return cudaErrorInvalidValue;
}

template <int LAW, int STORAGE>
cudaError_t launch_diag_t(const hx::MeshView &m, void *diag, cudaStream_t s) {
    auto kern = k_diagonal<LAW, STORAGE>;
    const size_t smem = (size_t)(3 + 3 + 9 + 18 + 18) * SZ * sizeof(Real);
    static cudaError_t attr = set_smem(kern, smem);
    if (attr != cudaSuccess) return attr;
    if (m.n_elem == 0) return cudaSuccess;
    kern<<<m.n_elem, threads_for(2), smem, s>>>(m, (Real *)diag);
    return cudaGetLastError();
}

cudaError_t op_diagonal(const hx::MeshView &m, int storage, void *diag, cudaStream_t s) {
#define HX_DIAG_CASE(L, S) \
    if (m.law == L && storage == S) return launch_diag_t<L, S>(m, diag, s);
    HX_DIAG_CASE(HX_CNH, HX_RECOMPUTE)
    HX_DIAG_CASE(HX_CNH, HX_CACHE_F)
    HX_DIAG_CASE(HX_CNH, HX_CACHE_TENSORS)
    HX_DIAG_CASE(HX_CNH, HX_SPATIAL_TENSORS)
    HX_DIAG_CASE(HX_INH, HX_RECOMPUTE)
    HX_DIAG_CASE(HX_INH, HX_CACHE_F)
    HX_DIAG_CASE(HX_INH, HX_CACHE_TENSORS)
    HX_DIAG_CASE(HX_INH, HX_SPATIAL_TENSORS)
    HX_DIAG_CASE(HX_FIBER, HX_RECOMPUTE)
    HX_DIAG_CASE(HX_FIBER, HX_CACHE_F)
    HX_DIAG_CASE(HX_FIBER, HX_CACHE_TENSORS)
    HX_DIAG_CASE(HX_FIBER, HX_SPATIAL_TENSORS)
#undef HX_DIAG_CASE
    return cudaErrorInvalidValue;
}

cudaError_t op_geometry(const hx::MeshView &m, const double *X, const int32_t *gconn, int g, double *geo64,
                        float *geo32, cudaStream_t s) {
    if (m.n_qp == 0) return cudaSuccess;
    k_geometry<<<2048, 256, 0, s>>>(m, X, gconn, g, geo64, geo32);
    return cudaGetLastError();
}

cudaError_t op_node_coords(const hx::MeshView &m, const double *X, const int32_t *gconn, int g, double *out,
                           cudaStream_t s) {
    if (m.n_elem == 0) return cudaSuccess;
    k_node_coords<<<2048, 256, 0, s>>>(m, X, gconn, g, out);
    return cudaGetLastError();
}

cudaError_t op_material_eval(const hx::MeshView &m, int e, int form, int64_t n, const double *G, const double *H,
                             double *S, double *P, double *dP, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n + 127) / 128, 4096);
#define HX_ME_CASE(L, F) \
    if (m.law == L && form == F) { k_material_eval<L, F><<<grid, 128, 0, s>>>(m, e, n, G, H, S, P, dP); return cudaGetLastError(); }
    HX_ME_CASE(HX_CNH, 0) HX_ME_CASE(HX_CNH, 1) HX_ME_CASE(HX_CNH, 2)
    HX_ME_CASE(HX_INH, 0) HX_ME_CASE(HX_INH, 1) HX_ME_CASE(HX_INH, 2)
    HX_ME_CASE(HX_FIBER, 0) HX_ME_CASE(HX_FIBER, 1) HX_ME_CASE(HX_FIBER, 2)
#undef HX_ME_CASE
    return cudaErrorInvalidValue;
}

#if !HX_UNIT_F32
cudaError_t op_body_force(const hx::MeshView &m, const double *b, double *f, cudaStream_t s) {
    constexpr int EPB = 2;
    constexpr size_t smem = (size_t)6 * EPB * SZ * sizeof(Real);
    if (m.n_elem == 0) return cudaSuccess;
    cudaError_t e = set_smem(k_body_force<EPB>, smem);
    if (e != cudaSuccess) return e;
    k_body_force<EPB><<<(m.n_elem + EPB - 1) / EPB, threads_for(EPB), smem, s>>>(m, b[0], b[1], b[2], f);
    return cudaGetLastError();
}
#endif

}  // namespace
}  // namespace hx_unit

extern "C++" const hx::PrecOps *HX_OPS_NAME() {
    using namespace hx_unit;

    static const hx::PrecOps ops = {
        HX_P,
        HX_UNIT_F32 ? 1 : 0,
        op_upload,
#if HX_UNIT_F32
        nullptr,
        nullptr,
#else
        op_geometry,
        op_node_coords,
#endif
        op_precompute,
        op_apply,
        op_residual,
        op_diagonal,
        op_material_eval,
#if HX_UNIT_F32
        nullptr,
#else
        op_body_force,
#endif
        6,
    };
    return &ops;
}
