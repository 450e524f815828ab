// hx_batch.cu -- many meshes of mixed polynomial degree in one persistent
// launch of the tangent apply. Compiled once per precision (HX_UNIT_F32).
//
// The per-degree body (hx_core.cuh) is included once per degree, each copy in
// its own namespace with its own constant-memory tables. The batch kernel
// walks a device work list of (mesh, tile) items -- sorted by degree so that a
// CTA mostly stays on one code path -- and dispatches each item to the tile
// function of its mesh's degree. All items share one block shape (BT threads);
// the tile size of a degree is the largest that fits BT threads and the
// shared-memory budget (two CTAs per SM). Items whose tile fits with its
// quadrature-point fields staged in shared memory take the staged path of the
// single-mesh apply, the copies issued when the item starts (one mbarrier per
// CTA). Batches run the caching strategies (the quadrature-point data of every
// mesh is refreshed by hx_precompute_qp).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "hx_internal.h"

#ifndef HX_UNIT_F32
#define HX_UNIT_F32 0
#endif

namespace hx_batch_unit {
#if HX_UNIT_F32
typedef float Real;
#else
typedef double Real;
#endif
constexpr int BT = 256;                    // threads per CTA of the batch kernel
constexpr size_t BATCH_SMEM = 112 * 1024;  // shared arrays per CTA at most (two CTAs per SM)
}  // namespace hx_batch_unit

#define HX_P 1
#define HXB_NS hxb1
#include "hx_batch_degree.cuh"
#undef HXB_NS
#undef HX_P

#define HX_P 2
#define HXB_NS hxb2
#include "hx_batch_degree.cuh"
#undef HXB_NS
#undef HX_P

#define HX_P 3
#define HXB_NS hxb3
#include "hx_batch_degree.cuh"
#undef HXB_NS
#undef HX_P

#define HX_P 4
#define HXB_NS hxb4
#include "hx_batch_degree.cuh"
#undef HXB_NS
#undef HX_P

#define HX_P 5
#define HXB_NS hxb5
#include "hx_batch_degree.cuh"
#undef HXB_NS
#undef HX_P

#define HX_P 6
#define HXB_NS hxb6
#include "hx_batch_degree.cuh"
#undef HXB_NS
#undef HX_P

namespace hx_batch_unit {
namespace {

template <int LAW, int STORAGE>
__global__ void __launch_bounds__(BT, 2) k_batch_apply(const hx::BatchMesh *__restrict__ meshes,
                                                     const int2 *__restrict__ items, int nitems) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ hx::MeshView mv;
    __shared__ const void *sdu;
    __shared__ void *sout;
    __shared__ __align__(8) uint64_t bar;  // staged items' bulk copies
    if (threadIdx.x == 0) hxb1::mbar_init(&bar, 1);
    uint32_t phase = 0;
    __shared__ int skip;
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const int2 it = items[w];
        __syncthreads();  // the previous item is done with mv and the shared arrays
        if (threadIdx.x == 0) {
            mv = meshes[it.x].m;
            sdu = meshes[it.x].du;
            sout = meshes[it.x].out;
            skip = meshes[it.x].active && !*meshes[it.x].active;
        }
        __syncthreads();
        if (skip) continue;  // a mesh of the batched CG that has converged
        int r;
        switch (mv.p) {
            case 1: r = hxb1::tile<LAW, STORAGE>(mv, it.y, sdu, sout, smem_raw, &bar, phase); break;
            case 2: r = hxb2::tile<LAW, STORAGE>(mv, it.y, sdu, sout, smem_raw, &bar, phase); break;
            case 3: r = hxb3::tile<LAW, STORAGE>(mv, it.y, sdu, sout, smem_raw, &bar, phase); break;
            case 4: r = hxb4::tile<LAW, STORAGE>(mv, it.y, sdu, sout, smem_raw, &bar, phase); break;
            case 5: r = hxb5::tile<LAW, STORAGE>(mv, it.y, sdu, sout, smem_raw, &bar, phase); break;
            default: r = hxb6::tile<LAW, STORAGE>(mv, it.y, sdu, sout, smem_raw, &bar, phase); break;
        }
        if (r < 0) return;  // every thread: the wait gave up (flag set by the tile)
        phase ^= (uint32_t)r;
    }
}

// out_i = 0 for every mesh i (grid.y = mesh)
__global__ void k_batch_zero(const hx::BatchMesh *__restrict__ meshes, int nmesh) {
    const int i = blockIdx.y;
    if (i >= nmesh) return;
    if (meshes[i].active && !*meshes[i].active) return;
    Real *o = (Real *)meshes[i].out;
    const int64_t n = meshes[i].n_dofs;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        o[j] = Real(0);
}

template <int LAW, int STORAGE>
constexpr size_t max_smem() {
    size_t s = hxb1::batch_smem<LAW, STORAGE>();
    s = s > hxb2::batch_smem<LAW, STORAGE>() ? s : hxb2::batch_smem<LAW, STORAGE>();
    s = s > hxb3::batch_smem<LAW, STORAGE>() ? s : hxb3::batch_smem<LAW, STORAGE>();
    s = s > hxb4::batch_smem<LAW, STORAGE>() ? s : hxb4::batch_smem<LAW, STORAGE>();
    s = s > hxb5::batch_smem<LAW, STORAGE>() ? s : hxb5::batch_smem<LAW, STORAGE>();
    s = s > hxb6::batch_smem<LAW, STORAGE>() ? s : hxb6::batch_smem<LAW, STORAGE>();
    return s;
}

int sm_count_b() {
    static int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

template <int LAW, int STORAGE>
cudaError_t launch_t(const hx::BatchMesh *meshes, const int2 *items, int nitems, cudaStream_t s) {
    auto kern = k_batch_apply<LAW, STORAGE>;
    constexpr size_t smem = max_smem<LAW, STORAGE>();
    static int per_sm = [&] {
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return 0;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, BT, smem) != cudaSuccess) return 0;
        return b;
    }();
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    if (nitems == 0) return cudaSuccess;
    const int grid = nitems < per_sm * sm_count_b() ? nitems : per_sm * sm_count_b();
    kern<<<grid, BT, smem, s>>>(meshes, items, nitems);
    return cudaGetLastError();
}

cudaError_t op_apply(int law, int storage, const hx::BatchMesh *meshes, const int2 *items, int nitems,
                     cudaStream_t s) {
#define HX_B_CASE(L, S) \
    if (law == L && storage == S) return launch_t<L, S>(meshes, items, nitems, s);
    HX_B_CASE(HX_CNH, HX_CACHE_F)
    HX_B_CASE(HX_CNH, HX_CACHE_TENSORS)
    HX_B_CASE(HX_INH, HX_CACHE_F)
    HX_B_CASE(HX_INH, HX_CACHE_TENSORS)
    HX_B_CASE(HX_FIBER, HX_CACHE_F)
    HX_B_CASE(HX_FIBER, HX_CACHE_TENSORS)
    HX_B_CASE(HX_CNH, HX_SPATIAL_TENSORS)
    HX_B_CASE(HX_INH, HX_SPATIAL_TENSORS)
    HX_B_CASE(HX_FIBER, HX_SPATIAL_TENSORS)
#undef HX_B_CASE
    return cudaErrorInvalidValue;
}

cudaError_t op_zero(const hx::BatchMesh *meshes, int nmesh, cudaStream_t s) {
    if (nmesh == 0) return cudaSuccess;
    k_batch_zero<<<dim3(256, nmesh), 256, 0, s>>>(meshes, nmesh);
    return cudaGetLastError();
}

template <int LAW>
int epb_law(int p, int storage) {
#define HX_B_EPB(P)                                                                              \
    case P:                                                                                      \
        return storage == HX_RECOMPUTE       ? hxb##P::batch_epb<LAW, HX_RECOMPUTE>()       \
               : storage == HX_CACHE_F       ? hxb##P::batch_epb<LAW, HX_CACHE_F>()         \
               : storage == HX_CACHE_TENSORS ? hxb##P::batch_epb<LAW, HX_CACHE_TENSORS>()   \
                                             : hxb##P::batch_epb<LAW, HX_SPATIAL_TENSORS>();
    switch (p) {
        HX_B_EPB(1)
        HX_B_EPB(2)
        HX_B_EPB(3)
        HX_B_EPB(4)
        HX_B_EPB(5)
        HX_B_EPB(6)
        default:
            return 0;
    }
#undef HX_B_EPB
}
int op_epb(int p, int law, int storage) {
    return law == HX_CNH ? epb_law<HX_CNH>(p, storage)
           : law == HX_INH ? epb_law<HX_INH>(p, storage)
                           : epb_law<HX_FIBER>(p, storage);
}

cudaError_t op_upload_p(int p, const double *B, const double *D, const double *Gd, const double *w,
                        const double *geoV, const double *geoD, const double *geoVn) {
    switch (p) {
        case 1: return hxb1::op_upload(B, D, Gd, w, geoV, geoD, geoVn);
        case 2: return hxb2::op_upload(B, D, Gd, w, geoV, geoD, geoVn);
        case 3: return hxb3::op_upload(B, D, Gd, w, geoV, geoD, geoVn);
        case 4: return hxb4::op_upload(B, D, Gd, w, geoV, geoD, geoVn);
        case 5: return hxb5::op_upload(B, D, Gd, w, geoV, geoD, geoVn);
        case 6: return hxb6::op_upload(B, D, Gd, w, geoV, geoD, geoVn);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace hx_batch_unit

#if HX_UNIT_F32
extern "C++" const hx::BatchOps *hx_batch_ops_f32() {
#else
extern "C++" const hx::BatchOps *hx_batch_ops_f64() {
#endif
    using namespace hx_batch_unit;
    static const hx::BatchOps ops = {HX_UNIT_F32 ? 1 : 0, op_upload_p, op_epb, op_apply, op_zero};
    return &ops;
}
