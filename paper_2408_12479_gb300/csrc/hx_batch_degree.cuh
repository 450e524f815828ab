// hx_batch_degree.cuh -- one degree of the batch unit: the per-degree core
// (hx_core.cuh) plus the batch tile of that degree, in namespace HXB_NS. The
// includer defines HX_P and HXB_NS; this file has no include guard on purpose.
namespace HXB_NS {
using Real = hx_batch_unit::Real;
namespace {
#include "hx_core.cuh"

// elements per work item: at most BT threads (n^2 per element) and at most
// BATCH_SMEM bytes of shared arrays
template <int STORAGE>
constexpr int batch_epb() {
    constexpr int arrays = ApplySmem<1, HX_CNH, STORAGE, false>::arrays;
    constexpr int by_threads = hx_batch_unit::BT / NN;
    constexpr int by_smem = (int)(hx_batch_unit::BATCH_SMEM / ((size_t)arrays * CES * sizeof(Real)));
    constexpr int e = by_threads < by_smem ? by_threads : by_smem;
    return e < 1 ? 1 : e;
}
template <int STORAGE>
constexpr size_t batch_smem() {
    return ApplySmem<batch_epb<STORAGE>(), HX_CNH, STORAGE, false>::bytes;
}
template <int LAW, int STORAGE>
__device__ __noinline__ void tile(const hx::MeshView &m, int t, const void *du, void *out, unsigned char *smem) {
    batch_tile<batch_epb<STORAGE>(), hx_batch_unit::BT, LAW, STORAGE>(m, t, (const Real *)du, (Real *)out, smem);
}
}  // namespace
}  // namespace HXB_NS
