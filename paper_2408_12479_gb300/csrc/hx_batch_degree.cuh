// hx_batch_degree.cuh -- one degree of the batch unit: the per-degree core
// (hx_core.cuh) plus the batch tile of that degree, in namespace HXB_NS. The
// includer defines HX_P and HXB_NS; this file has no include guard on purpose.
namespace HXB_NS {
using Real = hx_batch_unit::Real;
namespace {
#include "hx_core.cuh"

// Tile shape of a work item of this degree. Staged (the quadrature-point
// fields copied into shared memory by bulk copies, as in the single-mesh
// apply) where a tile that fits BATCH_SMEM with its stage still keeps at least
// half of the BT threads busy and starts on a 16-byte boundary; otherwise the
// register path, whose tile only needs the cubes. Elements per item: at most
// BT threads (n^2, or a warp per element in the row-swizzled layout).
template <int LAW, int STORAGE>
struct BatchCfg {
    static constexpr int arrays = ApplySmem<1, LAW, STORAGE, false>::arrays;
    static constexpr int tpe_s = ROWSW ? 32 : NN;  // threads per element, staged
    static constexpr size_t elem_s =
        ((size_t)arrays * Lay<ROWSW>::ES + (size_t)QpFields<LAW, STORAGE>::n * NQ) * sizeof(Real);
    static constexpr int epb_staged() {
        for (int e = hx_batch_unit::BT / tpe_s; e >= 1; --e)
            if ((size_t)e * elem_s + 16 <= hx_batch_unit::BATCH_SMEM && ((size_t)e * NQ * sizeof(Real)) % 16 == 0)
                return e;
        return 0;
    }
    static constexpr int epb_plain() {
        constexpr int by_threads = hx_batch_unit::BT / NN;
        constexpr int by_smem = (int)(hx_batch_unit::BATCH_SMEM / ((size_t)arrays * CES * sizeof(Real)));
        constexpr int e = by_threads < by_smem ? by_threads : by_smem;
        return e < 1 ? 1 : e;
    }
    static constexpr bool staged = STORAGE != HX_RECOMPUTE && 2 * epb_staged() * tpe_s >= hx_batch_unit::BT;
    static constexpr int epb = staged ? epb_staged() : epb_plain();
    static constexpr size_t smem =
        staged ? ApplySmem<(staged ? epb : 1), LAW, STORAGE, true>::bytes : ApplySmem<epb, LAW, STORAGE, false>::bytes;
};
template <int LAW, int STORAGE>
constexpr int batch_epb() {
    return BatchCfg<LAW, STORAGE>::epb;
}
template <int LAW, int STORAGE>
constexpr size_t batch_smem() {
    return BatchCfg<LAW, STORAGE>::smem;
}
// One work item: 0 done on the register path, 1 done on the staged path (one
// wait on bar at parity phase), -1 the staged copies never arrived.
template <int LAW, int STORAGE>
__device__ __noinline__ int tile(const hx::MeshView &m, int t, const void *du, void *out, unsigned char *smem,
                                 uint64_t *bar, uint32_t phase) {
    using C = BatchCfg<LAW, STORAGE>;
    if constexpr (C::staged) {
        return batch_tile_staged<C::epb, hx_batch_unit::BT, LAW, STORAGE>(m, t, (const Real *)du, (Real *)out, smem,
                                                                           bar, phase)
                   ? 1
                   : -1;
    } else {
        batch_tile<C::epb, hx_batch_unit::BT, LAW, STORAGE>(m, t, (const Real *)du, (Real *)out, smem);
        return 0;
    }
}
}  // namespace
}  // namespace HXB_NS
