// k_tile.cu -- fused tile-pass kernels (forward, and adjoint over psi and lambda).
#include <algorithm>
#include <atomic>

#include "k_tile_dev.cuh"

namespace qs {
namespace {

using namespace tiledev;

static_assert(sizeof(TileGroup) % 16 == 0 && sizeof(SGate<float>) % 16 == 0 && sizeof(SGate<double>) % 16 == 0,
              "per-pass shared-memory tables keep 16-byte alignment");

template <typename Real, bool ADJ>
__global__ void __launch_bounds__(kTileThreads, (ADJ && sizeof(Real) == 8) ? 1 : 2)
k_tile_pass(typename TileT<Real>::T2 *__restrict__ psi, typename TileT<Real>::T2 *__restrict__ lam, const TilePass P,
            const TileGroup *__restrict__ groups, const RegGate *__restrict__ gates, double *__restrict__ part,
            size_t part_stride) {
    using T2 = typename TileT<Real>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t T = 1u << P.k;
    T2 *tp = reinterpret_cast<T2 *>(smem_raw);
    T2 *tl = tp + T;  // adjoint: lambda tile
    Acc<Real> *acc = reinterpret_cast<Acc<Real> *>(smem_raw + (ADJ ? 2 : 1) * (size_t)T * sizeof(T2));  // [kTileMaxParam][8]
    TileGroup *sgroups = reinterpret_cast<TileGroup *>(acc + (ADJ ? kTileMaxParam * (kTileThreads / 32) : 0));
    SGate<Real> *sgates = reinterpret_cast<SGate<Real> *>(sgroups + P.group_count);  // tables sized for this pass
    uint64_t *g_j = reinterpret_cast<uint64_t *>(sgates + P.gate_count);
    uint32_t *s_j = reinterpret_cast<uint32_t *>(g_j + kTileMaxSteps);
    const int tid = threadIdx.x;
    if (ADJ)
        for (int i = tid; i < kTileMaxParam * (kTileThreads / 32); i += kTileThreads) acc[i] = Acc<Real>{};
    stage_pass<Real>(P, groups, gates, sgroups, sgates);
    const TileAddr ta = tile_addr<Real>(P, g_j, s_j);
    const SGate<Real> *G0 = sgates;
    for (uint64_t tau = blockIdx.x; tau < P.ntiles; tau += gridDim.x) {
        const uint64_t base = tile_base(P, tau);
        if (P.hctrl) {
            bool any = false;
            for (int g = 0; g < P.gate_count; ++g) any |= ((base & G0[g].hmask) == G0[g].hvals);
            if (!any) continue;  // no gate of the pass selects this tile
        }
        load_tile<Real>(ta, g_j, s_j, base, psi, tp);
        if (ADJ) load_tile<Real>(ta, g_j, s_j, base, lam, tl);
        __syncthreads();
        apply_groups<Real, ADJ>(tp, tl, base, P.k, sgroups, P.group_count, sgates, nullptr, acc);
        store_tile<Real>(ta, g_j, s_j, base, tp, psi);
        if (ADJ) store_tile<Real>(ta, g_j, s_j, base, tl, lam);
        __syncthreads();
    }
    if (ADJ) {
        __syncthreads();
        for (int p = tid; p < P.nparam; p += kTileThreads) {
            double s = 0.0;
            for (int w = 0; w < kTileThreads / 32; ++w) s += acc[p * (kTileThreads / 32) + w].value();
            part[(size_t)P.param_gslot[p] * part_stride + blockIdx.x] = s;
        }
    }
}

template <typename Real, bool ADJ>
cudaError_t go(void *psi, void *lam, const TilePass &p, const TileGroup *groups, const RegGate *gates, double *part,
               size_t part_stride, cudaStream_t st) {
    auto kern = k_tile_pass<Real, ADJ>;
    const size_t smem = tile_smem_bytes(sizeof(Real) == 4 ? QS_C64 : QS_C128, p.k, ADJ, p.group_count, p.gate_count);
    static std::atomic<size_t> configured[64];  // per device: dynamic shared memory allowed so far
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (smem > 48 * 1024 && smem > configured[dev].load()) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        size_t cur = configured[dev].load();
        while (cur < smem && !configured[dev].compare_exchange_weak(cur, smem)) {
        }
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTileThreads, smem) != cudaSuccess || occ < 1) occ = 1;
    uint64_t cap = (uint64_t)device_sm_count() * occ;
    if (ADJ) cap = std::min<uint64_t>(cap, part_stride);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(p.ntiles, cap));
    using T2 = typename TileT<Real>::T2;
    kern<<<grid, kTileThreads, smem, st>>>(reinterpret_cast<T2 *>(psi), reinterpret_cast<T2 *>(lam), p, groups, gates,
                                           part, part_stride);
    return cudaGetLastError();
}

}  // namespace

size_t tile_smem_bytes(int dtype, int k, bool adjoint, int groups, int gates) {
    const size_t es = dtype == QS_C64 ? 8 : 16;
    const size_t sg = dtype == QS_C64 ? sizeof(SGate<float>) : sizeof(SGate<double>);
    return (adjoint ? 2 : 1) * (size_t(1) << k) * es + (adjoint ? kTileMaxParam * (kTileThreads / 32) * sizeof(double) : 0) +
           (size_t)groups * sizeof(TileGroup) + (size_t)gates * sg + kTileMaxSteps * (sizeof(uint64_t) + sizeof(uint32_t));
}

cudaError_t launch_tile_pass(int dtype, void *psi, void *lam, const TilePass &p, const TileGroup *groups,
                             const RegGate *gates, double *part, size_t part_stride, cudaStream_t st) {
    const bool adj = lam != nullptr;
    if (dtype == QS_C64)
        return adj ? go<float, true>(psi, lam, p, groups, gates, part, part_stride, st)
                   : go<float, false>(psi, lam, p, groups, gates, part, part_stride, st);
    return adj ? go<double, true>(psi, lam, p, groups, gates, part, part_stride, st)
               : go<double, false>(psi, lam, p, groups, gates, part, part_stride, st);
}

}  // namespace qs
