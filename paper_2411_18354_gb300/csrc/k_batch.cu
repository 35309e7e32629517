// k_batch.cu -- one persistent kernel that runs forward pass, energy and adjoint gradient for
// many independent states of different sizes.
//
// Each CTA takes the next state from an atomic work queue (states ordered largest first, so
// the long ones start early) until the queue is empty; nothing waits on anything. Per state:
//  - the state's parameters become (cos, sin) of theta/2 in shared memory;
//  - small states (n <= small_bits) live in shared memory for the whole computation: start
//    from |0...0>, apply the forward program, form lambda = O psi with O = sum_i Z_i and the
//    energy <psi|O|psi> in one pass, then the reverse program un-applies every gate to psi and
//    lambda and accumulates Re <lambda| dU psi> per parameter (float64, one slot per warp);
//  - large states run the same programs as tile passes over this CTA's two workspace vectors
//    in global memory (tiles of 2^tile_bits amplitudes in shared memory).
// Every gate is applied on its reduced iteration set (Section III-B of arXiv 2411.18354).
#include <algorithm>

#include "k_batch.cuh"
#include "k_tile_dev.cuh"

namespace qs {
namespace {

using namespace tiledev;

template <typename Real>
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    __syncthreads();
    return s;
}

// lambda = O psi and E = <psi|O|psi> over amplitudes [0, N) of `src`, written to `dst`
// (both in shared memory with the tile swizzle `sw`, or both in global memory, sw = 0).
// Partial sums: per thread in the state's precision (compensated for complex64), float64
// across threads.
template <typename Real>
__device__ __forceinline__ double obs_pass(const typename TileT<Real>::T2 *src, typename TileT<Real>::T2 *dst, int n,
                                           double *red, int sw) {
    using T2 = typename TileT<Real>::T2;
    constexpr int U = 4;  // independent loads in flight per thread
    const uint64_t N = 1ull << n;
    Acc<Real> acc{};
    for (uint64_t k0 = threadIdx.x; k0 < N; k0 += (uint64_t)U * blockDim.x) {
        T2 v[U];
        uint64_t pos[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t k = k0 + (uint64_t)u * blockDim.x;
            pos[u] = k < N ? (sw ? tile_swizzle((uint32_t)k, sw) : k) : 0;
            if (k < N) v[u] = src[pos[u]];
        }
        Real run = 0;  // float over U terms, float64 above
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t k = k0 + (uint64_t)u * blockDim.x;
            if (k < N) {
                const Real w = (Real)(n - 2 * __popcll(k));
                run += w * (v[u].x * v[u].x + v[u].y * v[u].y);
                v[u].x *= w;
                v[u].y *= w;
                dst[pos[u]] = v[u];
            }
        }
        acc.add(run);
    }
    return block_sum<Real>(acc.value(), red);
}

template <typename Real>
__device__ void run_program_global(const BatchArgs &a, const BatchProg &pg, bool adjoint, typename TileT<Real>::T2 *psi,
                                   typename TileT<Real>::T2 *lam, typename TileT<Real>::T2 *tp,
                                   typename TileT<Real>::T2 *tl, const Real *cs, Acc<Real> *gacc, TileGroup *sgroups,
                                   SGate<Real> *sgates, TilePass *spass, uint64_t *g_j, uint32_t *s_j) {
    const int begin = adjoint ? pg.adj_begin : pg.fwd_begin;
    const int count = adjoint ? pg.adj_count : pg.fwd_count;
    for (int pi = begin; pi < begin + count; ++pi) {
        // the pass descriptor, its gates and the tile address tables go to shared memory
        for (int i = threadIdx.x; i < (int)(sizeof(TilePass) / 4); i += blockDim.x)
            reinterpret_cast<uint32_t *>(spass)[i] = reinterpret_cast<const uint32_t *>(a.passes + pi)[i];
        __syncthreads();
        const TilePass &P = *spass;
        stage_pass<Real>(P, a.groups, a.gates, sgroups, sgates, cs, adjoint);
        const TileAddr ta = tile_addr<Real>(P, g_j, s_j);
        const SGate<Real> *G0 = sgates;
        for (uint64_t tau = 0; tau < P.ntiles; ++tau) {
            const uint64_t base = tile_base(P, tau);
            if (P.hctrl) {
                bool any = false;
                for (int g = 0; g < P.gate_count; ++g) any |= ((base & G0[g].hmask) == G0[g].hvals);
                if (!any) continue;
            }
            load_tile<Real>(ta, g_j, s_j, base, psi, tp);
            if (adjoint) load_tile<Real>(ta, g_j, s_j, base, lam, tl);
            __syncthreads();
            if (adjoint)
                apply_groups<Real, true, kGroupBitsAdjoint, 1, true>(tp, tl, base, P.k, sgroups, P.group_count, sgates, cs, gacc);
            else
                apply_groups<Real, false, kGroupBits, 1, true>(tp, nullptr, base, P.k, sgroups, P.group_count, sgates, cs, nullptr);
            store_tile<Real>(ta, g_j, s_j, base, tp, psi);
            if (adjoint) store_tile<Real>(ta, g_j, s_j, base, tl, lam);
            __syncthreads();
        }
        __syncthreads();  // the next pass restages the gate table
    }
}

template <typename Real>
__global__ void __launch_bounds__(kBatchThreads, sizeof(Real) == 4 ? 2 : 1) k_batch(const BatchArgs a) {
    using T2 = typename TileT<Real>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t T = 1u << a.smem_bits;
    T2 *tp = reinterpret_cast<T2 *>(smem_raw);
    T2 *tl = tp + T;
    Real *cs = reinterpret_cast<Real *>(tl + T);                                   // [2 * max_params]
    Acc<Real> *gacc = reinterpret_cast<Acc<Real> *>(cs + 2 * ((a.max_params + 1) & ~1));  // [max_params * nwarps]
    double *red = reinterpret_cast<double *>(gacc + (size_t)a.max_params * (kBatchThreads / 32));  // [nwarps]
    TileGroup *sgroups = reinterpret_cast<TileGroup *>(red + kBatchThreads / 32);
    SGate<Real> *sgates = reinterpret_cast<SGate<Real> *>(sgroups + kTileMaxGates);
    TilePass *spass = reinterpret_cast<TilePass *>(sgates + kTileMaxGates);
    uint64_t *g_j = reinterpret_cast<uint64_t *>(spass + 1);
    uint32_t *s_j = reinterpret_cast<uint32_t *>(g_j + kTileMaxSteps);
    int *next = reinterpret_cast<int *>(s_j + kTileMaxSteps);
    const int tid = threadIdx.x;
    const int nwarps = kBatchThreads / 32;
    T2 *ws_psi = reinterpret_cast<T2 *>(a.workspace) + (size_t)blockIdx.x * 2 * a.ws_stride;
    T2 *ws_lam = ws_psi + a.ws_stride;
    for (;;) {
        if (tid == 0) *next = atomicAdd(a.queue, 1);
        __syncthreads();
        const int qi = *next;
        __syncthreads();
        if (qi >= a.num_states) break;
        const BatchState st = a.states[a.order[qi]];
        const BatchProg pg = a.progs[st.prog];
        const int n = st.n;
        for (int p = tid; p < st.nparam; p += kBatchThreads) {
            double s, c;
            sincos(0.5 * a.theta[st.param_off + p], &s, &c);
            cs[2 * p] = (Real)c;
            cs[2 * p + 1] = (Real)s;
        }
        for (int i = tid; i < st.nparam * nwarps; i += kBatchThreads) gacc[i] = Acc<Real>{};
        double energy;
        if (pg.small) {
            const uint32_t N = 1u << n;
            // |0...0>: element 0 sits at swizzled position 0, every other element is 0
            for (uint32_t k = tid; k < N; k += kBatchThreads) tp[k] = T2{(Real)(k == 0), (Real)0};
            __syncthreads();
            for (int pi = pg.fwd_begin; pi < pg.fwd_begin + pg.fwd_count; ++pi) {
                const TilePass &P = a.passes[pi];
                stage_pass<Real>(P, a.groups, a.gates, sgroups, sgates, cs, false);
                apply_groups<Real, false, kGroupBits, 1, true>(tp, nullptr, 0, n, sgroups, P.group_count, sgates, cs, nullptr);
                __syncthreads();
            }
            energy = obs_pass<Real>(tp, tl, n, red, TileT<Real>::SW);
            for (int pi = pg.adj_begin; pi < pg.adj_begin + pg.adj_count; ++pi) {
                const TilePass &P = a.passes[pi];
                stage_pass<Real>(P, a.groups, a.gates, sgroups, sgates, cs, true);
                apply_groups<Real, true, kGroupBitsAdjoint, 1, true>(tp, tl, 0, n, sgroups, P.group_count, sgates, cs, gacc);
                __syncthreads();
            }
        } else {
            const uint64_t N = 1ull << n;
            for (uint64_t k = tid; k < N; k += kBatchThreads) ws_psi[k] = T2{(Real)(k == 0), (Real)0};
            __syncthreads();
            run_program_global<Real>(a, pg, false, ws_psi, ws_lam, tp, tl, cs, nullptr, sgroups, sgates, spass, g_j, s_j);
            energy = obs_pass<Real>(ws_psi, ws_lam, n, red, 0);
            run_program_global<Real>(a, pg, true, ws_psi, ws_lam, tp, tl, cs, gacc, sgroups, sgates, spass, g_j, s_j);
        }
        __syncthreads();
        if (tid == 0) a.energy[a.order[qi]] = energy;
        for (int p = tid; p < st.nparam; p += kBatchThreads) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += gacc[p * nwarps + w].value();
            a.grad[st.param_off + p] = 2.0 * s;
        }
        __syncthreads();
    }
}

}  // namespace

size_t batch_smem_bytes(int dtype, int smem_bits, int max_params) {
    const size_t es = dtype == QS_C64 ? 8 : 16;
    const size_t rs = dtype == QS_C64 ? 4 : 8;
    const size_t sg = dtype == QS_C64 ? sizeof(SGate<float>) : sizeof(SGate<double>);
    return 2 * (size_t(1) << smem_bits) * es + 2 * (size_t)((max_params + 1) & ~1) * rs +
           (size_t)max_params * (kBatchThreads / 32) * sizeof(double) + (kBatchThreads / 32) * sizeof(double) +
           kTileMaxGates * (sizeof(TileGroup) + sg) + sizeof(TilePass) + kTileMaxSteps * (sizeof(uint64_t) + 4) + 16;
}

int batch_grid(int dtype, size_t smem) {
    int occ = 0;
    cudaError_t e;
    if (dtype == QS_C64) {
        e = cudaFuncSetAttribute(k_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<float>, kBatchThreads, smem);
    } else {
        e = cudaFuncSetAttribute(k_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<double>, kBatchThreads, smem);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return std::max(occ, 0) * device_sm_count();
}

cudaError_t launch_batch(int dtype, const BatchArgs &a, int grid, size_t smem, cudaStream_t st) {
    if (dtype == QS_C64) k_batch<float><<<grid, kBatchThreads, smem, st>>>(a);
    else k_batch<double><<<grid, kBatchThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace qs
