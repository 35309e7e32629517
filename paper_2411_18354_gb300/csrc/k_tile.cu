// k_tile.cu -- fused tile-pass kernels (forward, and adjoint over psi and lambda).
#include <algorithm>

#include "k_gate.cuh"
#include "k_tile.cuh"

namespace qs {
namespace {

template <typename Real> struct TileT;
template <> struct TileT<float> {
    using T2 = float2;
    using V = float4;  // 2 amplitudes per 16-byte vector
    static constexpr int VEC = 2;
};
template <> struct TileT<double> {
    using T2 = double2;
    using V = double2;  // 1 amplitude per 16-byte vector
    static constexpr int VEC = 1;
};

__device__ __forceinline__ uint64_t tile_base(const TilePass &P, uint64_t tau) {
    uint64_t b = 0;
    for (int s = 0; s < P.tnseg; ++s) b |= (tau << P.tshift[s]) & P.tmask[s];
    return b;
}

__device__ __forceinline__ uint64_t scatter_local(const TilePass &P, uint32_t o) {
    uint64_t g = 0;
    for (int r = 0; r < P.nruns; ++r)
        g |= (uint64_t)((o >> P.run_src[r]) & ((1u << P.run_len[r]) - 1u)) << P.run_dst[r];
    return g;
}

__device__ __forceinline__ uint32_t local_pair(const TileGate &G, uint32_t j) {
    uint32_t lo = G.ins;
    for (int s = 0; s < G.nseg; ++s) lo |= (j << G.shift[s]) & G.mask[s];
    return lo;
}

template <typename T2, typename Real>
__device__ __forceinline__ void apply_pair(int op, int side, const double *Ud, T2 &x, T2 &y) {
    if (op == OP_GEN) {
        const Real a0 = (Real)Ud[0], a1 = (Real)Ud[1], b0 = (Real)Ud[2], b1 = (Real)Ud[3];
        const Real c0 = (Real)Ud[4], c1 = (Real)Ud[5], d0 = (Real)Ud[6], d1 = (Real)Ud[7];
        T2 nx = cmac<T2, Real>(a0, a1, x, b0, b1, y);
        T2 ny = cmac<T2, Real>(c0, c1, x, d0, d1, y);
        x = nx;
        y = ny;
    } else if (op == OP_SWAP) {
        T2 t = x;
        x = y;
        y = t;
    } else if (op == OP_DIAG) {
        x = cmul<T2, Real>((Real)Ud[0], (Real)Ud[1], x);
        y = cmul<T2, Real>((Real)Ud[6], (Real)Ud[7], y);
    } else {  // OP_SIDE: scalar in U[0..1]
        if (side) y = cmul<T2, Real>((Real)Ud[0], (Real)Ud[1], y);
        else x = cmul<T2, Real>((Real)Ud[0], (Real)Ud[1], x);
    }
}

template <typename Real, bool ADJ>
__global__ void __launch_bounds__(kTileThreads)
k_tile_pass(typename TileT<Real>::T2 *__restrict__ psi, typename TileT<Real>::T2 *__restrict__ lam, const TilePass P,
            const TileGate *__restrict__ gates, double *__restrict__ part, size_t part_stride) {
    using T2 = typename TileT<Real>::T2;
    using V = typename TileT<Real>::V;
    constexpr int VEC = TileT<Real>::VEC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t T = 1u << P.k;
    T2 *tp = reinterpret_cast<T2 *>(smem_raw);
    T2 *tl = tp + T;  // adjoint: lambda tile
    double *acc = reinterpret_cast<double *>(smem_raw + (ADJ ? 2 : 1) * (size_t)T * sizeof(T2));  // [kTileMaxParam][8]
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (ADJ) {
        for (int i = tid; i < kTileMaxParam * (kTileThreads / 32); i += kTileThreads) acc[i] = 0.0;
        __syncthreads();
    }
    const TileGate *G0 = gates + P.gate_begin;
    const uint32_t nvec = T / VEC;
    for (uint64_t tau = blockIdx.x; tau < P.ntiles; tau += gridDim.x) {
        const uint64_t base = tile_base(P, tau);
        bool any = false;
        for (int g = 0; g < P.gate_count; ++g) any |= ((base & G0[g].hmask) == G0[g].hvals);
        if (!any) continue;  // no gate of the pass selects this tile
        for (uint32_t v = tid; v < nvec; v += kTileThreads) {
            const uint64_t gi = base | scatter_local(P, v * VEC);
            reinterpret_cast<V *>(tp)[v] = *reinterpret_cast<const V *>(psi + gi);
            if (ADJ) reinterpret_cast<V *>(tl)[v] = *reinterpret_cast<const V *>(lam + gi);
        }
        __syncthreads();
        for (int g = 0; g < P.gate_count; ++g) {
            const TileGate &G = G0[g];
            if ((base & G.hmask) != G.hvals) continue;  // uniform over the block
            const uint32_t pairs = 1u << G.log_pairs;
            Real dot = 0;
            for (uint32_t j = tid; j < pairs; j += kTileThreads) {
                const uint32_t lo = local_pair(G, j), hi = lo | G.tbit;
                T2 x = tp[lo], y = tp[hi];
                apply_pair<T2, Real>(G.op, G.side, G.U, x, y);
                tp[lo] = x;
                tp[hi] = y;
                if (ADJ) {
                    T2 a = tl[lo], b = tl[hi];
                    if (G.slot >= 0) {
                        T2 mx = x, my = y;
                        apply_pair<T2, Real>(G.op == OP_DIAG ? OP_DIAG : OP_GEN, 0, G.D, mx, my);
                        dot += a.x * mx.x + a.y * mx.y + b.x * my.x + b.y * my.y;
                    }
                    apply_pair<T2, Real>(G.op, G.side, G.U, a, b);
                    tl[lo] = a;
                    tl[hi] = b;
                }
            }
            if (ADJ && G.slot >= 0) {
                double d = (double)dot;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                if (lane == 0) acc[G.slot * (kTileThreads / 32) + warp] += d;
            }
            __syncthreads();
        }
        for (uint32_t v = tid; v < nvec; v += kTileThreads) {
            const uint64_t gi = base | scatter_local(P, v * VEC);
            *reinterpret_cast<V *>(psi + gi) = reinterpret_cast<const V *>(tp)[v];
            if (ADJ) *reinterpret_cast<V *>(lam + gi) = reinterpret_cast<const V *>(tl)[v];
        }
        __syncthreads();
    }
    if (ADJ) {
        __syncthreads();
        for (int p = tid; p < P.nparam; p += kTileThreads) {
            double s = 0.0;
            for (int w = 0; w < kTileThreads / 32; ++w) s += acc[p * (kTileThreads / 32) + w];
            part[(size_t)P.param_gslot[p] * part_stride + blockIdx.x] = s;
        }
    }
}

template <typename Real, bool ADJ>
cudaError_t go(void *psi, void *lam, const TilePass &p, const TileGate *gates, double *part, size_t part_stride,
               cudaStream_t st) {
    auto kern = k_tile_pass<Real, ADJ>;
    const size_t smem = tile_smem_bytes(sizeof(Real) == 4 ? QS_C64 : QS_C128, p.k, ADJ);
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTileThreads, smem) != cudaSuccess || occ < 1) occ = 1;
    uint64_t cap = (uint64_t)device_sm_count() * occ;
    if (ADJ) cap = std::min<uint64_t>(cap, part_stride);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(p.ntiles, cap));
    using T2 = typename TileT<Real>::T2;
    kern<<<grid, kTileThreads, smem, st>>>(reinterpret_cast<T2 *>(psi), reinterpret_cast<T2 *>(lam), p, gates, part,
                                           part_stride);
    return cudaGetLastError();
}

}  // namespace

size_t tile_smem_bytes(int dtype, int k, bool adjoint) {
    const size_t es = dtype == QS_C64 ? 8 : 16;
    return (adjoint ? 2 : 1) * (size_t(1) << k) * es + (adjoint ? kTileMaxParam * (kTileThreads / 32) * sizeof(double) : 0);
}

cudaError_t launch_tile_pass(int dtype, void *psi, void *lam, const TilePass &p, const TileGate *gates, double *part,
                             size_t part_stride, cudaStream_t st) {
    const bool adj = lam != nullptr;
    if (dtype == QS_C64)
        return adj ? go<float, true>(psi, lam, p, gates, part, part_stride, st)
                   : go<float, false>(psi, lam, p, gates, part, part_stride, st);
    return adj ? go<double, true>(psi, lam, p, gates, part, part_stride, st)
               : go<double, false>(psi, lam, p, gates, part, part_stride, st);
}

}  // namespace qs
