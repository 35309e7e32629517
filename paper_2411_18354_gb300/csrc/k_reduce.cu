// k_reduce.cu -- one-pass <Z_i> for every qubit and the squared norm.
//
// <Z_i> = sum_k |psi_k|^2 (1 - 2 bit_i(k)) = T - 2 S_i with T = sum_k |psi_k|^2 and
// S_i = sum over k with bit i set. One read of the state gives T and all S_i:
//  - a block works on tiles of 2^TB consecutive amplitudes; inside a tile the amplitude
//    offset is (j, thread, v) with v the element inside a 16-byte vector (complex64 only),
//    the thread index (lane bits, then warp bits) and the unrolled load index j (4 bits);
//  - each thread sums |psi|^2 over its 32 (complex64) or 16 (complex128) values, also per
//    v bit and per j bit (those bits are compile-time constants of the unrolled loop);
//  - warp shuffles reduce the per-thread sums and form the lane-bit sums;
//  - warp totals give the warp-bit sums; bits at or above TB are constant per tile and
//    take the tile total when set;
//  - thread b of the block owns output b and accumulates it over the block's tiles; a final
//    one-block pass adds the per-block results in float64 in a fixed order.
// Complex64: per-thread, per-warp and per-tile sums are float32 (at most 32, 1024 and 8192
// terms), the running sum over a block's tiles is a compensated (Kahan) float32 sum, and the
// sum over blocks is float64. Complex128: float64 everywhere. The result does not depend on
// scheduling (fixed tile-to-block assignment and fixed summation order).
// Complex128 is bound by the FP64 pipe (GB300 issues about 2 FP64 operations per SM per clock),
// so its sums are arranged for fewer operations: a thread's 16 values go through a pairwise
// tree whose partial sums also give the four j-bit sums (26 adds instead of 48); the warp
// forms the lane-bit sums on the way while it reduces the total (a butterfly: 15 shuffles and
// adds instead of 25) and reduces the four j-bit sums by a transposed reduce-scatter that
// leaves each in its own lanes (6 instead of 20).
#include <algorithm>

#include "k_gate.cuh"

namespace qs {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1024;
constexpr int kJ = 16;  // unrolled loads per thread per tile

template <typename Real> struct RedT;
template <> struct RedT<float> {
    using T2 = float2;
    static constexpr int VB = 1;  // log2(amplitudes per 16-byte load)
};
template <> struct RedT<double> {
    using T2 = double2;
    static constexpr int VB = 0;
};

template <typename A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename Real>
__global__ void __launch_bounds__(kRedThreads)
k_expz_tiles(const typename RedT<Real>::T2 *__restrict__ psi, int n, uint64_t ntiles, double *__restrict__ partials) {
    using A = Real;  // per-thread / per-warp accumulator type
    constexpr int VB = RedT<Real>::VB;
    constexpr int TB = VB + 8 + 4;
    // per-warp values: [0] total, [1..VB] v-bit, [1+VB .. 4+VB] j bits, [5+VB .. 9+VB] lane bits
    constexpr int NV = 1 + VB + 4 + 5;
    __shared__ A wpart[kRedThreads / 32][NV];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    Acc<Real> acc{};  // output `tid` of this block, over its tiles
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        A tot = 0, sv = 0, sj[4] = {0, 0, 0, 0};
        if constexpr (VB == 1) {
            const float4 *base = reinterpret_cast<const float4 *>(psi) + (tile << (TB - 1));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float4 q[kJ / 2];
#pragma unroll
                for (int jj = 0; jj < kJ / 2; ++jj) q[jj] = base[(h * (kJ / 2) + jj) * kRedThreads + tid];
#pragma unroll
                for (int jj = 0; jj < kJ / 2; ++jj) {
                    const int j = h * (kJ / 2) + jj;
                    const A p0 = (A)fmaf(q[jj].x, q[jj].x, q[jj].y * q[jj].y);
                    const A p1 = (A)fmaf(q[jj].z, q[jj].z, q[jj].w * q[jj].w);
                    const A s = p0 + p1;
                    tot += s;
                    sv += p1;
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if ((j >> b) & 1) sj[b] += s;
                }
            }
        } else {
            // complex128: |psi|^2 of the thread's 16 values, a pairwise tree, per-warp sums
            const double2 *base = reinterpret_cast<const double2 *>(psi) + (tile << TB);
            double p[kJ];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                double2 q[kJ / 2];
#pragma unroll
                for (int jj = 0; jj < kJ / 2; ++jj) q[jj] = base[(h * (kJ / 2) + jj) * kRedThreads + tid];
#pragma unroll
                for (int jj = 0; jj < kJ / 2; ++jj) p[h * (kJ / 2) + jj] = fma(q[jj].x, q[jj].x, q[jj].y * q[jj].y);
            }
            double a[8], b4[4], c2[2];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = p[2 * i] + p[2 * i + 1];
#pragma unroll
            for (int i = 0; i < 4; ++i) b4[i] = a[2 * i] + a[2 * i + 1];
            c2[0] = b4[0] + b4[1];
            c2[1] = b4[2] + b4[3];
            double t = c2[0] + c2[1];
            double sjt[4];  // sum over the thread's j with bit b set
            sjt[3] = c2[1];
            sjt[2] = b4[1] + b4[3];
            sjt[1] = (a[1] + a[3]) + (a[5] + a[7]);
            sjt[0] = ((p[1] + p[3]) + (p[5] + p[7])) + ((p[9] + p[11]) + (p[13] + p[15]));
            // butterfly over the lane bits: before step b, t sums the 2^b lanes that differ from
            // this one below bit b; the half with bit b set is this lane's t or its partner's
            double lb[5];
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                const double pt = __shfl_xor_sync(0xffffffffu, t, 1 << b);
#pragma unroll
                for (int c = 0; c < b; ++c) lb[c] += __shfl_xor_sync(0xffffffffu, lb[c], 1 << b);
                lb[b] = ((lane >> b) & 1) ? t : pt;
                t += pt;
            }
            // j-bit sums: lanes with lane bit 4 = 0 keep sums 0, 1 and lanes with bit 4 = 1 keep
            // 2, 3; then bit 3 splits those; bits 2..0 finish each sum. Sum q ends in the lanes
            // with (lane >> 3) == q.
            const bool h4 = (lane >> 4) & 1, h3 = (lane >> 3) & 1;
            const double k0 = (h4 ? sjt[2] : sjt[0]) + __shfl_xor_sync(0xffffffffu, h4 ? sjt[0] : sjt[2], 16);
            const double k1 = (h4 ? sjt[3] : sjt[1]) + __shfl_xor_sync(0xffffffffu, h4 ? sjt[1] : sjt[3], 16);
            double vj = (h3 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, h3 ? k0 : k1, 8);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) vj += __shfl_xor_sync(0xffffffffu, vj, o);
            if (lane == 0) {
                wpart[warp][0] = (A)t;
#pragma unroll
                for (int b = 0; b < 5; ++b) wpart[warp][5 + b] = (A)lb[b];
            }
            if ((lane & 7) == 0) wpart[warp][1 + (lane >> 3)] = (A)vj;
        }
        if constexpr (VB == 1) {
            // lane-bit sums before the total is reduced
            A sl[5];
#pragma unroll
            for (int b = 0; b < 5; ++b) sl[b] = warp_sum<A>(((lane >> b) & 1) ? tot : (A)0);
            tot = warp_sum<A>(tot);
            sv = warp_sum<A>(sv);
#pragma unroll
            for (int b = 0; b < 4; ++b) sj[b] = warp_sum<A>(sj[b]);
            if (lane == 0) {
                wpart[warp][0] = tot;
                wpart[warp][1] = sv;
#pragma unroll
                for (int b = 0; b < 4; ++b) wpart[warp][1 + VB + b] = sj[b];
#pragma unroll
                for (int b = 0; b < 5; ++b) wpart[warp][5 + VB + b] = sl[b];
            }
        }
        __syncthreads();
        if (tid <= n) {
            // output tid: tid == n -> total; else S_tid (sum over amplitudes with bit tid set)
            A v = 0;
            const int b = tid;
            if (b == n) {
                for (int w = 0; w < kRedThreads / 32; ++w) v += wpart[w][0];
            } else if (b < VB) {
                for (int w = 0; w < kRedThreads / 32; ++w) v += wpart[w][1];
            } else if (b < VB + 5) {
                for (int w = 0; w < kRedThreads / 32; ++w) v += wpart[w][5 + VB + (b - VB)];
            } else if (b < VB + 8) {
                for (int w = 0; w < kRedThreads / 32; ++w)
                    if ((w >> (b - VB - 5)) & 1) v += wpart[w][0];
            } else if (b < TB) {
                for (int w = 0; w < kRedThreads / 32; ++w) v += wpart[w][1 + VB + (b - VB - 8)];
            } else if ((tile >> (b - TB)) & 1ull) {
                for (int w = 0; w < kRedThreads / 32; ++w) v += wpart[w][0];
            }
            acc.add(v);
        }
        __syncthreads();
    }
    if (tid <= n) partials[(size_t)tid * gridDim.x + blockIdx.x] = acc.value();  // output-major
}

// Fixed-order sum of the per-block partials (output-major: partials[b * nblocks + g]); one
// block, a warp per output: lane l adds blocks l, l + 32, ... and the warp combines its lanes
// in a fixed shuffle order.
__global__ void k_expz_final(const double *__restrict__ partials, int nblocks, int n,
                             double *__restrict__ out_z, double *__restrict__ out_norm2) {
    __shared__ double sums[kMaxQubits + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b = warp; b <= n; b += nw) {
        double v = 0.0;
        for (int g = lane; g < nblocks; g += 32) v += partials[(size_t)b * nblocks + g];
        v = warp_sum<double>(v);
        if (lane == 0) sums[b] = v;
    }
    __syncthreads();
    const int b = threadIdx.x;
    if (b < n && out_z) out_z[b] = sums[n] - 2.0 * sums[b];
    if (b == n && out_norm2) *out_norm2 = sums[n];
}

// Small states (fewer amplitudes than one tile): one block, float64 per amplitude.
template <typename Real>
__global__ void __launch_bounds__(kRedThreads)
k_expz_small(const typename RedT<Real>::T2 *__restrict__ psi, int n, double *__restrict__ out_z,
             double *__restrict__ out_norm2) {
    constexpr int kMaxSmallBits = 13;
    __shared__ double red[kRedThreads / 32][kMaxSmallBits + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t N = 1ull << n;
    double tot = 0.0, s[kMaxSmallBits];
#pragma unroll
    for (int b = 0; b < kMaxSmallBits; ++b) s[b] = 0.0;
    for (uint64_t k = tid; k < N; k += kRedThreads) {
        const double re = (double)psi[k].x, im = (double)psi[k].y;
        const double p = re * re + im * im;
        tot += p;
#pragma unroll
        for (int b = 0; b < kMaxSmallBits; ++b)
            if (b < n && ((k >> b) & 1ull)) s[b] += p;
    }
    tot = warp_sum<double>(tot);
#pragma unroll
    for (int b = 0; b < kMaxSmallBits; ++b) s[b] = warp_sum<double>(s[b]);
    if (lane == 0) {
        red[warp][kMaxSmallBits] = tot;
#pragma unroll
        for (int b = 0; b < kMaxSmallBits; ++b) red[warp][b] = s[b];
    }
    __syncthreads();
    if (tid == 0) {
        double T = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) T += red[w][kMaxSmallBits];
        for (int b = 0; b < n; ++b) {
            double S = 0.0;
            for (int w = 0; w < kRedThreads / 32; ++w) S += red[w][b];
            if (out_z) out_z[b] = T - 2.0 * S;
        }
        if (out_norm2) *out_norm2 = T;
    }
}

template <typename Real>
cudaError_t expect_z_impl(const void *psi, int n, double *scratch, double *out_z, double *out_norm2,
                          cudaStream_t st) {
    using T2 = typename RedT<Real>::T2;
    constexpr int TB = RedT<Real>::VB + 8 + 4;
    const T2 *p = reinterpret_cast<const T2 *>(psi);
    if (n < TB) {
        k_expz_small<Real><<<1, kRedThreads, 0, st>>>(p, n, out_z, out_norm2);
        return cudaGetLastError();
    }
    static const int occ = [] {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_expz_tiles<Real>, kRedThreads, 0) != cudaSuccess || o < 1) o = 1;
        return o;
    }();
    const uint64_t ntiles = 1ull << (n - TB);
    const uint64_t cap = std::min<uint64_t>((uint64_t)kRedMaxBlocks, (uint64_t)device_sm_count() * occ);
    const int grid = (int)std::min<uint64_t>(ntiles, cap);
    k_expz_tiles<Real><<<grid, kRedThreads, 0, st>>>(p, n, ntiles, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_expz_final<<<1, 1024, 0, st>>>(scratch, grid, n, out_z, out_norm2);
    return cudaGetLastError();
}

}  // namespace

size_t reduce_scratch_doubles(int n) { return (size_t)kRedMaxBlocks * (size_t)(n + 1); }

cudaError_t launch_expect_z(int dtype, const void *psi, int n, double *scratch, double *out_z,
                            double *out_norm2, cudaStream_t st) {
    if (dtype == QS_Q30) return launch_expect_z_q30(psi, n, scratch, out_z, out_norm2, st);
    return dtype == QS_C64 ? expect_z_impl<float>(psi, n, scratch, out_z, out_norm2, st)
                           : expect_z_impl<double>(psi, n, scratch, out_z, out_norm2, st);
}

}  // namespace qs
