// k_gate_q30.cu -- the gate update and <Z_i> for fixed-point amplitudes (QS_Q30).
//
// The paper's conclusion names fixed-point amplitudes as a way to cut the FPGA's arithmetic
// cost. Here a QS_Q30 state stores each real and imaginary part as a signed 32-bit integer v
// meaning v / 2^30 (Q1.30: range [-2, 2), resolution 2^-30), 8 bytes per amplitude like
// complex64. The gate matrix is rounded once to the same format on the host. A selected pair
// is updated exactly in 64-bit integers and rounded once per output component:
//     x'_re = sat32((ar xr - ai xi + br yr - bi yi + 2^29) >> 30)      (and likewise im, y')
// i.e. round to nearest with ties toward +infinity, then saturation to the int32 range. With
// |components| <= 1 (2^30) and |matrix entries| <= 1 every product is below 2^60 in magnitude
// and the sum of four below 2^62, so the 64-bit sum never overflows. Exchanges (X, CNOT,
// Toffoli) move the integers unchanged. Every operation is exact integer arithmetic, so the
// GPU result equals the CPU oracle's (same formula) bit for bit. The pairs are scheduled on
// the reduced iteration set exactly as for the floating-point states (Section III-B).
#include <algorithm>

#include "k_gate.cuh"
#include "qs_debug.cuh"

namespace qs {
namespace {

struct Q30Gate {
    uint64_t mask[kMaxSeg];
    uint64_t ins, tbit, cmask, cvals;
    int32_t shift[kMaxSeg];
    int32_t m[8];  // a, b, c, d as (re, im), Q1.30
};

__device__ __forceinline__ int32_t q30_round(long long s) {
    long long r = (s + (1ll << 29)) >> 30;  // arithmetic shift: floor((s + 2^29) / 2^30)
    r = r > 2147483647ll ? 2147483647ll : (r < -2147483648ll ? -2147483648ll : r);
    return (int32_t)r;
}

// a x + b y for Q1.30 complex values (m = a.re, a.im, b.re, b.im).
__device__ __forceinline__ int2 q30_mac(const int32_t *m, int2 x, int2 y) {
    const long long re = (long long)m[0] * x.x - (long long)m[1] * x.y + (long long)m[2] * y.x - (long long)m[3] * y.y;
    const long long im = (long long)m[0] * x.y + (long long)m[1] * x.x + (long long)m[2] * y.y + (long long)m[3] * y.x;
    return make_int2(q30_round(re), q30_round(im));
}

template <bool SWAP>
__device__ __forceinline__ void q30_pair(int2 &x, int2 &y, const int32_t *m) {
    if (SWAP) {
        const int2 t = x;
        x = y;
        y = t;
    } else {
        const int2 nx = q30_mac(m, x, y), ny = q30_mac(m + 4, x, y);
        x = nx;
        y = ny;
    }
}

template <int NS>
__device__ __forceinline__ uint64_t q30_deposit(uint64_t j, const Q30Gate &g) {
    uint64_t r = g.ins;
#pragma unroll
    for (int s = 0; s < NS; ++s) r |= (j << g.shift[s]) & g.mask[s];
    return r;
}

constexpr int kQ30Threads = 256;

// One unit per thread per step (like k_gate): LAY_ADJ: R adjacent pairs from lo (t = 0);
// LAY_SPLIT: R consecutive amplitudes at lo and at lo + 2^t. MASKED: the baseline comparator.
template <int NS, int LAY, int R, bool SWAP, bool MASKED>
__global__ void __launch_bounds__(kQ30Threads) k_gate_q30(int2 *__restrict__ psi, const Q30Gate g, uint64_t units) {
    const int r = R == 2 ? 1 : 0;
    const uint64_t step = (uint64_t)gridDim.x * kQ30Threads;
    for (uint64_t u = (uint64_t)blockIdx.x * kQ30Threads + threadIdx.x; u < units; u += step) {
        const uint64_t lo = q30_deposit<NS>(u << r, g);
        if (MASKED && (lo & g.cmask) != g.cvals) continue;
        if (LAY == LAY_ADJ) {
            if (!QS_DBG_OK(lo, 2 * R)) continue;
            int2 v[2 * R];
#pragma unroll
            for (int i = 0; i < 2 * R; ++i) v[i] = psi[lo + i];
#pragma unroll
            for (int i = 0; i < R; ++i) q30_pair<SWAP>(v[2 * i], v[2 * i + 1], g.m);
#pragma unroll
            for (int i = 0; i < 2 * R; ++i) psi[lo + i] = v[i];
            QS_DBG_WRITE(lo, 2 * R);
        } else {
            if (!QS_DBG_OK(lo, R) || !QS_DBG_OK(lo | g.tbit, R)) continue;
            int2 x[R], y[R];
            if (R == 2) {
                const int4 a = *reinterpret_cast<const int4 *>(psi + lo);
                const int4 b = *reinterpret_cast<const int4 *>(psi + (lo | g.tbit));
                x[0] = make_int2(a.x, a.y);
                x[R - 1] = make_int2(a.z, a.w);
                y[0] = make_int2(b.x, b.y);
                y[R - 1] = make_int2(b.z, b.w);
            } else {
                x[0] = psi[lo];
                y[0] = psi[lo | g.tbit];
            }
#pragma unroll
            for (int i = 0; i < R; ++i) q30_pair<SWAP>(x[i], y[i], g.m);
            if (R == 2) {
                *reinterpret_cast<int4 *>(psi + lo) = make_int4(x[0].x, x[0].y, x[R - 1].x, x[R - 1].y);
                *reinterpret_cast<int4 *>(psi + (lo | g.tbit)) = make_int4(y[0].x, y[0].y, y[R - 1].x, y[R - 1].y);
            } else {
                psi[lo] = x[0];
                psi[lo | g.tbit] = y[0];
            }
            QS_DBG_WRITE(lo, R);
            QS_DBG_WRITE(lo | g.tbit, R);
        }
    }
}

// Round half away from zero, saturated: the Q1.30 value of a matrix entry.
int32_t quantize_q30(double v) {
    const double s = v * 1073741824.0;  // 2^30
    double r = s >= 0 ? std::floor(s + 0.5) : -std::floor(-s + 0.5);
    if (r > 2147483647.0) r = 2147483647.0;
    if (r < -2147483648.0) r = -2147483648.0;
    return (int32_t)r;
}

template <int NS, int LAY, int R, bool SWAP, bool MASKED>
cudaError_t go_q30(void *psi, const Q30Gate &g, uint64_t units, cudaStream_t st) {
    const uint64_t need = (units + kQ30Threads - 1) / kQ30Threads;
    const uint64_t cap = (uint64_t)device_sm_count() * 8;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(need, cap));
    k_gate_q30<NS, LAY, R, SWAP, MASKED><<<grid, kQ30Threads, 0, st>>>(static_cast<int2 *>(psi), g, units);
    return cudaGetLastError();
}

template <int NS, bool MASKED>
cudaError_t by_shape_q30(void *psi, const GatePlan &p, const Q30Gate &g, cudaStream_t st) {
    const bool swap = !MASKED && p.op == OP_SWAP;
    if (p.layout == LAY_ADJ)
        return swap ? go_q30<NS, LAY_ADJ, 1, true, MASKED>(psi, g, p.units, st)
                    : go_q30<NS, LAY_ADJ, 1, false, MASKED>(psi, g, p.units, st);
    if (p.r == 1)
        return swap ? go_q30<NS, LAY_SPLIT, 2, true, MASKED>(psi, g, p.units, st)
                    : go_q30<NS, LAY_SPLIT, 2, false, MASKED>(psi, g, p.units, st);
    return swap ? go_q30<NS, LAY_SPLIT, 1, true, MASKED>(psi, g, p.units, st)
                : go_q30<NS, LAY_SPLIT, 1, false, MASKED>(psi, g, p.units, st);
}

// <Z_i> and the squared norm: tiles of 2^12 amplitudes; a thread sums p_k = re^2 + im^2 (exact
// in 64 bits, then float64 scaled by 2^-60) over its 16 values (j bits 8..11 of the offset),
// warps form the lane-bit sums, thread 0 adds everything of the tile to the block's sums in a
// fixed order; one final pass adds the blocks' sums in order. States below 2^12 amplitudes use
// the same kernel with one partial tile.
constexpr int kQTile = 12;
constexpr int kQBlocks = 1024;

__global__ void __launch_bounds__(256) k_expz_q30(const int2 *__restrict__ psi, int n, uint64_t ntiles,
                                                  double *__restrict__ partials) {
    __shared__ double wpart[8][10];  // per warp: total, 5 lane bits, 4 j bits
    __shared__ double bsum[kMaxQubits + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t N = 1ull << n;
    for (int i = tid; i <= n; i += blockDim.x) bsum[i] = 0.0;
    __syncthreads();
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        double t = 0.0, sj[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint64_t k = (tile << kQTile) + ((uint64_t)j << 8) + tid;
            if (k < N) {
                const int2 v = psi[k];
                const double p = (double)((long long)v.x * v.x + (long long)v.y * v.y) * 8.673617379884035e-19;  // 2^-60
                t += p;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if ((j >> b) & 1) sj[b] += p;
            }
        }
        double w[10];
        w[0] = t;
#pragma unroll
        for (int b = 0; b < 5; ++b) w[1 + b] = ((lane >> b) & 1) ? t : 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) w[6 + b] = sj[b];
#pragma unroll
        for (int i = 0; i < 10; ++i)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w[i] += __shfl_xor_sync(0xffffffffu, w[i], o);
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < 10; ++i) wpart[warp][i] = w[i];
        __syncthreads();
        if (tid == 0) {
            double tt = 0.0;
            for (int q = 0; q < 8; ++q) tt += wpart[q][0];
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                if (i < 5) {
                    for (int q = 0; q < 8; ++q) s += wpart[q][1 + i];
                } else if (i < 8) {
                    for (int q = 0; q < 8; ++q)
                        if ((q >> (i - 5)) & 1) s += wpart[q][0];
                } else if (i < kQTile) {
                    for (int q = 0; q < 8; ++q) s += wpart[q][6 + (i - 8)];
                } else {
                    s = ((tile >> (i - kQTile)) & 1) ? tt : 0.0;
                }
                bsum[i] += s;
            }
            bsum[n] += tt;
        }
        __syncthreads();
    }
    for (int i = tid; i <= n; i += blockDim.x) partials[(uint64_t)i * gridDim.x + blockIdx.x] = bsum[i];
}

// out_z[i] = T - 2 S_i, out_norm2 = T, from the per-block sums (added in block order).
__global__ void k_expz_q30_final(const double *__restrict__ partials, int nblocks, int n, double *__restrict__ out_z,
                                 double *__restrict__ out_norm2) {
    __shared__ double tot;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += partials[(uint64_t)n * nblocks + b];
        tot = t;
        if (out_norm2) *out_norm2 = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[(uint64_t)i * nblocks + b];
        if (out_z) out_z[i] = tot - 2.0 * s;
    }
}

}  // namespace

cudaError_t launch_gate_q30(void *psi, const GatePlan &p, bool masked, uint64_t cmask, uint64_t cvals,
                            cudaStream_t st) {
    if (p.units == 0) return cudaSuccess;
    Q30Gate g;
    for (int s = 0; s < kMaxSeg; ++s) {
        g.mask[s] = s < p.map.nseg ? p.map.mask[s] : 0;
        g.shift[s] = s < p.map.nseg ? p.map.shift[s] : 0;
    }
    g.ins = p.map.ins;
    g.tbit = p.tbit;
    g.cmask = cmask;
    g.cvals = cvals;
    for (int i = 0; i < 8; ++i) g.m[i] = quantize_q30(p.Ufull[i]);
    const int ns = p.map.nseg;
    if (masked) {
        if (ns <= 2) return by_shape_q30<2, true>(psi, p, g, st);
        if (ns <= 4) return by_shape_q30<4, true>(psi, p, g, st);
        return by_shape_q30<kMaxSeg, true>(psi, p, g, st);
    }
    if (ns <= 2) return by_shape_q30<2, false>(psi, p, g, st);
    if (ns <= 4) return by_shape_q30<4, false>(psi, p, g, st);
    return by_shape_q30<kMaxSeg, false>(psi, p, g, st);
}

size_t reduce_scratch_doubles_q30(int n) { return (size_t)(n + 1) * kQBlocks; }

cudaError_t launch_expect_z_q30(const void *psi, int n, double *scratch, double *out_z, double *out_norm2,
                                cudaStream_t st) {
    const uint64_t ntiles = n >= kQTile ? (1ull << (n - kQTile)) : 1;
    const unsigned blocks = (unsigned)std::min<uint64_t>(ntiles, std::min<uint64_t>(kQBlocks, (uint64_t)device_sm_count() * 4));
    k_expz_q30<<<blocks, 256, 0, st>>>(static_cast<const int2 *>(psi), n, ntiles, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_expz_q30_final<<<1, 64, 0, st>>>(scratch, (int)blocks, n, out_z, out_norm2);
    return cudaGetLastError();
}

}  // namespace qs
