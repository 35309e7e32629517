// k_adjoint.cu -- adjoint (reverse-sweep) gradient kernels.
//
// For E = <psi|O|psi>, psi = U_G ... U_1 |psi_in>, O = sum_i Z_i:
//   lambda = O psi;  for g = G .. 1:  psi <- U_g^dagger psi;
//                                     if g has a parameter: grad += 2 Re <lambda| dU_g psi>;
//                                     lambda <- U_g^dagger lambda.
// No intermediate state is stored: un-applying a unitary gate recovers the state before
// it. One kernel does the three steps of one gate on the gate's reduced iteration set
// (the 2^(n-1-c) control-satisfied pairs, Section III-B of arXiv 2411.18354), reading
// and writing psi and lambda once. The inner product is summed per thread in the state's
// precision, per warp and block in float64, and per block written to a fixed slot; a
// final pass adds the slots in a fixed order.
#include <algorithm>

#include "k_gate.cuh"
#include "qs_debug.cuh"

namespace qs {

constexpr int kAdjMaxBlocks = 1024;

namespace {

template <typename Real> struct DevMat { Real m[8]; };

template <typename Real, typename Idx, int NS, int LAY, int R, int OP, bool PARAM>
__global__ void __launch_bounds__(kGateThreads)
k_adj_step(typename CxT<Real>::T *__restrict__ psi, typename CxT<Real>::T *__restrict__ lam,
           const DevGate<Real, Idx> g, const DevMat<Real> du, Idx units, double *__restrict__ part) {
    using T2 = typename CxT<Real>::T;
    constexpr int r = Log2<R>::v;
    constexpr int A = (LAY == LAY_ADJ) ? 2 * R : R;
    constexpr int DOP = (OP == OP_DIAG) ? OP_DIAG : (OP == OP_REAL) ? OP_REAL : OP_GEN;  // structure of dU
    Real acc = 0;
    const Idx step = (Idx)gridDim.x * kGateThreads;
    for (Idx u = (Idx)blockIdx.x * kGateThreads + threadIdx.x; u < units; u += step) {
        const Idx lo = deposit<Idx, NS>(u << r, g);
        if (LAY == LAY_ADJ ? !QS_DBG_OK(lo, A) : (!QS_DBG_OK(lo, R) || !QS_DBG_OK(lo | g.tbit, R))) continue;
        T2 px[A], py[(LAY == LAY_SPLIT) ? R : 1], lx[A], ly[(LAY == LAY_SPLIT) ? R : 1];
        if (LAY == LAY_ADJ) {
            Vec<Real, A>::ld(psi + lo, px);
            Vec<Real, A>::ld(lam + lo, lx);
        } else {
            Vec<Real, R>::ld(psi + lo, px);
            Vec<Real, R>::ld(psi + (lo | g.tbit), py);
            Vec<Real, R>::ld(lam + lo, lx);
            Vec<Real, R>::ld(lam + (lo | g.tbit), ly);
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            T2 &x = (LAY == LAY_ADJ) ? px[2 * i] : px[i];
            T2 &y = (LAY == LAY_ADJ) ? px[2 * i + 1] : py[i];
            T2 &a = (LAY == LAY_ADJ) ? lx[2 * i] : lx[i];
            T2 &b = (LAY == LAY_ADJ) ? lx[2 * i + 1] : ly[i];
            pair_update<OP, T2, Real>(x, y, g.m);  // psi <- U^dagger psi
            if (PARAM) {
                T2 mx = x, my = y;
                pair_update<DOP, T2, Real>(mx, my, du.m);  // mu = dU psi
                acc += a.x * mx.x + a.y * mx.y + b.x * my.x + b.y * my.y;  // Re <lambda|mu>
            }
            pair_update<OP, T2, Real>(a, b, g.m);  // lambda <- U^dagger lambda
        }
        if (LAY == LAY_ADJ) {
            Vec<Real, A>::st(psi + lo, px);
            Vec<Real, A>::st(lam + lo, lx);
            QS_DBG_WRITE(lo, A);
        } else {
            QS_DBG_WRITE(lo, R);
            QS_DBG_WRITE(lo | g.tbit, R);
            Vec<Real, R>::st(psi + lo, px);
            Vec<Real, R>::st(psi + (lo | g.tbit), py);
            Vec<Real, R>::st(lam + lo, lx);
            Vec<Real, R>::st(lam + (lo | g.tbit), ly);
        }
    }
    if (PARAM) {
        __shared__ double wsum[kGateThreads / 32];
        double v = (double)acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kGateThreads / 32; ++w) s += wsum[w];
            part[blockIdx.x] = s;
        }
    }
}

// lambda_k = (n - 2 popcount(k)) psi_k : O = sum_i Z_i is diagonal with that eigenvalue.
template <typename Real>
__global__ void k_obs_sumz(const typename CxT<Real>::T *__restrict__ psi, typename CxT<Real>::T *__restrict__ lam,
                           int n, uint64_t N) {
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += step) {
        const Real w = (Real)(n - 2 * __popcll(k));
        typename CxT<Real>::T v = psi[k];
        v.x *= w;
        v.y *= w;
        lam[k] = v;
    }
}

__global__ void k_sum_vec(const double *__restrict__ z, int n, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += z[i];
        *out = s;
    }
}

// slot_sum[s] = sum over blocks of part[s][b] (fixed order).
__global__ void k_slot_sums(const double *__restrict__ part, int nslots, double *__restrict__ slot_sum) {
    // a warp per slot: lane l adds blocks l, l + 32, ... (coalesced), then a fixed-order
    // shuffle reduction
    const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= nslots) return;  // uniform over the warp
    double v = 0.0;
    for (int b = lane; b < kAdjMaxBlocks; b += 32) v += part[(size_t)s * kAdjMaxBlocks + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) slot_sum[s] = v;
}

// grad[p] = 2 * sum of slot sums whose parameter is p (slots in gate order).
__global__ void k_grad_gather(const double *__restrict__ slot_sum, const int *__restrict__ slot_param, int nslots,
                              double *__restrict__ grad, int nparams) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nparams) return;
    double v = 0.0;
    for (int s = 0; s < nslots; ++s)
        if (slot_param[s] == p) v += slot_sum[s];
    grad[p] = 2.0 * v;
}

template <typename K>
int occ_of(K kern) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kGateThreads, 0) != cudaSuccess || o < 1) o = 1;
    return o;
}

template <typename Real, typename Idx, int NS, int LAY, int R, int OP, bool PARAM>
cudaError_t go(void *psi, void *lam, const GatePlan &p, const double *dU, double *part, cudaStream_t st) {
    auto kern = k_adj_step<Real, Idx, NS, LAY, R, OP, PARAM>;
    static const int occ = occ_of(kern);
    const uint64_t need = (p.units + kGateThreads - 1) / kGateThreads;
    const uint64_t cap = std::min<uint64_t>((uint64_t)device_sm_count() * occ, (uint64_t)kAdjMaxBlocks);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(need, cap));
    DevGate<Real, Idx> g;
    for (int s = 0; s < kMaxSeg; ++s) {
        g.mask[s] = (Idx)(s < p.map.nseg ? p.map.mask[s] : 0);
        g.shift[s] = s < p.map.nseg ? p.map.shift[s] : 0;
    }
    g.ins = (Idx)p.map.ins;
    g.tbit = (Idx)p.tbit;
    g.cmask = 0;
    g.cvals = 0;
    for (int i = 0; i < 8; ++i) g.m[i] = (Real)p.U[i];
    DevMat<Real> d;
    for (int i = 0; i < 8; ++i) d.m[i] = dU ? (Real)dU[i] : (Real)0;
    using T2 = typename CxT<Real>::T;
    kern<<<grid, kGateThreads, 0, st>>>(reinterpret_cast<T2 *>(psi), reinterpret_cast<T2 *>(lam), g, d, (Idx)p.units, part);
    return cudaGetLastError();
}

template <typename Real, typename Idx, int NS>
cudaError_t by_shape(void *psi, void *lam, const GatePlan &p, const double *dU, double *part, cudaStream_t st) {
    constexpr bool F = sizeof(Real) == 4;
    const bool param = dU != nullptr;
#define QS_ADJ_OPS(LAY, R)                                                                            \
    if (param) {                                                                                      \
        if (p.op == OP_GEN) return go<Real, Idx, NS, LAY, R, OP_GEN, true>(psi, lam, p, dU, part, st);   \
        if (p.op == OP_DIAG) return go<Real, Idx, NS, LAY, R, OP_DIAG, true>(psi, lam, p, dU, part, st); \
        if (p.op == OP_REAL) return go<Real, Idx, NS, LAY, R, OP_REAL, true>(psi, lam, p, dU, part, st); \
    } else {                                                                                          \
        if (p.op == OP_REAL) return go<Real, Idx, NS, LAY, R, OP_REAL, false>(psi, lam, p, dU, part, st); \
        if (p.op == OP_GEN) return go<Real, Idx, NS, LAY, R, OP_GEN, false>(psi, lam, p, dU, part, st);  \
        if (p.op == OP_DIAG) return go<Real, Idx, NS, LAY, R, OP_DIAG, false>(psi, lam, p, dU, part, st); \
        if (p.op == OP_SWAP) return go<Real, Idx, NS, LAY, R, OP_SWAP, false>(psi, lam, p, dU, part, st); \
    }
    if (p.layout == LAY_SPLIT) {
        if (p.r == 0) { QS_ADJ_OPS(LAY_SPLIT, 1) }
        else if (p.r == 1 && F) { QS_ADJ_OPS(LAY_SPLIT, 2) }
    } else if (p.r == 0) {
        QS_ADJ_OPS(LAY_ADJ, 1)
    }
#undef QS_ADJ_OPS
    return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t adj_step_impl(void *psi, void *lam, const GatePlan &p, const double *dU, double *part, cudaStream_t st) {
    if (p.units == 0) return cudaSuccess;
    const bool narrow = p.n <= 32;
    if (p.map.nseg <= 4)
        return narrow ? by_shape<Real, uint32_t, 4>(psi, lam, p, dU, part, st)
                      : by_shape<Real, uint64_t, 4>(psi, lam, p, dU, part, st);
    return narrow ? by_shape<Real, uint32_t, kMaxSeg>(psi, lam, p, dU, part, st)
                  : by_shape<Real, uint64_t, kMaxSeg>(psi, lam, p, dU, part, st);
}

}  // namespace

size_t adj_partials_per_slot() { return kAdjMaxBlocks; }

cudaError_t launch_adj_step(int dtype, void *psi, void *lam, const GatePlan &p, const double *dU, double *part,
                            cudaStream_t st) {
    return dtype == QS_C64 ? adj_step_impl<float>(psi, lam, p, dU, part, st)
                           : adj_step_impl<double>(psi, lam, p, dU, part, st);
}

cudaError_t launch_obs_sumz(int dtype, const void *psi, void *lam, int n, cudaStream_t st) {
    const uint64_t N = 1ull << n;
    const unsigned grid = (unsigned)std::min<uint64_t>((N + 255) / 256, (uint64_t)device_sm_count() * 8);
    if (dtype == QS_C64)
        k_obs_sumz<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(psi), reinterpret_cast<float2 *>(lam), n, N);
    else
        k_obs_sumz<double><<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(psi), reinterpret_cast<double2 *>(lam), n, N);
    return cudaGetLastError();
}

cudaError_t launch_sum_vec(const double *z, int n, double *out, cudaStream_t st) {
    k_sum_vec<<<1, 32, 0, st>>>(z, n, out);
    return cudaGetLastError();
}

cudaError_t launch_grad_final(const double *part, int nslots, double *slot_sum, const int *slot_param,
                              double *grad, int nparams, cudaStream_t st) {
    if (nslots > 0) {
        k_slot_sums<<<(nslots + 7) / 8, 256, 0, st>>>(part, nslots, slot_sum);  // 8 slots (warps) per block
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nparams > 0) {
        k_grad_gather<<<(nparams + 127) / 128, 128, 0, st>>>(slot_sum, slot_param, nslots, grad, nparams);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace qs
