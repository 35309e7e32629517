// k_batch_major.cu -- helper kernels of the batch's pass-major path (qs_batch_run with
// QS_FLAG_JIT): the states of one batch program (same qubit count and gate list) live side by
// side in one buffer, and every pass of the program runs over all of them in one launch of a
// kernel compiled for that pass (qs_jit.cu). These kernels prepare the states and angles,
// form lambda = O psi with the energies, and sum the per-tile gradient partials.
#include "k_batch_major.cuh"
#include "k_gate.cuh"

namespace qs {
namespace {

constexpr int kBmThreads = 256;
constexpr uint32_t kObsChunk = 1u << 14;  // amplitudes per block of the energy pass

// psi_s = |0...0> for every state; cs[s][p] = (cos, sin) of theta / 2 for its parameters.
template <typename Real>
__global__ void __launch_bounds__(kBmThreads) k_bm_init(typename CxT<Real>::T *__restrict__ psi, int n, int S,
                                                       Real *__restrict__ cs, int nparam,
                                                       const double *__restrict__ theta,
                                                       const uint64_t *__restrict__ param_off,
                                                       const int *__restrict__ gstate) {
    using T2 = typename CxT<Real>::T;
    const uint64_t N = 1ull << n, total = (uint64_t)S << n;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step) {
        T2 v;
        v.x = (i & (N - 1)) == 0 ? (Real)1 : (Real)0;
        v.y = 0;
        psi[i] = v;
    }
    const uint64_t np = (uint64_t)S * nparam;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += step) {
        const uint64_t s = j / nparam, p = j % nparam;
        double sn, c;
        sincos(0.5 * theta[param_off[gstate[s]] + p], &sn, &c);
        cs[2 * j] = (Real)c;
        cs[2 * j + 1] = (Real)sn;
    }
}

// lambda = O psi with O = sum_i Z_i (weight n - 2 popcount(k) on amplitude k) and the
// partial sums of <psi|O|psi>, one block per chunk of a state: part[s * chunks + c].
template <typename Real>
__global__ void __launch_bounds__(kBmThreads) k_bm_obs(const typename CxT<Real>::T *__restrict__ psi,
                                                      typename CxT<Real>::T *__restrict__ lam, int n, uint32_t chunks,
                                                      double *__restrict__ part) {
    using T2 = typename CxT<Real>::T;
    __shared__ double red[kBmThreads / 32];
    const uint64_t s = blockIdx.x / chunks, c = blockIdx.x % chunks;
    const uint64_t N = 1ull << n;
    const uint64_t len = N / chunks;  // chunks divides N (both powers of two)
    const uint64_t k0 = c * len;
    const T2 *src = psi + s * N;
    T2 *dst = lam + s * N;
    Acc<Real> acc{};
    constexpr int U = 4;
    for (uint64_t k = threadIdx.x; k < len; k += (uint64_t)U * kBmThreads) {
        T2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t kk = k + (uint64_t)u * kBmThreads;
            if (kk < len) v[u] = src[k0 + kk];
        }
        Real run = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t kk = k + (uint64_t)u * kBmThreads;
            if (kk < len) {
                const Real w = (Real)(n - 2 * __popcll(k0 + kk));
                run += w * (v[u].x * v[u].x + v[u].y * v[u].y);
                v[u].x *= w;
                v[u].y *= w;
                dst[k0 + kk] = v[u];
            }
        }
        acc.add(run);
    }
    double t = acc.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int w = 0; w < kBmThreads / 32; ++w) e += red[w];
        part[blockIdx.x] = e;
    }
}

// energy of each state: its chunks' partials added in order.
__global__ void __launch_bounds__(kBmThreads) k_bm_energy(const double *__restrict__ part, int S, uint32_t chunks,
                                                         double *__restrict__ energy, const int *__restrict__ gstate) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        double e = 0.0;
        for (uint32_t c = 0; c < chunks; ++c) e += part[(uint64_t)s * chunks + c];
        energy[gstate[s]] = e;
    }
}

// dE/dtheta_p = 2 sum over the gates p drives (in program order) of the per-tile partials of
// Re <lambda| dU psi>: block per state, thread per parameter. items[csr_ptr[p] .. csr_ptr[p+1])
// are the offsets of p's gates' partial blocks ([J][state][tile] of their sweep pass).
__global__ void __launch_bounds__(kBmThreads) k_bm_grad(const double *__restrict__ part, const int *__restrict__ csr_ptr,
                                                       const uint64_t *__restrict__ items, int nparam, int S,
                                                       uint32_t tiles, double *__restrict__ grad,
                                                       const uint64_t *__restrict__ param_off,
                                                       const int *__restrict__ gstate) {
    const int s = blockIdx.x;
    for (int p = threadIdx.x; p < nparam; p += blockDim.x) {
        double g = 0.0;
        for (int it = csr_ptr[p]; it < csr_ptr[p + 1]; ++it) {
            const double *q = part + items[it] + (uint64_t)s * tiles;
            for (uint32_t t = 0; t < tiles; ++t) g += q[t];
        }
        grad[param_off[gstate[s]] + p] = 2.0 * g;
    }
}

template <typename Real>
cudaError_t init_impl(void *psi, int n, int S, void *cs, int nparam, const double *theta, const uint64_t *param_off,
                      const int *gstate, cudaStream_t st) {
    const uint64_t work = std::max<uint64_t>((uint64_t)S << n, (uint64_t)S * nparam);
    const unsigned grid = (unsigned)std::min<uint64_t>((work + kBmThreads - 1) / kBmThreads,
                                                       (uint64_t)device_sm_count() * 8);
    k_bm_init<Real><<<std::max(1u, grid), kBmThreads, 0, st>>>(static_cast<typename CxT<Real>::T *>(psi), n, S,
                                                                static_cast<Real *>(cs), nparam, theta, param_off,
                                                                gstate);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t obs_impl(const void *psi, void *lam, int n, int S, double *part, double *energy, const int *gstate,
                     cudaStream_t st) {
    const uint64_t N = 1ull << n;
    const uint32_t chunks = (uint32_t)std::max<uint64_t>(1, N / kObsChunk);
    k_bm_obs<Real><<<(unsigned)((uint64_t)S * chunks), kBmThreads, 0, st>>>(
        static_cast<const typename CxT<Real>::T *>(psi), static_cast<typename CxT<Real>::T *>(lam), n, chunks, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bm_energy<<<(S + kBmThreads - 1) / kBmThreads, kBmThreads, 0, st>>>(part, S, chunks, energy, gstate);
    return cudaGetLastError();
}

}  // namespace

size_t bm_obs_partials(int n, int S) {
    const uint64_t N = 1ull << n;
    return (size_t)S * (size_t)std::max<uint64_t>(1, N / kObsChunk);
}

cudaError_t launch_bm_init(int dtype, void *psi, int n, int S, void *cs, int nparam, const double *theta,
                           const uint64_t *param_off, const int *gstate, cudaStream_t st) {
    return dtype == QS_C64 ? init_impl<float>(psi, n, S, cs, nparam, theta, param_off, gstate, st)
                           : init_impl<double>(psi, n, S, cs, nparam, theta, param_off, gstate, st);
}

cudaError_t launch_bm_obs(int dtype, const void *psi, void *lam, int n, int S, double *part, double *energy,
                          const int *gstate, cudaStream_t st) {
    return dtype == QS_C64 ? obs_impl<float>(psi, lam, n, S, part, energy, gstate, st)
                           : obs_impl<double>(psi, lam, n, S, part, energy, gstate, st);
}

cudaError_t launch_bm_grad(const double *part, const int *csr_ptr, const uint64_t *items, int nparam, int S,
                           uint32_t tiles, double *grad, const uint64_t *param_off, const int *gstate, cudaStream_t st) {
    if (nparam == 0) return cudaSuccess;
    k_bm_grad<<<S, kBmThreads, 0, st>>>(part, csr_ptr, items, nparam, S, tiles, grad, param_off, gstate);
    return cudaGetLastError();
}

}  // namespace qs
