// k_batch_major.cuh -- helper kernels of the batch's pass-major path (see k_batch_major.cu).
#pragma once

#include <algorithm>
#include <cstdint>

#include "qs_internal.cuh"

namespace qs {

// Every state of a program (S states of n qubits, stored 2^n amplitudes apart at psi) set to
// |0...0>; cs (S x nparam pairs in the state precision) = (cos, sin) of theta / 2, theta of
// state s at theta[param_off[gstate[s]]].
cudaError_t launch_bm_init(int dtype, void *psi, int n, int S, void *cs, int nparam, const double *theta,
                           const uint64_t *param_off, const int *gstate, cudaStream_t st);

// lambda = O psi (O = sum_i Z_i) and energy[gstate[s]] = <psi_s|O|psi_s> for every state; `part`
// holds bm_obs_partials(n, S) doubles (fixed-order partial sums).
size_t bm_obs_partials(int n, int S);
cudaError_t launch_bm_obs(int dtype, const void *psi, void *lam, int n, int S, double *part, double *energy,
                          const int *gstate, cudaStream_t st);

// grad[param_off[gstate[s]] + p] = 2 * sum over items[csr_ptr[p] .. csr_ptr[p+1]) of the
// `tiles` partials at part + item + s * tiles.
cudaError_t launch_bm_grad(const double *part, const int *csr_ptr, const uint64_t *items, int nparam, int S,
                           uint32_t tiles, double *grad, const uint64_t *param_off, const int *gstate, cudaStream_t st);

}  // namespace qs
