// k_gate_c128.cu -- complex128 (float64 arithmetic) instantiations of the gate kernels.
#include "k_gate_dispatch.cuh"

namespace qs {
cudaError_t launch_gate_c128(void *psi, const GatePlan &p, bool masked, uint64_t cmask,
                             uint64_t cvals, cudaStream_t st) {
    return gate_detail::launch<double>(psi, p, masked, cmask, cvals, st);
}
}  // namespace qs
