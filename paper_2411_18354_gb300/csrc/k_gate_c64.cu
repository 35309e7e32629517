// k_gate_c64.cu -- complex64 (float32 arithmetic) instantiations of the gate kernels.
#include "k_gate_dispatch.cuh"

namespace qs {
cudaError_t launch_gate_c64(void *psi, const GatePlan &p, bool masked, uint64_t cmask,
                            uint64_t cvals, cudaStream_t st) {
    return gate_detail::launch<float>(psi, p, masked, cmask, cvals, st);
}
}  // namespace qs
