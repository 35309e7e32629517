// qs_debug.cu -- the debug build's status word and its C entry points (stubs returning
// QS_EUNSUPPORTED in the release build).
#include "qs_debug.cuh"
#include "qs_internal.cuh"

namespace qs {
qs_status set_error(qs_status st, const char *msg);
qs_status cuda_fail(cudaError_t e, const char *what);
#ifdef QS_DEBUG_CHECKS
__device__ DebugState g_qs_debug;

// Device address of the status word (compiled passes receive it as a kernel parameter).
void *debug_state_address() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_qs_debug) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
#else
void *debug_state_address() { return nullptr; }
#endif
}  // namespace qs

using namespace qs;

extern "C" {

int qs_debug_build(void) {
#ifdef QS_DEBUG_CHECKS
    return 1;
#else
    return 0;
#endif
}

qs_status qs_debug_configure(uint64_t n_amps, unsigned int *counts, uint64_t count_n) {
#ifdef QS_DEBUG_CHECKS
    DebugState d{};
    d.n_amps = n_amps;
    d.counts = counts;
    d.count_n = counts ? count_n : 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_qs_debug, &d, sizeof(d));
    if (e != cudaSuccess) return cuda_fail(e, "qs_debug_configure");
    return QS_OK;
#else
    (void)n_amps;
    (void)counts;
    (void)count_n;
    return set_error(QS_EUNSUPPORTED, "qs_debug_configure: not a debug build (QS_DEBUG_CHECKS)");
#endif
}

qs_status qs_debug_status(unsigned int *status, uint64_t *first_bad) {
#ifdef QS_DEBUG_CHECKS
    DebugState d{};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&d, g_qs_debug, sizeof(d));
    if (e != cudaSuccess) return cuda_fail(e, "qs_debug_status");
    if (status) *status = d.status;
    if (first_bad) *first_bad = d.first_bad;
    return QS_OK;
#else
    (void)status;
    (void)first_bad;
    return set_error(QS_EUNSUPPORTED, "qs_debug_status: not a debug build (QS_DEBUG_CHECKS)");
#endif
}

}  // extern "C"
