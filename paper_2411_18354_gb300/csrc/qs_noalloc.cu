// qs_noalloc.cu -- qs_expect_z_noalloc: the <Z_i> / norm reduction for callers that cannot
// allocate device memory.
//
// Who needs this: code whose device memory is owned by someone else's allocator (a
// framework's memory pool or a fixed arena that must not be fragmented or overcommitted),
// code that runs on a latency budget where a cudaMalloc (which may synchronise the device)
// is not acceptable, and code that must not fail for lack of memory halfway through a job.
// qs_expect_z needs a per-state scratch buffer for its per-block partial sums, which it
// allocates on first use; this variant instead uses one fixed array that lives in the
// library's device image, so a call allocates nothing at all.
//
// The array is a file-scope __device__ variable. Host code cannot use its name as a device
// address (the host-side symbol is only a stand-in), so on the first call on each device
// the library asks the runtime for the array's device address with cudaGetSymbolAddress,
// with that device current, and passes that address to the kernels. That first call
// therefore makes a runtime query; make it before any stream capture.
//
// Every call on a device shares the one array, and the array keeps whatever the last call
// left in it. The kernels write every partial they later read, so nothing has to be
// cleared between calls. Calls that can overlap on the GPU (different streams, or the same
// array used from several host threads on different streams) race on the array and give
// wrong results: serialise them.
//
// The looked-up address belongs to the device's current CUDA context. A cudaDeviceReset
// destroys that context (and the array with it); the cached address is not looked up again,
// so after a reset this entry point must not be called again in the same process.
#include <cstdio>
#include <mutex>

#include "qs_internal.cuh"

namespace qs {
qs_status set_error(qs_status st, const char *msg);
qs_status cuda_fail(cudaError_t e, const char *what);
}  // namespace qs

using namespace qs;

namespace {

// Room for the per-block partial sums of a state of up to 40 qubits: at most 1024 blocks
// with 41 doubles each (n outputs + the total): 1024 * 41 * 8 = 335,872 bytes per device.
constexpr size_t kNoAllocScratchDoubles = 1024 * 41;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices] = {};

qs_status scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "qs_expect_z_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(QS_EUNSUPPORTED, "qs_expect_z_noalloc: device index >= 64");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // device `dev` is current here
        if (e != cudaSuccess || !p) return cuda_fail(e, "qs_expect_z_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return QS_OK;
}

// The kernels read `p` (or write it) from the current device: it must be device memory (or
// managed memory) of that device. A host pointer, or memory of another device, would make the
// kernels fault instead of failing cleanly, so both are rejected before anything is launched.
// cudaPointerGetAttributes is a host-side query; it allocates nothing.
qs_status check_device_pointer(const void *p, int dev, const char *what) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[160];
        std::snprintf(msg, sizeof(msg), "qs_expect_z_noalloc: %s is not a pointer the CUDA runtime knows", what);
        return set_error(QS_EINVAL, msg);
    }
    if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "qs_expect_z_noalloc: %s must be device (or managed) memory of the current device %d", what,
                      dev);
        return set_error(QS_EINVAL, msg);
    }
    return QS_OK;
}

}  // namespace

extern "C" qs_status qs_expect_z_noalloc(const void *psi, int n, qs_dtype dtype, void *stream, double *out_z,
                                         double *out_norm2) {
    if (!psi) return set_error(QS_EINVAL, "qs_expect_z_noalloc: psi is NULL");
    if (reinterpret_cast<uintptr_t>(psi) % 16 != 0) return set_error(QS_EINVAL, "qs_expect_z_noalloc: psi is not 16-byte aligned");
    if (dtype != QS_C64 && dtype != QS_C128) return set_error(QS_EINVAL, "qs_expect_z_noalloc: bad dtype");
    if (n < 1 || n > kMaxQubits) return set_error(QS_EINVAL, "qs_expect_z_noalloc: n out of range [1, 40]");
    if (!out_z && !out_norm2) return set_error(QS_EINVAL, "qs_expect_z_noalloc: both outputs are NULL");
    if (reduce_scratch_doubles(n) > kNoAllocScratchDoubles)
        return set_error(QS_EINVAL, "qs_expect_z_noalloc: the partial sums for this n do not fit the fixed "
                                    "scratch array of 1024 * 41 doubles");
    int dev = 0;
    cudaError_t ge = cudaGetDevice(&dev);
    if (ge != cudaSuccess) return cuda_fail(ge, "qs_expect_z_noalloc: cudaGetDevice");
    qs_status st = check_device_pointer(psi, dev, "psi");
    if (st == QS_OK && out_z) st = check_device_pointer(out_z, dev, "out_z");
    if (st == QS_OK && out_norm2) st = check_device_pointer(out_norm2, dev, "out_norm2");
    if (st != QS_OK) return st;
    double *scratch = nullptr;
    st = scratch_for_current_device(&scratch);
    if (st != QS_OK) return st;
    cudaError_t e = launch_expect_z(dtype, psi, n, scratch, out_z, out_norm2, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "qs_expect_z_noalloc launch");
    return QS_OK;
}
