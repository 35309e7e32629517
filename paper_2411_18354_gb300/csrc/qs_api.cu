// qs_api.cu -- the extern "C" entry points declared in include/qs.h.
//
// Every entry point validates its arguments completely before enqueuing anything, maps
// CUDA failures to QS_ECUDA with the CUDA message, and records the message of the last
// failure per thread.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "qs_internal.cuh"
#include "qs_state.cuh"

namespace {

thread_local char g_err[1024] = "";

qs_status fail(qs_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

}  // namespace

namespace qs {

qs_status set_error(qs_status st, const char *msg) { return fail(st, "%s", msg); }

qs_status cuda_fail(cudaError_t e, const char *what) {
    return fail(QS_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

size_t elem_bytes(int dtype) { return dtype == QS_C128 ? 16 : 8; }

// L2 fetch size for DRAM misses (cudaLimitMaxL2FetchGranularity of this process's context).
// A gate with controls on low qubits selects runs of 8-64 bytes; with the device's default
// fetch size each such run pulls a 128-byte block from DRAM, so the limit is set to one
// 32-byte sector per device the library works on (QS_L2_FETCH_BYTES or qs_set_l2_fetch_bytes
// choose another value; 0 leaves the context's limit alone).
static std::mutex g_l2_mutex;
static int g_l2_bytes = -1;           // configured value, -1 = not read from the environment yet
static int g_l2_applied[64];          // per device: value applied (0 = none yet)

static bool valid_l2_bytes(int b) { return b == 0 || b == 32 || b == 64 || b == 128; }

static int l2_configured_locked() {
    if (g_l2_bytes < 0) {
        g_l2_bytes = 32;
        if (const char *env = std::getenv("QS_L2_FETCH_BYTES")) {
            const int v = std::atoi(env);
            if (valid_l2_bytes(v)) g_l2_bytes = v;
        }
    }
    return g_l2_bytes;
}

void apply_l2_fetch(int device) {
    std::lock_guard<std::mutex> lock(g_l2_mutex);
    const int want = l2_configured_locked();
    if (want == 0 || device < 0 || device >= 64 || g_l2_applied[device] == want) return;
    if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)want) == cudaSuccess)
        g_l2_applied[device] = want;
    cudaGetLastError();  // a hint: a context that refuses it keeps its default
}

qs_status ensure_reduce_scratch(qs_state *s) {
    const size_t need = reduce_scratch_doubles(s->n) + 64;
    if (s->red_scratch && s->red_scratch_n >= need) return QS_OK;
    if (s->red_scratch) {
        cudaFree(s->red_scratch);
        s->red_scratch = nullptr;
        s->red_scratch_n = 0;
    }
    cudaError_t e = cudaMalloc(&s->red_scratch, need * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->red_scratch = nullptr;
        return fail(QS_ENOMEM, "reduction scratch of %zu bytes: %s", need * sizeof(double), cudaGetErrorString(e));
    }
    s->red_scratch_n = need;
    return QS_OK;
}

}  // namespace qs

using namespace qs;

// ------------------------------------------------------------------------------------
// Basis-state kernel
// ------------------------------------------------------------------------------------
namespace {
__global__ void k_set_one(void *psi, uint64_t k, int dtype) {
    if (dtype == QS_Q30) reinterpret_cast<int2 *>(psi)[k] = make_int2(1 << 30, 0);
    else if (dtype == QS_C64) reinterpret_cast<float2 *>(psi)[k] = make_float2(1.0f, 0.0f);
    else reinterpret_cast<double2 *>(psi)[k] = make_double2(1.0, 0.0);
}

qs_status check_state(const qs_state *s) {
    if (!s) return fail(QS_EINVAL, "state is NULL");
    if (s->magic != kStateMagic) return fail(QS_EINVAL, "state handle is not valid (freed or corrupt)");
    return QS_OK;
}
}  // namespace

extern "C" {

const char *qs_last_error(void) { return g_err; }

qs_status qs_set_l2_fetch_bytes(int bytes) {
    if (!valid_l2_bytes(bytes)) return fail(QS_EINVAL, "qs_set_l2_fetch_bytes: %d is not 0, 32, 64 or 128", bytes);
    std::lock_guard<std::mutex> lock(g_l2_mutex);
    g_l2_bytes = bytes;
    return QS_OK;
}

int qs_get_l2_fetch_bytes(void) {
    std::lock_guard<std::mutex> lock(g_l2_mutex);
    return l2_configured_locked();
}

const char *qs_build_info(void) {
    return "libqs: sm_103a state-vector kernels (reduced iteration scheduling, Section III-B of arXiv 2411.18354)";
}

qs_status qs_state_alloc(int n, qs_dtype dtype, void *stream, qs_state **out) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxQubits) return fail(QS_EINVAL, "n=%d out of range [1, %d]", n, kMaxQubits);
    if (dtype != QS_C64 && dtype != QS_C128 && dtype != QS_Q30) return fail(QS_EINVAL, "bad dtype %d", (int)dtype);
    const size_t bytes = (size_t(1) << n) * elem_bytes(dtype);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "cudaMalloc(%zu bytes) for n=%d: %s", bytes, n, cudaGetErrorString(e));
    }
    qs_state *s = new (std::nothrow) qs_state();
    if (!s) {
        cudaFree(p);
        return fail(QS_ENOMEM, "host allocation of the state handle failed");
    }
    s->n = n;
    s->dtype = dtype;
    s->psi = p;
    s->bytes = bytes;
    s->owned = true;
    s->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&s->device);
    apply_l2_fetch(s->device);
    qs_status st = qs_state_set_basis(s, 0);
    if (st != QS_OK) {
        qs_state_free(s);
        return st;
    }
    *out = s;
    return QS_OK;
}

qs_status qs_state_wrap(void *dev_ptr, size_t bytes, int n, qs_dtype dtype, void *stream, qs_state **out) {
    if (!out) return fail(QS_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxQubits) return fail(QS_EINVAL, "n=%d out of range [1, %d]", n, kMaxQubits);
    if (dtype != QS_C64 && dtype != QS_C128 && dtype != QS_Q30) return fail(QS_EINVAL, "bad dtype %d", (int)dtype);
    if (!dev_ptr) return fail(QS_EINVAL, "dev_ptr is NULL");
    if (reinterpret_cast<uintptr_t>(dev_ptr) % 256 != 0) return fail(QS_EINVAL, "dev_ptr is not 256-byte aligned");
    const size_t need = (size_t(1) << n) * elem_bytes(dtype);
    if (bytes < need) return fail(QS_EINVAL, "buffer of %zu bytes is smaller than 2^%d amplitudes (%zu bytes)", bytes, n, need);
    qs_state *s = new (std::nothrow) qs_state();
    if (!s) return fail(QS_ENOMEM, "host allocation of the state handle failed");
    s->n = n;
    s->dtype = dtype;
    s->psi = dev_ptr;
    s->bytes = need;
    s->owned = false;
    s->stream = reinterpret_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&s->device) == cudaSuccess) apply_l2_fetch(s->device);
    cudaGetLastError();
    *out = s;
    return QS_OK;
}

qs_status qs_state_free(qs_state *s) {
    if (!s) return QS_OK;
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    cudaStreamSynchronize(s->stream);
    release_state_buffers(s);
    if (s->owned && s->psi) cudaFree(s->psi);
    s->magic = 0;
    delete s;
    cudaGetLastError();
    return QS_OK;
}

qs_status qs_state_info(const qs_state *s, int *n, qs_dtype *dtype, void **dev_ptr) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (n) *n = s->n;
    if (dtype) *dtype = s->dtype;
    if (dev_ptr) *dev_ptr = s->psi;
    return QS_OK;
}

qs_status qs_state_set_stream(qs_state *s, void *stream) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    s->stream = reinterpret_cast<cudaStream_t>(stream);
    return QS_OK;
}

qs_status qs_state_set_basis(qs_state *s, uint64_t k) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (k >> s->n) return fail(QS_EINVAL, "basis index %llu >= 2^%d", (unsigned long long)k, s->n);
    cudaError_t e = cudaMemsetAsync(s->psi, 0, s->bytes, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    k_set_one<<<1, 1, 0, s->stream>>>(s->psi, k, (int)s->dtype);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "set_basis launch");
    return QS_OK;
}

qs_status qs_state_copy_to_host(const qs_state *s, void *dst, size_t bytes) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (!dst) return fail(QS_EINVAL, "dst is NULL");
    if (bytes != s->bytes) return fail(QS_EINVAL, "bytes=%zu, the state holds %zu", bytes, s->bytes);
    cudaError_t e = cudaMemcpyAsync(dst, s->psi, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy_to_host");
    return QS_OK;
}

qs_status qs_state_copy_from_host(qs_state *s, const void *src, size_t bytes) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (!src) return fail(QS_EINVAL, "src is NULL");
    if (bytes != s->bytes) return fail(QS_EINVAL, "bytes=%zu, the state holds %zu", bytes, s->bytes);
    cudaError_t e = cudaMemcpyAsync(s->psi, src, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy_from_host");
    return QS_OK;
}

qs_status qs_state_copy_from_host_async(qs_state *s, const void *src, size_t bytes) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (!src) return fail(QS_EINVAL, "src is NULL");
    if (bytes != s->bytes) return fail(QS_EINVAL, "bytes=%zu, the state holds %zu", bytes, s->bytes);
    cudaError_t e = cudaMemcpyAsync(s->psi, src, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy_from_host_async");
    return QS_OK;
}

qs_status qs_state_copy_to_host_async(const qs_state *s, void *dst, size_t bytes) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    if (!dst) return fail(QS_EINVAL, "dst is NULL");
    if (bytes != s->bytes) return fail(QS_EINVAL, "bytes=%zu, the state holds %zu", bytes, s->bytes);
    cudaError_t e = cudaMemcpyAsync(dst, s->psi, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy_to_host_async");
    return QS_OK;
}

qs_status qs_state_synchronize(const qs_state *s) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qs_state_synchronize");
    return QS_OK;
}

qs_status qs_apply_gate(qs_state *s, int target, uint64_t ctrl_mask, uint64_t ctrl_vals, const double U[8]) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    GatePlan p;
    char err[256];
    if (!plan_gate(s->n, s->dtype, target, ctrl_mask, ctrl_vals, U, QS_GATE_U, -1, &p, err, sizeof(err)))
        return fail(QS_EINVAL, "qs_apply_gate: %s", err);
    cudaError_t e = launch_gate(s->dtype, s->psi, p, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qs_apply_gate launch");
    return QS_OK;
}

qs_status qs_apply_x(qs_state *s, int target, uint64_t ctrl_mask, uint64_t ctrl_vals) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    GatePlan p;
    char err[256];
    if (!plan_gate(s->n, s->dtype, target, ctrl_mask, ctrl_vals, nullptr, QS_GATE_X, -1, &p, err, sizeof(err)))
        return fail(QS_EINVAL, "qs_apply_x: %s", err);
    cudaError_t e = launch_gate(s->dtype, s->psi, p, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qs_apply_x launch");
    return QS_OK;
}

qs_status qs_apply_gate_masked(qs_state *s, int target, uint64_t ctrl_mask, uint64_t ctrl_vals, const double U[8]) {
    qs_status st = check_state(s);
    if (st != QS_OK) return st;
    GatePlan p, pm;
    char err[256];
    if (!plan_gate(s->n, s->dtype, target, ctrl_mask, ctrl_vals, U, QS_GATE_U, -1, &p, err, sizeof(err)))
        return fail(QS_EINVAL, "qs_apply_gate_masked: %s", err);
    plan_masked(p, &pm);
    std::memcpy(pm.U, U, sizeof(pm.U));
    cudaError_t e = launch_gate_masked(s->dtype, s->psi, pm, ctrl_mask, ctrl_vals, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qs_apply_gate_masked launch");
    return QS_OK;
}

qs_status qs_expect_z(const qs_state *cs, double *out, double *out_norm2, int flags) {
    qs_status st = check_state(cs);
    if (st != QS_OK) return st;
    qs_state *s = const_cast<qs_state *>(cs);
    if (!out && !out_norm2) return fail(QS_EINVAL, "qs_expect_z: both outputs are NULL");
    st = ensure_reduce_scratch(s);
    if (st != QS_OK) return st;
    const bool on_dev = (flags & QS_FLAG_OUT_DEVICE) != 0;
    double *dz = on_dev ? out : s->red_scratch;            // n values
    double *dn = on_dev ? out_norm2 : s->red_scratch + s->n;  // 1 value
    double *part = s->red_scratch + 64;
    cudaError_t e = launch_expect_z(s->dtype, s->psi, s->n, part, dz, dn, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qs_expect_z launch");
    if (!on_dev) {
        double host[kMaxQubits + 1];
        e = cudaMemcpyAsync(host, s->red_scratch, (s->n + 1) * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "qs_expect_z copy-out");
        if (out) std::memcpy(out, host, s->n * sizeof(double));
        if (out_norm2) *out_norm2 = host[s->n];
    }
    return QS_OK;
}

}  // extern "C"
