// qs_state.cuh -- the opaque qs_state handle and helpers shared by the entry points.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "qs_internal.cuh"

namespace qs {

constexpr uint32_t kStateMagic = 0x51535354u;  // "QSST"

struct GraphCacheEntry {
    uint64_t key;                 // hash of `bytes` (the lookup key)
    std::vector<unsigned char> bytes;  // everything the key hashes, compared on a hash hit
    cudaGraphExec_t exec;
    void *table;  // device gate table of the fused passes recorded in the graph (or null)
};

}  // namespace qs

struct qs_state {
    uint32_t magic = qs::kStateMagic;
    int n = 0;
    qs_dtype dtype = QS_C64;
    void *psi = nullptr;     // amplitudes (device)
    size_t bytes = 0;        // 2^n * element size
    bool owned = false;      // psi allocated by the library
    cudaStream_t stream = nullptr;
    int device = 0;
    // library-owned scratch (device)
    double *red_scratch = nullptr;  // reduction partials and outputs
    size_t red_scratch_n = 0;
    void *lam = nullptr;            // adjoint: second vector (lambda), same size as psi
    double *grad_scratch = nullptr; // adjoint: per-gate, per-block partial inner products
    size_t grad_scratch_n = 0;
    void *tile_table = nullptr;     // fused passes: device copy of the tile gate table
    size_t tile_table_bytes = 0;
    // CUDA graphs of circuits, keyed by a hash of the gate list, theta and flags
    cudaStream_t capture_stream = nullptr;
    std::vector<qs::GraphCacheEntry> graphs;
};

namespace qs {

qs_status set_error(qs_status st, const char *msg);
qs_status cuda_fail(cudaError_t e, const char *what);
size_t elem_bytes(int dtype);
// Sets the L2 fetch size limit once per device (see qs_set_l2_fetch_bytes).
void apply_l2_fetch(int device);
qs_status ensure_reduce_scratch(qs_state *s);
void release_state_buffers(qs_state *s);  // scratch, lambda, graphs, capture stream

}  // namespace qs
