// k_batch.cuh -- descriptors of the batched persistent kernel.
#pragma once

#include "k_tile.cuh"

namespace qs {

constexpr int kBatchThreads = 256;

struct BatchState {
    int32_t n;
    int32_t prog;      // index of the state's program
    int32_t nparam;    // parameters of this state
    int32_t pad;
    uint64_t param_off;  // offset of the state's parameters in theta / grad
};

struct BatchProg {
    int32_t fwd_begin, fwd_count;  // passes of the forward program
    int32_t adj_begin, adj_count;  // passes of the reverse sweep
    int32_t small;                 // 1: the whole state fits in shared memory
    int32_t n;
};

struct BatchArgs {
    const BatchState *states;
    const int32_t *order;   // queue position -> state index (largest first)
    const BatchProg *progs;
    const TilePass *passes;
    const TileGroup *groups;
    const RegGate *gates;
    const double *theta;
    double *energy;
    double *grad;
    void *workspace;        // per CTA: psi and lambda, ws_stride amplitudes each
    uint64_t ws_stride;
    int *queue;
    int num_states;
    int smem_bits;          // shared-memory tile: 2^smem_bits amplitudes (x2: psi, lambda)
    int max_params;
};

size_t batch_smem_bytes(int dtype, int smem_bits, int max_params);
int batch_grid(int dtype, size_t smem);  // resident CTAs on the device for that shared memory size
cudaError_t launch_batch(int dtype, const BatchArgs &a, int grid, size_t smem, cudaStream_t st);

}  // namespace qs
