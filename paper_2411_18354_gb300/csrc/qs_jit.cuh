// qs_jit.cuh -- tile passes compiled for their exact shape at run time.
//
// The interpreted tile pass (k_tile_pass) reads each gate's descriptor from shared memory,
// decodes it and dispatches through a switch on (operation, target place, in-row controls)
// for every row of every tile; that per-gate loop, not the arithmetic, bounds it. Here the
// host writes the CUDA source of one kernel per pass shape instead: the tile map, the
// register groups (row deposits, swizzled element offsets, folded exchanges), every gate's
// operation, target place and control pattern become compile-time constants, so each gate is
// straight-line code (its pair updates, predicated on row controls and guarded by its tile
// predicate). Only the gate matrices (and, in the adjoint sweep, their derivatives) are kernel
// parameters: they live in the constant bank, where the FMA instructions read them directly,
// and a circuit with the same structure but other angles reuses the compiled kernel.
//
// Sources are compiled with NVRTC for sm_103a into a cubin, cached by source text (a process-
// wide map; compiled once per distinct pass shape), and loaded with the runtime's library API
// (context-independent: each device loads it on first launch).
#pragma once

#include <string>
#include <vector>

#include "qs_fuse.cuh"

namespace qs {

// A compiled pass kernel: index into the process-wide cache, and its launch parameters.
struct JitPass {
    int entry = -1;           // cache entry (module) index
    int kernel = -1;          // kernel index inside the module
    size_t smem = 0;          // dynamic shared memory of one block
    size_t arg_bytes = 0;     // size of the parameter block (matrices)
    bool batched = false;     // runs over the states of a batch program
    int nparam_gates = 0;     // batch: parameterised gates of the pass
};

// One program to compile: its passes, forward or reverse sweep, single state or batch.
struct JitRequest {
    const FusedProgram *prog;
    bool adjoint;
    bool batched;
    std::vector<JitPass> *out;
};

// Compile the passes of several programs at once (new kernels compiled concurrently).
bool jit_prepare_programs(int dtype, const std::vector<JitRequest> &reqs, std::string *err,
                          double *compile_seconds = nullptr, int *compiled_modules = nullptr);

// Generate (and compile, on a cache miss) the kernels of every tile pass of `prog`. Forward
// programs: lam_mode = false; adjoint sweep: true. Fills `out` with one JitPass per pass.
// Needs no device (compilation only). Returns false with `err` on a compile failure.
bool jit_prepare_program(int dtype, bool adjoint, const FusedProgram &prog, std::vector<JitPass> *out,
                         std::string *err, double *compile_seconds = nullptr, int *compiled_modules = nullptr);

// Load the compiled kernels of these passes on the current device and set their launch
// attributes (done before a stream capture records launches of them).
cudaError_t jit_load(const std::vector<JitPass> &passes);

// Launch pass `p` of `prog` with its compiled kernel. Adjoint: lam, part (gradient partials
// [slot][part_stride]) as for launch_tile_pass.
cudaError_t launch_jit_pass(int dtype, const JitPass &jp, const FusedProgram &prog, int p, void *psi, void *lam,
                            double *part, size_t part_stride, cudaStream_t st);

// Launch batched pass `p` over `nstates` states whose vectors start `stride` amplitudes apart at
// psi (and lam, sweep), with their (cos, sin) of theta/2 at cs (cs_stride reals per state);
// sweep: part receives per tile and parameterised gate J the partial of Re <lambda| dU psi> at
// [(J * nstates + state) * tiles_per_state + tile].
cudaError_t launch_jit_pass_batched(int dtype, const JitPass &jp, const FusedProgram &prog, int p, void *psi,
                                    void *lam, double *part, uint64_t stride, uint64_t nstates, const void *cs,
                                    uint32_t cs_stride, cudaStream_t st);

// Whether the kernel of a pass with 2^k-amplitude tiles double-buffers them.
bool jit_double_buffer(int dtype, bool adjoint, int k);

// The generated source of one pass (exposed for tests of the generator).
// batched: the kernel runs the pass over `nstates` states of one batch program at once (tile
// index = state * tiles per state + tile), each state's vectors `stride` amplitudes apart,
// the parameterised gates' matrices formed per tile from that state's (cos, sin) of theta/2
// (RegGate pkind / pkind2 / pidx / pidx2), and in the sweep the gradient partial of every
// parameterised gate written per tile.
std::string jit_pass_source(int dtype, bool adjoint, const TilePass &P, const TileGroup *groups,
                            const RegGate *gates, const char *kname, bool batched = false);

}  // namespace qs
