// k_tile.cuh -- fused tile pass: a run of consecutive gates applied to shared-memory tiles
// of the state in one HBM round trip.
//
// A pass chooses k "local" qubits L (always including the lowest ones, so that tile rows are
// contiguous in memory, plus the targets of its gates). A tile is the 2^k amplitudes that
// share the values of the n - k non-local qubits. Inside a tile every gate of the pass is
// applied on its reduced iteration set in local coordinates (Section III-B of arXiv
// 2411.18354: target and local controls inserted into a compact counter); controls on
// non-local qubits are constant over the tile and become a tile predicate, so a tile that no
// gate of the pass selects is neither read nor written.
#pragma once

#include "qs_internal.cuh"

namespace qs {

constexpr int kTileMaxBits = 14;
constexpr int kTileSeg = kTileMaxBits + 1;
constexpr int kTileMaxParam = 64;  // parameterised gates per adjoint pass
constexpr int kTileMaxGates = 96;  // gates per pass
constexpr int kTileThreads = 256;

// One gate of a pass, in the pass's local coordinates.
struct TileGate {
    uint32_t mask[kTileSeg];  // local pair counter -> local index (segments)
    uint8_t shift[kTileSeg];
    uint8_t nseg;
    uint32_t ins;             // inserted local control values
    uint32_t tbit;            // local target bit
    uint32_t log_pairs;       // log2 of the pairs selected inside a tile
    int32_t op;               // GateOp
    int32_t side;             // OP_SIDE: which side is scaled
    int32_t slot;             // adjoint: accumulator index inside the pass, -1 if no parameter
    int32_t pkind;            // batch: QS_GATE_RY / QS_GATE_RZ -> matrices from theta[pidx]; 0 = fixed
    int32_t pidx;             // batch: parameter index inside the state
    int32_t pad;
    uint64_t hmask, hvals;    // non-local controls: the tile predicate (global bits)
    double U[8];              // forward: U; adjoint: U^dagger
    double D[8];              // adjoint: dU/dtheta (parameterised gates)
    float Uf[8];              // the same, rounded once to float32 for complex64 states
    float Df[8];
};

struct TilePass {
    int n, k;
    int nruns;                 // local offset -> global bits, by runs of consecutive bits
    uint8_t run_src[kTileMaxBits], run_len[kTileMaxBits], run_dst[kTileMaxBits];
    uint64_t tmask[kMaxSeg];   // tile index -> base address (non-local positions)
    int32_t tshift[kMaxSeg];
    int32_t tnseg;
    uint64_t ntiles;
    int32_t gate_begin, gate_count;
    int32_t nparam;            // adjoint: parameterised gates of this pass
    int32_t param_gslot[kTileMaxParam];  // adjoint: global gradient slot of each accumulator
};

// Launch one pass. `gates` is the device copy of the gate table; `part` the gradient partial
// array [slot][kAdjMaxBlocks] (adjoint only).
cudaError_t launch_tile_pass(int dtype, void *psi, void *lam, const TilePass &p, const TileGate *gates,
                             double *part, size_t part_stride, cudaStream_t st);
size_t tile_smem_bytes(int dtype, int k, bool adjoint);

}  // namespace qs
