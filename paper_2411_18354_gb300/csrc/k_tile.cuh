// k_tile.cuh -- fused tile pass: a run of consecutive gates applied to shared-memory tiles
// of the state in one HBM round trip.
//
// A pass chooses k "local" qubits L (always including the lowest ones, so that tile rows are
// contiguous in memory, plus the targets of its gates). A tile is the 2^k amplitudes that
// share the values of the n - k non-local qubits. Controls on non-local qubits are constant
// over a tile and become a tile predicate, so a tile that no gate of the pass selects is
// neither read nor written.
//
// Inside a tile the gates run in register groups: consecutive gates whose targets lie in a
// set Q of (at most) 4 local qubits. Each thread takes one row -- the 16 amplitudes that
// differ only in Q -- into registers, applies every gate of the group to it (pairs 2^p apart
// inside the row, p = the target's place in Q; controls in Q select elements, controls on
// other local qubits select rows), and writes it back: one shared-memory round trip per
// group instead of one per gate. Tiles are stored in shared memory with an XOR swizzle of
// the low index bits so that the rows of a warp fall on distinct banks.
#pragma once

#include "qs_internal.cuh"

namespace qs {

constexpr int kTileMaxBits = 14;
constexpr int kGroupBits = 4;      // register qubits per group, at most (16 amplitudes per row)
constexpr int kGroupBitsAdjoint = 3;  // in the adjoint sweep (psi and lambda rows in registers)
constexpr int kTileMaxParam = 64;  // parameterised gates per adjoint pass
constexpr int kTileMaxGates = 64;   // gates (and so at most as many groups) per pass of the batched kernel
constexpr int kPassMaxGates = 128;  // the same for a single-state tile pass (tables sized per pass)
constexpr int kTileThreads = 256;

// One gate inside a register group.
struct RegGate {
    uint8_t p;                // target: bit p of the row element index
    uint8_t cqm, cqv;         // controls on group qubits: element e selected iff (e & cqm) == cqv
    uint8_t pad0;
    uint32_t crm, crv;        // controls on other local qubits: row selected iff (row & crm) == crv
    int32_t op;               // GateOp
    int32_t side;             // OP_SIDE: which side is scaled
    int32_t slot;             // adjoint: accumulator index, -1 if no parameter
    int32_t pkind;            // batch: QS_GATE_RY / QS_GATE_RZ -> matrices from theta[pidx]; 0 = fixed
    int32_t pidx;             // batch: parameter index inside the state
    int32_t pkind2, pidx2;    // batch forward: a second rotation applied after the first (0 = none)
    int32_t pad1;
    uint64_t hmask, hvals;    // non-local controls: the tile predicate (global bits)
    double U[8];              // forward: U; adjoint: U^dagger
    double D[8];              // adjoint: dU/dtheta (parameterised gates)
    float Uf[8];              // the same, rounded once to float32 for complex64 states
    float Df[8];
};

// A register group: which local qubits are in registers, how a row number becomes a local
// index (the other local qubits), and its gates.
struct TileGroup {
    uint8_t q[kGroupBits];    // local positions of the group qubits (element bit i <-> q[i])
    uint8_t r;                // number of group qubits (< 4 only for tiles of fewer than 4 qubits)
    uint8_t nrseg;            // row -> local index segments
    uint8_t rshift[kGroupBits + 1];
    uint32_t rmask[kGroupBits + 1];
    uint32_t qsw[kGroupBits];  // shared-memory offset (swizzled) of each group qubit's bit
    int32_t gate_begin, gate_count;  // into the RegGate table
    int32_t hctrl;             // some gate of the group has a non-local control
    // Exchanges at the start / end of the group whose controls all sit in the group permute its
    // elements; they are folded into the row copies: element e is read from offset gperm[e]
    // (has_g) and written to offset sperm[e] (has_s) instead of its own position.
    uint16_t gperm[1 << kGroupBits], sperm[1 << kGroupBits];
    uint8_t has_g, has_s, pad[2];
};

struct TilePass {
    int n, k;
    int nruns;                 // local offset -> global bits, by runs of consecutive bits
    uint8_t run_src[kTileMaxBits], run_len[kTileMaxBits], run_dst[kTileMaxBits];
    uint64_t tmask[kMaxSeg];   // tile index -> base address (non-local positions)
    int32_t tshift[kMaxSeg];
    int32_t tnseg;
    uint64_t ntiles;
    int32_t gate_begin, gate_count;    // all RegGates of the pass
    int32_t group_begin, group_count;  // its register groups
    int32_t hctrl;                     // some gate of the pass has a non-local control
    int32_t nparam;            // adjoint: parameterised gates of this pass
    int32_t param_gslot[kTileMaxParam];  // adjoint: global gradient slot of each accumulator
};

// Launch one pass. `groups` / `gates` are the device copies of the group and gate tables;
// `part` the gradient partial array [slot][part_stride] (adjoint only).
cudaError_t launch_tile_pass(int dtype, void *psi, void *lam, const TilePass &p, const TileGroup *groups,
                             const RegGate *gates, double *part, size_t part_stride, cudaStream_t st);
// Dynamic shared memory of one k_tile_pass block: the 2^k-amplitude tile (psi and lambda for
// the adjoint), the adjoint's accumulators, and the pass's group and gate tables.
size_t tile_smem_bytes(int dtype, int k, bool adjoint, int groups, int gates);
constexpr size_t kTileMaxSmem = 227 * 1024;  // opt-in shared memory per block

// Shared-memory position of local index a (XOR swizzle of the low `sw` bits with the folded
// higher bits; sw = 4 for complex64, 3 for complex128). A bijection on [0, 2^k).
__host__ __device__ __forceinline__ uint32_t tile_swizzle(uint32_t a, int sw) {
    uint32_t x = a >> sw, f = 0;
    for (int i = 0; i < kTileMaxBits; i += sw) f ^= x >> i;
    return a ^ (f & ((1u << sw) - 1u));
}

}  // namespace qs
