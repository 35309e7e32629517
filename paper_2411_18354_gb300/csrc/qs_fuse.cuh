// qs_fuse.cuh -- fused program: a sequence of single-gate launches and tile passes.
#pragma once

#include <vector>

#include "k_tile.cuh"

namespace qs {

struct FusedOp {
    int pass;  // >= 0: index into passes; -1: single gate
    int gate;  // single gate: index into the plan list
};

struct FusedProgram {
    std::vector<FusedOp> ops;
    std::vector<TilePass> passes;
    std::vector<TileGate> gates;  // all passes' gates, uploaded to the device once
    std::vector<int> gate_src;    // plan index each TileGate came from
};

// Plan the gates plans[seq[0]], plans[seq[1]], ... (execution order). For the adjoint
// sweep, `dus[g]` is dU/dtheta of gate g (nullptr when g has no parameter) and `gslots[g]` its
// gradient slot; pass nullptr for both in forward mode. k = local qubits per tile.
// max_gates bounds the gates of one pass (fusion depth); with allow_single == false every gate
// goes into a pass, also when the pass holds only that gate.
bool plan_fused(int n, int dtype, int k, const std::vector<int> &seq, const std::vector<GatePlan> &plans,
                const std::vector<const double *> *dus, const std::vector<int> *gslots, FusedProgram *prog,
                int max_gates = kTileMaxGates, bool allow_single = true);

}  // namespace qs
