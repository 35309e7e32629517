// qs_fuse.cuh -- fused program: a sequence of single-gate launches and tile passes.
#pragma once

#include <vector>

#include "k_diag.cuh"
#include "k_tile.cuh"

namespace qs {

struct FusedOp {
    int pass;       // >= 0: index into passes; -1: single gate or diagonal run
    int gate;       // single gate: index into the plan list
    int drun = -1;  // >= 0: index into druns (a run of diagonal gates in one pass, k_diag)
};

struct DiagRun {
    int begin, count;  // into FusedProgram::dgates (sorted by class)
    DiagCounts nc;
};

struct FusedProgram {
    std::vector<FusedOp> ops;
    std::vector<TilePass> passes;
    std::vector<TileGroup> groups;  // all passes' register groups
    std::vector<RegGate> gates;     // all groups' gates
    std::vector<int> gate_src;      // plan index each RegGate came from
    std::vector<int> order;         // plan indices in the order the program applies them
    std::vector<DiagRun> druns;
    std::vector<DiagGate> dgates;   // all diagonal runs' gates
    double model_cost = 0.0;        // planner's cost estimate (units of one state read + write)
};

// Modelled cost of launching gate p alone (fraction of the state it moves), and the fixed
// latency of one launch on an n-qubit state, both in units of one state read + write.
double single_launch_cost(const GatePlan &p, int dtype);
double launch_latency_cost(int n, int dtype);

// Fraction of the tiles pass `pass` reads and writes: those at least one of its gates selects
// (all of them when exchanges are folded into its row copies).
double pass_touched_fraction(const FusedProgram &prog, int pass);

// Byte size and packing of a program's device table: groups, then gates, then the diagonal
// runs' gates (each part 16-byte aligned).
size_t program_table_bytes(const FusedProgram &p);
void pack_program_table(const FusedProgram &p, void *host_dst);
// Device pointers of the two parts, given the table's device base address.
const TileGroup *table_groups(const FusedProgram &p, const void *dev_base);
const RegGate *table_gates(const FusedProgram &p, const void *dev_base);
const DiagGate *table_dgates(const FusedProgram &p, const void *dev_base);

// Plan the gates plans[seq[0]], plans[seq[1]], ... (the circuit's order; the program may apply
// gates that commute in another order, see `order`). For the adjoint
// sweep, `dus[g]` is dU/dtheta of gate g (nullptr when g has no parameter) and `gslots[g]` its
// gradient slot; pass nullptr for both in forward mode. k = local qubits per tile.
// max_gates bounds the gates of one pass (fusion depth); with allow_single == false every gate
// goes into a pass, also when the pass holds only that gate.
bool plan_fused(int n, int dtype, int k, const std::vector<int> &seq, const std::vector<GatePlan> &plans,
                const std::vector<const double *> *dus, const std::vector<int> *gslots, FusedProgram *prog,
                int max_gates = kPassMaxGates, bool allow_single = true, int group_bits = 0, bool jit = false);
// group_bits: register qubits per group; 0 = kGroupBits for forward programs and
// kGroupBitsAdjoint when dus != nullptr. The kernel that runs the program must use the same.
// Forward programs with allow_single (not the batched kernel) may also put consecutive
// diagonal gates, optionally after one uncontrolled gate, into diagonal-run ops.
// jit: the passes will run as kernels compiled for their shape (QS_FLAG_JIT), whose per-gate
// cost is lower (and depends on the gate's operation), so passes may hold more gates.

}  // namespace qs
