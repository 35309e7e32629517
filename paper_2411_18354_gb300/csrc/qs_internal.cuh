// qs_internal.cuh -- shared declarations of the libqs translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "qs.h"

namespace qs {

// Largest number of non-empty free-bit segments a counter can be split into: with m
// inserted positions and n - m free bits there are at most min(m + 1, n - m) non-empty
// segments, which is at most 21 for n <= 40.
constexpr int kMaxSeg = 21;
constexpr int kMaxQubits = 40;

// Gate operation classes chosen on the host from the exact structure of U.
enum GateOp : int {
    OP_GEN = 0,   // general 2x2: (x, y) -> (a x + b y, c x + d y)
    OP_SWAP = 1,  // (x, y) -> (y, x), no arithmetic
    OP_DIAG = 2,  // (x, y) -> (a x, d y)
    OP_SIDE = 3,  // one side only: z -> s z on the amplitudes whose bit t equals `side`
    OP_REAL = 4,  // general 2x2 with real entries (e.g. RY, H): half the multiplications
};

// Layout classes of one work unit (see k_gate.cu).
enum UnitLayout : int {
    LAY_SPLIT = 0,  // unit = R consecutive amplitudes at lo and R at lo + 2^t
    LAY_ADJ = 1,    // t == 0: unit = R consecutive (x, y) pairs, 2R contiguous amplitudes
};

// Counter -> amplitude index map of one gate: idx(j) = ins | OR_s ((j << shift_s) & mask_s).
// Segment s holds the free amplitude bits between the (s-1)-th and s-th inserted
// position (inserted = target and controls, ascending), so every counter bit moves up by
// the number of inserted positions below it. This is Eq. 4 of Section III-B (insert the
// control bits, ascending) followed by ithCleared (insert a 0 at the target) written as
// masks: inserting at ascending positions p_0 < p_1 < ... moves the bits of segment s up
// by s.
struct IndexMap {
    uint64_t mask[kMaxSeg];
    uint64_t ins;      // inserted bit values: control values (target bit is 0)
    int32_t shift[kMaxSeg];
    int32_t nseg;      // number of non-empty segments actually used
    int32_t pad;
};

struct GatePlan {
    int n;
    int t;
    int c;              // number of controls
    uint64_t tbit;      // 1 << t
    int op;             // GateOp
    int side;           // OP_SIDE: 0 = lo side (a), 1 = hi side (d)
    int layout;         // UnitLayout
    int r;              // log2 of amplitudes (SPLIT) or pairs (ADJ) per unit
    uint64_t units;     // number of work units
    IndexMap map;       // counter -> first amplitude of the unit
    double U[8];        // matrix (for OP_SIDE: U[0..1] = scalar)
    uint64_t ctrl_mask; // the gate as given (for the fused tile pass)
    uint64_t ctrl_vals;
    double Ufull[8];    // full matrix (exchange: [[0,1],[1,0]])
};

// Host planning (qs_plan.cpp): builds the sorted insertion positions and picks op/layout.
// Returns false and writes `err` if the gate is invalid.
// force_op >= 0 skips the structure analysis and uses that GateOp with the full U.
bool plan_gate(int n, int dtype, int target, uint64_t ctrl_mask, uint64_t ctrl_vals,
               const double U[8], int kind, int force_op, GatePlan *out, char *err, size_t errlen);
// Counter -> index segments for inserted positions pos[0..m-1] (ascending, values `ins`).
void build_map(int n, const int *pos, int m, uint64_t ins, IndexMap *map);
// Same plan with all 2^(n-1) pairs scheduled and masked (baseline comparator).
void plan_masked(const GatePlan &compact, GatePlan *out);

int device_sm_count();

// Launchers (return the CUDA error of the launch).
cudaError_t launch_gate(int dtype, void *psi, const GatePlan &p, cudaStream_t st);
cudaError_t launch_gate_masked(int dtype, void *psi, const GatePlan &p, uint64_t ctrl_mask,
                               uint64_t ctrl_vals, cudaStream_t st);
cudaError_t launch_set_basis(int dtype, void *psi, int n, uint64_t k, cudaStream_t st);

// Fixed-point (QS_Q30) gate kernel: matrix from p.Ufull rounded to Q1.30 (k_gate_q30.cu).
cudaError_t launch_gate_q30(void *psi, const GatePlan &p, bool masked, uint64_t cmask, uint64_t cvals,
                            cudaStream_t st);
cudaError_t launch_expect_z_q30(const void *psi, int n, double *scratch, double *out_z, double *out_norm2,
                                cudaStream_t st);

// Reductions: partial sums per block, then a fixed-order final pass (deterministic).
// `scratch` must hold reduce_scratch_doubles(n) doubles.
size_t reduce_scratch_doubles(int n);
cudaError_t launch_expect_z(int dtype, const void *psi, int n, double *scratch,
                            double *out_z /*device, n*/, double *out_norm2 /*device, 1*/,
                            cudaStream_t st);

}  // namespace qs
