// k_diag.cuh -- runs of diagonal gates applied in one pass.
//
// A gate diag(a, d) on target t with controls (mask, vals) multiplies amplitude k by
//   f(k) = a  if (k & mask) == vals and bit t of k is 0,
//          d  if (k & mask) == vals and bit t of k is 1,
//          1  otherwise,
// so consecutive diagonal gates commute and their product is the diagonal operator
// prod_g f_g(k). One pass applies it: every thread owns chunks of 8 consecutive amplitudes
// (index bits 0-2 vary inside a chunk), evaluates each gate's factor once per chunk where the
// factor does not depend on bits 0-2, and loads / stores a chunk only when some factor in it
// differs from 1.
#pragma once

#include <cstdint>

#include "qs_internal.cuh"

namespace qs {

constexpr int kDiagChunkBits = 3;   // amplitudes per chunk: 8
constexpr int kDiagMaxGates = 64;   // gates per launch (staged in shared memory)

// The chunks of a launch are visited through a compact counter with the launch's fixed bits
// inserted (index bits >= 3 on which every gate needs the same value for its factor to differ
// from 1, as the controls of a single gate are inserted into its pair counter): the 32 chunks of
// a warp then differ only in the five lowest free chunk bits, the warp's "lane bits".
enum DiagClass : int32_t {
    DIAG_WARP = 0, // factor independent of bits 0-2 and the lane bits: the same for a whole warp
    DIAG_WT = 1,   // controls off bits 0-2 and the lane bits, target t in them, t shared by all
                   // DIAG_WT gates of a launch: the warp forms the products for bit t = 0 and 1
    DIAG_HI = 2,   // independent of bits 0-2: one scalar per chunk
    DIAG_LO1 = 3,  // on one bit u < 3 (and bits >= 3): a scalar per value of bit u
    DIAG_LOM = 4,  // on two or more bits < 3: per element
};
constexpr int kDiagClasses = 5;
constexpr int kDiagMaxFixed = 8;

// Host-built description of one diagonal gate (device table entry).
struct DiagGate {
    uint64_t hm, hv;      // condition on bits >= 3 (controls): (k & hm) == hv
    uint64_t thi;         // 1 << t when t >= 3, else 0
    int32_t cls;          // DiagClass
    int32_t u;            // DIAG_LO1: the low bit
    int32_t ut;           // DIAG_LO1: 1 if u is the target, 0 if u is a control with value cv
    int32_t cv;
    int32_t lm, lv;       // DIAG_LOM: controls on bits < 3
    int32_t tlo;          // 1 << t when t < 3, else 0
    int32_t aone, done;   // a == 1, d == 1 exactly
    int32_t t;
    double a[2], d[2];
};

// Classify gate plan p (op DIAG or SIDE) into a DiagGate (never DIAG_WT: that needs the whole
// launch, see assign_diag_classes). Returns false for other ops.
bool make_diag_gate(const GatePlan &p, DiagGate *out);

// One launch: gates sorted by class, ncls[c] = gates of class c, wt = the DIAG_WT target;
// nfix fixed bits at chunk-level positions fix_pos (ascending) with values fix_val (bit i for
// fix_pos[i]); warp classes only when the compact counter has >= 32 values.
// lead_t >= 0: the pass first applies the uncontrolled 2x2 gate lu (row-major, interleaved
// re / im) on target lead_t to every amplitude (then no bits are fixed: every chunk changes).
struct DiagCounts {
    int32_t ncls[kDiagClasses];
    int32_t wt;
    int32_t nfix;
    int32_t fix_pos[kDiagMaxFixed];
    uint32_t fix_val;
    int32_t lead_t;
    double lu[8];
};

// Find the launch's fixed bits (none with a leading gate on lead_t >= 0), classify its gates
// (sorted by class in place) and count them.
DiagCounts assign_diag_classes(DiagGate *gates, int count, int n, int lead_t = -1);

// Apply gates[0..count) (device table), after the leading gate if counts.lead_t >= 0, to the
// 2^n amplitudes at psi.
cudaError_t launch_diag_run(int dtype, void *psi, int n, const DiagGate *gates, int count, DiagCounts counts,
                            cudaStream_t st);

}  // namespace qs
