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

enum DiagClass : int32_t {
    DIAG_WARP = 0, // factor depends on bits >= 8 only: the same for the 32 chunks of a warp
    DIAG_HI = 1,   // on bits >= 3 only: one scalar per chunk
    DIAG_LO1 = 2,  // on bits >= 3 and one bit u < 3: a scalar per value of bit u
    DIAG_LOM = 3,  // on two or more bits < 3: per element
};
// A warp's 32 consecutive chunks differ only in index bits 3-7.
constexpr int kDiagWarpBits = kDiagChunkBits + 5;

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
    int32_t pad;
    double a[2], d[2];
};

// Classify gate plan p (op DIAG or SIDE) into a DiagGate. Returns false for other ops.
bool make_diag_gate(const GatePlan &p, DiagGate *out);

// Gates of one launch, sorted by class (DIAG_WARP first, then HI, LO1, LOM); ncls[c] = gates of
// class c. count <= kDiagMaxGates; DIAG_WARP gates need n >= kDiagWarpBits.
struct DiagCounts {
    int32_t ncls[4];
};

// Apply gates[0..count) (device table) to the 2^n amplitudes at psi.
cudaError_t launch_diag_run(int dtype, void *psi, int n, const DiagGate *gates, int count, DiagCounts counts,
                            cudaStream_t st);

}  // namespace qs
