// qs_debug.cuh -- checks of the library's debug build (compiled with QS_DEBUG_CHECKS).
//
// compute-sanitizer is not available for these kernels, so the debug build checks two things
// itself, without trapping: every global-memory access of the gate, tile-pass and
// diagonal-run kernels (and of compiled passes) lies inside the state under test, and, when a
// per-amplitude counter array is given, how often each amplitude is written. An access outside
// the state is not made: its index is recorded in a device status word that the host reads
// back (qs_debug_status), and the kernel carries on. In the release build the macros are empty.
#pragma once

#include <cstdint>

namespace qs {

struct DebugState {
    unsigned int status;          // bit 0: an access outside [0, n_amps) was skipped
    unsigned int pad;
    unsigned long long n_amps;    // amplitudes of the state under test (0: no bounds check)
    unsigned int *counts;         // writes per amplitude (nullptr: not counted)
    unsigned long long count_n;   // length of counts
    unsigned long long first_bad; // an index that failed the check
};

#ifdef QS_DEBUG_CHECKS
extern __device__ DebugState g_qs_debug;

// True if amplitudes [idx, idx + span) are inside the state; otherwise records idx and
// returns false (the caller skips the access).
__device__ __forceinline__ bool dbg_in_range(uint64_t idx, int span) {
    const unsigned long long n = g_qs_debug.n_amps;
    if (n == 0 || idx + (uint64_t)span <= n) return true;
    g_qs_debug.first_bad = idx;
    atomicOr(&g_qs_debug.status, 1u);
    return false;
}

// Counts one write of each amplitude in [idx, idx + span).
__device__ __forceinline__ void dbg_count(uint64_t idx, int span) {
    unsigned int *c = g_qs_debug.counts;
    if (!c) return;
    for (int i = 0; i < span; ++i)
        if (idx + i < g_qs_debug.count_n) atomicAdd(c + idx + i, 1u);
}
#define QS_DBG_OK(idx, span) ::qs::dbg_in_range((uint64_t)(idx), (span))
#define QS_DBG_WRITE(idx, span) ::qs::dbg_count((uint64_t)(idx), (span))
#else
#define QS_DBG_OK(idx, span) true
#define QS_DBG_WRITE(idx, span) ((void)0)
#endif

}  // namespace qs
