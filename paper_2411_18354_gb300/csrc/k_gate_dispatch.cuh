// k_gate_dispatch.cuh -- picks the k_gate instantiation for a GatePlan and launches it.
// Included once per precision (k_gate_c64.cu, k_gate_c128.cu) so the two instantiation
// sets compile in parallel.
#pragma once

#include <algorithm>

#include "k_gate.cuh"

namespace qs {
namespace gate_detail {

template <typename Real, typename Idx>
DevGate<Real, Idx> make_dev(const GatePlan &p, uint64_t cmask, uint64_t cvals) {
    DevGate<Real, Idx> g;
    for (int s = 0; s < kMaxSeg; ++s) {
        g.mask[s] = (Idx)(s < p.map.nseg ? p.map.mask[s] : 0);
        g.shift[s] = s < p.map.nseg ? p.map.shift[s] : 0;
    }
    g.ins = (Idx)p.map.ins;
    g.tbit = (Idx)p.tbit;
    g.cmask = (Idx)cmask;
    g.cvals = (Idx)cvals;
    for (int i = 0; i < 8; ++i) g.m[i] = (Real)p.U[i];
    return g;
}

template <typename K>
int occupancy_of(K kern) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kGateThreads, 0) != cudaSuccess || occ < 1)
        occ = 1;
    return occ;
}

template <typename Real, typename Idx, int NS, int LAY, int R, int OP, bool MASKED>
cudaError_t go(void *psi, const GatePlan &p, uint64_t cmask, uint64_t cvals, cudaStream_t st) {
    // units in flight per thread: 2 with a vector on each side, 4 with one vector per unit
    constexpr int UNR = (LAY == LAY_ADJ || OP == OP_SIDE) ? 4 : 2;
    auto kern = k_gate<Real, Idx, NS, LAY, R, OP, MASKED, UNR>;
    static const int occ = occupancy_of(kern);
    const uint64_t per_block = (uint64_t)kGateThreads * UNR;
    const uint64_t need = (p.units + per_block - 1) / per_block;
    const uint64_t cap = (uint64_t)device_sm_count() * (uint64_t)occ;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(need, cap));
    using T2 = typename CxT<Real>::T;
    // small gates (at most 2^15 pair counters per block of the grid: c >= 4 at n = 30) start as
    // programmatic dependents of the previous kernel, hiding their launch behind its tail; large
    // ones launch normally (their blocks would only wait on the SMs while the previous gate drains)
    const bool dependent = (p.units << p.r) <= (uint64_t)grid << 15;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kGateThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = dependent ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, reinterpret_cast<T2 *>(psi), make_dev<Real, Idx>(p, cmask, cvals),
                              (Idx)p.units, p.side);
}

template <typename Real, typename Idx, int NS, bool MASKED>
cudaError_t by_shape(void *psi, const GatePlan &p, uint64_t cmask, uint64_t cvals, cudaStream_t st) {
    constexpr bool F = sizeof(Real) == 4;
    const int op = MASKED ? (int)OP_GEN : p.op;
#define QS_OPS(LAY, R)                                                                        \
    switch (op) {                                                                             \
        case OP_GEN: return go<Real, Idx, NS, LAY, R, OP_GEN, MASKED>(psi, p, cmask, cvals, st); \
        case OP_REAL: if (!MASKED) return go<Real, Idx, NS, LAY, R, OP_REAL, false>(psi, p, cmask, cvals, st); break; \
        case OP_SWAP: if (!MASKED) return go<Real, Idx, NS, LAY, R, OP_SWAP, false>(psi, p, cmask, cvals, st); break; \
        case OP_DIAG: if (!MASKED) return go<Real, Idx, NS, LAY, R, OP_DIAG, false>(psi, p, cmask, cvals, st); break; \
        case OP_SIDE: if (!MASKED && LAY == LAY_SPLIT) return go<Real, Idx, NS, LAY_SPLIT, R, OP_SIDE, false>(psi, p, cmask, cvals, st); break; \
        default: break;                                                                       \
    }
    if (p.layout == LAY_SPLIT) {
        if (p.r == 0) { QS_OPS(LAY_SPLIT, 1) }
        else if (p.r == 1 && F) { QS_OPS(LAY_SPLIT, 2) }
    } else if (p.r == 0) {
        QS_OPS(LAY_ADJ, 1)
    }
#undef QS_OPS
    return cudaErrorInvalidValue;
}

template <typename Real, typename Idx, bool MASKED>
cudaError_t by_nseg(void *psi, const GatePlan &p, uint64_t cmask, uint64_t cvals, cudaStream_t st) {
    const int ns = p.map.nseg;
    if (ns <= 2) return by_shape<Real, Idx, 2, MASKED>(psi, p, cmask, cvals, st);
    if (ns <= 4) return by_shape<Real, Idx, 4, MASKED>(psi, p, cmask, cvals, st);
    if (ns <= 10) return by_shape<Real, Idx, 10, MASKED>(psi, p, cmask, cvals, st);
    return by_shape<Real, Idx, kMaxSeg, MASKED>(psi, p, cmask, cvals, st);
}

template <typename Real>
cudaError_t launch(void *psi, const GatePlan &p, bool masked, uint64_t cmask, uint64_t cvals,
                   cudaStream_t st) {
    if (p.units == 0) return cudaSuccess;
    const bool narrow = p.n <= 32;  // every amplitude index fits in 32 bits
    if (masked)
        return narrow ? by_nseg<Real, uint32_t, true>(psi, p, cmask, cvals, st)
                      : by_nseg<Real, uint64_t, true>(psi, p, cmask, cvals, st);
    return narrow ? by_nseg<Real, uint32_t, false>(psi, p, cmask, cvals, st)
                  : by_nseg<Real, uint64_t, false>(psi, p, cmask, cvals, st);
}

}  // namespace gate_detail
}  // namespace qs
