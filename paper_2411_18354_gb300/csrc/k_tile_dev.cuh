// k_tile_dev.cuh -- device code shared by the fused tile pass and the batched kernel:
// applying register groups of gates to one shared-memory tile (and, for the adjoint sweep,
// to the matching lambda tile, with the gradient inner products).
#pragma once

#include "k_gate.cuh"
#include "k_tile.cuh"

namespace qs {
namespace tiledev {

template <typename Real> struct TileT;
template <> struct TileT<float> {
    using T2 = float2;
    using V = float4;  // 2 amplitudes per 16-byte global vector
    static constexpr int VEC = 2;
    static constexpr int SW = 4;  // 16 amplitudes of 8 bytes per 128-byte bank row
    __device__ static const float *U(const RegGate &G) { return G.Uf; }
    __device__ static const float *D(const RegGate &G) { return G.Df; }
};
template <> struct TileT<double> {
    using T2 = double2;
    using V = double2;
    static constexpr int VEC = 1;
    static constexpr int SW = 3;  // 8 amplitudes of 16 bytes per bank row
    __device__ static const double *U(const RegGate &G) { return G.U; }
    __device__ static const double *D(const RegGate &G) { return G.D; }
};

// Compact copy of a RegGate in shared memory (matrices in the state's precision), staged once
// per pass so that every row reads its gates with broadcast shared-memory loads.
template <typename Real> struct alignas(16) SGate {
    uint64_t hmask, hvals;
    // crm, crv, meta, pidx -- one 16-byte load; meta = code | cqm << 8 | cqv << 12 | side << 16 |
    // pkind << 17 | (slot + 1) << 20, code = (op * 4 + p) * 2 + (cqm != 0)
    uint32_t crm, crv, meta, pidx;
    Real u[8], d[8];
};

template <typename Real>
__device__ __forceinline__ void param_matrices(int kind, Real c, Real s, bool adjoint, Real *u, Real *d);

template <typename Real>
__device__ __forceinline__ void stage_gate(const RegGate &G, SGate<Real> &S, const Real *cs, bool adjoint) {
    S.hmask = G.hmask;
    S.hvals = G.hvals;
    S.crm = G.crm;
    S.crv = G.crv;
    const uint32_t code = (uint32_t)((G.op * 4 + G.p) * 2 + (G.cqm != 0));
    int pkind = G.pkind;
    S.pidx = (uint32_t)G.pidx;
    if (G.pkind != 0 && cs) {  // the state's parameter: matrices built once per pass
        param_matrices<Real>(G.pkind, cs[2 * G.pidx], cs[2 * G.pidx + 1], adjoint, S.u, S.d);
        if (G.pkind2 != 0) {  // forward only: a second rotation on the same qubit, u <- u2 u
            Real u2[8], d2[8], w[8];
            param_matrices<Real>(G.pkind2, cs[2 * G.pidx2], cs[2 * G.pidx2 + 1], false, u2, d2);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const Real *a0 = u2 + 4 * i, *b0 = S.u + 2 * j, *b1 = S.u + 4 + 2 * j;
                    w[4 * i + 2 * j] = a0[0] * b0[0] - a0[1] * b0[1] + a0[2] * b1[0] - a0[3] * b1[1];
                    w[4 * i + 2 * j + 1] = a0[0] * b0[1] + a0[1] * b0[0] + a0[2] * b1[1] + a0[3] * b1[0];
                }
#pragma unroll
            for (int i = 0; i < 8; ++i) S.u[i] = w[i];
        }
        pkind = 0;
    } else {
        const Real *u = TileT<Real>::U(G);
        const Real *d = TileT<Real>::D(G);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            S.u[i] = u[i];
            S.d[i] = d[i];
        }
    }
    S.meta = code | ((uint32_t)G.cqm << 8) | ((uint32_t)G.cqv << 12) | ((uint32_t)(G.side & 1) << 16) |
             ((uint32_t)(pkind & 7) << 17) | ((uint32_t)(G.slot + 1) << 20);
}

// Copy a pass's groups and gates to shared memory (group gate indices become pass-relative).
// Ends with a block barrier.
template <typename Real>
__device__ __forceinline__ void stage_pass(const TilePass &P, const TileGroup *groups, const RegGate *gates,
                                           TileGroup *sgroups, SGate<Real> *sgates, const Real *cs = nullptr,
                                           bool adjoint = false) {
    for (int i = threadIdx.x; i < P.group_count; i += blockDim.x) {
        TileGroup g = groups[P.group_begin + i];
        g.gate_begin -= P.gate_begin;
        sgroups[i] = g;
    }
    for (int i = threadIdx.x; i < P.gate_count; i += blockDim.x)
        stage_gate<Real>(gates[P.gate_begin + i], sgates[i], cs, adjoint);
    __syncthreads();
}

// Gate fields kept in registers while a row is processed.
template <typename Real> struct GateRegs {
    uint32_t crm, crv;
    int cqm, cqv, side, slot, code;
    Real u[8], d[8];
};

// Parameterised matrices from (c, s) = (cos(theta/2), sin(theta/2)):
//  RY = [[c, -s], [s, c]]             RY^dagger = [[c, s], [-s, c]]   dRY = 1/2 [[-s, -c], [c, -s]]
//  RZ = diag(c - i s, c + i s)        RZ^dagger = diag(c + i s, c - i s)
//  dRZ = diag((-s - i c) / 2, (-s + i c) / 2)
template <typename Real>
__device__ __forceinline__ void param_matrices(int kind, Real c, Real s, bool adjoint, Real *u, Real *d) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        u[i] = 0;
        d[i] = 0;
    }
    const Real h = (Real)0.5;
    if (kind == QS_GATE_RY) {
        u[0] = c;
        u[6] = c;
        u[2] = adjoint ? s : -s;
        u[4] = adjoint ? -s : s;
        d[0] = -h * s;
        d[2] = -h * c;
        d[4] = h * c;
        d[6] = -h * s;
    } else {
        u[0] = c;
        u[6] = c;
        u[1] = adjoint ? s : -s;
        u[7] = adjoint ? -s : s;
        d[0] = -h * s;
        d[1] = -h * c;
        d[6] = -h * s;
        d[7] = h * c;
    }
}

// Raw copy of a staged gate (one 16-byte control word and the matrices).
template <typename Real> struct GateRaw {
    uint4 w;  // crm, crv, meta, pidx
    Real u[8], d[8];
};

template <typename Real, bool ADJ>
__device__ __forceinline__ void fetch_gate(const SGate<Real> &G, GateRaw<Real> &r) {
    using V = typename TileT<Real>::V;  // 16 bytes
    constexpr int PER = 16 / sizeof(Real);
    r.w = *reinterpret_cast<const uint4 *>(&G.crm);
#pragma unroll
    for (int i = 0; i < 8; i += PER) *reinterpret_cast<V *>(&r.u[i]) = *reinterpret_cast<const V *>(&G.u[i]);
    if (ADJ) {
#pragma unroll
        for (int i = 0; i < 8; i += PER) *reinterpret_cast<V *>(&r.d[i]) = *reinterpret_cast<const V *>(&G.d[i]);
    }
}

template <typename Real>
__device__ __forceinline__ void decode_gate(const GateRaw<Real> &g, GateRegs<Real> &r, const Real *cs, bool adjoint) {
    r.crm = g.w.x;
    r.crv = g.w.y;
    const uint32_t meta = g.w.z;
    r.code = (int)(meta & 0xffu);
    r.cqm = (int)((meta >> 8) & 0xfu);
    r.cqv = (int)((meta >> 12) & 0xfu);
    r.side = (int)((meta >> 16) & 1u);
    const int pkind = (int)((meta >> 17) & 7u);
    r.slot = (int)(meta >> 20) - 1;
    if (pkind != 0 && cs) {
        param_matrices<Real>(pkind, cs[2 * g.w.w], cs[2 * g.w.w + 1], adjoint, r.u, r.d);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) r.u[i] = g.u[i];
        if (adjoint) {
#pragma unroll
            for (int i = 0; i < 8; ++i) r.d[i] = g.d[i];
        }
    }
}

__device__ __forceinline__ uint64_t tile_base(const TilePass &P, uint64_t tau) {
    uint64_t b = 0;
    for (int s = 0; s < P.tnseg; ++s) b |= (tau << P.tshift[s]) & P.tmask[s];
    return b;
}

__device__ __forceinline__ uint64_t scatter_local(const TilePass &P, uint32_t o) {
    uint64_t g = 0;
    for (int r = 0; r < P.nruns; ++r)
        g |= (uint64_t)((o >> P.run_src[r]) & ((1u << P.run_len[r]) - 1u)) << P.run_dst[r];
    return g;
}

template <int OP, typename T2, typename Real>
__device__ __forceinline__ void op_pair(T2 &x, T2 &y, const Real *u, int side) {
    if (OP == OP_SIDE) {
        if (side) y = cmul<T2, Real>(u[0], u[1], y);
        else x = cmul<T2, Real>(u[0], u[1], x);
    } else {
        pair_update<OP, T2, Real>(x, y, u);
    }
}

// All pairs (e, e | 2^P) of the thread's RPT rows for one gate with operation OP; CQ: the
// gate has controls on group qubits (else every pair of a selected row is updated); UNI: every
// row is selected (no per-row predicate). RPT independent rows per thread share one decoded
// gate (the kernels use RPT = 1: with 2 rows the register budget of 2 CTAs per SM spills).
// Rows of tiles with fewer than GB qubits
// are padded with zero elements that pair only with each other, so they stay zero and add
// nothing to the inner products.
template <int P, int OP, bool ADJ, int GB, bool CQ, int RPT, bool UNI, typename T2, typename Real>
__device__ __forceinline__ void row_pairs(T2 (&v)[RPT][1 << GB], T2 (&w)[RPT][ADJ ? (1 << GB) : 1],
                                          const GateRegs<Real> &R, const bool (&ok)[RPT], Real &dot) {
    constexpr int DOP = OP == OP_DIAG ? OP_DIAG : (OP == OP_REAL ? OP_REAL : OP_GEN);
#pragma unroll
    for (int e = 0; e < (1 << GB); ++e) {
        if ((e >> P) & 1) continue;
        const int e2 = e | (1 << P);
        if (!CQ || ((e & R.cqm) == R.cqv)) {
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                if (!UNI && !ok[j]) continue;
                op_pair<OP, T2, Real>(v[j][e], v[j][e2], R.u, R.side);
                if (ADJ) {
                    if (R.slot >= 0) {
                        T2 mx = v[j][e], my = v[j][e2];
                        pair_update<DOP, T2, Real>(mx, my, R.d);
                        dot += w[j][e].x * mx.x + w[j][e].y * mx.y + w[j][e2].x * my.x + w[j][e2].y * my.y;
                    }
                    op_pair<OP, T2, Real>(w[j][e], w[j][e2], R.u, R.side);
                }
            }
        }
    }
}

// Gate dispatch. FOLD: one switch on (staged code << 1 | pred) selects operation, target
// place, in-row controls and whether rows need a per-thread predicate (fewer live registers:
// the batched kernel, which holds both sweep directions). Otherwise a uniform branch on pred
// picks one of two switches on the staged code (faster in the tile pass).
template <bool ADJ, int GB, int RPT, bool UNI, typename T2, typename Real>
__device__ __forceinline__ void row_switch(T2 (&v)[RPT][1 << GB], T2 (&w)[RPT][ADJ ? (1 << GB) : 1],
                                          const GateRegs<Real> &R, const bool (&ok)[RPT], Real &dot) {
#define QS_ROW1(OP, P, CQ)                                                                                   \
    case (((OP)*4 + (P)) * 2 + (CQ)):                                                                        \
        if ((P) < GB) row_pairs<((P) < GB ? (P) : 0), OP, ADJ, GB, CQ, RPT, UNI, T2, Real>(v, w, R, ok, dot); \
        break;
#define QS_ROW(OP, P) QS_ROW1(OP, P, 0) QS_ROW1(OP, P, 1)
#define QS_ROW_OP(OP) QS_ROW(OP, 0) QS_ROW(OP, 1) QS_ROW(OP, 2) QS_ROW(OP, 3)
    switch (R.code) {
        QS_ROW_OP(OP_GEN)
        QS_ROW_OP(OP_SWAP)
        QS_ROW_OP(OP_DIAG)
        QS_ROW_OP(OP_SIDE)
        QS_ROW_OP(OP_REAL)
        default: break;
    }
#undef QS_ROW_OP
#undef QS_ROW
#undef QS_ROW1
}

template <bool ADJ, int GB, int RPT, typename T2, typename Real>
__device__ __forceinline__ void row_switch_folded(T2 (&v)[RPT][1 << GB], T2 (&w)[RPT][ADJ ? (1 << GB) : 1],
                                                 const GateRegs<Real> &R, const bool (&ok)[RPT], bool pred,
                                                 Real &dot) {
#define QS_ROW1(OP, P, CQ, PR)                                                                                  \
    case ((((OP)*4 + (P)) * 2 + (CQ)) << 1) | (PR):                                                             \
        if ((P) < GB) row_pairs<((P) < GB ? (P) : 0), OP, ADJ, GB, CQ, RPT, !(PR), T2, Real>(v, w, R, ok, dot); \
        break;
#define QS_ROW(OP, P) QS_ROW1(OP, P, 0, 0) QS_ROW1(OP, P, 0, 1) QS_ROW1(OP, P, 1, 0) QS_ROW1(OP, P, 1, 1)
#define QS_ROW_OP(OP) QS_ROW(OP, 0) QS_ROW(OP, 1) QS_ROW(OP, 2) QS_ROW(OP, 3)
    switch ((R.code << 1) | (pred ? 1 : 0)) {
        QS_ROW_OP(OP_GEN)
        QS_ROW_OP(OP_SWAP)
        QS_ROW_OP(OP_DIAG)
        QS_ROW_OP(OP_SIDE)
        QS_ROW_OP(OP_REAL)
        default: break;
    }
#undef QS_ROW_OP
#undef QS_ROW
#undef QS_ROW1
}

template <bool ADJ, int GB, int RPT, bool FOLD, typename T2, typename Real>
__device__ __forceinline__ void row_gate(T2 (&v)[RPT][1 << GB], T2 (&w)[RPT][ADJ ? (1 << GB) : 1],
                                         const GateRegs<Real> &R, const bool (&ok)[RPT], bool pred, Real &dot) {
    if (FOLD) row_switch_folded<ADJ, GB, RPT, T2, Real>(v, w, R, ok, pred, dot);
    else if (!pred) row_switch<ADJ, GB, RPT, true, T2, Real>(v, w, R, ok, dot);
    else row_switch<ADJ, GB, RPT, false, T2, Real>(v, w, R, ok, dot);
}

// Register qubits per group: 4 for forward passes, 3 for the adjoint sweep (psi and lambda
// rows both live in registers there).
template <bool ADJ> struct GroupBits { static constexpr int v = ADJ ? 3 : kGroupBits; };

// Apply the pass's register groups to the tile tp (and lambda tile tl if ADJ) whose global
// base index is `base`. Each thread holds RPT rows of 2^GB elements at a time. Adjoint: for a
// gate with slot >= 0 the warp partial of Re <lambda| dU psi> (summed over the warp in the
// state's precision) is added to acc[slot * nwarps + warp]. Every executed group ends with a
// block barrier.
template <typename Real, bool ADJ, int GB = GroupBits<ADJ>::v, int RPT = 1, bool FOLD = false>
__device__ __forceinline__ void apply_groups(typename TileT<Real>::T2 *tp, typename TileT<Real>::T2 *tl, uint64_t base,
                                             int k, const TileGroup *groups, int group_count, const SGate<Real> *gates,
                                             const Real *cs, Acc<Real> *acc) {
    using T2 = typename TileT<Real>::T2;
    constexpr int SW = TileT<Real>::SW;
    constexpr int E = 1 << GB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int gi = 0; gi < group_count; ++gi) {
        const TileGroup &Gr = groups[gi];
        if (Gr.hctrl && !Gr.has_g && !Gr.has_s) {  // (folded exchanges act on every tile)
            bool any = false;
            for (int g = 0; g < Gr.gate_count; ++g)
                any |= (base & gates[Gr.gate_begin + g].hmask) == gates[Gr.gate_begin + g].hvals;
            if (!any) continue;  // uniform: nothing of this group touches the tile
        }
        const int r = Gr.r;
        // The swizzle is linear over XOR (a ^ f(a) with f built from shifts and XORs), so the
        // position of (row bits | element bits) is swz(row) ^ swz(element bits); the group
        // qubits' offsets come precomputed.
        uint32_t qs_[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) qs_[i] = Gr.qsw[i];
        const uint32_t rows = 1u << (k - r);
        const uint32_t step = blockDim.x * RPT;
        const bool all_rows = (rows % step) == 0;  // uniform: no thread idles in any row block
        for (uint32_t rb = 0; rb < rows; rb += step) {
            uint32_t ra[RPT], rs[RPT];
            bool active[RPT];
            T2 v[RPT][E], w[RPT][ADJ ? E : 1];
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const uint32_t rho = rb + j * blockDim.x + tid;
                active[j] = rho < rows;
                ra[j] = 0;
                for (int s = 0; s < Gr.nrseg; ++s) ra[j] |= (rho << Gr.rshift[s]) & Gr.rmask[s];
                rs[j] = tile_swizzle(ra[j], SW);
                const bool gp = Gr.has_g;  // uniform: exchanges folded into the gather
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t ps = rs[j] ^ (gp ? (uint32_t)Gr.gperm[e]
                                                    : (((e & 1) ? qs_[0] : 0u) ^ ((e & 2) ? qs_[1] : 0u) ^
                                                       ((e & 4) ? qs_[2] : 0u) ^ ((e & 8) ? qs_[3] : 0u)));
                    if (active[j] && e < (1 << r)) {
                        v[j][e] = tp[ps];
                        if (ADJ) w[j][e] = tl[ps];
                    } else {
                        v[j][e] = T2{0, 0};
                        if (ADJ) w[j][e] = T2{0, 0};
                    }
                }
            }
            const int gb = Gr.gate_begin, gc = Gr.gate_count;
            for (int g = 0; g < gc; ++g) {
                if (Gr.hctrl && (base & gates[gb + g].hmask) != gates[gb + g].hvals) continue;  // uniform
                GateRaw<Real> cr;
                fetch_gate<Real, ADJ>(gates[gb + g], cr);
                GateRegs<Real> R;
                decode_gate<Real>(cr, R, cs, ADJ);
                Real dot = 0;
                bool ok[RPT];
#pragma unroll
                for (int j = 0; j < RPT; ++j) ok[j] = active[j] && ((ra[j] & R.crm) == R.crv);
                // uniform: without row controls and with every thread on a row, no predicate
                row_gate<ADJ, GB, RPT, FOLD, T2, Real>(v, w, R, ok, !(all_rows && R.crm == 0), dot);
                if (ADJ && R.slot >= 0) {
                    Real d = dot;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                    if (lane == 0) acc[R.slot * nwarps + warp].add(d);
                }
            }
            const bool sp = Gr.has_s;  // uniform: exchanges folded into the scatter
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t ps = rs[j] ^ (sp ? (uint32_t)Gr.sperm[e]
                                                    : (((e & 1) ? qs_[0] : 0u) ^ ((e & 2) ? qs_[1] : 0u) ^
                                                       ((e & 4) ? qs_[2] : 0u) ^ ((e & 8) ? qs_[3] : 0u)));
                    if (active[j] && e < (1 << r)) {
                        tp[ps] = v[j][e];
                        if (ADJ) tl[ps] = w[j][e];
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Global <-> shared copies of one tile (swizzled in shared memory). Loads are asynchronous
// copies (cp.async, one per amplitude: 8 bytes for complex64, 16 for complex128) that need no
// registers, so every thread has all its copies of the tile in flight at once; the caller's
// block barrier follows the final wait.
__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Address tables of a pass's tile copies. Element o = VEC * (tid + j * blockDim) + i of a tile:
// both its global offset (a bit deposit) and its shared-memory position (the swizzle) are
// XOR-linear over disjoint bit fields, so they split into a per-thread part (registers), a
// per-step part (a small shared table, the same for all threads) and the element bit i.
constexpr int kTileMaxSteps = (1 << kTileMaxBits) / kTileThreads;  // 64

struct TileAddr {
    uint64_t g_t;   // this thread's part of the global offset
    uint32_t s_t;   // this thread's part of the shared-memory position
    uint32_t s_1;   // position offset of element bit i = 1 (complex64 pairs)
    uint32_t steps; // blockDim-strided steps that cover the tile (0 for threads past a small tile)
};

// Fills the per-step tables g_j / s_j (shared, kTileMaxSteps entries) and returns the thread's
// part. Ends with a block barrier.
template <typename Real>
__device__ __forceinline__ TileAddr tile_addr(const TilePass &P, uint64_t *g_j, uint32_t *s_j) {
    constexpr int VEC = TileT<Real>::VEC, SW = TileT<Real>::SW;
    const uint32_t nvec = (1u << P.k) / VEC;
    TileAddr a;
    const uint32_t o_t = threadIdx.x * VEC;
    a.g_t = scatter_local(P, o_t);
    a.s_t = tile_swizzle(o_t, SW);
    a.s_1 = tile_swizzle(1u, SW);
    a.steps = threadIdx.x < nvec ? (nvec + blockDim.x - 1) / blockDim.x : 0u;
    const uint32_t nsteps = (nvec + blockDim.x - 1) / blockDim.x;
    for (uint32_t j = threadIdx.x; j < nsteps; j += blockDim.x) {
        const uint32_t o_j = j * blockDim.x * VEC;  // disjoint from o_t: blockDim * VEC is a power of two
        g_j[j] = scatter_local(P, o_j);
        s_j[j] = tile_swizzle(o_j, SW);
    }
    __syncthreads();
    return a;
}

template <typename Real>
__device__ __forceinline__ void load_tile(const TileAddr &ta, const uint64_t *g_j, const uint32_t *s_j, uint64_t base,
                                          const typename TileT<Real>::T2 *src, typename TileT<Real>::T2 *dst) {
    const uint64_t g0 = base | ta.g_t;
    for (uint32_t j = 0; j < ta.steps; ++j) {
        if (!QS_DBG_OK(g0 | g_j[j], TileT<Real>::VEC)) continue;
        const typename TileT<Real>::T2 *g = src + (g0 | g_j[j]);
        const uint32_t s = ta.s_t ^ s_j[j];
        if (sizeof(Real) == 4) {
            cp_async_8(dst + s, g);
            cp_async_8(dst + (s ^ ta.s_1), g + 1);
        } else {
            cp_async_16(dst + s, g);
        }
    }
    cp_async_wait_all();
}

template <typename Real>
__device__ __forceinline__ void store_tile(const TileAddr &ta, const uint64_t *g_j, const uint32_t *s_j, uint64_t base,
                                           const typename TileT<Real>::T2 *src, typename TileT<Real>::T2 *dst) {
    using V = typename TileT<Real>::V;
    using T2 = typename TileT<Real>::T2;
    constexpr int VEC = TileT<Real>::VEC;
    const uint64_t g0 = base | ta.g_t;
    for (uint32_t j = 0; j < ta.steps; ++j) {
        if (!QS_DBG_OK(g0 | g_j[j], VEC)) continue;
        QS_DBG_WRITE(g0 | g_j[j], VEC);
        const uint32_t s = ta.s_t ^ s_j[j];
        V x;
        T2 *xs = reinterpret_cast<T2 *>(&x);
        xs[0] = src[s];
        if (VEC == 2) xs[VEC - 1] = src[s ^ ta.s_1];
        *reinterpret_cast<V *>(dst + (g0 | g_j[j])) = x;
    }
}

}  // namespace tiledev
}  // namespace qs
