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

template <typename Real>
__device__ __forceinline__ void load_gate(const SGate<Real> &G, GateRegs<Real> &r, const Real *cs, bool adjoint) {
    const uint4 w = *reinterpret_cast<const uint4 *>(&G.crm);
    r.crm = w.x;
    r.crv = w.y;
    const uint32_t meta = w.z;
    r.code = (int)(meta & 0xffu);
    r.cqm = (int)((meta >> 8) & 0xfu);
    r.cqv = (int)((meta >> 12) & 0xfu);
    r.side = (int)((meta >> 16) & 1u);
    const int pkind = (int)((meta >> 17) & 7u);
    r.slot = (int)(meta >> 20) - 1;
    if (pkind != 0 && cs) {
        param_matrices<Real>(pkind, cs[2 * w.w], cs[2 * w.w + 1], adjoint, r.u, r.d);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) r.u[i] = G.u[i];
        if (adjoint && r.slot >= 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) r.d[i] = G.d[i];
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

// All pairs (e, e | 2^P) of one row for one gate with operation OP; CQ: the gate has
// controls on group qubits (else every pair of a selected row is updated). Rows of tiles with
// fewer than GB qubits are padded with zero elements that pair only with each other, so they
// stay zero and add nothing to the inner products.
template <int P, int OP, bool ADJ, int GB, bool CQ, typename T2, typename Real>
__device__ __forceinline__ void row_pairs(T2 *v, T2 *w, const GateRegs<Real> &R, bool row_ok, Real &dot) {
    constexpr int DOP = OP == OP_DIAG ? OP_DIAG : (OP == OP_REAL ? OP_REAL : OP_GEN);
    if (!row_ok) return;
#pragma unroll
    for (int e = 0; e < (1 << GB); ++e) {
        if ((e >> P) & 1) continue;
        const int e2 = e | (1 << P);
        if (!CQ || ((e & R.cqm) == R.cqv)) {
            op_pair<OP, T2, Real>(v[e], v[e2], R.u, R.side);
            if (ADJ) {
                if (R.slot >= 0) {
                    T2 mx = v[e], my = v[e2];
                    pair_update<DOP, T2, Real>(mx, my, R.d);
                    dot += w[e].x * mx.x + w[e].y * mx.y + w[e2].x * my.x + w[e2].y * my.y;
                }
                op_pair<OP, T2, Real>(w[e], w[e2], R.u, R.side);
            }
        }
    }
}

// One switch on the staged dispatch code selects (operation, target place, in-row controls).
template <bool ADJ, int GB, typename T2, typename Real>
__device__ __forceinline__ void row_gate(T2 *v, T2 *w, const GateRegs<Real> &R, bool row_ok, Real &dot) {
#define QS_ROW(OP, P)                                                                                    \
    case ((OP)*4 + (P)) * 2 + 0:                                                                         \
        if ((P) < GB) row_pairs<((P) < GB ? (P) : 0), OP, ADJ, GB, false, T2, Real>(v, w, R, row_ok, dot); \
        break;                                                                                           \
    case ((OP)*4 + (P)) * 2 + 1:                                                                         \
        if ((P) < GB) row_pairs<((P) < GB ? (P) : 0), OP, ADJ, GB, true, T2, Real>(v, w, R, row_ok, dot);  \
        break;
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
}

// Register qubits per group: 4 for forward passes, 3 for the adjoint sweep (psi and lambda
// rows both live in registers there).
template <bool ADJ> struct GroupBits { static constexpr int v = ADJ ? 3 : 4; };

// Apply the pass's register groups to the tile tp (and lambda tile tl if ADJ) whose global
// base index is `base`. Adjoint: for a gate with slot >= 0 the warp partial of
// Re <lambda| dU psi> (summed over the warp in the state's precision) is added to
// acc[slot * nwarps + warp]. Every executed group ends with a block barrier.
template <typename Real, bool ADJ, int GB = GroupBits<ADJ>::v>
__device__ __forceinline__ void apply_groups(typename TileT<Real>::T2 *tp, typename TileT<Real>::T2 *tl, uint64_t base,
                                             int k, const TileGroup *groups, int group_count, const SGate<Real> *gates,
                                             const Real *cs, Acc<Real> *acc) {
    using T2 = typename TileT<Real>::T2;
    constexpr int SW = TileT<Real>::SW;
    constexpr int E = 1 << GB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int gi = 0; gi < group_count; ++gi) {
        const TileGroup &Gr = groups[gi];
        if (Gr.hctrl) {
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
        for (uint32_t rb = 0; rb < rows; rb += blockDim.x) {
            const uint32_t rho = rb + tid;
            const bool active = rho < rows;
            uint32_t ra = 0;
            for (int s = 0; s < Gr.nrseg; ++s) ra |= (rho << Gr.rshift[s]) & Gr.rmask[s];
            const uint32_t rs = tile_swizzle(ra, SW);
            T2 v[E], w[ADJ ? E : 1];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint32_t ps = rs ^ ((e & 1) ? qs_[0] : 0u) ^ ((e & 2) ? qs_[1] : 0u) ^ ((e & 4) ? qs_[2] : 0u) ^
                                    ((e & 8) ? qs_[3] : 0u);
                if (active && e < (1 << r)) {
                    v[e] = tp[ps];
                    if (ADJ) w[e] = tl[ps];
                } else {
                    v[e] = T2{0, 0};
                    if (ADJ) w[e] = T2{0, 0};
                }
            }
            for (int g = 0; g < Gr.gate_count; ++g) {
                const SGate<Real> &G = gates[Gr.gate_begin + g];
                if (Gr.hctrl && (base & G.hmask) != G.hvals) continue;  // uniform
                GateRegs<Real> R;
                load_gate<Real>(G, R, cs, ADJ);
                const bool row_ok = active && ((ra & R.crm) == R.crv);
                Real dot = 0;
                row_gate<ADJ, GB, T2, Real>(v, w, R, row_ok, dot);
                if (ADJ && R.slot >= 0) {
                    Real d = dot;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                    if (lane == 0) acc[R.slot * nwarps + warp].add(d);
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint32_t ps = rs ^ ((e & 1) ? qs_[0] : 0u) ^ ((e & 2) ? qs_[1] : 0u) ^ ((e & 4) ? qs_[2] : 0u) ^
                                    ((e & 8) ? qs_[3] : 0u);
                if (active && e < (1 << r)) {
                    tp[ps] = v[e];
                    if (ADJ) tl[ps] = w[e];
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
