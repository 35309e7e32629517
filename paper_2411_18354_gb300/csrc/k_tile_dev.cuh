// k_tile_dev.cuh -- device code shared by the fused tile pass and the batched kernel:
// applying a list of TileGates to one shared-memory tile (and, for the adjoint sweep, to the
// matching lambda tile with the gradient inner products).
#pragma once

#include "k_gate.cuh"
#include "k_tile.cuh"

namespace qs {
namespace tiledev {

template <typename Real> struct TileT;
template <> struct TileT<float> {
    using T2 = float2;
    using V = float4;  // 2 amplitudes per 16-byte vector
    static constexpr int VEC = 2;
    __device__ static const float *U(const TileGate &G) { return G.Uf; }
    __device__ static const float *D(const TileGate &G) { return G.Df; }
};
template <> struct TileT<double> {
    using T2 = double2;
    using V = double2;  // 1 amplitude per 16-byte vector
    static constexpr int VEC = 1;
    __device__ static const double *U(const TileGate &G) { return G.U; }
    __device__ static const double *D(const TileGate &G) { return G.D; }
};

// Gate fields a thread keeps in registers while it works through the gate's pairs.
template <typename Real> struct GateRegs {
    uint32_t mask[4];
    uint32_t shift[4];
    uint32_t ins, tbit, pairs;
    int nseg, op, side, slot;
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
__device__ __forceinline__ void load_gate(const TileGate &G, GateRegs<Real> &r, const Real *cs, bool adjoint) {
    r.nseg = G.nseg;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        r.mask[s] = s < r.nseg ? G.mask[s] : 0u;
        r.shift[s] = s < r.nseg ? G.shift[s] : 0u;
    }
    r.ins = G.ins;
    r.tbit = G.tbit;
    r.pairs = 1u << G.log_pairs;
    r.op = G.op;
    r.side = G.side;
    r.slot = G.slot;
    if (G.pkind != 0 && cs) {
        param_matrices<Real>(G.pkind, cs[2 * G.pidx], cs[2 * G.pidx + 1], adjoint, r.u, r.d);
    } else {
        const Real *u = TileT<Real>::U(G);
        const Real *d = TileT<Real>::D(G);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            r.u[i] = u[i];
            r.d[i] = d[i];
        }
    }
}

// Local pair index: up to 4 counter segments from registers, the rest from the table.
template <typename Real>
__device__ __forceinline__ uint32_t local_pair(const GateRegs<Real> &r, const TileGate &G, uint32_t j) {
    uint32_t lo = r.ins;
#pragma unroll
    for (int s = 0; s < 4; ++s) lo |= (j << r.shift[s]) & r.mask[s];
    for (int s = 4; s < r.nseg; ++s) lo |= (j << G.shift[s]) & G.mask[s];
    return lo;
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

template <typename T2, typename Real>
__device__ __forceinline__ void apply_pair(int op, int side, const Real *u, T2 &x, T2 &y) {
    if (op == OP_GEN) {
        T2 nx = cmac<T2, Real>(u[0], u[1], x, u[2], u[3], y);
        T2 ny = cmac<T2, Real>(u[4], u[5], x, u[6], u[7], y);
        x = nx;
        y = ny;
    } else if (op == OP_REAL) {
        pair_update<OP_REAL, T2, Real>(x, y, u);
    } else if (op == OP_SWAP) {
        T2 t = x;
        x = y;
        y = t;
    } else if (op == OP_DIAG) {
        x = cmul<T2, Real>(u[0], u[1], x);
        y = cmul<T2, Real>(u[6], u[7], y);
    } else {  // OP_SIDE: scalar in u[0..1]
        if (side) y = cmul<T2, Real>(u[0], u[1], y);
        else x = cmul<T2, Real>(u[0], u[1], x);
    }
}

// Apply gates G0[0..count) to the tile tp (and, if ADJ, the lambda tile tl) whose global base
// index is `base`. Adjoint: for a gate with slot >= 0, the warp partial of Re <lambda|dU psi>
// is added to acc[slot * nwarps + warp] (float64). Ends with a block barrier.
template <typename Real, bool ADJ>
__device__ __forceinline__ void apply_gates(typename TileT<Real>::T2 *tp, typename TileT<Real>::T2 *tl, uint64_t base,
                                            const TileGate *G0, int count, const Real *cs, double *acc) {
    using T2 = typename TileT<Real>::T2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int g = 0; g < count; ++g) {
        const TileGate &G = G0[g];
        if ((base & G.hmask) != G.hvals) continue;  // uniform over the block
        GateRegs<Real> R;
        load_gate<Real>(G, R, cs, ADJ);
        const int dop = R.op == OP_DIAG ? OP_DIAG : R.op == OP_REAL ? OP_REAL : OP_GEN;
        Real dot = 0;
        for (uint32_t j = tid; j < R.pairs; j += blockDim.x) {
            const uint32_t lo = local_pair<Real>(R, G, j), hi = lo | R.tbit;
            T2 x = tp[lo], y = tp[hi];
            apply_pair<T2, Real>(R.op, R.side, R.u, x, y);
            tp[lo] = x;
            tp[hi] = y;
            if (ADJ) {
                T2 a = tl[lo], b = tl[hi];
                if (R.slot >= 0) {
                    T2 mx = x, my = y;
                    apply_pair<T2, Real>(dop, 0, R.d, mx, my);
                    dot += a.x * mx.x + a.y * mx.y + b.x * my.x + b.y * my.y;
                }
                apply_pair<T2, Real>(R.op, R.side, R.u, a, b);
                tl[lo] = a;
                tl[hi] = b;
            }
        }
        if (ADJ && R.slot >= 0) {
            double d = (double)dot;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if (lane == 0) acc[R.slot * nwarps + warp] += d;
        }
        __syncthreads();
    }
}

}  // namespace tiledev
}  // namespace qs
