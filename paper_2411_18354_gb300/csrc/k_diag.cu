// k_diag.cu -- one pass over the state for a run of diagonal gates (see k_diag.cuh).
#include <algorithm>
#include <cstring>

#include "k_diag.cuh"
#include "qs_debug.cuh"
#include "k_gate.cuh"

namespace qs {

bool make_diag_gate(const GatePlan &p, DiagGate *g) {
    if (p.op != OP_DIAG && p.op != OP_SIDE) return false;
    std::memset(g, 0, sizeof(*g));
    const double *U = p.Ufull;  // diag(a, d): a = U[0..1], d = U[6..7]
    g->a[0] = U[0];
    g->a[1] = U[1];
    g->d[0] = U[6];
    g->d[1] = U[7];
    g->aone = U[0] == 1.0 && U[1] == 0.0;
    g->done = U[6] == 1.0 && U[7] == 0.0;
    g->t = p.t;
    const uint64_t lo = (1ull << kDiagChunkBits) - 1ull;
    g->hm = p.ctrl_mask & ~lo;
    g->hv = p.ctrl_vals & ~lo;
    const uint64_t clo = p.ctrl_mask & lo;
    const bool tlo = p.t < kDiagChunkBits;
    g->thi = tlo ? 0ull : (1ull << p.t);
    g->tlo = tlo ? (1 << p.t) : 0;
    const int nlo = __builtin_popcountll(clo) + (tlo ? 1 : 0);
    if (nlo == 0) {
        g->cls = DIAG_HI;
    } else if (nlo == 1) {
        g->cls = DIAG_LO1;
        if (tlo) {
            g->u = p.t;
            g->ut = 1;
        } else {
            g->u = __builtin_ctzll(clo);
            g->ut = 0;
            g->cv = (int32_t)((p.ctrl_vals >> g->u) & 1ull);
        }
    } else {
        g->cls = DIAG_LOM;
        g->lm = (int32_t)clo;
        g->lv = (int32_t)(p.ctrl_vals & lo);
    }
    return true;
}

// Index bits >= 3 a gate needs for its factor to differ from 1: its controls, and its target
// when one side of the matrix is exactly 1.
static void necessary_bits(const DiagGate &g, uint64_t *mask, uint64_t *vals) {
    *mask = g.hm;
    *vals = g.hv;
    if (g.thi && g.aone != g.done) {
        *mask |= g.thi;
        if (g.aone) *vals |= g.thi;  // only the bit-1 side changes
    }
}

DiagCounts assign_diag_classes(DiagGate *g, int count, int n, int lead_t) {
    DiagCounts nc;
    std::memset(&nc, 0, sizeof(nc));
    nc.wt = -1;
    nc.lead_t = lead_t;
    // fixed bits: necessary for every gate, with the same value
    uint64_t fm = ~0ull, fv = 0;
    for (int i = 0; i < count; ++i) {
        uint64_t m, v;
        necessary_bits(g[i], &m, &v);
        if (i == 0) {
            fm = m;
            fv = v;
        } else {
            fm &= m & ~(fv ^ v);
            fv &= fm;
        }
    }
    if (count == 0 || lead_t >= 0) fm = 0;  // a leading gate changes every chunk
    int nfix = 0;
    for (int b = kDiagChunkBits; b < n && nfix < kDiagMaxFixed; ++b)
        if ((fm >> b) & 1ull) {
            nc.fix_pos[nfix] = b - kDiagChunkBits;
            nc.fix_val |= (uint32_t)((fv >> b) & 1ull) << nfix;
            ++nfix;
        }
    nc.nfix = nfix;
    uint64_t fixed = 0;
    for (int i = 0; i < nfix; ++i) fixed |= 1ull << (nc.fix_pos[i] + kDiagChunkBits);
    // lane bits: the five lowest free chunk-level bits (the pair bit of a leading gate on a bit
    // >= 3 is not free: each thread holds both of its values)
    if (lead_t >= kDiagChunkBits) fixed |= 1ull << lead_t;
    uint64_t lanes = 0;
    int nl = 0;
    for (int b = kDiagChunkBits; b < n && nl < 5; ++b)
        if (!((fixed >> b) & 1ull)) {
            lanes |= 1ull << b;
            ++nl;
        }
    const bool warp_ok = nl == 5;  // the compact counter has >= 32 values
    const uint64_t varying = lanes | ((1ull << kDiagChunkBits) - 1ull);
    int wt = -1;
    bool one_target = true;
    for (int i = 0; i < count; ++i) {
        DiagGate &G = g[i];
        if (!warp_ok || G.cls == DIAG_LOM) continue;
        const uint64_t ctrl = (G.hm | (G.cls == DIAG_LO1 && !G.ut ? (1ull << G.u) : 0ull)) & ~fixed;
        const uint64_t tb = (1ull << G.t) & ~fixed;
        if ((ctrl & varying) != 0) continue;
        if ((tb & varying) == 0) {
            G.cls = DIAG_WARP;  // controls and target constant over the warp (fixed or above the lanes)
        } else if (G.cls == DIAG_HI || (G.cls == DIAG_LO1 && G.ut)) {
            if (wt < 0) wt = G.t;
            else if (wt != G.t) one_target = false;
        }
    }
    if (wt >= 0 && one_target) {
        for (int i = 0; i < count; ++i) {
            DiagGate &G = g[i];
            if (G.cls == DIAG_WARP || G.cls == DIAG_LOM || G.t != wt) continue;
            const uint64_t ctrl = (G.hm | (G.cls == DIAG_LO1 && !G.ut ? (1ull << G.u) : 0ull)) & ~fixed;
            if ((ctrl & varying) == 0 && (G.cls == DIAG_HI || (G.cls == DIAG_LO1 && G.ut))) G.cls = DIAG_WT;
        }
        nc.wt = wt;
    }
    std::stable_sort(g, g + count, [](const DiagGate &a, const DiagGate &b) { return a.cls < b.cls; });
    for (int i = 0; i < count; ++i) ++nc.ncls[g[i].cls];
    return nc;
}

namespace {

template <typename Real> struct SDiag {
    uint64_t hm, hv, thi;
    int32_t cls, u, ut, cv, lm, lv, tlo, aone, done, t;
    Real a[2], d[2];
};

// A chunk of 8 amplitudes: four 16-byte vectors (complex64) or eight (complex128).
__device__ __forceinline__ void ld8(const float2 *p, float2 *v) {
    Vec<float, 4>::ld(p, v);
    Vec<float, 4>::ld(p + 4, v + 4);
}
__device__ __forceinline__ void st8(float2 *p, const float2 *v) {
    Vec<float, 4>::st(p, v);
    Vec<float, 4>::st(p + 4, v + 4);
}
__device__ __forceinline__ void ld8(const double2 *p, double2 *v) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = p[i];
}
__device__ __forceinline__ void st8(double2 *p, const double2 *v) {
#pragma unroll
    for (int i = 0; i < 8; ++i) p[i] = v[i];
}

template <typename T2, typename Real>
__device__ __forceinline__ T2 cm(const Real *f, T2 x) {
    return cmul<T2, Real>(f[0], f[1], x);
}

// s0[u], s1[u]: chunk scalars for elements whose bit u is 0 / 1 (u = 0, 1, 2), unrolled so
// they stay in registers.
template <typename T2, typename Real>
__device__ __forceinline__ void mul_bit(T2 (&s0)[3], T2 (&s1)[3], int u, int val, const Real *f) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (b == u) {
            if (val) s1[b] = cm<T2, Real>(f, s1[b]);
            else s0[b] = cm<T2, Real>(f, s0[b]);
        }
    }
}

// Per-element factors f[0..7] of the chunk at `base` (the product of every gate's factor);
// returns whether some factor differs from 1. Called by all 32 lanes of a warp together (the
// warp classes exchange partial products).
template <typename Real>
__device__ __forceinline__ bool chunk_factors(uint64_t base, const SDiag<Real> *sg, int count, const DiagCounts &nc,
                                              int lane, typename CxT<Real>::T (&f)[1 << kDiagChunkBits]) {
    using T2 = typename CxT<Real>::T;
    constexpr int E = 1 << kDiagChunkBits;
    const int w_end = nc.ncls[DIAG_WARP], wt_end = w_end + nc.ncls[DIAG_WT], h_end = wt_end + nc.ncls[DIAG_HI],
              l1_end = h_end + nc.ncls[DIAG_LO1];
    const int wt = nc.wt;
    const bool any_lo1 = nc.ncls[DIAG_LO1] > 0 || (nc.ncls[DIAG_WT] > 0 && wt < kDiagChunkBits);
    const bool any_lom = nc.ncls[DIAG_LOM] > 0;
    T2 s = T2{1, 0};
    bool touched = false;
    if (w_end > 0) {
        // factors constant over the warp: each lane takes every 32nd gate, then the warp
        // multiplies the partial products
        for (int g = lane; g < w_end; g += 32) {
            const SDiag<Real> &G = sg[g];
            if ((base & G.hm) != G.hv) continue;
            const bool tb = (base & G.thi) != 0;
            if (tb ? !G.done : !G.aone) {
                s = cm<T2, Real>(tb ? G.d : G.a, s);
                touched = true;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T2 q;
            q.x = __shfl_xor_sync(0xffffffffu, s.x, o);
            q.y = __shfl_xor_sync(0xffffffffu, s.y, o);
            s = cmul<T2, Real>(q.x, q.y, s);
        }
        touched = __any_sync(0xffffffffu, touched);
    }
    T2 s0[3] = {T2{1, 0}, T2{1, 0}, T2{1, 0}}, s1[3] = {T2{1, 0}, T2{1, 0}, T2{1, 0}};
    if (wt_end > w_end) {
        // controls constant over the warp, one target in the lane or element bits: the warp
        // forms the products for target bit 0 (p0) and 1 (p1) the same way
        T2 p0 = T2{1, 0}, p1 = T2{1, 0};
        bool n0 = false, n1 = false;
        for (int g = w_end + lane; g < wt_end; g += 32) {
            const SDiag<Real> &G = sg[g];
            if ((base & G.hm) != G.hv) continue;
            if (!G.aone) {
                p0 = cm<T2, Real>(G.a, p0);
                n0 = true;
            }
            if (!G.done) {
                p1 = cm<T2, Real>(G.d, p1);
                n1 = true;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T2 q0, q1;
            q0.x = __shfl_xor_sync(0xffffffffu, p0.x, o);
            q0.y = __shfl_xor_sync(0xffffffffu, p0.y, o);
            q1.x = __shfl_xor_sync(0xffffffffu, p1.x, o);
            q1.y = __shfl_xor_sync(0xffffffffu, p1.y, o);
            p0 = cmul<T2, Real>(q0.x, q0.y, p0);
            p1 = cmul<T2, Real>(q1.x, q1.y, p1);
        }
        n0 = __any_sync(0xffffffffu, n0);
        n1 = __any_sync(0xffffffffu, n1);
        if (wt >= kDiagChunkBits) {  // the target bit is constant in this chunk
            const bool tb = (base >> wt) & 1ull;
            s = cmul<T2, Real>(tb ? p1.x : p0.x, tb ? p1.y : p0.y, s);
            touched |= tb ? n1 : n0;
        } else {                     // the target bit varies inside the chunk
#pragma unroll
            for (int b = 0; b < kDiagChunkBits; ++b) {
                if (b == wt) {
                    s0[b] = p0;
                    s1[b] = p1;
                }
            }
            touched |= n0 || n1;
        }
    }
    for (int g = wt_end; g < h_end; ++g) {
        const SDiag<Real> &G = sg[g];
        if ((base & G.hm) != G.hv) continue;
        const bool tb = (base & G.thi) != 0;
        if (tb ? !G.done : !G.aone) {
            s = cm<T2, Real>(tb ? G.d : G.a, s);
            touched = true;
        }
    }
    for (int g = h_end; g < l1_end; ++g) {
        const SDiag<Real> &G = sg[g];
        if ((base & G.hm) != G.hv) continue;
        const bool tb = (base & G.thi) != 0;
        if (G.ut) {  // bit u is the target: a where it is 0, d where it is 1
            if (!G.aone) mul_bit<T2, Real>(s0, s1, G.u, 0, G.a);
            if (!G.done) mul_bit<T2, Real>(s0, s1, G.u, 1, G.d);
            touched |= !(G.aone && G.done);
        } else if (tb ? !G.done : !G.aone) {  // bit u is a control with value cv
            mul_bit<T2, Real>(s0, s1, G.u, G.cv, tb ? G.d : G.a);
            touched = true;
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) f[e] = s;
    if (any_lo1) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            f[e] = cmul<T2, Real>((e & 1) ? s1[0].x : s0[0].x, (e & 1) ? s1[0].y : s0[0].y, f[e]);
            f[e] = cmul<T2, Real>((e & 2) ? s1[1].x : s0[1].x, (e & 2) ? s1[1].y : s0[1].y, f[e]);
            f[e] = cmul<T2, Real>((e & 4) ? s1[2].x : s0[2].x, (e & 4) ? s1[2].y : s0[2].y, f[e]);
        }
    }
    if (any_lom) {
        for (int g = l1_end; g < count; ++g) {
            const SDiag<Real> &G = sg[g];
            if ((base & G.hm) != G.hv) continue;
            const bool tb = (base & G.thi) != 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if ((e & G.lm) != G.lv) continue;
                const bool bt = G.tlo ? (e & G.tlo) != 0 : tb;
                if (bt ? !G.done : !G.aone) {
                    f[e] = cm<T2, Real>(bt ? G.d : G.a, f[e]);
                    touched = true;
                }
            }
        }
    }
    return touched;
}

// The leading gate on bit T of the chunk (compile-time element indices keep x in registers).
template <int T, typename T2, typename Real>
__device__ __forceinline__ void lead_in_chunk(T2 (&x)[1 << kDiagChunkBits], const Real *L) {
#pragma unroll
    for (int e = 0; e < (1 << kDiagChunkBits); ++e)
        if (!((e >> T) & 1)) pair_update<OP_GEN, T2, Real>(x[e], x[e | (1 << T)], L);
}

// LEAD: 0 = diagonal run only; 1 = first an uncontrolled 2x2 gate on a target inside the chunk
// (bits 0-2); 2 = first an uncontrolled 2x2 gate on target t0 >= 3, each thread holding the
// two chunks that differ in bit t0.
template <typename Real, int LEAD>
__global__ void __launch_bounds__(256) k_diag_run(typename CxT<Real>::T *__restrict__ psi, const DiagGate *__restrict__ gates,
                                                  int count, DiagCounts nc, uint64_t nunits) {
    using T2 = typename CxT<Real>::T;
    constexpr int E = 1 << kDiagChunkBits;
    __shared__ SDiag<Real> sg[kDiagMaxGates];
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const DiagGate &G = gates[i];
        SDiag<Real> &S = sg[i];
        S.hm = G.hm;
        S.hv = G.hv;
        S.thi = G.thi;
        S.cls = G.cls;
        S.u = G.u;
        S.ut = G.ut;
        S.cv = G.cv;
        S.lm = G.lm;
        S.lv = G.lv;
        S.tlo = G.tlo;
        S.aone = G.aone;
        S.done = G.done;
        S.t = G.t;
        S.a[0] = (Real)G.a[0];
        S.a[1] = (Real)G.a[1];
        S.d[0] = (Real)G.d[0];
        S.d[1] = (Real)G.d[1];
    }
    __syncthreads();
    Real L[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) L[i] = (Real)nc.lu[i];
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;  // a multiple of 32: warps stay aligned
    for (uint64_t cc = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; cc < nunits; cc += stride) {
        if (LEAD == 2) {
            const int p = nc.lead_t - kDiagChunkBits;  // the pair bit, chunk level
            const uint64_t c0 = ((cc >> p) << (p + 1)) | (cc & ((1ull << p) - 1ull));
            const uint64_t b0 = c0 << kDiagChunkBits, b1 = b0 | (1ull << nc.lead_t);
            T2 x[E], y[E], f[E];
            if (!QS_DBG_OK(b0, E) || !QS_DBG_OK(b1, E)) continue;
            ld8(psi + b0, x);
            ld8(psi + b1, y);
#pragma unroll
            for (int e = 0; e < E; ++e) pair_update<OP_GEN, T2, Real>(x[e], y[e], L);
            if (chunk_factors<Real>(b0, sg, count, nc, lane, f)) {
#pragma unroll
                for (int e = 0; e < E; ++e) x[e] = cmul<T2, Real>(f[e].x, f[e].y, x[e]);
            }
            if (chunk_factors<Real>(b1, sg, count, nc, lane, f)) {
#pragma unroll
                for (int e = 0; e < E; ++e) y[e] = cmul<T2, Real>(f[e].x, f[e].y, y[e]);
            }
            st8(psi + b0, x);
            st8(psi + b1, y);
            QS_DBG_WRITE(b0, E);
            QS_DBG_WRITE(b1, E);
        } else {
            uint64_t c = cc;  // insert the fixed bits, lowest position first
            for (int i = 0; i < nc.nfix; ++i) {
                const int p = nc.fix_pos[i];
                c = ((c >> p) << (p + 1)) | (c & ((1ull << p) - 1ull)) | ((uint64_t)((nc.fix_val >> i) & 1u) << p);
            }
            const uint64_t base = c << kDiagChunkBits;
            // the chunk's loads are issued before its factors are formed, so that their latency
            // overlaps that work (the compact counter leaves few chunks whose factors are all 1)
            T2 x[E], f[E];
            if (!QS_DBG_OK(base, E)) continue;
            ld8(psi + base, x);
            const bool touched = chunk_factors<Real>(base, sg, count, nc, lane, f);
            if (LEAD == 0 && !touched) continue;  // every factor of this chunk is 1: no store
            if (LEAD == 1) {
                if (nc.lead_t == 0) lead_in_chunk<0, T2, Real>(x, L);
                else if (nc.lead_t == 1) lead_in_chunk<1, T2, Real>(x, L);
                else lead_in_chunk<2, T2, Real>(x, L);
            }
            if (touched) {
#pragma unroll
                for (int e = 0; e < E; ++e) x[e] = cmul<T2, Real>(f[e].x, f[e].y, x[e]);
            }
            st8(psi + base, x);
            QS_DBG_WRITE(base, E);
        }
    }
}

}  // namespace

cudaError_t launch_diag_run(int dtype, void *psi, int n, const DiagGate *gates, int count, DiagCounts nc,
                            cudaStream_t st) {
    if (count <= 0 && nc.lead_t < 0) return cudaSuccess;
    int total = 0;
    for (int c = 0; c < kDiagClasses; ++c) total += nc.ncls[c];
    const int lead = nc.lead_t < 0 ? 0 : (nc.lead_t < kDiagChunkBits ? 1 : 2);
    const int free_bits = n - kDiagChunkBits - nc.nfix - (lead == 2 ? 1 : 0);  // bits of the unit counter
    if (count < 0 || count > kDiagMaxGates || n < kDiagChunkBits || total != count || nc.nfix < 0 ||
        nc.nfix > kDiagMaxFixed || (lead != 0 && nc.nfix != 0) || nc.lead_t >= n || free_bits < 0 ||
        ((nc.ncls[DIAG_WARP] > 0 || nc.ncls[DIAG_WT] > 0) && free_bits < 5) ||
        (nc.ncls[DIAG_WT] > 0 && (nc.wt < 0 || nc.wt >= n)))
        return cudaErrorInvalidValue;
    const uint64_t nunits = 1ull << free_bits;
    const uint64_t cap = (uint64_t)device_sm_count() * 8;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((nunits + 255) / 256, cap));
#define QS_DIAG_GO(R, T2)                                                                                       \
    switch (lead) {                                                                                            \
        case 0: k_diag_run<R, 0><<<grid, 256, 0, st>>>(reinterpret_cast<T2 *>(psi), gates, count, nc, nunits); break; \
        case 1: k_diag_run<R, 1><<<grid, 256, 0, st>>>(reinterpret_cast<T2 *>(psi), gates, count, nc, nunits); break; \
        default: k_diag_run<R, 2><<<grid, 256, 0, st>>>(reinterpret_cast<T2 *>(psi), gates, count, nc, nunits); break; \
    }
    if (dtype == QS_C64) {
        QS_DIAG_GO(float, float2)
    } else {
        QS_DIAG_GO(double, double2)
    }
#undef QS_DIAG_GO
    return cudaGetLastError();
}

}  // namespace qs
