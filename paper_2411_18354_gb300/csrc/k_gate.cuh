// k_gate.cuh -- controlled single-qubit gate kernels on the reduced iteration set.
//
// Section III-B of arXiv 2411.18354 schedules only the 2^(n-1-c) iterations whose control
// bits hold: a reduced iteration index i_r is mapped to a global iteration index by Eq. 4
// (controls in ascending order, adjusted by Eq. 3), and ithCleared inserts a 0 at the
// target to give the first element of the pair; the second element is 2^t above it.
// Here the same map is one bit deposit: the counter's bits are spread over the free
// (non-target, non-control) positions and the control values are OR-ed in. A counter is
// scheduled per work unit, not per pair: a unit covers R consecutive free-bit values,
// which are R consecutive amplitudes (or R consecutive adjacent pairs when t = 0), so that
// each thread moves 16- or 32-byte vectors and a warp touches contiguous memory whenever
// the lowest inserted position allows it.
//
// Update per pair (Section III, Eq. 2): x' = a x + b y, y' = c x + d y with x = C_k,
// y = C_{k+2^t}; specialised variants exchange (X/CNOT/Toffoli), scale both sides
// (diagonal) or scale one side only (diagonal with a 1 on the other side).
#pragma once

#include "qs_debug.cuh"
#include "qs_internal.cuh"

namespace qs {

template <typename Real> struct CxT;
template <> struct CxT<float> { using T = float2; };
template <> struct CxT<double> { using T = double2; };

// R consecutive complex values, moved with the widest aligned vector type.
template <typename Real, int R> struct Vec;
template <> struct Vec<float, 1> {
    __device__ __forceinline__ static void ld(const float2 *p, float2 *v) { v[0] = *p; }
    __device__ __forceinline__ static void st(float2 *p, const float2 *v) { *p = v[0]; }
};
template <> struct Vec<float, 2> {
    __device__ __forceinline__ static void ld(const float2 *p, float2 *v) {
        float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = make_float2(q.x, q.y);
        v[1] = make_float2(q.z, q.w);
    }
    __device__ __forceinline__ static void st(float2 *p, const float2 *v) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    }
};
template <> struct Vec<float, 4> {
    __device__ __forceinline__ static void ld(const float2 *p, float2 *v) {
        Vec<float, 2>::ld(p, v);
        Vec<float, 2>::ld(p + 2, v + 2);
    }
    __device__ __forceinline__ static void st(float2 *p, const float2 *v) {
        Vec<float, 2>::st(p, v);
        Vec<float, 2>::st(p + 2, v + 2);
    }
};
template <> struct Vec<double, 1> {
    __device__ __forceinline__ static void ld(const double2 *p, double2 *v) { v[0] = *p; }
    __device__ __forceinline__ static void st(double2 *p, const double2 *v) { *p = v[0]; }
};
template <> struct Vec<double, 2> {
    __device__ __forceinline__ static void ld(const double2 *p, double2 *v) { v[0] = p[0]; v[1] = p[1]; }
    __device__ __forceinline__ static void st(double2 *p, const double2 *v) { p[0] = v[0]; p[1] = v[1]; }
};

// Device copy of a gate: index map in the index width, matrix in the state's precision.
template <typename Real, typename Idx> struct DevGate {
    Idx mask[kMaxSeg];
    Idx ins;
    Idx tbit;
    Idx cmask;  // masked comparator only: control mask / values tested per unit
    Idx cvals;
    int32_t shift[kMaxSeg];
    Real m[8];  // a, b, c, d as (re, im)
};

template <typename Idx, int NS, typename G>
__device__ __forceinline__ Idx deposit(Idx j, const G &g) {
    Idx r = g.ins;
#pragma unroll
    for (int s = 0; s < NS; ++s) r |= (j << g.shift[s]) & g.mask[s];
    return r;
}

// a x + b y for complex a = (ar, ai), b = (br, bi).
template <typename T2, typename Real>
__device__ __forceinline__ T2 cmac(Real ar, Real ai, const T2 &x, Real br, Real bi, const T2 &y) {
    T2 o;
    o.x = fma(ar, x.x, fma(-ai, x.y, fma(br, y.x, -bi * y.y)));
    o.y = fma(ar, x.y, fma(ai, x.x, fma(br, y.y, bi * y.x)));
    return o;
}
template <typename T2, typename Real>
__device__ __forceinline__ T2 cmul(Real ar, Real ai, const T2 &x) {
    T2 o;
    o.x = fma(ar, x.x, -ai * x.y);
    o.y = fma(ar, x.y, ai * x.x);
    return o;
}

template <int OP, typename T2, typename Real>
__device__ __forceinline__ void pair_update(T2 &x, T2 &y, const Real *m) {
    if (OP == OP_GEN) {
        T2 nx = cmac<T2, Real>(m[0], m[1], x, m[2], m[3], y);
        T2 ny = cmac<T2, Real>(m[4], m[5], x, m[6], m[7], y);
        x = nx;
        y = ny;
    } else if (OP == OP_REAL) {
        T2 nx, ny;
        nx.x = fma(m[0], x.x, m[2] * y.x);
        nx.y = fma(m[0], x.y, m[2] * y.y);
        ny.x = fma(m[4], x.x, m[6] * y.x);
        ny.y = fma(m[4], x.y, m[6] * y.y);
        x = nx;
        y = ny;
    } else if (OP == OP_SWAP) {
        T2 tmp = x;
        x = y;
        y = tmp;
    } else if (OP == OP_DIAG) {
        x = cmul<T2, Real>(m[0], m[1], x);
        y = cmul<T2, Real>(m[6], m[7], y);
    }
}

// Running sum in the state's precision, 8 bytes either way: float64 for complex128; for
// complex64 a float sum with its compensation term (Kahan), because float64 arithmetic runs
// at a small fraction of the float32 rate on this GPU. All-zero bits = 0.
template <typename Real> struct Acc;
template <> struct Acc<double> {
    double s;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s, c;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

constexpr int kGateThreads = 256;

template <int R> struct Log2;
template <> struct Log2<1> { static constexpr int v = 0; };
template <> struct Log2<2> { static constexpr int v = 1; };
template <> struct Log2<4> { static constexpr int v = 2; };

// One work unit per thread per inner step, UNR units in flight per thread.
//  LAY_SPLIT: unit u covers counters (u << r) .. (u << r) + R - 1, i.e. the R amplitudes
//             lo .. lo+R-1 and their partners lo+2^t ..; requires r <= lowest inserted bit.
//  LAY_ADJ:   t == 0; unit u covers R adjacent pairs = 2R amplitudes from lo.
//  OP_SIDE:   only the amplitudes at lo + side*2^t are read, scaled and written.
//  MASKED:    baseline comparator: the map inserts only the target; units whose first
//             amplitude fails the control test return without touching memory.
template <typename Real, typename Idx, int NS, int LAY, int R, int OP, bool MASKED, int UNR>
__global__ void __launch_bounds__(kGateThreads)
k_gate(typename CxT<Real>::T *__restrict__ psi, const DevGate<Real, Idx> g, Idx units, int side) {
    using T2 = typename CxT<Real>::T;
    constexpr int r = Log2<R>::v;
    constexpr int A = (LAY == LAY_ADJ) ? 2 * R : R;  // amplitudes per load group
    // When launched as a programmatic dependent of the previous kernel on the stream, this block
    // may start while that kernel drains: the state is touched only after it has completed and
    // its writes are visible (grid dependency barrier; immediate for a normal launch). The next
    // gate may be scheduled right away.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const Idx step = (Idx)gridDim.x * kGateThreads * UNR;
    for (Idx u0 = (Idx)blockIdx.x * kGateThreads * UNR + threadIdx.x; u0 < units; u0 += step) {
        T2 x[UNR][A];
        T2 y[UNR][(LAY == LAY_SPLIT && OP != OP_SIDE) ? R : 1];
        Idx lo[UNR];
        bool on[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const Idx u = u0 + (Idx)k * kGateThreads;
            on[k] = u < units;
            lo[k] = deposit<Idx, NS>(u << r, g);
            if (MASKED) on[k] = on[k] && ((lo[k] & g.cmask) == g.cvals);
#ifdef QS_DEBUG_CHECKS
            if (on[k]) {
                if (LAY == LAY_ADJ) on[k] = QS_DBG_OK(lo[k], A);
                else if (OP == OP_SIDE) on[k] = QS_DBG_OK(lo[k] | (side ? g.tbit : (Idx)0), R);
                else on[k] = QS_DBG_OK(lo[k], R) && QS_DBG_OK(lo[k] | g.tbit, R);
            }
#endif
            if (on[k]) {
                if (LAY == LAY_ADJ) {
                    Vec<Real, A>::ld(psi + lo[k], x[k]);
                } else if (OP == OP_SIDE) {
                    Vec<Real, R>::ld(psi + (lo[k] | (side ? g.tbit : (Idx)0)), x[k]);
                } else {
                    Vec<Real, R>::ld(psi + lo[k], x[k]);
                    Vec<Real, R>::ld(psi + (lo[k] | g.tbit), y[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            if (!on[k]) continue;
            if (LAY == LAY_ADJ) {
#pragma unroll
                for (int i = 0; i < R; ++i) pair_update<OP, T2, Real>(x[k][2 * i], x[k][2 * i + 1], g.m);
                Vec<Real, A>::st(psi + lo[k], x[k]);
                QS_DBG_WRITE(lo[k], A);
            } else if (OP == OP_SIDE) {
#pragma unroll
                for (int i = 0; i < R; ++i) x[k][i] = cmul<T2, Real>(g.m[0], g.m[1], x[k][i]);
                Vec<Real, R>::st(psi + (lo[k] | (side ? g.tbit : (Idx)0)), x[k]);
                QS_DBG_WRITE(lo[k] | (side ? g.tbit : (Idx)0), R);
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) pair_update<OP, T2, Real>(x[k][i], y[k][i], g.m);
                Vec<Real, R>::st(psi + lo[k], x[k]);
                Vec<Real, R>::st(psi + (lo[k] | g.tbit), y[k]);
                QS_DBG_WRITE(lo[k], R);
                QS_DBG_WRITE(lo[k] | g.tbit, R);
            }
        }
    }
}

}  // namespace qs
