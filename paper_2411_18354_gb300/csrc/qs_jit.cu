// qs_jit.cu -- tile passes generated for their exact shape and compiled at run time (NVRTC).
//
// What a generated kernel computes is what k_tile_pass computes for the same TilePass, groups
// and gates (the same tile map, swizzle, register groups, folded exchanges, predicates and
// pair updates, Section III Eq. 2 per selected pair); only the per-gate interpretation is
// gone. See qs_jit.cuh.
#include <nvrtc.h>
#include <sys/stat.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "k_tile.cuh"
#include "qs_jit.cuh"

namespace qs {

int device_sm_count();
void *debug_state_address();

#ifdef QS_DEBUG_CHECKS
constexpr bool kDebugBuild = true;
#else
constexpr bool kDebugBuild = false;
#endif

namespace {

struct Out {
    std::string s;
    void f(const char *fmt, ...) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        const int m = std::vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        if (m < (int)sizeof(buf)) {
            s += buf;
        } else {
            std::vector<char> big((size_t)m + 1);
            va_start(ap, fmt);
            std::vsnprintf(big.data(), big.size(), fmt, ap);
            va_end(ap);
            s += big.data();
        }
    }
};

// Local tile offset o -> global amplitude offset (the pass's runs of consecutive local bits).
uint64_t scatter_host(const TilePass &P, uint32_t o) {
    uint64_t g = 0;
    for (int r = 0; r < P.nruns; ++r)
        g |= (uint64_t)((o >> P.run_src[r]) & ((1u << P.run_len[r]) - 1u)) << P.run_dst[r];
    return g;
}

// Types, copies and pair updates shared by every generated kernel (one precision).
void preamble(Out &o, bool dbl) {
    o.f("typedef unsigned int u32;\ntypedef unsigned long long u64;\n");
    if (dbl) {
        o.f("typedef double R;\nstruct alignas(16) T2 { double x, y; };\n");
        o.f("__device__ __forceinline__ R F(R a, R b, R c) { return __fma_rn(a, b, c); }\n");
    } else {
        o.f("typedef float R;\nstruct alignas(8) T2 { float x, y; };\nstruct alignas(16) T4 { float x, y, z, w; };\n");
        o.f("__device__ __forceinline__ R F(R a, R b, R c) { return __fmaf_rn(a, b, c); }\n");
    }
    // the same operation order as the interpreted pass (k_gate.cuh cmac / cmul / pair_update)
    if (dbl) {
        o.f("__device__ __forceinline__ void u_gen(T2 &x, T2 &y, const R *m) {\n"
            "  T2 a, b;\n"
            "  a.x = F(m[0], x.x, F(-m[1], x.y, F(m[2], y.x, -m[3] * y.y)));\n"
            "  a.y = F(m[0], x.y, F(m[1], x.x, F(m[2], y.y, m[3] * y.x)));\n"
            "  b.x = F(m[4], x.x, F(-m[5], x.y, F(m[6], y.x, -m[7] * y.y)));\n"
            "  b.y = F(m[4], x.y, F(m[5], x.x, F(m[6], y.y, m[7] * y.x)));\n"
            "  x = a; y = b;\n}\n");
        o.f("__device__ __forceinline__ void u_real(T2 &x, T2 &y, const R *m) {\n"
            "  T2 a, b;\n"
            "  a.x = F(m[0], x.x, m[2] * y.x); a.y = F(m[0], x.y, m[2] * y.y);\n"
            "  b.x = F(m[4], x.x, m[6] * y.x); b.y = F(m[4], x.y, m[6] * y.y);\n"
            "  x = a; y = b;\n}\n");
    } else {
        // float32: the real-matrix update takes the real and imaginary parts of a pair through
        // one packed two-lane instruction (fma.rn.f32x2 / mul.rn.f32x2, each lane rounded like
        // the scalar operation): the same results, half the instructions. (The general update
        // stays scalar: packed, it saves a quarter of its instructions but makes the register
        // allocation of long passes take minutes to compile.)
        o.f("__device__ __forceinline__ u64 pk(float a, float b) { u64 r; asm(\"mov.b64 %%0, {%%1, %%2};\" : \"=l\"(r) : "
            "\"f\"(a), \"f\"(b)); return r; }\n");
        o.f("__device__ __forceinline__ T2 upk(u64 r) { T2 a; asm(\"mov.b64 {%%0, %%1}, %%2;\" : \"=f\"(a.x), \"=f\"(a.y) : "
            "\"l\"(r)); return a; }\n");
        o.f("__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) { u64 d; asm(\"fma.rn.f32x2 %%0, %%1, %%2, %%3;\" : "
            "\"=l\"(d) : \"l\"(a), \"l\"(b), \"l\"(c)); return d; }\n");
        o.f("__device__ __forceinline__ u64 mul2(u64 a, u64 b) { u64 d; asm(\"mul.rn.f32x2 %%0, %%1, %%2;\" : \"=l\"(d) : "
            "\"l\"(a), \"l\"(b)); return d; }\n");
        o.f("__device__ __forceinline__ void u_gen(T2 &x, T2 &y, const R *m) {\n"
            "  T2 a, b;\n"
            "  a.x = F(m[0], x.x, F(-m[1], x.y, F(m[2], y.x, -m[3] * y.y)));\n"
            "  a.y = F(m[0], x.y, F(m[1], x.x, F(m[2], y.y, m[3] * y.x)));\n"
            "  b.x = F(m[4], x.x, F(-m[5], x.y, F(m[6], y.x, -m[7] * y.y)));\n"
            "  b.y = F(m[4], x.y, F(m[5], x.x, F(m[6], y.y, m[7] * y.x)));\n"
            "  x = a; y = b;\n}\n");
        o.f("__device__ __forceinline__ void u_real(T2 &x, T2 &y, const R *m) {\n"
            "  const u64 X = pk(x.x, x.y), Y = pk(y.x, y.y);\n"
            "  const u64 a = fma2(pk(m[0], m[0]), X, mul2(pk(m[2], m[2]), Y));\n"
            "  const u64 b = fma2(pk(m[4], m[4]), X, mul2(pk(m[6], m[6]), Y));\n"
            "  x = upk(a); y = upk(b);\n}\n");
    }
    o.f("__device__ __forceinline__ void u_mul(T2 &x, R ar, R ai) {\n"
        "  T2 a; a.x = F(ar, x.x, -ai * x.y); a.y = F(ar, x.y, ai * x.x); x = a;\n}\n");
    o.f("__device__ __forceinline__ void u_diag(T2 &x, T2 &y, const R *m) { u_mul(x, m[0], m[1]); u_mul(y, m[6], m[7]); }\n");
    o.f("__device__ __forceinline__ void u_swap(T2 &x, T2 &y) { T2 t = x; x = y; y = t; }\n");
    // a parameterised gate from (c, s) = (cos, sin) of theta / 2: kind 2 = RY = [[c, -s], [s, c]],
    // kind 3 = RZ = diag(c - i s, c + i s); adj: the dagger; d: dU/dtheta of the gate itself
    o.f("__device__ __forceinline__ void pmat(int kind, R c, R s, int adj, R *u, R *d) {\n"
        "  for (int i = 0; i < 8; ++i) { u[i] = 0; d[i] = 0; }\n"
        "  const R h = (R)0.5;\n"
        "  u[0] = c; u[6] = c;\n"
        "  if (kind == 2) { u[2] = adj ? s : -s; u[4] = adj ? -s : s; d[0] = -h * s; d[2] = -h * c; d[4] = h * c; "
        "d[6] = -h * s; }\n"
        "  else { u[1] = adj ? s : -s; u[7] = adj ? -s : s; d[0] = -h * s; d[1] = -h * c; d[6] = -h * s; d[7] = h * c; }\n"
        "}\n");
    // w = a b for row-major complex 2x2 matrices (interleaved re, im)
    o.f("__device__ __forceinline__ void mat2(const R *a, const R *b, R *w) {\n"
        "  for (int i = 0; i < 2; ++i) for (int j = 0; j < 2; ++j) {\n"
        "    const R *x = a + 4 * i, *y0 = b + 2 * j, *y1 = b + 4 + 2 * j;\n"
        "    w[4 * i + 2 * j] = x[0] * y0[0] - x[1] * y0[1] + x[2] * y1[0] - x[3] * y1[1];\n"
        "    w[4 * i + 2 * j + 1] = x[0] * y0[1] + x[1] * y0[0] + x[2] * y1[1] + x[3] * y1[0];\n"
        "  }\n}\n");
    o.f("__device__ __forceinline__ void cp8(void *s, const void *g) {\n"
        "  asm volatile(\"cp.async.ca.shared.global [%%0], [%%1], 8;\\n\" :: \"r\"((u32)__cvta_generic_to_shared(s)), "
        "\"l\"(g) : \"memory\");\n}\n");
    o.f("__device__ __forceinline__ void cp16(void *s, const void *g) {\n"
        "  asm volatile(\"cp.async.cg.shared.global [%%0], [%%1], 16;\\n\" :: \"r\"((u32)__cvta_generic_to_shared(s)), "
        "\"l\"(g) : \"memory\");\n}\n");
    o.f("__device__ __forceinline__ void cpcommit() { asm volatile(\"cp.async.commit_group;\\n\" ::: \"memory\"); }\n");
    o.f("__device__ __forceinline__ void cpwait0() { asm volatile(\"cp.async.wait_group 0;\\n\" ::: \"memory\"); }\n");
    o.f("__device__ __forceinline__ void cpwait1() { asm volatile(\"cp.async.wait_group 1;\\n\" ::: \"memory\"); }\n");
}

// Expression of the tile swizzle of `a` (the same bijection as tile_swizzle, k_tile.cuh).
std::string swz_expr(const char *a, int sw) {
    std::string x = std::string("(") + a + " >> " + std::to_string(sw) + ")";
    std::string f = x;
    for (int i = sw; i < kTileMaxBits; i += sw) f += " ^ (" + x + " >> " + std::to_string(i) + ")";
    return std::string("(") + a + " ^ ((" + f + ") & " + std::to_string((1u << sw) - 1u) + "u))";
}

// Tile predicate of a set of gates: "" if some gate has no non-local control (every tile
// is selected), else the condition that one of them selects the tile at `bv` (a variable).
std::string any_selects(const RegGate *g, int count, const char *bv = "base") {
    std::vector<std::pair<uint64_t, uint64_t>> seen;
    std::string c;
    for (int i = 0; i < count; ++i) {
        if (g[i].hmask == 0) return "";
        bool dup = false;
        for (auto &s : seen) dup |= s.first == g[i].hmask && s.second == g[i].hvals;
        if (dup) continue;
        seen.push_back({g[i].hmask, g[i].hvals});
        char b[96];
        std::snprintf(b, sizeof(b), "%s((%s & 0x%llxull) == 0x%llxull)", c.empty() ? "" : " || ", bv,
                      (unsigned long long)g[i].hmask, (unsigned long long)g[i].hvals);
        c += b;
    }
    return c;
}

// Expressions of the gates' matrices (m), derivatives (d) and gradient accumulator indices.
struct Refs {
    std::vector<std::string> m, d;
    std::vector<int> acc;
};

// The pair updates of one gate on row registers v (and, adjoint, w with the derivative dot
// when the gate has a parameter). A rotation U = exp(-i theta P / 2) about the Pauli P = Y or Z
// (pauli 'Y' / 'Z') has dU/dtheta = (-i/2) P U, so with psi' = U^dagger psi (the amplitudes
// after the un-apply) Re <lambda| dU psi'> = Re <lambda| (-i/2) P psi> = Im <lambda| P psi> / 2:
// it is taken from the pair before the un-apply, 4 products per pair, no derivative matrix
// (the caller halves the sum). pauli == 0: the derivative matrix is applied to a copy of the
// un-applied pair and dotted with lambda.
void emit_gate_pairs(Out &o, const RegGate &G, int gi, int E, bool adjoint, bool param, char pauli, const char *v,
                     const char *w, const Refs &refs) {
    const char *M = refs.m[gi].c_str();
    const int p = G.p;
    int dop = G.op == OP_DIAG ? OP_DIAG : (G.op == OP_REAL ? OP_REAL : OP_GEN);
    for (int e = 0; e < E; ++e) {
        if ((e >> p) & 1) continue;
        if ((e & G.cqm) != G.cqv) continue;
        const int e2 = e | (1 << p);
        auto op = [&](const char *a) {
            switch (G.op) {
            case OP_GEN: o.f("u_gen(%s[%d], %s[%d], %s);\n", a, e, a, e2, M); break;
            case OP_REAL: o.f("u_real(%s[%d], %s[%d], %s);\n", a, e, a, e2, M); break;
            case OP_DIAG: o.f("u_diag(%s[%d], %s[%d], %s);\n", a, e, a, e2, M); break;
            case OP_SWAP: o.f("u_swap(%s[%d], %s[%d]);\n", a, e, a, e2); break;
            case OP_SIDE: o.f("u_mul(%s[%d], %s[0], %s[1]);\n", a, G.side ? e2 : e, M, M); break;
            default: break;
            }
        };
        if (adjoint && param && pauli == 'Y')  // Im <l|Y p> = (l1 . p0) - (l0 . p1), real dot products
            o.f("dot += (%s[%d].x * %s[%d].x + %s[%d].y * %s[%d].y) - (%s[%d].x * %s[%d].x + %s[%d].y * %s[%d].y);\n", w, e2, v,
                e, w, e2, v, e, w, e, v, e2, w, e, v, e2);
        else if (adjoint && param && pauli == 'Z')  // Im <l|Z p> = Im(conj(l0) p0) - Im(conj(l1) p1)
            o.f("dot += (%s[%d].x * %s[%d].y - %s[%d].y * %s[%d].x) - (%s[%d].x * %s[%d].y - %s[%d].y * %s[%d].x);\n", w, e, v,
                e, w, e, v, e, w, e2, v, e2, w, e2, v, e2);
        op(v);
        if (adjoint) {
            if (param && !pauli) {
                o.f("{ T2 mx = %s[%d], my = %s[%d]; ", v, e, v, e2);
                o.f("%s(mx, my, %s); ", dop == OP_DIAG ? "u_diag" : (dop == OP_REAL ? "u_real" : "u_gen"),
                    refs.d[gi].c_str());
                o.f("dot += %s[%d].x * mx.x + %s[%d].y * mx.y + %s[%d].x * my.x + %s[%d].y * my.y; }\n", w, e, w, e, w,
                    e2, w, e2);
            }
            op(w);
        }
    }
}

// A run of consecutive diagonal gates (diag(a, d) or one side only) in a register group: they
// commute, so their product is applied at once. The gates are sorted into classes by the
// element bits their factor depends on (target place, in-row controls); per row, each class
// multiplies its gates' factors (a for target bit 0, d for bit 1) where the gate's tile and row
// predicates hold, and each element is then multiplied by the factors of the classes that
// select it: one complex product per gate and row plus one per selected element and class,
// instead of one per selected element and gate.
void emit_diag_run(Out &o, const RegGate *gs, int gi0, int count, int E, bool adjoint, const Refs &refs) {
    struct Cls {
        int p, cqm, cqv;
        bool has_a = false, has_d = false;
    };
    std::vector<Cls> cls;
    std::vector<int> cls_of(count);
    for (int i = 0; i < count; ++i) {
        const RegGate &R = gs[i];
        int c = -1;
        for (size_t j = 0; j < cls.size(); ++j)
            if (cls[j].p == R.p && cls[j].cqm == R.cqm && cls[j].cqv == R.cqv) c = (int)j;
        if (c < 0) {
            cls.push_back(Cls{R.p, R.cqm, R.cqv});
            c = (int)cls.size() - 1;
        }
        cls_of[i] = c;
        const bool a = R.op == OP_DIAG || (R.op == OP_SIDE && R.side == 0);
        const bool d = R.op == OP_DIAG || (R.op == OP_SIDE && R.side == 1);
        cls[c].has_a |= a;
        cls[c].has_d |= d;
    }
    o.f("      { // %d diagonal gates in %zu classes\n", count, cls.size());
    for (size_t c = 0; c < cls.size(); ++c) {
        if (cls[c].has_a) o.f("        T2 fa%zu; fa%zu.x = 1; fa%zu.y = 0;\n", c, c, c);
        if (cls[c].has_d) o.f("        T2 fd%zu; fd%zu.x = 1; fd%zu.y = 0;\n", c, c, c);
    }
    for (int i = 0; i < count; ++i) {
        const RegGate &R = gs[i];
        const int gi = gi0 + i, c = cls_of[i];
        std::string cond;
        char t[128];
        if (R.hmask) {
            std::snprintf(t, sizeof(t), "((base & 0x%llxull) == 0x%llxull)", (unsigned long long)R.hmask,
                          (unsigned long long)R.hvals);
            cond = t;
        }
        if (R.crm) {
            std::snprintf(t, sizeof(t), "%s((ra & 0x%xu) == 0x%xu)", cond.empty() ? "" : " && ", R.crm, R.crv);
            cond += t;
        }
        o.f("        if (%s) {", cond.empty() ? "true" : cond.c_str());
        const char *M = refs.m[gi].c_str();
        if (R.op == OP_DIAG)
            o.f(" u_mul(fa%d, %s[0], %s[1]); u_mul(fd%d, %s[6], %s[7]);", c, M, M, c, M, M);
        else
            o.f(" u_mul(f%c%d, %s[0], %s[1]);", R.side ? 'd' : 'a', c, M, M);
        o.f(" }\n");
    }
    for (int e = 0; e < E; ++e) {
        for (size_t c = 0; c < cls.size(); ++c) {
            if ((e & cls[c].cqm) != cls[c].cqv) continue;
            const bool hi = (e >> cls[c].p) & 1;
            if (hi ? !cls[c].has_d : !cls[c].has_a) continue;
            const char f = hi ? 'd' : 'a';
            o.f("        u_mul(v[%d], f%c%zu.x, f%c%zu.y);\n", e, f, c, f, c);
            if (adjoint) o.f("        u_mul(w[%d], f%c%zu.x, f%c%zu.y);\n", e, f, c, f, c);
        }
    }
    o.f("      }\n");
}

// The Pauli of a parameterised gate of the sweep: its rotation kind (batch), or the structure
// the planner forces on rotations (RY: real, RZ: diagonal); 0 when neither.
char pauli_of(const RegGate &R, bool batched) {
    if (batched) return R.pkind == QS_GATE_RY ? 'Y' : R.pkind == QS_GATE_RZ ? 'Z' : 0;
    return R.op == OP_REAL ? 'Y' : R.op == OP_DIAG ? 'Z' : 0;
}

}  // namespace

// Two tile buffers per block (the next tile's copies in flight while the current one is
// computed) where both still leave room for two blocks per SM.
bool jit_double_buffer(int dtype, bool adjoint, int k) {
    const size_t tile = (size_t(1) << k) * (dtype == QS_C64 ? 8 : 16) * (adjoint ? 2 : 1);
    return 2 * tile <= 100 * 1024;
}

std::string jit_pass_source(int dtype, bool adjoint, const TilePass &P, const TileGroup *groups,
                            const RegGate *gates, const char *kname, bool batched) {
    const bool dbl = dtype == QS_C128;
    const int SW = dbl ? 3 : 4;
    const int VEC = dbl ? 1 : 2;
    const int T = kTileThreads;
    const int k = P.k;
    const uint32_t nvec = (1u << k) / VEC;
    const uint32_t steps = (nvec + T - 1) / T;
    const int G = P.gate_count;
    const RegGate *pg = gates + P.gate_begin;
    // Matrix (and derivative) of each gate as an expression: parameters of the kernel (single
    // state), or, in a batch, shared-memory rows formed per tile from the tile's state's angles
    // for the parameterised gates (pm_, pd_; J = index among them).
    std::vector<int> pj(G, -1);
    int NPG = 0;
    if (batched)
        for (int i = 0; i < G; ++i)
            if (pg[i].pkind != 0) pj[i] = NPG++;
    const int NP = adjoint ? (batched ? NPG : P.nparam) : 0;  // gradient accumulators
    Refs refs;
    refs.m.resize(G);
    refs.d.resize(G);
    for (int i = 0; i < G; ++i) {
        char b[48];
        if (pj[i] >= 0) std::snprintf(b, sizeof(b), "(pm_ + %d)", 8 * pj[i]);
        else std::snprintf(b, sizeof(b), "a.m[%d]", i);
        refs.m[i] = b;
        if (pj[i] >= 0) std::snprintf(b, sizeof(b), "(pd_ + %d)", 8 * pj[i]);
        else std::snprintf(b, sizeof(b), "a.d[%d]", pg[i].slot);
        refs.d[i] = b;
        refs.acc.push_back(batched ? pj[i] : pg[i].slot);
    }
    // debug build: every global access checked against the state's size (2^n), writes counted
    const bool dbg = kDebugBuild && !batched;
    Out o;
    preamble(o, dbl);
    if (dbg) {
        o.f("struct DebugState { unsigned status, pad; u64 n_amps; unsigned *counts; u64 count_n; u64 first_bad; };\n");
        o.f("__device__ __forceinline__ bool dok(DebugState *d, u64 i, int span) {\n"
            "  if (d->n_amps == 0 || i + span <= d->n_amps) return true;\n"
            "  d->first_bad = i; atomicOr(&d->status, 1u); return false;\n}\n");
        o.f("__device__ __forceinline__ void dcount(DebugState *d, u64 i, int span) {\n"
            "  if (!d->counts) return;\n"
            "  for (int j = 0; j < span; ++j) if (i + j < d->count_n) atomicAdd(d->counts + i + j, 1u);\n}\n");
    }
    // parameter block: the fixed matrices of the pass's gates (U, or U^dagger in the adjoint
    // sweep); single state: the derivatives of its parameterised gates and their global
    // gradient slots; batch: the parameter indices of the parameterised gates
    o.f("struct alignas(16) A {\n  R m[%d][8];\n", G > 0 ? G : 1);
    if (adjoint && !batched) o.f("  R d[%d][8];\n  int gs[%d];\n", NP > 0 ? NP : 1, NP > 0 ? NP : 1);
    if (batched) o.f("  int pix[%d][2];\n", G > 0 ? G : 1);
    o.f("};\n");
    o.f("__device__ __forceinline__ u32 swz(u32 a) { return %s; }\n", swz_expr("a", SW).c_str());
    const int minb = (adjoint && dbl) ? 1 : 2;
    if (batched)
        o.f("extern \"C\" __global__ void __launch_bounds__(%d, %d) %s(T2 *__restrict__ psi, T2 *__restrict__ lam, "
            "double *__restrict__ part, u64 stride, u64 nstates, const R *__restrict__ cs, u32 cs_stride, "
            "const __grid_constant__ A a) {\n",
            T, minb, kname);
    else if (adjoint)
        o.f("extern \"C\" __global__ void __launch_bounds__(%d, %d) %s(T2 *__restrict__ psi, T2 *__restrict__ lam, "
            "double *__restrict__ part, u64 part_stride, const __grid_constant__ A a%s) {\n",
            T, minb, kname, dbg ? ", DebugState *dbg" : "");
    else
        o.f("extern \"C\" __global__ void __launch_bounds__(%d, %d) %s(T2 *__restrict__ psi, const __grid_constant__ A a%s) {\n",
            T, minb, kname, dbg ? ", DebugState *dbg" : "");
    const bool db = jit_double_buffer(dtype, adjoint, k);
    const uint32_t TILE = 1u << k;
    const uint32_t BUF = (adjoint ? 2 : 1) * TILE;  // one buffer: psi tile (and lambda tile)
    o.f("  extern __shared__ __align__(16) unsigned char sm_[];\n");
    o.f("  T2 *const sm0 = reinterpret_cast<T2 *>(sm_);\n");
    o.f("  R *const sr_ = reinterpret_cast<R *>(sm0 + %u);\n", (db ? 2 : 1) * BUF);
    if (batched) {
        o.f("  R *const pm_ = sr_;\n");
        if (adjoint) o.f("  R *const pd_ = pm_ + %d;\n", 8 * (NPG > 0 ? NPG : 1));
    }
    const int pm_words = batched ? (adjoint ? 2 : 1) * 8 * (NPG > 0 ? NPG : 1) : 0;
    if (adjoint) {
        o.f("  R *acc_s = sr_ + %d;\n", pm_words);
        o.f("  R *acc_c = acc_s + %d;\n", (NP > 0 ? NP : 1) * (T / 32));
        o.f("  for (int i = threadIdx.x; i < %d; i += %d) { acc_s[i] = 0; acc_c[i] = 0; }\n", (NP > 0 ? NP : 1) * (T / 32), T);
        o.f("  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;\n");
    }
    o.f("  const u32 tid = threadIdx.x;\n");
    // this thread's part of the copy addresses (XOR-linear in the element index)
    o.f("  const u32 o_t = tid * %d;\n", VEC);
    {
        std::string g = "0ull";
        for (int r = 0; r < P.nruns; ++r) {
            char b[160];
            std::snprintf(b, sizeof(b), " | ((u64)((o_t >> %d) & %uu) << %d)", P.run_src[r], (1u << P.run_len[r]) - 1u,
                          P.run_dst[r]);
            g += b;
        }
        o.f("  const u64 g_t = %s;\n", g.c_str());
    }
    o.f("  const u32 s_t = swz(o_t);\n");
    const bool cp_guard = nvec < (uint32_t)T;
    int logt = 0;
    while ((1ull << logt) < P.ntiles) ++logt;
    if (batched)
        o.f("  const u64 ntiles = nstates << %d;  // %llu tiles per state\n", logt, (unsigned long long)P.ntiles);
    else
        o.f("  const u64 ntiles = %lluull;\n", (unsigned long long)P.ntiles);
    {
        std::string b = "0ull";
        for (int s = 0; s < P.tnseg; ++s) {
            char t[96];
            std::snprintf(t, sizeof(t), " | ((t_ << %d) & 0x%llxull)", P.tshift[s], (unsigned long long)P.tmask[s]);
            b += t;
        }
        if (batched)  // the tile index within its state: the low bits of the batch-wide index
            o.f("  auto tile_base = [](u64 t_) -> u64 { t_ &= %lluull; return %s; };\n",
                (unsigned long long)(P.ntiles - 1), b.c_str());
        else
            o.f("  auto tile_base = [](u64 t_) -> u64 { return %s; };\n", b.c_str());
    }
    if (batched) {
        o.f("  auto gvec = [&](T2 *v_, u64 t_) -> T2 * { return v_ + (t_ >> %d) * stride; };\n", logt);
    } else {
        o.f("  auto gvec = [](T2 *v_, u64) -> T2 * { return v_; };\n");
    }
    std::string sel;
    if (P.hctrl) sel = any_selects(pg, G, "b_");
    if (!sel.empty()) o.f("  auto selected = [](u64 b_) -> bool { return %s; };\n", sel.c_str());
    // tile copies (asynchronous loads into swizzled shared-memory positions; stores from registers)
    const uint32_t s1 = tile_swizzle(1u, SW);
    auto copies = [&](bool load, const char *gname, const char *tname, const char *bname) {
        if (cp_guard) o.f("    if (tid < %uu) {\n", nvec);
        for (uint32_t j = 0; j < steps; ++j) {
            const uint32_t oj = j * T * VEC;
            const unsigned long long gj = (unsigned long long)scatter_host(P, oj);
            const uint32_t sj = tile_swizzle(oj, SW);
            if (dbg) {
                o.f("    if (dok(dbg, %s | g_t | 0x%llxull, %d)) ", bname, gj, VEC);
                if (!load) o.f("{ dcount(dbg, %s | g_t | 0x%llxull, %d); ", bname, gj, VEC);
            }
            if (load && !dbl)
                o.f("    { const T2 *g = %s + (%s | g_t | 0x%llxull); const u32 s = s_t ^ %uu; "
                    "cp8(%s + s, g); cp8(%s + (s ^ %uu), g + 1); }\n",
                    gname, bname, gj, sj, tname, tname, s1);
            else if (load)
                o.f("    cp16(%s + (s_t ^ %uu), %s + (%s | g_t | 0x%llxull));\n", tname, sj, gname, bname, gj);
            else if (!dbl)
                o.f("    { const u32 s = s_t ^ %uu; const T2 x0 = %s[s], x1 = %s[s ^ %uu]; T4 q; q.x = x0.x; "
                    "q.y = x0.y; q.z = x1.x; q.w = x1.y; *reinterpret_cast<T4 *>(%s + (%s | g_t | 0x%llxull)) = q; }\n",
                    sj, tname, tname, s1, gname, bname, gj);
            else
                o.f("    %s[%s | g_t | 0x%llxull] = %s[s_t ^ %uu];\n", gname, bname, gj, tname, sj);
            if (dbg && !load) o.f("    }\n");
        }
        if (cp_guard) o.f("    }\n");
    };
    auto loads = [&](const char *tname, const char *bname, const char *tau_name) {
        o.f("    {\n    T2 *tq = %s;\n    const T2 *gp_ = gvec(psi, %s);\n", tname, tau_name);
        copies(true, "gp_", "tq", bname);
        if (adjoint) {
            o.f("    T2 *tr = tq + %u;\n    const T2 *gl_ = gvec(lam, %s);\n", TILE, tau_name);
            copies(true, "gl_", "tr", bname);
        }
        o.f("    }\n    cpcommit();\n");
    };
    // batch: the matrices of the parameterised gates for the state of tile tau_ (one thread
    // per gate), from that state's (cos, sin) of theta / 2
    auto stage_params = [&](const char *tau_name) {
        if (!batched || NPG == 0) return;
        o.f("    {\n      const R *cq = cs + (%s >> %d) * (u64)cs_stride;\n", tau_name, logt);
        for (int i = 0; i < G; ++i) {
            if (pj[i] < 0) continue;
            const RegGate &R = pg[i];
            o.f("      if (tid == %d) { R u1[8], d1[8]; pmat(%d, cq[2 * a.pix[%d][0]], cq[2 * a.pix[%d][0] + 1], %d, u1, d1);",
                pj[i] % T, R.pkind, i, i, adjoint ? 1 : 0);
            if (!adjoint && R.pkind2 != 0)
                o.f(" R u2[8], d2[8]; pmat(%d, cq[2 * a.pix[%d][1]], cq[2 * a.pix[%d][1] + 1], 0, u2, d2);"
                    " mat2(u2, u1, pm_ + %d);",
                    R.pkind2, i, i, 8 * pj[i]);
            else
                o.f(" for (int q_ = 0; q_ < 8; ++q_) pm_[%d + q_] = u1[q_];", 8 * pj[i]);
            if (adjoint && !pauli_of(R, true)) o.f(" for (int q_ = 0; q_ < 8; ++q_) pd_[%d + q_] = d1[q_];", 8 * pj[i]);
            o.f(" }\n");
        }
        o.f("    }\n");
    };
    const char *skip_next = sel.empty() ? "" : "    while (nxt < ntiles && !selected(tile_base(nxt))) nxt += gridDim.x;\n";
    o.f("  u64 tau = blockIdx.x;\n");
    if (!sel.empty()) o.f("  while (tau < ntiles && !selected(tile_base(tau))) tau += gridDim.x;\n");
    if (db) o.f("  int cur = 0;\n");
    if (db) {
        o.f("  if (tau < ntiles) {\n    const u64 b0 = tile_base(tau);\n");
        loads("sm0", "b0", "tau");
        o.f("  }\n");
    }
    o.f("  while (tau < ntiles) {\n");
    o.f("    const u64 base = tile_base(tau);\n");
    o.f("    u64 nxt = tau + gridDim.x;\n%s", skip_next);
    if (db)
        o.f("    T2 *tp = sm0 + cur * %u;\n", BUF);
    else
        o.f("    T2 *tp = sm0;  // one buffer\n");
    if (adjoint) o.f("    T2 *tl = tp + %u;\n", TILE);
    stage_params("tau");
    if (db) {
        o.f("    if (nxt < ntiles) {\n      const u64 nb = tile_base(nxt);\n      T2 *tn = sm0 + (cur ^ 1) * %u;\n", BUF);
        loads("tn", "nb", "nxt");
        o.f("      cpwait1();\n    } else {\n      cpwait0();\n    }\n");
    } else {
        loads("tp", "base", "tau");
        o.f("    cpwait0();\n");
    }
    o.f("    __syncthreads();\n");

    for (int gi_ = 0; gi_ < P.group_count; ++gi_) {
        const TileGroup &Gr = groups[P.group_begin + gi_];
        const int r = Gr.r;
        const int E = 1 << r;
        const uint32_t rows = 1u << (k - r);
        const uint32_t rblocks = (rows + T - 1) / T;
        const int gb = Gr.gate_begin - P.gate_begin;  // pass-relative
        o.f("    // register group %d: qubits", gi_);
        for (int q = 0; q < r; ++q) o.f(" %d", Gr.q[q]);
        o.f(", %d gates\n", Gr.gate_count);
        std::string gcond;
        if (Gr.hctrl && !Gr.has_g && !Gr.has_s) gcond = any_selects(pg + gb, Gr.gate_count);
        o.f("    if (%s) {\n", gcond.empty() ? "true" : gcond.c_str());
        // element offsets of the gather and the scatter
        std::vector<uint32_t> og(E), os(E);
        for (int e = 0; e < E; ++e) {
            uint32_t off = 0;
            for (int q = 0; q < r; ++q)
                if ((e >> q) & 1) off ^= Gr.qsw[q];
            og[e] = Gr.has_g ? Gr.gperm[e] : off;
            os[e] = Gr.has_s ? Gr.sperm[e] : off;
        }
        for (uint32_t rb = 0; rb < rblocks; ++rb) {
            o.f("    {\n      const u32 rho = %uu + tid;\n", rb * T);
            const bool guard = rows < (rb + 1) * (uint32_t)T;
            std::string ra = "0u";
            for (int s = 0; s < Gr.nrseg; ++s) {
                char t[80];
                std::snprintf(t, sizeof(t), " | ((rho << %d) & 0x%xu)", Gr.rshift[s], Gr.rmask[s]);
                ra += t;
            }
            o.f("      const u32 ra = %s;\n      const u32 rs = swz(ra);\n", ra.c_str());
            o.f("      const bool act = %s;\n", guard ? (std::string("rho < ") + std::to_string(rows) + "u").c_str() : "true");
            o.f("      T2 v[%d];\n", E);
            if (adjoint) o.f("      T2 w[%d];\n", E);
            o.f("      if (act) {\n");
            for (int e = 0; e < E; ++e) {
                o.f("        v[%d] = tp[rs ^ %uu];\n", e, og[e]);
                if (adjoint) o.f("        w[%d] = tl[rs ^ %uu];\n", e, og[e]);
            }
            o.f("      } else {\n");
            for (int e = 0; e < E; ++e) {
                o.f("        v[%d].x = 0; v[%d].y = 0;\n", e, e);
                if (adjoint) o.f("        w[%d].x = 0; w[%d].y = 0;\n", e, e);
            }
            o.f("      }\n");
            auto mergeable = [&](int g) {
                const RegGate &R = pg[gb + g];
                return (R.op == OP_DIAG || R.op == OP_SIDE) && !(adjoint && R.slot >= 0);
            };
            for (int g = 0; g < Gr.gate_count; ++g) {
                if (g + 1 < Gr.gate_count && mergeable(g) && mergeable(g + 1)) {
                    int h = g;
                    while (h < Gr.gate_count && mergeable(h)) ++h;
                    emit_diag_run(o, pg + gb + g, gb + g, h - g, E, adjoint, refs);
                    g = h - 1;
                    continue;
                }
                const RegGate &R = pg[gb + g];
                const int gi = gb + g;  // pass-relative gate index
                const int slot = adjoint && R.slot >= 0 ? refs.acc[gi] : -1;
                o.f("      // gate %d: op %d, place %d, cq %x/%x, rows %x/%x\n", gi, R.op, R.p, R.cqm, R.cqv, R.crm, R.crv);
                const bool tile_guard = R.hmask != 0;
                if (tile_guard)
                    o.f("      if ((base & 0x%llxull) == 0x%llxull) {\n", (unsigned long long)R.hmask,
                        (unsigned long long)R.hvals);
                else
                    o.f("      {\n");
                if (slot >= 0) o.f("        R dot = 0;\n");
                std::string rc = "act";
                if (R.crm) {
                    char t[80];
                    std::snprintf(t, sizeof(t), "act && ((ra & 0x%xu) == 0x%xu)", R.crm, R.crv);
                    rc = t;
                }
                const bool need_rc = guard || R.crm;
                if (need_rc) o.f("        if (%s) {\n", rc.c_str());
                const char pauli = slot >= 0 ? pauli_of(R, batched) : 0;
                emit_gate_pairs(o, R, gi, E, adjoint, slot >= 0, pauli, "v", "w", refs);
                if (need_rc) o.f("        }\n");
                if (slot >= 0 && pauli) o.f("        dot *= (R)0.5;\n");
                if (slot >= 0) {
                    o.f("        for (int of = 16; of > 0; of >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, of);\n");
                    o.f("        if (lane == 0) { R *s_ = acc_s + %d * %d + warp, *c_ = acc_c + %d * %d + warp; "
                        "const R y = dot - *c_; const R t = *s_ + y; *c_ = (t - *s_) - y; *s_ = t; }\n",
                        slot, T / 32, slot, T / 32);
                }
                o.f("      }\n");
            }
            o.f("      if (act) {\n");
            for (int e = 0; e < E; ++e) {
                o.f("        tp[rs ^ %uu] = v[%d];\n", os[e], e);
                if (adjoint) o.f("        tl[rs ^ %uu] = w[%d];\n", os[e], e);
            }
            o.f("      }\n    }\n");
        }
        o.f("    }\n    __syncthreads();\n");
    }
    o.f("    {\n    T2 *gp_ = gvec(psi, tau);\n");
    copies(false, "gp_", "tp", "base");
    if (adjoint) {
        o.f("    T2 *gl_ = gvec(lam, tau);\n");
        copies(false, "gl_", "tl", "base");
    }
    o.f("    }\n    __syncthreads();\n");
    if (adjoint && batched && NP > 0) {
        // this tile's gradient partials (sum over the block's warps), then fresh accumulators;
        // the loop's next block barrier orders them before the next tile adds to them
        o.f("    for (int p = threadIdx.x; p < %d; p += %d) {\n", NP, T);
        o.f("      double s = 0.0;\n");
        o.f("      for (int w_ = 0; w_ < %d; ++w_) { s += (double)acc_s[p * %d + w_] - (double)acc_c[p * %d + w_]; "
            "acc_s[p * %d + w_] = 0; acc_c[p * %d + w_] = 0; }\n",
            T / 32, T / 32, T / 32, T / 32, T / 32);
        o.f("      part[((u64)p * nstates + (tau >> %d)) * %lluull + (tau & %lluull)] = s;\n    }\n", logt,
            (unsigned long long)P.ntiles, (unsigned long long)(P.ntiles - 1));
    }
    o.f("    tau = nxt;\n%s  }\n", db ? "    cur ^= 1;\n" : "");
    if (adjoint && !batched && NP > 0) {
        o.f("  __syncthreads();\n");
        o.f("  for (int p = threadIdx.x; p < %d; p += %d) {\n", NP, T);
        o.f("    double s = 0.0;\n");
        o.f("    for (int w_ = 0; w_ < %d; ++w_) s += (double)acc_s[p * %d + w_] - (double)acc_c[p * %d + w_];\n", T / 32,
            T / 32, T / 32);
        o.f("    part[(u64)a.gs[p] * part_stride + blockIdx.x] = s;\n  }\n");
    }
    o.f("}\n");
    return o.s;
}

namespace {

// ---------------------------------------------------------------------------------------------
// Compile cache
// ---------------------------------------------------------------------------------------------

struct Module {
    std::string source;       // all kernels of the module
    std::vector<char> cubin;
    std::vector<std::string> names;
    cudaLibrary_t lib = nullptr;  // loaded on first launch
    std::vector<cudaKernel_t> kernels;
    std::vector<size_t> smem_set[64];  // per device: dynamic shared memory configured per kernel
    std::vector<int> occ[64];          // per device: resident blocks per SM per kernel (0 = unknown)
};

std::mutex g_mu;
std::vector<std::unique_ptr<Module>> g_modules;
std::unordered_map<std::string, std::pair<int, int>> g_by_source;  // kernel source -> (module, kernel)
std::unordered_map<std::string, std::pair<int, int>> g_by_shape;   // shape key -> (module, kernel)

// Everything a pass's generated source depends on, as bytes (the matrices excluded): looking
// this up costs far less than generating the source, so a repeated circuit finds its kernels
// without writing them again.
std::string shape_key(int dtype, bool adjoint, bool batched, const TilePass &P, const TileGroup *groups,
                      const RegGate *gates) {
    std::string k;
    auto put = [&k](const void *p, size_t n) { k.append(static_cast<const char *>(p), n); };
    const int hdr[5] = {dtype, adjoint ? 1 : 0, batched ? 1 : 0, P.gate_count, P.group_count};
    put(hdr, sizeof(hdr));
    put(&P.n, sizeof(P.n));
    put(&P.k, sizeof(P.k));
    put(&P.nruns, sizeof(P.nruns));
    put(P.run_src, sizeof(P.run_src));
    put(P.run_len, sizeof(P.run_len));
    put(P.run_dst, sizeof(P.run_dst));
    put(P.tmask, sizeof(P.tmask));
    put(P.tshift, sizeof(P.tshift));
    put(&P.tnseg, sizeof(P.tnseg));
    put(&P.ntiles, sizeof(P.ntiles));
    put(&P.hctrl, sizeof(P.hctrl));
    put(&P.nparam, sizeof(P.nparam));
    for (int i = 0; i < P.group_count; ++i) {
        TileGroup g = groups[P.group_begin + i];
        g.gate_begin -= P.gate_begin;
        put(&g, sizeof(g));
    }
    for (int i = 0; i < P.gate_count; ++i) {
        const RegGate &g = gates[P.gate_begin + i];
        put(&g.p, 4);  // p, cqm, cqv, pad0
        put(&g.crm, sizeof(g.crm));
        put(&g.crv, sizeof(g.crv));
        put(&g.op, sizeof(g.op));
        put(&g.side, sizeof(g.side));
        put(&g.slot, sizeof(g.slot));
        put(&g.hmask, sizeof(g.hmask));
        put(&g.hvals, sizeof(g.hvals));
        if (batched) {  // the kinds of the rotations whose matrices the kernel forms
            const int kinds[2] = {g.pkind, g.pkind2};
            put(kinds, sizeof(kinds));
        }
    }
    return k;
}

bool compile_cubin(const std::string &src, std::vector<char> *cubin, std::string *err) {
    nvrtcProgram prog;
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "qs_jit_pass.cu", 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS) {
        *err = std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r);
        return false;
    }
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=true", "-DQS_JIT=1"};
    r = nvrtcCompileProgram(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    if (r != NVRTC_SUCCESS) {
        size_t ls = 0;
        nvrtcGetProgramLogSize(prog, &ls);
        std::string log(ls, '\0');
        if (ls) nvrtcGetProgramLog(prog, &log[0]);
        *err = std::string("NVRTC compile failed: ") + nvrtcGetErrorString(r) + "\n" + log.substr(0, 4000);
        nvrtcDestroyProgram(&prog);
        return false;
    }
    size_t n = 0;
    r = nvrtcGetCUBINSize(prog, &n);
    if (r == NVRTC_SUCCESS) {
        cubin->resize(n);
        r = nvrtcGetCUBIN(prog, cubin->data());
    }
    nvrtcDestroyProgram(&prog);
    if (r != NVRTC_SUCCESS) {
        *err = std::string("nvrtcGetCUBIN: ") + nvrtcGetErrorString(r);
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------------------------
// On-disk kernel cache (QS_JIT_CACHE_DIR)
// ---------------------------------------------------------------------------------------------
// With QS_JIT_CACHE_DIR=<directory> every compiled kernel is also written there, one file per
// kernel source, and a later process loads it instead of compiling. A file holds a header, the
// kernel's full source and its cubin; it is used only when the stored source equals the
// wanted one byte for byte (so neither a name collision nor a stale file can give another
// kernel), and written under a temporary name then renamed (readers never see a partial one).
constexpr char kDiskMagic[8] = {'Q', 'S', 'J', 'I', 'T', 'C', '1', '\n'};

std::string disk_cache_dir() {
    const char *d = std::getenv("QS_JIT_CACHE_DIR");
    return (d && *d) ? std::string(d) : std::string();
}

// File of a kernel source: FNV-1a of the source, the compile options and the NVRTC version.
std::string disk_path(const std::string &dir, const std::string &src) {
    int major = 0, minor = 0;
    nvrtcVersion(&major, &minor);
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](const char *p, size_t n) {
        for (size_t i = 0; i < n; ++i) {
            h ^= (unsigned char)p[i];
            h *= 1099511628211ull;
        }
    };
    char v[64];
    const int m = std::snprintf(v, sizeof(v), "sm_103a;c++17;fmad;nvrtc %d.%d;", major, minor);
    mix(v, (size_t)m);
    mix(src.data(), src.size());
    char name[64];
    std::snprintf(name, sizeof(name), "/qs_jit_%016llx.bin", (unsigned long long)h);
    return dir + name;
}

bool disk_load(const std::string &path, const std::string &src, std::vector<char> *cubin) {
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return false;
    std::vector<char> all;
    char buf[1 << 16];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) all.insert(all.end(), buf, buf + got);
    std::fclose(f);
    const size_t hdr = sizeof(kDiskMagic) + sizeof(uint64_t);
    if (all.size() < hdr || std::memcmp(all.data(), kDiskMagic, sizeof(kDiskMagic)) != 0) return false;
    uint64_t len = 0;
    std::memcpy(&len, all.data() + sizeof(kDiskMagic), sizeof(len));
    if (len != src.size() || all.size() <= hdr + len || std::memcmp(all.data() + hdr, src.data(), len) != 0) return false;
    cubin->assign(all.begin() + (ptrdiff_t)(hdr + len), all.end());
    return true;
}

void disk_store(const std::string &path, const std::string &src, const std::vector<char> &cubin) {
    const std::string tmp = path + ".tmp" + std::to_string((unsigned long long)std::hash<std::thread::id>()(
                                                std::this_thread::get_id()));
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;  // not writable: the cache is an optimisation only
    const uint64_t len = src.size();
    bool ok = std::fwrite(kDiskMagic, 1, sizeof(kDiskMagic), f) == sizeof(kDiskMagic) &&
              std::fwrite(&len, 1, sizeof(len), f) == sizeof(len) && std::fwrite(src.data(), 1, src.size(), f) == src.size() &&
              std::fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) std::remove(tmp.c_str());
}

}  // namespace

bool jit_prepare_programs(int dtype, const std::vector<JitRequest> &reqs, std::string *err, double *compile_seconds,
                          int *compiled_modules) {
    if (compile_seconds) *compile_seconds = 0.0;
    if (compiled_modules) *compiled_modules = 0;
    const size_t es = dtype == QS_C64 ? 8 : 16, rs = dtype == QS_C64 ? 4 : 8;
    // every pass of every request, in order
    struct Item {
        const FusedProgram *prog;
        int pass;
        bool adjoint, batched;
        size_t req;
    };
    std::vector<Item> items;
    for (size_t ri = 0; ri < reqs.size(); ++ri) {
        const JitRequest &r = reqs[ri];
        r.out->assign(r.prog->passes.size(), JitPass{});
        for (size_t p = 0; p < r.prog->passes.size(); ++p) items.push_back({r.prog, (int)p, r.adjoint, r.batched, ri});
    }
    // one source per pass (kernel name fixed: the source text alone keys the cache); a pass
    // whose shape was seen before needs no source
    std::vector<std::string> srcs(items.size()), keys(items.size());
    std::vector<char> known(items.size(), 0);
    std::lock_guard<std::mutex> lock(g_mu);
    for (size_t i = 0; i < items.size(); ++i) {
        const Item &it = items[i];
        const FusedProgram &prog = *it.prog;
        keys[i] = shape_key(dtype, it.adjoint, it.batched, prog.passes[it.pass], prog.groups.data(), prog.gates.data());
        if (g_by_shape.count(keys[i])) {
            known[i] = 1;
            continue;
        }
        srcs[i] = jit_pass_source(dtype, it.adjoint, prog.passes[it.pass], prog.groups.data(), prog.gates.data(),
                                  "qs_pass", it.batched);
    }
    // passes whose source is not cached yet go into new modules (renamed kernels)
    std::vector<int> missing;
    std::unordered_map<std::string, int> first_of;
    for (size_t p = 0; p < srcs.size(); ++p) {
        if (known[p] || g_by_source.count(srcs[p])) continue;
        if (first_of.count(srcs[p])) continue;
        first_of[srcs[p]] = (int)p;
        missing.push_back((int)p);
    }
    const std::string dir = disk_cache_dir();
    if (!missing.empty() && !dir.empty()) {
        ::mkdir(dir.c_str(), 0755);  // if missing (one level; an error leaves the cache unused)
        // one module per kernel: loaded from the directory where present, else compiled
        // (concurrently) and written there
        auto t0 = std::chrono::steady_clock::now();
        std::vector<std::unique_ptr<Module>> mods(missing.size());
        std::vector<size_t> todo;
        for (size_t i = 0; i < missing.size(); ++i) {
            mods[i] = std::make_unique<Module>();
            mods[i]->source = srcs[missing[i]];
            mods[i]->names.push_back("qs_pass");
            if (!disk_load(disk_path(dir, mods[i]->source), mods[i]->source, &mods[i]->cubin)) todo.push_back(i);
        }
        std::vector<std::string> errs(mods.size());
        std::vector<char> ok(mods.size(), 1);
        unsigned hw = std::thread::hardware_concurrency();
        if (hw == 0) hw = 4;
        std::atomic<size_t> next{0};
        {
            std::vector<std::thread> th;
            for (unsigned w = 0; w < std::min<size_t>(hw, todo.size()); ++w)
                th.emplace_back([&] {
                    for (size_t q; (q = next.fetch_add(1)) < todo.size();) {
                        Module &m = *mods[todo[q]];
                        ok[todo[q]] = compile_cubin(m.source, &m.cubin, &errs[todo[q]]) ? 1 : 0;
                        if (ok[todo[q]]) disk_store(disk_path(dir, m.source), m.source, m.cubin);
                    }
                });
            for (auto &t : th) t.join();
        }
        for (size_t i = 0; i < mods.size(); ++i)
            if (!ok[i]) {
                *err = errs[i];
                return false;
            }
        for (size_t i = 0; i < mods.size(); ++i) {
            g_by_source[srcs[missing[i]]] = {(int)g_modules.size(), 0};
            g_modules.push_back(std::move(mods[i]));
        }
        if (compile_seconds)
            *compile_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (compiled_modules) *compiled_modules = (int)todo.size();
        missing.clear();
    }
    if (!missing.empty()) {
        auto t0 = std::chrono::steady_clock::now();
        // split the new kernels into modules compiled concurrently (NVRTC is thread-safe):
        // contiguous chunks of about equal source size, one per hardware thread at most
        size_t total = 0;
        for (int p : missing) total += srcs[p].size();
        unsigned hw = std::thread::hardware_concurrency();
        if (hw == 0) hw = 4;
        const size_t nmod = std::max<size_t>(1, std::min<size_t>({(size_t)hw, missing.size(), 32}));
        std::vector<std::unique_ptr<Module>> mods;
        std::vector<std::vector<int>> members;
        {
            size_t acc = 0, cur = 0;
            mods.push_back(std::make_unique<Module>());
            members.emplace_back();
            for (size_t i = 0; i < missing.size(); ++i) {
                const std::string &src = srcs[missing[i]];
                if (acc >= (cur + 1) * total / nmod && !members.back().empty() && cur + 1 < nmod) {
                    ++cur;
                    mods.push_back(std::make_unique<Module>());
                    members.emplace_back();
                }
                Module &m = *mods.back();
                const size_t idx = m.names.size();
                const std::string nm = "qs_pass_" + std::to_string(idx);
                std::string s2 = src;
                const size_t at = s2.find(" qs_pass(");
                s2.replace(at, 9, " " + nm + "(");
                m.source += "namespace m" + std::to_string(idx) + " {\n" + s2 + "}\n";
                m.names.push_back(nm);
                members.back().push_back(missing[i]);
                acc += src.size();
            }
        }
        // QS_JIT_DUMP=<directory>: write each compiled module's source there (diagnostics)
        if (const char *dir = std::getenv("QS_JIT_DUMP")) {
            if (*dir) {
                for (size_t i = 0; i < mods.size(); ++i) {
                    const std::string path =
                        std::string(dir) + "/qs_jit_module_" + std::to_string(g_modules.size() + i) + ".cu";
                    if (FILE *f = std::fopen(path.c_str(), "w")) {
                        std::fwrite(mods[i]->source.data(), 1, mods[i]->source.size(), f);
                        std::fclose(f);
                    }
                }
            }
        }
        std::vector<std::string> errs(mods.size());
        std::vector<char> ok(mods.size(), 0);
        {
            std::vector<std::thread> th;
            for (size_t i = 0; i < mods.size(); ++i)
                th.emplace_back([&, i] { ok[i] = compile_cubin(mods[i]->source, &mods[i]->cubin, &errs[i]) ? 1 : 0; });
            for (auto &t : th) t.join();
        }
        for (size_t i = 0; i < mods.size(); ++i)
            if (!ok[i]) {
                *err = errs[i];
                return false;
            }
        for (size_t i = 0; i < mods.size(); ++i) {
            const int mi = (int)g_modules.size();
            for (size_t j = 0; j < members[i].size(); ++j) g_by_source[srcs[members[i][j]]] = {mi, (int)j};
            g_modules.push_back(std::move(mods[i]));
        }
        if (compile_seconds)
            *compile_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (compiled_modules) *compiled_modules = (int)mods.size();
    }
    for (size_t i = 0; i < items.size(); ++i) {
        if (!known[i]) g_by_shape[keys[i]] = g_by_source.at(srcs[i]);
        const auto &mk = g_by_shape.at(keys[i]);
        const Item &it = items[i];
        const FusedProgram &prog = *it.prog;
        JitPass &j = (*reqs[it.req].out)[it.pass];
        j.entry = mk.first;
        j.kernel = mk.second;
        const TilePass &P = prog.passes[it.pass];
        const size_t T = size_t(1) << P.k;
        int npg = 0;  // batch: parameterised gates of the pass
        if (it.batched)
            for (int g = P.gate_begin; g < P.gate_begin + P.gate_count; ++g) npg += prog.gates[g].pkind != 0;
        const size_t NP = it.adjoint ? (size_t)std::max(1, it.batched ? npg : P.nparam) : 0;
        const size_t pm = it.batched ? (it.adjoint ? 2 : 1) * 8 * (size_t)std::max(1, npg) : 0;
        j.smem = (jit_double_buffer(dtype, it.adjoint, P.k) ? 2 : 1) * (it.adjoint ? 2 : 1) * T * es +
                 (pm + 2 * NP * (kTileThreads / 32)) * rs;
        j.nparam_gates = npg;
        const size_t G = P.gate_count > 0 ? P.gate_count : 1;
        size_t bytes = G * 8 * rs;
        if (it.adjoint && !it.batched) {
            bytes += NP * 8 * rs;
            bytes += NP * sizeof(int);
        }
        if (it.batched) bytes = ((bytes + 3) & ~size_t(3)) + G * 2 * sizeof(int);
        j.arg_bytes = (bytes + 15) & ~size_t(15);
        j.batched = it.batched;
    }
    return true;
}

bool jit_prepare_program(int dtype, bool adjoint, const FusedProgram &prog, std::vector<JitPass> *out,
                         std::string *err, double *compile_seconds, int *compiled_modules) {
    return jit_prepare_programs(dtype, {JitRequest{&prog, adjoint, false, out}}, err, compile_seconds, compiled_modules);
}

namespace {

// The kernel of a compiled pass on the current device: loaded on first use, its dynamic shared
// memory allowed, its resident blocks per SM looked up once.
cudaError_t jit_kernel(const JitPass &jp, cudaKernel_t *kern, int *occ) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lock(g_mu);
    if (jp.entry < 0 || jp.entry >= (int)g_modules.size()) return cudaErrorInvalidValue;
    Module *m = g_modules[jp.entry].get();
    if (!m->lib) {
        cudaError_t e = cudaLibraryLoadData(&m->lib, m->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (e != cudaSuccess) return e;
        m->kernels.resize(m->names.size());
        for (size_t i = 0; i < m->names.size(); ++i) {
            e = cudaLibraryGetKernel(&m->kernels[i], m->lib, m->names[i].c_str());
            if (e != cudaSuccess) return e;
        }
    }
    *kern = m->kernels[jp.kernel];
    auto &ss = m->smem_set[dev];
    auto &oc = m->occ[dev];
    if (ss.size() < m->kernels.size()) {
        ss.resize(m->kernels.size(), 0);
        oc.resize(m->kernels.size(), 0);
    }
    if (jp.smem > 48 * 1024 && ss[jp.kernel] < jp.smem) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(*kern),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jp.smem);
        if (e != cudaSuccess) return e;
        ss[jp.kernel] = jp.smem;
        oc[jp.kernel] = 0;
    }
    if (oc[jp.kernel] == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, reinterpret_cast<const void *>(*kern), kTileThreads,
                                                          jp.smem) != cudaSuccess ||
            v < 1) {
            cudaGetLastError();
            v = 1;
        }
        oc[jp.kernel] = v;
    }
    *occ = oc[jp.kernel];
    return cudaSuccess;
}

// The fixed matrices of a pass's gates (state precision), row-major 8 reals each.
void put_matrices(int dtype, const FusedProgram &prog, const TilePass &P, unsigned char *dst) {
    const size_t rs = dtype == QS_C64 ? 4 : 8;
    const RegGate *g = prog.gates.data() + P.gate_begin;
    for (int i = 0; i < P.gate_count; ++i) {
        if (dtype == QS_C64)
            std::memcpy(dst + (size_t)i * 8 * rs, g[i].Uf, 8 * rs);
        else
            std::memcpy(dst + (size_t)i * 8 * rs, g[i].U, 8 * rs);
    }
}

}  // namespace

cudaError_t jit_load(const std::vector<JitPass> &passes) {
    for (const JitPass &jp : passes) {
        cudaKernel_t kern;
        int occ = 0;
        cudaError_t e = jit_kernel(jp, &kern, &occ);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_jit_pass(int dtype, const JitPass &jp, const FusedProgram &prog, int p, void *psi, void *lam,
                            double *part, size_t part_stride, cudaStream_t st) {
    cudaKernel_t kern;
    int occ = 1;
    cudaError_t e = jit_kernel(jp, &kern, &occ);
    if (e != cudaSuccess) return e;
    const TilePass &P = prog.passes[p];
    const bool adjoint = lam != nullptr;
    // parameter block: matrices (state precision), derivatives, gradient slots
    std::vector<unsigned char> blk(jp.arg_bytes, 0);
    const int G = P.gate_count;
    const RegGate *g = prog.gates.data() + P.gate_begin;
    const size_t rs = dtype == QS_C64 ? 4 : 8;
    const size_t G1 = G > 0 ? G : 1;
    put_matrices(dtype, prog, P, blk.data());
    if (adjoint) {
        const size_t NP1 = P.nparam > 0 ? P.nparam : 1;
        unsigned char *d = &blk[G1 * 8 * rs];
        for (int i = 0; i < G; ++i) {
            if (g[i].slot < 0) continue;
            if (dtype == QS_C64)
                std::memcpy(d + (size_t)g[i].slot * 8 * rs, g[i].Df, 8 * rs);
            else
                std::memcpy(d + (size_t)g[i].slot * 8 * rs, g[i].D, 8 * rs);
        }
        int *gs = reinterpret_cast<int *>(d + NP1 * 8 * rs);
        for (int i = 0; i < P.nparam; ++i) gs[i] = P.param_gslot[i];
    }
    uint64_t cap = (uint64_t)device_sm_count() * occ;
    if (adjoint) cap = std::min<uint64_t>(cap, part_stride);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(P.ntiles, cap));
    unsigned long long stride = part_stride;
    void *dbg = debug_state_address();  // debug build only: the generated kernels take it last
    void *args_fwd[] = {&psi, blk.data(), &dbg};
    void *args_adj[] = {&psi, &lam, &part, &stride, blk.data(), &dbg};
    return cudaLaunchKernel(reinterpret_cast<const void *>(kern), dim3(grid), dim3(kTileThreads),
                            adjoint ? args_adj : args_fwd, jp.smem, st);
}

cudaError_t launch_jit_pass_batched(int dtype, const JitPass &jp, const FusedProgram &prog, int p, void *psi,
                                    void *lam, double *part, uint64_t stride, uint64_t nstates, const void *cs,
                                    uint32_t cs_stride, cudaStream_t st) {
    if (!jp.batched) return cudaErrorInvalidValue;
    cudaKernel_t kern;
    int occ = 1;
    cudaError_t e = jit_kernel(jp, &kern, &occ);
    if (e != cudaSuccess) return e;
    const TilePass &P = prog.passes[p];
    std::vector<unsigned char> blk(jp.arg_bytes, 0);
    const int G = P.gate_count;
    const size_t rs = dtype == QS_C64 ? 4 : 8;
    const size_t G1 = G > 0 ? G : 1;
    put_matrices(dtype, prog, P, blk.data());
    int *pix = reinterpret_cast<int *>(blk.data() + ((G1 * 8 * rs + 3) & ~size_t(3)));
    const RegGate *g = prog.gates.data() + P.gate_begin;
    for (int i = 0; i < G; ++i) {
        pix[2 * i] = g[i].pidx;
        pix[2 * i + 1] = g[i].pidx2;
    }
    const uint64_t total = nstates * P.ntiles;
    const uint64_t cap = (uint64_t)device_sm_count() * occ;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(total, cap));
    unsigned long long stride_ = stride, nst = nstates;
    unsigned cs_st = cs_stride;
    void *args[] = {&psi, &lam, &part, &stride_, &nst, const_cast<void **>(&cs), &cs_st, blk.data()};
    return cudaLaunchKernel(reinterpret_cast<const void *>(kern), dim3(grid), dim3(kTileThreads), args, jp.smem, st);
}

}  // namespace qs
