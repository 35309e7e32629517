// qs_circuit.cu -- qs_apply_circuit and qs_adjoint_grad: whole gate lists, validated
// up front, launched per gate (or per fused tile pass) on the state's stream, optionally
// recorded once into a CUDA graph and replayed.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "qs_fuse.cuh"
#include "qs_internal.cuh"
#include "qs_jit.cuh"
#include "qs_state.cuh"

namespace qs {

size_t adj_partials_per_slot();
cudaError_t launch_adj_step(int dtype, void *psi, void *lam, const GatePlan &p, const double *dU, double *part,
                            cudaStream_t st);
cudaError_t launch_obs_sumz(int dtype, const void *psi, void *lam, int n, cudaStream_t st);
cudaError_t launch_sum_vec(const double *z, int n, double *out, cudaStream_t st);
cudaError_t launch_grad_final(const double *part, int nslots, double *slot_sum, const int *slot_param,
                              double *grad, int nparams, cudaStream_t st);

void release_state_buffers(qs_state *s) {
    for (auto &g : s->graphs) {
        cudaGraphExecDestroy(g.exec);
        if (g.table) cudaFree(g.table);
    }
    s->graphs.clear();
    if (s->tile_table) cudaFree(s->tile_table);
    s->tile_table = nullptr;
    s->tile_table_bytes = 0;
    if (s->capture_stream) cudaStreamDestroy(s->capture_stream);
    s->capture_stream = nullptr;
    if (s->red_scratch) cudaFree(s->red_scratch);
    s->red_scratch = nullptr;
    s->red_scratch_n = 0;
    if (s->lam) cudaFree(s->lam);
    s->lam = nullptr;
    if (s->grad_scratch) cudaFree(s->grad_scratch);
    s->grad_scratch = nullptr;
    s->grad_scratch_n = 0;
}

// RY(theta) = [[c, -s], [s, c]], RZ(theta) = diag(c - i s, c + i s), c = cos(theta/2),
// s = sin(theta/2): exp(-i theta P / 2) for P = Y, Z.
static void rot_matrix(int kind, double theta, double U[8]) {
    const double c = std::cos(0.5 * theta), s = std::sin(0.5 * theta);
    std::memset(U, 0, 8 * sizeof(double));
    if (kind == QS_GATE_RY) {
        U[0] = c; U[2] = -s; U[4] = s; U[6] = c;
    } else {
        U[0] = c; U[1] = -s; U[6] = c; U[7] = s;
    }
}

// d/dtheta of the matrices above: dRY = 1/2 [[-s, -c], [c, -s]],
// dRZ = diag(-i/2 (c - i s), i/2 (c + i s)) = diag((-s - i c)/2, (-s + i c)/2).
static void rot_derivative(int kind, double theta, double D[8]) {
    const double c = std::cos(0.5 * theta), s = std::sin(0.5 * theta);
    std::memset(D, 0, 8 * sizeof(double));
    if (kind == QS_GATE_RY) {
        D[0] = -0.5 * s; D[2] = -0.5 * c; D[4] = 0.5 * c; D[6] = -0.5 * s;
    } else {
        D[0] = -0.5 * s; D[1] = -0.5 * c; D[6] = -0.5 * s; D[7] = 0.5 * c;
    }
}

static void dagger(const double U[8], double D[8]) {
    // [a b; c d]^dagger = [a* c*; b* d*]
    D[0] = U[0]; D[1] = -U[1];
    D[2] = U[4]; D[3] = -U[5];
    D[4] = U[2]; D[5] = -U[3];
    D[6] = U[6]; D[7] = -U[7];
}

// Resolve one gate record into a forward plan (validating it). `theta` may be NULL if
// no gate is parameterised.
static bool plan_record(const qs_state *s, const qs_gate &g, const double *theta, size_t n_theta, size_t index,
                        GatePlan *p, char *err, size_t errlen) {
    char e2[200];
    if (g.reserved != 0) {
        std::snprintf(err, errlen, "gate %zu: reserved field must be 0", index);
        return false;
    }
    double U[8];
    int kind = g.kind;
    if (kind == QS_GATE_RY || kind == QS_GATE_RZ) {
        if (!theta || g.param < 0 || (size_t)g.param >= n_theta) {
            std::snprintf(err, errlen, "gate %zu: parameter index %d outside theta[%zu]", index, g.param, n_theta);
            return false;
        }
        if (!std::isfinite(theta[g.param])) {
            std::snprintf(err, errlen, "gate %zu: theta[%d] is not finite", index, g.param);
            return false;
        }
        rot_matrix(kind, theta[g.param], U);
        kind = QS_GATE_U;
    } else if (kind == QS_GATE_U) {
        std::memcpy(U, g.U, sizeof(U));
    } else if (kind != QS_GATE_X) {
        std::snprintf(err, errlen, "gate %zu: unknown kind %d", index, g.kind);
        return false;
    }
    if (!plan_gate(s->n, s->dtype, g.target, g.ctrl_mask, g.ctrl_vals, kind == QS_GATE_X ? nullptr : U, kind, -1, p,
                   e2, sizeof(e2))) {
        std::snprintf(err, errlen, "gate %zu: %s", index, e2);
        return false;
    }
    return true;
}

static uint64_t fnv1a(uint64_t h, const void *data, size_t n) {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Bytes one single-gate launch must move: every selected amplitude read and written
// (2 * 2^(n-c) * s); a one-sided diagonal gate touches only its changed side.
static double gate_algorithmic_bytes(const GatePlan &p, int dtype) {
    const double s = dtype == QS_C64 ? 8.0 : 16.0;
    const double b = 2.0 * std::ldexp(s, p.n - __builtin_popcountll(p.ctrl_mask));
    return p.op == OP_SIDE ? 0.5 * b : b;
}

// Floating-point operations of one gate's update (per selected pair: general 28, real or
// diagonal 12, one-sided 6, exchange 0), and of a sweep's derivative product (8 per pair).
static double gate_algorithmic_flops(const GatePlan &p) {
    if (p.units == 0) return 0.0;
    const double per = p.op == OP_GEN ? 28.0 : (p.op == OP_REAL || p.op == OP_DIAG) ? 12.0 : p.op == OP_SIDE ? 6.0 : 0.0;
    return per * std::ldexp(1.0, p.n - 1 - __builtin_popcountll(p.ctrl_mask));
}

static int tile_bits(int dtype, bool adjoint, bool jit = false);

// The bytes a recorded graph depends on: the gate records, the parameters, the flags, the
// state buffer and the tile size, each run preceded by its length so that different splits
// of the same bytes differ.
static void graph_key_bytes(const qs_state *s, const qs_gate *gates, size_t count, const double *theta,
                            size_t n_theta, int flags, std::vector<unsigned char> *out) {
    const int tb = tile_bits(s->dtype, false);
    const uint64_t nt = theta ? (uint64_t)n_theta : 0, ng = (uint64_t)count;
    out->clear();
    auto put = [out](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        out->insert(out->end(), b, b + n);
    };
    put(&ng, sizeof(ng));
    if (count > 0) put(gates, count * sizeof(qs_gate));
    put(&nt, sizeof(nt));
    if (nt > 0) put(theta, n_theta * sizeof(double));
    put(&flags, sizeof(flags));
    put(&s->psi, sizeof(s->psi));
    put(&tb, sizeof(tb));
}

// FNV-1a over the key bytes. QS_TEST_GRAPH_KEY (a test hook) replaces the hash with a fixed
// value so that a test can make different circuits collide on it.
static uint64_t graph_key_hash(const std::vector<unsigned char> &bytes) {
    const char *forced = std::getenv("QS_TEST_GRAPH_KEY");
    if (forced && *forced) return std::strtoull(forced, nullptr, 0);
    return fnv1a(1469598103934665603ull, bytes.data(), bytes.size());
}

// Forward application only: runs of consecutive gates with the same target and the same
// controls act on the same pairs, so their product (U_last ... U_first, formed in double
// precision) replaces them; e.g. RY then RZ on one qubit become one launch or one tile-pass
// gate. Exchange products that are the identity drop out. The baseline comparator
// (QS_FLAG_MASKED) and the adjoint sweep keep every gate.
static void cmatmul2(const double *A, const double *B, double *C) {  // C = A B, row-major 2x2
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < 2; ++k) {
                const double ar = A[2 * (2 * i + k)], ai = A[2 * (2 * i + k) + 1];
                const double br = B[2 * (2 * k + j)], bi = B[2 * (2 * k + j) + 1];
                re += ar * br - ai * bi;
                im += ar * bi + ai * br;
            }
            C[2 * (2 * i + j)] = re;
            C[2 * (2 * i + j) + 1] = im;
        }
}

// Float32 instructions per selected pair of one gate's update inside a compiled complex64 pass
// (general 16; real 4, as packed two-lane instructions; diagonal 8; one-sided 4; exchange and
// identity 0).
static int compiled_update_cost(const GatePlan &p) {
    if (p.units == 0) return 0;
    switch (p.op) {
    case OP_GEN: return 16;
    case OP_REAL: return 4;
    case OP_DIAG: return 8;
    case OP_SIDE: return 4;
    default: return 0;
    }
}

// flags: with QS_FLAG_FUSE | QS_FLAG_JIT on complex64 states a run is merged only where its
// product costs a compiled pass fewer instructions than its gates apart (RY then RZ: a general
// product, 16 per pair, against 4 + 8 apart; two diagonal or two real gates: merged).
static void merge_runs(const qs_state *s, std::vector<GatePlan> &plans, std::vector<int> *first_rec = nullptr,
                       int flags = 0) {
    const bool compiled = (flags & QS_FLAG_FUSE) && (flags & QS_FLAG_JIT) && s->dtype == QS_C64;
    std::vector<GatePlan> out;
    out.reserve(plans.size());
    if (first_rec) first_rec->clear();
    size_t i = 0;
    while (i < plans.size()) {
        size_t j = i + 1;
        while (j < plans.size() && plans[j].t == plans[i].t && plans[j].ctrl_mask == plans[i].ctrl_mask &&
               plans[j].ctrl_vals == plans[i].ctrl_vals)
            ++j;
        if (j == i + 1) {
            if (first_rec) first_rec->push_back((int)i);
            out.push_back(plans[i]);
        } else {
            double U[8], T[8];
            std::memcpy(U, plans[i].Ufull, sizeof(U));
            for (size_t q = i + 1; q < j; ++q) {
                cmatmul2(plans[q].Ufull, U, T);
                std::memcpy(U, T, sizeof(U));
            }
            GatePlan m;
            char e2[200];
            // an exact exchange product stays an exchange (bit-exact), else the planner
            // classifies the product's structure
            bool merge = plan_gate(s->n, s->dtype, plans[i].t, plans[i].ctrl_mask, plans[i].ctrl_vals, U, QS_GATE_U, -1,
                                   &m, e2, sizeof(e2));
            if (merge && compiled) {
                int apart = 0;
                for (size_t q = i; q < j; ++q) apart += compiled_update_cost(plans[q]);
                merge = compiled_update_cost(m) < apart;
            }
            if (merge) {
                if (first_rec) first_rec->push_back((int)i);
                out.push_back(m);
            } else {
                for (size_t q = i; q < j && first_rec; ++q) first_rec->push_back((int)q);
                out.insert(out.end(), plans.begin() + i, plans.begin() + j);  // not finite: keep the run
            }
        }
        i = j;
    }
    if (first_rec) first_rec->push_back((int)plans.size());
    plans.swap(out);
}

// With QS_FLAG_FUSE | QS_FLAG_JIT on complex64 states: an uncontrolled diagonal gate with
// entries of modulus 1, diag(a, d), is the global phase a times the one-sided gate diag(1, d/a),
// which a compiled pass applies in half the operations (4 float32 operations per pair instead of
// 8; RZ(theta) in particular). Global phases commute with every gate, so all but the first such
// gate become one-sided and the first takes the product of their phases: the same state up to
// rounding, global phase included.
static void fold_phases(const qs_state *s, std::vector<GatePlan> &plans, int flags) {
    if (!(flags & QS_FLAG_FUSE) || !(flags & QS_FLAG_JIT) || s->dtype != QS_C64) return;
    auto unit = [](double re, double im) { return std::fabs(re * re + im * im - 1.0) <= 1e-12; };
    int first = -1;
    double gr = 1.0, gi = 0.0;  // product of the phases taken out
    char e2[200];
    for (size_t i = 0; i < plans.size(); ++i) {
        const GatePlan &p = plans[i];
        if (p.units == 0 || p.op != OP_DIAG || p.ctrl_mask != 0) continue;
        const double ar = p.Ufull[0], ai = p.Ufull[1], dr = p.Ufull[6], di = p.Ufull[7];
        if (!unit(ar, ai) || !unit(dr, di)) continue;
        if (first < 0) {
            first = (int)i;
            continue;
        }
        // d / a = d conj(a) for |a| = 1
        const double U[8] = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0, dr * ar + di * ai, di * ar - dr * ai};
        GatePlan q;
        if (!plan_gate(s->n, s->dtype, p.t, 0, 0, U, QS_GATE_U, -1, &q, e2, sizeof(e2))) continue;
        const double nr = gr * ar - gi * ai, ni = gr * ai + gi * ar;
        gr = nr;
        gi = ni;
        plans[i] = q;
    }
    if (first < 0 || (gr == 1.0 && gi == 0.0)) return;
    const GatePlan &p = plans[first];
    const double ar = p.Ufull[0], ai = p.Ufull[1], dr = p.Ufull[6], di = p.Ufull[7];
    const double U[8] = {gr * ar - gi * ai, gr * ai + gi * ar, 0.0, 0.0, 0.0, 0.0, gr * dr - gi * di, gr * di + gi * dr};
    GatePlan q;
    if (plan_gate(s->n, s->dtype, p.t, 0, 0, U, QS_GATE_U, -1, &q, e2, sizeof(e2))) plans[first] = q;
}

static qs_status launch_plans(qs_state *s, const std::vector<GatePlan> &plans, cudaStream_t st,
                              bool masked = false) {
    for (size_t i = 0; i < plans.size(); ++i) {
        cudaError_t e = masked ? launch_gate_masked(s->dtype, s->psi, plans[i], plans[i].ctrl_mask,
                                                    plans[i].ctrl_vals, st)
                               : launch_gate(s->dtype, s->psi, plans[i], st);
        if (e != cudaSuccess) {
            char what[128];
            std::snprintf(what, sizeof(what), "qs_apply_circuit launch (gate %zu: t=%d op=%d layout=%d r=%d)", i,
                          plans[i].t, plans[i].op, plans[i].layout, plans[i].r);
            return cuda_fail(e, what);
        }
    }
    return QS_OK;
}

// Tuned tile sizes per (dtype, adjoint), set by qs_set_tile_bits (0 = default).
static std::atomic<int> g_tile_bits[2][2] = {{{0}, {0}}, {{0}, {0}}};

// Largest tile (local qubits) whose block fits the shared memory of one SM with the longest
// pass's gate tables: complex64 14 forward / 13 adjoint, complex128 13 / 12.
static int max_tile_bits(int dtype, bool adjoint) {
    int k = kTileMaxBits;
    while (k > 5 && tile_smem_bytes(dtype, k, adjoint, kPassMaxGates, kPassMaxGates) > kTileMaxSmem) --k;
    return k;
}

// Local qubits per tile of a fused pass (shared memory per CTA: 2^k amplitudes, twice that
// for the adjoint's psi and lambda tiles): QS_TILE_BITS if set (at most the largest tile that
// fits), else the tuned value, else the default.
// jit: the sweep's passes will be compiled for their shape; their default tile is smaller
// (2^11 amplitudes of psi and lambda: two tile buffers and two blocks fit one SM).
static int tile_bits(int dtype, bool adjoint, bool jit) {
    const char *env = std::getenv("QS_TILE_BITS");
    if (env && *env) {
        const int v = std::atoi(env);
        if (v >= 2 && v <= kTileMaxBits) return std::min(v, max_tile_bits(dtype, adjoint));
    }
    const int tuned = g_tile_bits[dtype == QS_C64 ? 0 : 1][adjoint ? 1 : 0].load();
    if (tuned > 0) return tuned;
    if (dtype == QS_C64) return adjoint && jit ? 11 : 12;
    return adjoint ? 10 : 11;
}

// Make sure `*buf` (device) holds `bytes`; grow-only. The old buffer may still be read by
// work queued on `st`, so the stream is drained before it is freed.
static qs_status ensure_device(void **buf, size_t *cap, size_t bytes, cudaStream_t st, const char *what) {
    if (*buf && *cap >= bytes) return QS_OK;
    if (*buf) {
        cudaStreamSynchronize(st);
        cudaFree(*buf);
    }
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(buf, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return set_error(QS_ENOMEM, what);
    }
    *cap = std::max<size_t>(bytes, 256);
    return QS_OK;
}

// Launch a fused program. Forward: `lam` == nullptr. Adjoint: single gates use the sweep
// kernel with dus[g] / part + slot * P, passes use the adjoint tile kernel.
static qs_status launch_program(qs_state *s, const FusedProgram &prog, const std::vector<GatePlan> &plans,
                                const void *dev_table, void *lam, const std::vector<const double *> *dus,
                                const std::vector<int> *slots, double *part, size_t P, cudaStream_t st,
                                const std::vector<JitPass> *jit = nullptr) {
    const TileGroup *groups = dev_table ? table_groups(prog, dev_table) : nullptr;
    const RegGate *gates = dev_table ? table_gates(prog, dev_table) : nullptr;
    const DiagGate *dgates = dev_table ? table_dgates(prog, dev_table) : nullptr;
    for (const FusedOp &op : prog.ops) {
        const bool bad = op.drun >= 0 ? (op.drun >= (int)prog.druns.size() || !dgates)
                                      : (op.pass >= (int)prog.passes.size() ||
                                         (op.pass < 0 && (op.gate < 0 || (size_t)op.gate >= plans.size())));
        if (bad) return set_error(QS_EINVAL, "fused program refers to a gate or pass it does not hold");
        cudaError_t e;
        if (op.drun >= 0) {
            const DiagRun &r = prog.druns[op.drun];
            e = launch_diag_run(s->dtype, s->psi, s->n, dgates + r.begin, r.count, r.nc, st);
        } else if (op.pass >= 0 && jit) {
            e = launch_jit_pass(s->dtype, (*jit)[op.pass], prog, op.pass, s->psi, lam, part, P, st);
        } else if (op.pass >= 0) {
            e = launch_tile_pass(s->dtype, s->psi, lam, prog.passes[op.pass], groups, gates, part, P, st);
        } else if (!lam) {
            e = launch_gate(s->dtype, s->psi, plans[op.gate], st);
        } else {
            const int slot = (*slots)[op.gate];
            e = launch_adj_step(s->dtype, s->psi, lam, plans[op.gate], (*dus)[op.gate],
                                slot >= 0 ? part + (size_t)slot * P : nullptr, st);
        }
        if (e != cudaSuccess) {
            char what[160];
            if (op.drun >= 0)
                std::snprintf(what, sizeof(what), "fused program launch (diagonal run %d, %d gates)", op.drun,
                              prog.druns[op.drun].count);
            else if (op.pass >= 0)
                std::snprintf(what, sizeof(what), "fused program launch (tile pass %d, k=%d, %d gates)", op.pass,
                              prog.passes[op.pass].k, prog.passes[op.pass].gate_count);
            else
                std::snprintf(what, sizeof(what), "fused program launch (gate %d: t=%d op=%d layout=%d r=%d)", op.gate,
                              plans[op.gate].t, plans[op.gate].op, plans[op.gate].layout, plans[op.gate].r);
            return cuda_fail(e, what);
        }
    }
    return QS_OK;
}

// Plans of one gradient: the forward gates (same-target runs merged), the sweep's gates
// (U^dagger, and dU/dtheta for parameterised ones with their gradient slots) and, with
// QS_FLAG_FUSE, the fused forward and sweep programs.
struct AdjPlan {
    std::vector<GatePlan> fwd, adj;
    std::vector<int> slot_of, slot_param;
    std::vector<double> dus;  // 8 doubles per slot
    std::vector<const double *> dusp;
    FusedProgram pf, pa;
};

// The per-gate plans of a gradient: forward (then merged), sweep (U^dagger), the parameter
// slots and derivative matrices.
static bool plan_adjoint_gates(const qs_state *s, const qs_gate *gates, size_t count, const double *theta,
                               size_t n_theta, int flags, AdjPlan *ap, char *err, size_t errlen) {
    std::vector<GatePlan> &fwd = ap->fwd, &adj = ap->adj;
    fwd.assign(count, GatePlan{});
    adj.assign(count, GatePlan{});
    ap->slot_of.assign(count, -1);
    std::vector<int> &slot_of = ap->slot_of, &slot_param = ap->slot_param;
    std::vector<double> &dus = ap->dus;
    slot_param.clear();
    dus.clear();
    char e2[200];
    for (size_t i = 0; i < count; ++i) {
        const qs_gate &g = gates[i];
        if (!plan_record(s, g, theta, n_theta, i, &fwd[i], err, errlen)) return false;
        double U[8], Ud[8];
        int force = -1;
        if (g.kind == QS_GATE_X) {
            force = OP_SWAP;
            std::memset(Ud, 0, sizeof(Ud));
            Ud[2] = 1.0;
            Ud[4] = 1.0;
        } else {
            if (g.kind == QS_GATE_RY || g.kind == QS_GATE_RZ) rot_matrix(g.kind, theta[g.param], U);
            else std::memcpy(U, g.U, sizeof(U));
            dagger(U, Ud);
            if (g.kind == QS_GATE_RY) force = OP_REAL;
            else if (g.kind == QS_GATE_RZ) force = OP_DIAG;
        }
        if (!plan_gate(s->n, s->dtype, g.target, g.ctrl_mask, g.ctrl_vals, Ud, QS_GATE_U, force, &adj[i], e2,
                       sizeof(e2))) {
            std::snprintf(err, errlen, "%s", e2);
            return false;
        }
        if (adj[i].op == OP_SIDE) {  // the sweep kernels scale both sides
            GatePlan q;
            plan_gate(s->n, s->dtype, g.target, g.ctrl_mask, g.ctrl_vals, Ud, QS_GATE_U, OP_DIAG, &q, e2, sizeof(e2));
            adj[i] = q;
        }
        if (g.kind == QS_GATE_RY || g.kind == QS_GATE_RZ) {
            slot_of[i] = (int)slot_param.size();
            slot_param.push_back(g.param);
            double D[8];
            rot_derivative(g.kind, theta[g.param], D);
            dus.insert(dus.end(), D, D + 8);
        }
    }
    ap->dusp.assign(count, nullptr);
    for (size_t i = 0; i < count; ++i)
        if (slot_of[i] >= 0) ap->dusp[i] = &dus[8 * slot_of[i]];
    merge_runs(s, fwd, nullptr, flags);  // the forward pass needs no per-gate state
    fold_phases(s, fwd, flags);
    return true;
}

// The fused forward and sweep programs of a gradient whose per-gate plans ap holds.
static void plan_adjoint_programs(const qs_state *s, int flags, AdjPlan *ap) {
    const size_t count = ap->adj.size();
    std::vector<int> seq(ap->fwd.size());
    for (size_t i = 0; i < ap->fwd.size(); ++i) seq[i] = (int)i;
    const bool jit = (flags & QS_FLAG_JIT) != 0;
    plan_fused(s->n, s->dtype, tile_bits(s->dtype, false), seq, ap->fwd, nullptr, nullptr, &ap->pf, kPassMaxGates, true,
               0, jit);
    seq.resize(count);
    for (size_t i = 0; i < count; ++i) seq[i] = (int)(count - 1 - i);
    // sweep passes keep psi and lambda rows of kGroupBitsAdjoint group qubits in registers
    // (compiled passes too: with 4, their long straight-line groups spill registers)
    plan_fused(s->n, s->dtype, tile_bits(s->dtype, true, jit), seq, ap->adj, &ap->dusp, &ap->slot_of, &ap->pa,
               kPassMaxGates, true, 0, jit);
}

static bool plan_adjoint(const qs_state *s, const qs_gate *gates, size_t count, const double *theta, size_t n_theta,
                         int flags, AdjPlan *ap, char *err, size_t errlen) {
    if (!plan_adjoint_gates(s, gates, count, theta, n_theta, flags, ap, err, errlen)) return false;
    if (flags & QS_FLAG_FUSE) plan_adjoint_programs(s, flags, ap);
    return true;
}

// ---------------------------------------------------------------------------------------------
// Plan cache
// ---------------------------------------------------------------------------------------------
// A training loop applies or differentiates the same circuit with new angles again and again.
// A fused program depends on the angles only through the gates' matrices, as long as every
// gate keeps its structure (operation class, one-sided side, identity or not): the last
// kPlanCacheEntries programs (of qs_apply_circuit: one; of qs_adjoint_grad: forward and sweep)
// are kept process-wide, keyed by everything else they depend on (entry point, size,
// precision, flags, tile sizes, the gate records), and a call whose per-gate structure equals
// the cached one takes them and copies its own matrices in. Programs with diagonal-run
// launches (whose factor classes follow the values) are not kept.
namespace {

constexpr size_t kPlanCacheEntries = 8;
constexpr size_t kPlanCacheMaxGates = 65536;  // gates of a kept entry's programs

struct PlanCacheEntry {
    std::vector<unsigned char> key;
    std::vector<uint64_t> sig;
    FusedProgram pf, pa;
    std::vector<JitPass> jf, ja;
    uint64_t used = 0;
};

std::mutex g_plan_mu;
std::vector<PlanCacheEntry> g_plan_cache;
uint64_t g_plan_clock = 0;

std::vector<unsigned char> plan_cache_key(char entry, const qs_state *s, const qs_gate *gates, size_t count,
                                          size_t n_theta, int flags) {
    std::vector<unsigned char> k(1, (unsigned char)entry);
    auto put = [&k](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        k.insert(k.end(), b, b + n);
    };
    const bool jit = (flags & QS_FLAG_JIT) != 0;
    const int64_t hdr[7] = {s->n, (int64_t)s->dtype, flags & (QS_FLAG_FUSE | QS_FLAG_JIT), tile_bits(s->dtype, false),
                            tile_bits(s->dtype, true, jit), (int64_t)count, (int64_t)n_theta};
    put(hdr, sizeof(hdr));
    if (count > 0) put(gates, count * sizeof(qs_gate));
    return k;
}

// The structure of per-gate plans (what a program built from them depends on besides values).
void plans_signature(const std::vector<GatePlan> &plans, std::vector<uint64_t> *sig) {
    sig->push_back(plans.size());
    for (const GatePlan &p : plans) {
        sig->push_back((uint64_t)(uint32_t)p.op | ((uint64_t)(uint32_t)p.side << 8) | ((uint64_t)(p.units == 0) << 16) |
                       ((uint64_t)(uint32_t)p.t << 24));
        sig->push_back(p.ctrl_mask);
        sig->push_back(p.ctrl_vals);
    }
}

std::vector<uint64_t> adj_signature(const AdjPlan &ap) {
    std::vector<uint64_t> sig;
    plans_signature(ap.fwd, &sig);
    plans_signature(ap.adj, &sig);
    for (int x : ap.slot_of) sig.push_back((uint64_t)(int64_t)x);
    return sig;
}

// The matrices of a program's gates from the current plans (and derivative matrices).
void refresh_matrices(FusedProgram &prog, const std::vector<GatePlan> &plans, const std::vector<const double *> *dusp) {
    for (size_t gi = 0; gi < prog.gates.size(); ++gi) {
        RegGate &R = prog.gates[gi];
        const int src = prog.gate_src[gi];
        std::memcpy(R.U, plans[src].U, sizeof(R.U));
        for (int q = 0; q < 8; ++q) R.Uf[q] = (float)R.U[q];
        if (dusp && R.slot >= 0 && (*dusp)[src]) {
            std::memcpy(R.D, (*dusp)[src], sizeof(R.D));
            for (int q = 0; q < 8; ++q) R.Df[q] = (float)R.D[q];
        }
    }
}

// Copies of the kept programs for this key and structure (pa / ja may be null for an entry
// with one program).
bool plan_cache_take(const std::vector<unsigned char> &key, const std::vector<uint64_t> &sig, FusedProgram *pf,
                     FusedProgram *pa, std::vector<JitPass> *jf, std::vector<JitPass> *ja) {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    for (PlanCacheEntry &e : g_plan_cache) {
        if (e.key != key || e.sig != sig) continue;
        e.used = ++g_plan_clock;
        *pf = e.pf;
        *jf = e.jf;
        if (pa) *pa = e.pa;
        if (ja) *ja = e.ja;
        return true;
    }
    return false;
}

void plan_cache_put(std::vector<unsigned char> key, std::vector<uint64_t> sig, const FusedProgram &pf,
                    const FusedProgram *pa, const std::vector<JitPass> &jf, const std::vector<JitPass> *ja) {
    if (!pf.druns.empty() || (pa && !pa->druns.empty())) return;
    // at most ~15 MB of gate tables per entry (larger programs are planned on every call)
    if (pf.gates.size() + (pa ? pa->gates.size() : 0) > kPlanCacheMaxGates) return;
    std::lock_guard<std::mutex> lock(g_plan_mu);
    PlanCacheEntry *slot = nullptr;
    if (g_plan_cache.size() < kPlanCacheEntries) {
        g_plan_cache.emplace_back();
        slot = &g_plan_cache.back();
    } else {
        slot = &g_plan_cache[0];
        for (PlanCacheEntry &e : g_plan_cache)
            if (e.used < slot->used) slot = &e;
    }
    slot->key = std::move(key);
    slot->sig = std::move(sig);
    slot->pf = pf;
    slot->pa = pa ? *pa : FusedProgram{};
    slot->jf = jf;
    slot->ja = ja ? *ja : std::vector<JitPass>{};
    slot->used = ++g_plan_clock;
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" {

qs_status qs_set_tile_bits(qs_dtype dtype, int adjoint, int bits) {
    if (dtype != QS_C64 && dtype != QS_C128) return set_error(QS_EINVAL, "qs_set_tile_bits: bad dtype");
    if (bits != 0 && (bits < 5 || bits > max_tile_bits(dtype, adjoint != 0))) {
        char msg[128];
        std::snprintf(msg, sizeof(msg), "qs_set_tile_bits: bits must be 0 or 5..%d for this precision and direction",
                      max_tile_bits(dtype, adjoint != 0));
        return set_error(QS_EINVAL, msg);
    }
    g_tile_bits[dtype == QS_C64 ? 0 : 1][adjoint ? 1 : 0].store(bits);
    return QS_OK;
}

int qs_get_tile_bits(qs_dtype dtype, int adjoint) { return tile_bits(dtype, adjoint != 0); }

// The launches of qs_adjoint_grad: the forward program, the energy reduction and lambda = O psi
// (one read of psi; one read of psi and a write of lambda), the reverse sweep over psi and lambda
// (a sweep step or pass reads and writes both vectors), the gradient sums.
static qs_status adjoint_schedule(const qs_state *shape, const qs_gate *gates, size_t count, const double *theta,
                                  size_t n_theta, int flags, qs_schedule *out) {
    AdjPlan ap;
    char err[256];
    if (!plan_adjoint(shape, gates, count, theta, n_theta, flags, &ap, err, sizeof(err)))
        return set_error(QS_EINVAL, err);
    qs_schedule r;
    std::memset(&r, 0, sizeof(r));
    const int n = shape->n, dtype = shape->dtype;
    const double state_bytes = std::ldexp(dtype == QS_C64 ? 8.0 : 16.0, n);
    r.gates = (int32_t)(ap.fwd.size() + ap.adj.size());
    auto add_program = [&](const FusedProgram &prog, const std::vector<GatePlan> &plans, double vectors) {
        r.model_cost += prog.model_cost * vectors;
        for (const TilePass &P : prog.passes) r.pass_gates += P.gate_count;
        for (const FusedOp &op : prog.ops) {
            if (op.drun >= 0) {
                ++r.diag_runs;
                r.algorithmic_bytes += vectors * state_bytes * std::ldexp(2.0, -prog.druns[op.drun].nc.nfix);
            } else if (op.pass >= 0) {
                ++r.tile_passes;
                r.algorithmic_bytes += vectors * 2.0 * state_bytes * pass_touched_fraction(prog, op.pass);
            } else {
                ++r.single_gates;
                r.algorithmic_bytes += vectors * gate_algorithmic_bytes(plans[op.gate], dtype);
            }
        }
    };
    for (const GatePlan &p : ap.fwd) r.algorithmic_flops += gate_algorithmic_flops(p);
    for (size_t i = 0; i < ap.adj.size(); ++i) {
        const GatePlan &p = ap.adj[i];
        r.algorithmic_flops += 2.0 * gate_algorithmic_flops(p);
        if (ap.slot_of[i] >= 0) r.algorithmic_flops += 8.0 * std::ldexp(1.0, n - 1 - __builtin_popcountll(p.ctrl_mask));
    }
    r.algorithmic_flops += 8.0 * std::ldexp(1.0, n);
    if (flags & QS_FLAG_FUSE) {
        add_program(ap.pf, ap.fwd, 1.0);
        add_program(ap.pa, ap.adj, 2.0);
    } else {
        for (const auto *pl : {&ap.fwd, &ap.adj}) {
            const double vectors = pl == &ap.adj ? 2.0 : 1.0;
            for (const GatePlan &p : *pl) {
                if (p.units == 0 && pl == &ap.fwd) continue;
                ++r.single_gates;
                // a sweep step of a parameterised gate reads both sides even when it is diagonal
                const double b = p.op == OP_SIDE && pl == &ap.fwd ? 0.5 : 1.0;
                r.algorithmic_bytes += vectors * b * 2.0 * std::ldexp(dtype == QS_C64 ? 8.0 : 16.0,
                                                                      n - __builtin_popcountll(p.ctrl_mask));
                r.model_cost += vectors * (single_launch_cost(p, dtype) + launch_latency_cost(n, dtype));
            }
        }
    }
    r.algorithmic_bytes += 3.0 * state_bytes;  // energy: read psi; lambda = O psi: read psi, write lambda
    r.launches = r.single_gates + r.tile_passes + r.diag_runs + 4;  // + reductions, lambda, gradient sums
    *out = r;
    return QS_OK;
}

qs_status qs_circuit_schedule(int n, qs_dtype dtype, const qs_gate *gates, size_t count, const double *theta,
                              size_t n_theta, int flags, qs_schedule *out) {
    if (!out) return set_error(QS_EINVAL, "qs_circuit_schedule: out is NULL");
    if (dtype != QS_C64 && dtype != QS_C128 && dtype != QS_Q30)
        return set_error(QS_EINVAL, "qs_circuit_schedule: bad dtype");
    if (dtype == QS_Q30 && (flags & (QS_FLAG_FUSE | QS_FLAG_ADJOINT)))
        return set_error(QS_EUNSUPPORTED, "qs_circuit_schedule: fused passes and gradients are not built for QS_Q30");
    if (n < 1 || n > kMaxQubits) return set_error(QS_EINVAL, "qs_circuit_schedule: n out of range");
    if (count > 0 && !gates) return set_error(QS_EINVAL, "qs_circuit_schedule: gates is NULL");
    if (flags & ~(QS_FLAG_FUSE | QS_FLAG_GRAPH | QS_FLAG_MASKED | QS_FLAG_JIT | QS_FLAG_ADJOINT))
        return set_error(QS_EINVAL, "qs_circuit_schedule: unknown flags");
    if ((flags & QS_FLAG_FUSE) && (flags & QS_FLAG_MASKED))
        return set_error(QS_EINVAL, "qs_circuit_schedule: QS_FLAG_MASKED cannot be combined with QS_FLAG_FUSE");
    if ((flags & QS_FLAG_ADJOINT) && (flags & QS_FLAG_MASKED))
        return set_error(QS_EINVAL, "qs_circuit_schedule: QS_FLAG_MASKED cannot be combined with QS_FLAG_ADJOINT");
    qs_state shape;  // planning reads only the state's size and precision
    shape.n = n;
    shape.dtype = dtype;
    if (flags & QS_FLAG_ADJOINT) return adjoint_schedule(&shape, gates, count, theta, n_theta, flags, out);
    std::vector<GatePlan> plans(count);
    char err[256];
    for (size_t i = 0; i < count; ++i)
        if (!plan_record(&shape, gates[i], theta, n_theta, i, &plans[i], err, sizeof(err)))
            return set_error(QS_EINVAL, err);
    const bool masked = (flags & QS_FLAG_MASKED) != 0;
    if (!masked && dtype != QS_Q30) merge_runs(&shape, plans, nullptr, flags);
    fold_phases(&shape, plans, flags);
    qs_schedule r;
    std::memset(&r, 0, sizeof(r));
    r.gates = (int32_t)plans.size();
    for (const GatePlan &p : plans) r.algorithmic_flops += gate_algorithmic_flops(p);
    const double state_bytes = std::ldexp(dtype == QS_C64 ? 8.0 : 16.0, n);
    if (flags & QS_FLAG_FUSE) {
        std::vector<int> seq(plans.size());
        for (size_t i = 0; i < plans.size(); ++i) seq[i] = (int)i;
        FusedProgram prog;
        plan_fused(n, dtype, tile_bits(dtype, false), seq, plans, nullptr, nullptr, &prog, kPassMaxGates, true, 0,
                   (flags & QS_FLAG_JIT) != 0);
        for (const FusedOp &op : prog.ops) {
            if (op.drun >= 0)
                ++r.diag_runs;
            else if (op.pass >= 0)
                ++r.tile_passes;
            else
                ++r.single_gates;
        }
        for (const TilePass &P : prog.passes) r.pass_gates += P.gate_count;
        r.model_cost = prog.model_cost;
        for (const FusedOp &op : prog.ops) {
            if (op.drun >= 0)
                r.algorithmic_bytes += state_bytes * std::ldexp(2.0, -prog.druns[op.drun].nc.nfix);
            else if (op.pass >= 0)
                r.algorithmic_bytes += 2.0 * state_bytes * pass_touched_fraction(prog, op.pass);
            else
                r.algorithmic_bytes += gate_algorithmic_bytes(plans[op.gate], dtype);
        }
    } else {
        for (const GatePlan &p : plans) {
            if (p.units == 0) continue;
            ++r.single_gates;
            r.model_cost += (masked ? 1.0 : single_launch_cost(p, dtype)) + launch_latency_cost(n, dtype);
            r.algorithmic_bytes += masked ? 2.0 * state_bytes : gate_algorithmic_bytes(p, dtype);
        }
    }
    r.launches = r.single_gates + r.tile_passes + r.diag_runs;
    *out = r;
    return QS_OK;
}

qs_status qs_circuit_order(int n, qs_dtype dtype, const qs_gate *gates, size_t count, const double *theta,
                           size_t n_theta, int flags, int32_t *order) {
    if (count > 0 && !order) return set_error(QS_EINVAL, "qs_circuit_order: order is NULL");
    qs_schedule sched;  // the same validation as the schedule
    const qs_status st = qs_circuit_schedule(n, dtype, gates, count, theta, n_theta, flags, &sched);
    if (st != QS_OK) return st;
    qs_state shape;
    shape.n = n;
    shape.dtype = dtype;
    std::vector<int> out;
    out.reserve(count);
    std::vector<char> placed(count, 0);
    auto put = [&](int r) {
        if (r >= 0 && (size_t)r < count && !placed[r]) {
            placed[r] = 1;
            out.push_back(r);
        }
    };
    char err[256];
    const bool fuse = (flags & QS_FLAG_FUSE) != 0;
    if (flags & QS_FLAG_ADJOINT) {
        AdjPlan ap;
        if (fuse) {
            if (!plan_adjoint(&shape, gates, count, theta, n_theta, flags, &ap, err, sizeof(err)))
                return set_error(QS_EINVAL, err);
            for (int g : ap.pa.order) put(g);  // sweep plans are one per gate record
        }
        for (size_t i = count; i-- > 0;) put((int)i);
    } else {
        if (fuse) {
            std::vector<GatePlan> plans(count);
            for (size_t i = 0; i < count; ++i)
                if (!plan_record(&shape, gates[i], theta, n_theta, i, &plans[i], err, sizeof(err)))
                    return set_error(QS_EINVAL, err);
            std::vector<int> first_rec;
            merge_runs(&shape, plans, &first_rec, flags);
            fold_phases(&shape, plans, flags);
            std::vector<int> seq(plans.size());
            for (size_t i = 0; i < plans.size(); ++i) seq[i] = (int)i;
            FusedProgram prog;
            plan_fused(n, dtype, tile_bits(dtype, false), seq, plans, nullptr, nullptr, &prog, kPassMaxGates, true, 0,
                       (flags & QS_FLAG_JIT) != 0);
            for (int pl : prog.order)
                for (int r = first_rec[pl]; r < first_rec[pl + 1]; ++r) put(r);
        }
        for (size_t i = 0; i < count; ++i) {  // identities (and everything, unfused) in the given order
            if (!placed[i]) put((int)i);
        }
    }
    for (size_t i = 0; i < count; ++i) order[i] = out[i];
    return QS_OK;
}

qs_status qs_circuit_compile(int n, qs_dtype dtype, const qs_gate *gates, size_t count, const double *theta,
                             size_t n_theta, int flags, int adjoint, double *compile_seconds, int *passes) {
    if (dtype != QS_C64 && dtype != QS_C128) return set_error(QS_EINVAL, "qs_circuit_compile: bad dtype");
    if (n < 1 || n > kMaxQubits) return set_error(QS_EINVAL, "qs_circuit_compile: n out of range");
    if (count > 0 && !gates) return set_error(QS_EINVAL, "qs_circuit_compile: gates is NULL");
    if (flags & ~(QS_FLAG_FUSE | QS_FLAG_GRAPH | QS_FLAG_JIT | QS_FLAG_OUT_DEVICE))
        return set_error(QS_EINVAL, "qs_circuit_compile: unknown flags");
    qs_state shape;  // planning reads only the state's size and precision
    shape.n = n;
    shape.dtype = dtype;
    std::vector<const FusedProgram *> progs;
    std::vector<bool> adj_of;
    char err[256];
    std::vector<GatePlan> plans;
    FusedProgram prog;
    AdjPlan ap;
    const int fl = flags | QS_FLAG_FUSE | QS_FLAG_JIT;
    if (!adjoint) {
        plans.resize(count);
        for (size_t i = 0; i < count; ++i)
            if (!plan_record(&shape, gates[i], theta, n_theta, i, &plans[i], err, sizeof(err)))
                return set_error(QS_EINVAL, err);
        merge_runs(&shape, plans, nullptr, fl);
        fold_phases(&shape, plans, fl);
        std::vector<int> seq(plans.size());
        for (size_t i = 0; i < plans.size(); ++i) seq[i] = (int)i;
        plan_fused(n, dtype, tile_bits(dtype, false), seq, plans, nullptr, nullptr, &prog, kPassMaxGates, true, 0,
                   (fl & QS_FLAG_JIT) != 0);
        progs.push_back(&prog);
        adj_of.push_back(false);
    } else {
        if (!plan_adjoint(&shape, gates, count, theta, n_theta, fl, &ap, err, sizeof(err)))
            return set_error(QS_EINVAL, err);
        progs.push_back(&ap.pf);
        adj_of.push_back(false);
        progs.push_back(&ap.pa);
        adj_of.push_back(true);
    }
    double secs = 0.0;
    int np = 0;
    for (size_t i = 0; i < progs.size(); ++i) {
        std::vector<JitPass> jit;
        std::string jerr;
        double t = 0.0;
        if (!jit_prepare_program(dtype, adj_of[i], *progs[i], &jit, &jerr, &t))
            return set_error(QS_ECUDA, ("qs_circuit_compile: " + jerr).c_str());
        secs += t;
        np += (int)progs[i]->passes.size();
    }
    if (compile_seconds) *compile_seconds = secs;
    if (passes) *passes = np;
    return QS_OK;
}

qs_status qs_apply_circuit(qs_state *s, const qs_gate *gates, size_t count, const double *theta, size_t n_theta,
                           int flags) {
    if (!s || s->magic != kStateMagic) return set_error(QS_EINVAL, "state is NULL or not valid");
    if (count > 0 && !gates) return set_error(QS_EINVAL, "qs_apply_circuit: gates is NULL");
    if (flags & ~(QS_FLAG_FUSE | QS_FLAG_GRAPH | QS_FLAG_MASKED | QS_FLAG_JIT))
        return set_error(QS_EINVAL, "qs_apply_circuit: unknown flags");
    if ((flags & QS_FLAG_FUSE) && (flags & QS_FLAG_MASKED))
        return set_error(QS_EINVAL, "qs_apply_circuit: QS_FLAG_MASKED cannot be combined with QS_FLAG_FUSE");
    if ((flags & QS_FLAG_JIT) && !(flags & QS_FLAG_FUSE))
        return set_error(QS_EINVAL, "qs_apply_circuit: QS_FLAG_JIT needs QS_FLAG_FUSE");
    if (s->dtype == QS_Q30 && (flags & QS_FLAG_FUSE))
        return set_error(QS_EUNSUPPORTED, "qs_apply_circuit: fused passes are not built for QS_Q30 states");
    // CUDA graph: one per distinct (gates, theta, flags, buffer, tile size). A recorded one is
    // launched before any validation or planning (its gates passed both when it was recorded):
    // the hash picks the candidate, the stored key bytes must then match exactly.
    std::vector<unsigned char> key_bytes;
    uint64_t key = 0;
    if (flags & QS_FLAG_GRAPH) {
        graph_key_bytes(s, gates, count, theta, n_theta, flags, &key_bytes);
        key = graph_key_hash(key_bytes);
        for (auto &g : s->graphs)
            if (g.key == key && g.bytes == key_bytes) {
                cudaError_t e = cudaGraphLaunch(g.exec, s->stream);
                if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
                return QS_OK;
            }
    }
    std::vector<GatePlan> plans(count);
    char err[256];
    for (size_t i = 0; i < count; ++i)
        if (!plan_record(s, gates[i], theta, n_theta, i, &plans[i], err, sizeof(err)))
            return set_error(QS_EINVAL, err);
    const bool masked = (flags & QS_FLAG_MASKED) != 0;
    // (fixed point rounds every gate: a merged product would round once and differ)
    if (!masked && s->dtype != QS_Q30) merge_runs(s, plans, nullptr, flags);
    fold_phases(s, plans, flags);
    if (masked) {
        // baseline schedule: every pair iteration launched, the controls tested per unit,
        // the general update with the full matrix (as the Section III-A kernel does)
        for (GatePlan &p : plans) {
            GatePlan pm;
            plan_masked(p, &pm);
            std::memcpy(pm.U, p.Ufull, sizeof(pm.U));
            p = pm;
        }
    }
    const bool fuse = (flags & QS_FLAG_FUSE) != 0;
    FusedProgram prog;
    std::vector<JitPass> jit;
    if (fuse) {
        std::vector<unsigned char> pkey = plan_cache_key('F', s, gates, count, n_theta, flags);
        std::vector<uint64_t> sig;
        plans_signature(plans, &sig);
        if (plan_cache_take(pkey, sig, &prog, nullptr, &jit, nullptr)) {
            refresh_matrices(prog, plans, nullptr);
        } else {
            std::vector<int> seq(plans.size());  // after merging: fewer plans than records
            for (size_t i = 0; i < plans.size(); ++i) seq[i] = (int)i;
            plan_fused(s->n, s->dtype, tile_bits(s->dtype, false), seq, plans, nullptr, nullptr, &prog, kPassMaxGates,
                       true, 0, (flags & QS_FLAG_JIT) != 0);
            if (flags & QS_FLAG_JIT) {
                std::string jerr;
                if (!jit_prepare_program(s->dtype, false, prog, &jit, &jerr))
                    return set_error(QS_ECUDA, ("qs_apply_circuit: " + jerr).c_str());
            }
            plan_cache_put(std::move(pkey), std::move(sig), prog, nullptr, jit, nullptr);
        }
    }
    if (flags & QS_FLAG_JIT) {
        cudaError_t e = jit_load(jit);  // before any stream capture below
        if (e != cudaSuccess) return cuda_fail(e, "qs_apply_circuit: loading compiled passes");
    }
    const std::vector<JitPass> *jp = (flags & QS_FLAG_JIT) ? &jit : nullptr;
    const size_t table_bytes = fuse ? program_table_bytes(prog) : 0;
    std::vector<char> table_host(table_bytes);
    if (table_bytes) pack_program_table(prog, table_host.data());

    if (!(flags & QS_FLAG_GRAPH)) {
        if (!fuse) return launch_plans(s, plans, s->stream, masked);
        qs_status st = ensure_device(&s->tile_table, &s->tile_table_bytes, table_bytes, s->stream,
                                     "qs_apply_circuit: cannot allocate the fused gate table");
        if (st != QS_OK) return st;
        if (table_bytes) {
            // stream-ordered: earlier passes on this stream have read the previous table
            cudaError_t e = cudaMemcpyAsync(s->tile_table, table_host.data(), table_bytes, cudaMemcpyHostToDevice,
                                            s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "qs_apply_circuit: gate table upload");
        }
        return launch_program(s, prog, plans, s->tile_table, nullptr, nullptr, nullptr, nullptr, 0, s->stream, jp);
    }

    // CUDA graph not recorded yet (the lookup above missed): record it, keep it, launch it.
    cudaGraphExec_t exec = nullptr;
    {
        cudaError_t e;
        void *table = nullptr;
        if (table_bytes) {
            e = cudaMalloc(&table, table_bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return set_error(QS_ENOMEM, "qs_apply_circuit: cannot allocate the graph's gate table");
            }
            e = cudaMemcpy(table, table_host.data(), table_bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(table);
                return cuda_fail(e, "qs_apply_circuit: gate table upload");
            }
        }
        if (!s->capture_stream) {
            e = cudaStreamCreateWithFlags(&s->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                if (table) cudaFree(table);
                return cuda_fail(e, "capture stream");
            }
        }
        e = cudaStreamBeginCapture(s->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            if (table) cudaFree(table);
            return cuda_fail(e, "cudaStreamBeginCapture");
        }
        qs_status st = fuse ? launch_program(s, prog, plans, table, nullptr, nullptr, nullptr, nullptr, 0,
                                             s->capture_stream, jp)
                            : launch_plans(s, plans, s->capture_stream, masked);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(s->capture_stream, &graph);
        if (st != QS_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (table) cudaFree(table);
            return st != QS_OK ? st : cuda_fail(e, "cudaStreamEndCapture");
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            if (table) cudaFree(table);
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        if (s->graphs.size() >= 16) {  // bounded cache: drop the oldest after the stream is idle
            cudaStreamSynchronize(s->stream);
            cudaGraphExecDestroy(s->graphs.front().exec);
            if (s->graphs.front().table) cudaFree(s->graphs.front().table);
            s->graphs.erase(s->graphs.begin());
        }
        s->graphs.push_back({key, std::move(key_bytes), exec, table});
    }
    cudaError_t e = cudaGraphLaunch(exec, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return QS_OK;
}

qs_status qs_adjoint_grad(qs_state *s, const qs_gate *gates, size_t count, const double *theta, size_t n_theta,
                          double *energy, double *grad, int flags) {
    if (!s || s->magic != kStateMagic) return set_error(QS_EINVAL, "state is NULL or not valid");
    if (count > 0 && !gates) return set_error(QS_EINVAL, "qs_adjoint_grad: gates is NULL");
    if (flags & ~(QS_FLAG_FUSE | QS_FLAG_GRAPH | QS_FLAG_OUT_DEVICE | QS_FLAG_JIT))
        return set_error(QS_EINVAL, "qs_adjoint_grad: unknown flags");
    if ((flags & QS_FLAG_JIT) && !(flags & QS_FLAG_FUSE))
        return set_error(QS_EINVAL, "qs_adjoint_grad: QS_FLAG_JIT needs QS_FLAG_FUSE");
    if (s->dtype == QS_Q30) return set_error(QS_EUNSUPPORTED, "qs_adjoint_grad: not built for QS_Q30 states");
    if (n_theta > 0 && !grad) return set_error(QS_EINVAL, "qs_adjoint_grad: grad is NULL");
    if (n_theta > (size_t)(1 << 24)) return set_error(QS_EINVAL, "qs_adjoint_grad: n_theta too large");
    const bool on_dev = (flags & QS_FLAG_OUT_DEVICE) != 0;
    AdjPlan ap;
    {
        char err[256];
        if (!plan_adjoint_gates(s, gates, count, theta, n_theta, flags, &ap, err, sizeof(err)))
            return set_error(QS_EINVAL, err);
    }
    std::vector<GatePlan> &fwd = ap.fwd, &adj = ap.adj;
    std::vector<int> &slot_of = ap.slot_of, &slot_param = ap.slot_param;
    std::vector<double> &dus = ap.dus;
    std::vector<const double *> &dusp = ap.dusp;
    FusedProgram &pf = ap.pf, &pa = ap.pa;
    const int nslots = (int)slot_param.size();
    const bool fuse = (flags & QS_FLAG_FUSE) != 0;
    std::vector<JitPass> jf, ja;
    const bool use_jit = (flags & QS_FLAG_JIT) != 0;
    if (fuse) {
        std::vector<unsigned char> key = plan_cache_key('A', s, gates, count, n_theta, flags);
        std::vector<uint64_t> sig = adj_signature(ap);
        if (plan_cache_take(key, sig, &pf, &pa, &jf, &ja)) {
            refresh_matrices(pf, fwd, nullptr);
            refresh_matrices(pa, adj, &dusp);
        } else {
            plan_adjoint_programs(s, flags, &ap);
            if (use_jit) {
                std::string jerr;
                if (!jit_prepare_program(s->dtype, false, pf, &jf, &jerr) ||
                    !jit_prepare_program(s->dtype, true, pa, &ja, &jerr))
                    return set_error(QS_ECUDA, ("qs_adjoint_grad: " + jerr).c_str());
            }
            plan_cache_put(std::move(key), std::move(sig), pf, &pa, jf, &ja);
        }
    }

    // Buffers: lambda, partials [nslots][P], slot sums, slot->param map, outputs.
    cudaError_t e;
    if (!s->lam) {
        e = cudaMalloc(&s->lam, s->bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->lam = nullptr;
            return set_error(QS_ENOMEM, "qs_adjoint_grad: cannot allocate the lambda vector");
        }
    }
    const size_t P = adj_partials_per_slot();
    const size_t need = (size_t)nslots * P + (size_t)nslots + (size_t)nslots + n_theta + 64 + 8;
    if (s->grad_scratch_n < need) {
        if (s->grad_scratch) cudaFree(s->grad_scratch);
        s->grad_scratch = nullptr;
        s->grad_scratch_n = 0;
        e = cudaMalloc(&s->grad_scratch, need * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->grad_scratch = nullptr;
            return set_error(QS_ENOMEM, "qs_adjoint_grad: cannot allocate gradient scratch");
        }
        s->grad_scratch_n = need;
    }
    qs_status st = ensure_reduce_scratch(s);
    if (st != QS_OK) return st;
    double *part = s->grad_scratch;
    double *slot_sum = part + (size_t)nslots * P;
    int *slot_param_dev = reinterpret_cast<int *>(slot_sum + nslots);  // nslots ints fit in nslots doubles
    double *grad_dev = slot_sum + 2 * (size_t)nslots;
    double *energy_dev = grad_dev + n_theta;
    cudaStream_t stm = s->stream;

    // Tables of the fused forward and sweep programs (one upload, stream-ordered).
    const size_t bf = fuse ? (program_table_bytes(pf) + 255) & ~size_t(255) : 0;
    const size_t ba = fuse ? program_table_bytes(pa) : 0;
    if (fuse && bf + ba > 0) {
        st = ensure_device(&s->tile_table, &s->tile_table_bytes, bf + ba, stm,
                           "qs_adjoint_grad: cannot allocate the fused gate table");
        if (st != QS_OK) return st;
        std::vector<char> both(bf + ba);
        pack_program_table(pf, both.data());
        pack_program_table(pa, both.data() + bf);
        e = cudaMemcpyAsync(s->tile_table, both.data(), both.size(), cudaMemcpyHostToDevice, stm);
        if (e != cudaSuccess) return cuda_fail(e, "qs_adjoint_grad: gate table upload");
    }
    const void *tab_f = s->tile_table;
    const void *tab_a = tab_f ? static_cast<const char *>(tab_f) + bf : nullptr;
    // Forward pass.
    st = fuse ? launch_program(s, pf, fwd, tab_f, nullptr, nullptr, nullptr, nullptr, 0, stm, use_jit ? &jf : nullptr)
              : launch_plans(s, fwd, stm);
    if (st != QS_OK) return st;
    // Energy and lambda = O psi.
    double *z = s->red_scratch;
    e = launch_expect_z(s->dtype, s->psi, s->n, s->red_scratch + 64, z, nullptr, stm);
    if (e == cudaSuccess) e = launch_sum_vec(z, s->n, (on_dev && energy) ? energy : energy_dev, stm);
    if (e == cudaSuccess) e = launch_obs_sumz(s->dtype, s->psi, s->lam, s->n, stm);
    if (e == cudaSuccess && nslots > 0)
        e = cudaMemsetAsync(part, 0, (size_t)nslots * P * sizeof(double), stm);
    if (e == cudaSuccess && nslots > 0)
        e = cudaMemcpyAsync(slot_param_dev, slot_param.data(), nslots * sizeof(int), cudaMemcpyHostToDevice, stm);
    if (e != cudaSuccess) return cuda_fail(e, "qs_adjoint_grad setup");
    // Reverse sweep.
    if (fuse) {
        st = launch_program(s, pa, adj, tab_a, s->lam, &dusp, &slot_of, part, P, stm, use_jit ? &ja : nullptr);
        if (st != QS_OK) return st;
    } else {
        for (size_t ii = count; ii-- > 0;) {
            const int slot = slot_of[ii];
            e = launch_adj_step(s->dtype, s->psi, s->lam, adj[ii], slot >= 0 ? &dus[8 * slot] : nullptr,
                                slot >= 0 ? part + (size_t)slot * P : nullptr, stm);
            if (e != cudaSuccess) return cuda_fail(e, "qs_adjoint_grad sweep launch");
        }
    }
    e = launch_grad_final(part, nslots, slot_sum, slot_param_dev, on_dev ? grad : grad_dev, (int)n_theta, stm);
    if (e != cudaSuccess) return cuda_fail(e, "qs_adjoint_grad final");
    if (!on_dev) {
        if (n_theta > 0) e = cudaMemcpyAsync(grad, grad_dev, n_theta * sizeof(double), cudaMemcpyDeviceToHost, stm);
        if (e == cudaSuccess && energy)
            e = cudaMemcpyAsync(energy, energy_dev, sizeof(double), cudaMemcpyDeviceToHost, stm);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
        if (e != cudaSuccess) return cuda_fail(e, "qs_adjoint_grad copy-out");
    }
    return QS_OK;
}

}  // extern "C"
