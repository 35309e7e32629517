// qs_batch.cu -- qs_batch_create / qs_batch_run / qs_batch_free: forward energy and adjoint
// gradient of many independent states in one persistent launch, recorded in a CUDA graph.
//
// Host side: every state's gate list is validated; states with identical (n, gate list) share
// one program; a program is the forward gate sequence and the reverse sweep, each planned into
// tile passes (the whole state is one tile when n <= small_bits, otherwise passes of
// tile_bits local qubits). Parameterised gates keep their parameter index; the kernel builds
// their matrices from theta. Tuning (small_bits, tile_bits, max_pass_gates) comes from the
// caller, normally the autotuner; 0 selects the library defaults.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <map>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "k_batch.cuh"
#include "k_batch_major.cuh"
#include "qs_fuse.cuh"
#include "qs_internal.cuh"
#include "qs_jit.cuh"
#include "qs_state.cuh"

namespace qs {
size_t elem_bytes(int dtype);
}  // namespace qs

using namespace qs;

namespace {
constexpr uint32_t kBatchMagic = 0x51534254u;  // "QSBT"
constexpr int kBatchMaxQubits = 30;
constexpr int kBatchMaxParams = 4096;
}  // namespace

// A program of the pass-major path (QS_FLAG_JIT): its states side by side in one buffer, every
// pass run over all of them by a kernel compiled for the pass.
struct BatchJitProg {
    int n = 0, nparam = 0;
    std::vector<int> states;        // global state indices
    qs::FusedProgram pf, pa;        // forward and sweep programs (rotation kinds / indices filled in)
    std::vector<qs::JitPass> jf, ja;
    void *psi = nullptr, *lam = nullptr, *cs = nullptr;
    double *part = nullptr, *obs = nullptr;  // sweep gradient partials, energy partials
    int *d_states = nullptr, *d_csr = nullptr;
    uint64_t *d_items = nullptr;
    std::vector<size_t> pass_off;   // per sweep pass: offset (doubles) of its partials in part
    uint32_t tiles = 1;             // tiles per state
};

struct qs_batch {
    uint32_t magic = kBatchMagic;
    qs_dtype dtype = QS_C64;
    int num_states = 0;
    uint64_t num_params = 0;
    cudaStream_t stream = nullptr;
    BatchArgs args{};
    int grid = 0;
    size_t smem = 0;
    int small_bits = 0, tile_bits = 0, max_pass_gates = 0;
    // device buffers
    void *d_states = nullptr, *d_order = nullptr, *d_progs = nullptr, *d_passes = nullptr, *d_gates = nullptr;
    void *d_groups = nullptr;
    void *workspace = nullptr;
    int *queue = nullptr;
    // graph of (queue reset + kernel) for the last (theta, energy, grad) pointers
    cudaGraphExec_t exec = nullptr;
    const double *g_theta = nullptr;
    double *g_energy = nullptr, *g_grad = nullptr;
    int g_flags = 0;
    cudaStream_t capture_stream = nullptr;
    // pass-major path (QS_FLAG_JIT): programs of the states above small_bits, prepared on first use
    std::vector<BatchJitProg> jprogs;
    std::vector<int32_t> small_order;  // the states at or below small_bits, largest first
    int *d_small_order = nullptr;
    uint64_t *d_param_off = nullptr;
    std::vector<uint64_t> param_off_host;
    bool jit_ready = false;
    double jit_compile_s = 0.0;
};

namespace {

void free_batch(qs_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (BatchJitProg &jp : b->jprogs)
        for (void *p : {jp.psi, jp.lam, jp.cs, (void *)jp.part, (void *)jp.obs, (void *)jp.d_states, (void *)jp.d_csr,
                        (void *)jp.d_items})
            if (p) cudaFree(p);
    if (b->d_small_order) cudaFree(b->d_small_order);
    if (b->d_param_off) cudaFree(b->d_param_off);
    for (void *p : {b->d_states, b->d_order, b->d_progs, b->d_passes, b->d_gates, b->d_groups, b->workspace,
                    (void *)b->queue})
        if (p) cudaFree(p);
    b->magic = 0;
    delete b;
}

template <typename T>
qs_status upload(const std::vector<T> &v, void **dst) {
    const size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return set_error(QS_ENOMEM, "qs_batch_create: device allocation failed");
    }
    if (!v.empty()) {
        e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "qs_batch_create: upload");
    }
    return QS_OK;
}

void dagger8(const double U[8], double D[8]) {
    D[0] = U[0]; D[1] = -U[1];
    D[2] = U[4]; D[3] = -U[5];
    D[4] = U[2]; D[5] = -U[3];
    D[6] = U[6]; D[7] = -U[7];
}

// Plans of one gate for the forward program (fwd) and the sweep (adj).
bool plan_pair(int n, int dtype, const qs_gate &g, int nparam, GatePlan *fwd, GatePlan *adj, char *err, size_t el) {
    double U[8] = {0}, Ud[8] = {0};
    if (g.kind == QS_GATE_RY || g.kind == QS_GATE_RZ) {
        if (g.param < 0 || g.param >= nparam) {
            std::snprintf(err, el, "parameter index %d outside the state's %d parameters", g.param, nparam);
            return false;
        }
        // placeholder matrices (the kernel builds the real ones from theta); only the structure counts
        const int op = g.kind == QS_GATE_RY ? OP_REAL : OP_DIAG;
        U[0] = U[6] = 0.5;
        if (g.kind == QS_GATE_RY) { U[2] = -0.5; U[4] = 0.5; }
        dagger8(U, Ud);
        return plan_gate(n, dtype, g.target, g.ctrl_mask, g.ctrl_vals, U, QS_GATE_U, op, fwd, err, el) &&
               plan_gate(n, dtype, g.target, g.ctrl_mask, g.ctrl_vals, Ud, QS_GATE_U, op, adj, err, el);
    }
    if (g.kind == QS_GATE_X) {
        if (!plan_gate(n, dtype, g.target, g.ctrl_mask, g.ctrl_vals, nullptr, QS_GATE_X, -1, fwd, err, el)) return false;
        *adj = *fwd;
        return true;
    }
    if (g.kind != QS_GATE_U) {
        std::snprintf(err, el, "unknown gate kind %d", g.kind);
        return false;
    }
    if (!plan_gate(n, dtype, g.target, g.ctrl_mask, g.ctrl_vals, g.U, QS_GATE_U, -1, fwd, err, el)) return false;
    dagger8(g.U, Ud);
    if (!plan_gate(n, dtype, g.target, g.ctrl_mask, g.ctrl_vals, Ud, QS_GATE_U, -1, adj, err, el)) return false;
    return true;
}

// Compile the pass-major path's kernels and allocate its buffers (first QS_FLAG_JIT run).
qs_status ensure_jit(qs_batch *b) {
    if (b->jit_ready) return QS_OK;
    const size_t es = elem_bytes(b->dtype), rs = es / 2;
    std::vector<JitRequest> reqs;
    for (BatchJitProg &jp : b->jprogs) {
        reqs.push_back({&jp.pf, false, true, &jp.jf});
        reqs.push_back({&jp.pa, true, true, &jp.ja});
    }
    std::string err;
    if (!reqs.empty() && !jit_prepare_programs(b->dtype, reqs, &err, &b->jit_compile_s))
        return set_error(QS_ECUDA, ("qs_batch_run: " + err).c_str());
    for (BatchJitProg &jp : b->jprogs) {  // loaded before any stream capture records them
        cudaError_t e = jit_load(jp.jf);
        if (e == cudaSuccess) e = jit_load(jp.ja);
        if (e != cudaSuccess) return cuda_fail(e, "qs_batch_run: loading compiled passes");
    }
    auto dev_alloc = [](void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        return true;
    };
    for (BatchJitProg &jp : b->jprogs) {
        const int S = (int)jp.states.size();
        const size_t N = size_t(1) << jp.n;
        jp.tiles = jp.pa.passes.empty() ? (jp.pf.passes.empty() ? 1u : (uint32_t)jp.pf.passes[0].ntiles)
                                        : (uint32_t)jp.pa.passes[0].ntiles;
        // sweep partials: per pass, [J][state][tile]; per parameter, the blocks of its gates
        jp.pass_off.clear();
        size_t total = 0;
        std::vector<std::vector<uint64_t>> items(jp.nparam);
        for (size_t i = 0; i < jp.pa.passes.size(); ++i) {
            const TilePass &P = jp.pa.passes[i];
            jp.pass_off.push_back(total);
            int J = 0;
            for (int g = P.gate_begin; g < P.gate_begin + P.gate_count; ++g) {
                const RegGate &G = jp.pa.gates[g];
                if (G.pkind == 0) continue;
                if (G.slot >= 0 && G.slot < jp.nparam)
                    items[G.slot].push_back(total + (uint64_t)J * S * (uint64_t)P.ntiles);
                ++J;
            }
            total += (size_t)J * S * (size_t)P.ntiles;
            if (P.ntiles != jp.tiles) return set_error(QS_EUNSUPPORTED, "qs_batch_run: passes of unequal tile counts");
        }
        std::vector<int> csr(jp.nparam + 1, 0);
        std::vector<uint64_t> flat;
        for (int q = 0; q < jp.nparam; ++q) {
            csr[q] = (int)flat.size();
            flat.insert(flat.end(), items[q].begin(), items[q].end());
        }
        csr[jp.nparam] = (int)flat.size();
        if (!dev_alloc(&jp.psi, (size_t)S * N * es) || !dev_alloc(&jp.lam, (size_t)S * N * es) ||
            !dev_alloc(&jp.cs, (size_t)S * std::max(1, jp.nparam) * 2 * rs) ||
            !dev_alloc((void **)&jp.part, total * sizeof(double)) ||
            !dev_alloc((void **)&jp.obs, bm_obs_partials(jp.n, S) * sizeof(double)))
            return set_error(QS_ENOMEM, "qs_batch_run: cannot allocate the pass-major state buffers");
        qs_status st;
        if ((st = upload(jp.states, (void **)&jp.d_states)) != QS_OK || (st = upload(csr, (void **)&jp.d_csr)) != QS_OK ||
            (st = upload(flat, (void **)&jp.d_items)) != QS_OK)
            return st;
        jp.pass_off.push_back(total);  // end marker: total partials
    }
    qs_status st;
    if ((st = upload(b->small_order, (void **)&b->d_small_order)) != QS_OK) return st;
    if ((st = upload(b->param_off_host, (void **)&b->d_param_off)) != QS_OK) return st;
    b->jit_ready = true;
    return QS_OK;
}

// Enqueue one pass-major run on `st`: the small states in the persistent kernel, then every
// larger program's passes over all its states.
cudaError_t enqueue_jit(qs_batch *b, const BatchArgs &a0, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (!b->small_order.empty()) {
        BatchArgs a = a0;
        a.order = b->d_small_order;
        a.num_states = (int)b->small_order.size();
        e = cudaMemsetAsync(b->queue, 0, sizeof(int), st);
        if (e == cudaSuccess) e = launch_batch(b->dtype, a, b->grid, b->smem, st);
        if (e != cudaSuccess) return e;
    }
    for (BatchJitProg &jp : b->jprogs) {
        const int S = (int)jp.states.size();
        const uint64_t N = 1ull << jp.n;
        e = launch_bm_init(b->dtype, jp.psi, jp.n, S, jp.cs, jp.nparam, a0.theta, b->d_param_off, jp.d_states, st);
        for (size_t i = 0; e == cudaSuccess && i < jp.pf.passes.size(); ++i)
            e = launch_jit_pass_batched(b->dtype, jp.jf[i], jp.pf, (int)i, jp.psi, nullptr, nullptr, N, S, jp.cs,
                                        2u * (uint32_t)jp.nparam, st);
        if (e == cudaSuccess)
            e = launch_bm_obs(b->dtype, jp.psi, jp.lam, jp.n, S, jp.obs, a0.energy, jp.d_states, st);
        if (e == cudaSuccess && jp.pass_off.back() > 0)
            e = cudaMemsetAsync(jp.part, 0, jp.pass_off.back() * sizeof(double), st);
        for (size_t i = 0; e == cudaSuccess && i < jp.pa.passes.size(); ++i)
            e = launch_jit_pass_batched(b->dtype, jp.ja[i], jp.pa, (int)i, jp.psi, jp.lam, jp.part + jp.pass_off[i], N,
                                        S, jp.cs, 2u * (uint32_t)jp.nparam, st);
        if (e == cudaSuccess)
            e = launch_bm_grad(jp.part, jp.d_csr, jp.d_items, jp.nparam, S, jp.tiles, a0.grad, b->d_param_off,
                               jp.d_states, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

qs_status qs_batch_create(int num_states, const int *n_qubits, const qs_gate *gates, const uint64_t *gate_offsets,
                          const uint64_t *param_offsets, qs_dtype dtype, int small_bits, int tile_bits,
                          int max_pass_gates, void *stream, qs_batch **out) {
    if (!out) return set_error(QS_EINVAL, "qs_batch_create: out is NULL");
    *out = nullptr;
    if (num_states < 1 || !n_qubits || !gate_offsets || !param_offsets)
        return set_error(QS_EINVAL, "qs_batch_create: need num_states >= 1 and the size / offset arrays");
    if (dtype == QS_Q30) return set_error(QS_EUNSUPPORTED, "qs_batch_create: batches are not built for QS_Q30 states");
    if (dtype != QS_C64 && dtype != QS_C128) return set_error(QS_EINVAL, "qs_batch_create: bad dtype");
    const int es = (int)elem_bytes(dtype);
    if (small_bits <= 0) small_bits = dtype == QS_C64 ? 12 : 11;
    if (tile_bits <= 0) tile_bits = dtype == QS_C64 ? 11 : 10;
    if (max_pass_gates <= 0 || max_pass_gates > kTileMaxGates) max_pass_gates = kTileMaxGates;  // its tables' size
    if (small_bits > kTileMaxBits || tile_bits > kTileMaxBits || tile_bits < 5)
        return set_error(QS_EINVAL, "qs_batch_create: small_bits / tile_bits out of range (tile_bits 5..14)");
    if (gate_offsets[0] != 0 || param_offsets[0] != 0) return set_error(QS_EINVAL, "qs_batch_create: offsets must start at 0");
    if (gate_offsets[num_states] > 0 && !gates) return set_error(QS_EINVAL, "qs_batch_create: gates is NULL");

    std::vector<BatchState> states(num_states);
    std::vector<BatchProg> progs;
    std::vector<TilePass> passes;
    std::vector<RegGate> tgates;
    std::vector<TileGroup> tgroups;
    std::map<std::string, int> prog_of;
    std::vector<std::pair<FusedProgram, FusedProgram>> host_progs;  // per program: forward, sweep
    int max_params = 1, max_large_n = 0, max_small_n = 0, smem_bits = 5;
    char err[256], e2[512];
    for (int s = 0; s < num_states; ++s) {
        const int n = n_qubits[s];
        if (n < 1 || n > kBatchMaxQubits) {
            std::snprintf(e2, sizeof(e2), "qs_batch_create: state %d has n=%d outside [1, %d]", s, n, kBatchMaxQubits);
            return set_error(QS_EINVAL, e2);
        }
        if (gate_offsets[s + 1] < gate_offsets[s] || param_offsets[s + 1] < param_offsets[s])
            return set_error(QS_EINVAL, "qs_batch_create: offsets must be non-decreasing");
        const uint64_t np = param_offsets[s + 1] - param_offsets[s];
        if (np > (uint64_t)kBatchMaxParams) return set_error(QS_EINVAL, "qs_batch_create: more than 4096 parameters in a state");
        const qs_gate *gs = gates + gate_offsets[s];
        const size_t gc = gate_offsets[s + 1] - gate_offsets[s];
        std::string key((const char *)&n, sizeof(n));
        key.append((const char *)&np, sizeof(np));
        key.append((const char *)gs, gc * sizeof(qs_gate));
        auto it = prog_of.find(key);
        int pid;
        if (it != prog_of.end()) {
            pid = it->second;
        } else {
            std::vector<GatePlan> fwd(gc), adj(gc);
            std::vector<const double *> dus(gc, nullptr);
            std::vector<int> slots(gc, -1);
            static const double kMarker[8] = {0};
            for (size_t i = 0; i < gc; ++i) {
                if (gs[i].reserved != 0) return set_error(QS_EINVAL, "qs_batch_create: reserved field must be 0");
                if (!plan_pair(n, dtype, gs[i], (int)np, &fwd[i], &adj[i], err, sizeof(err))) {
                    std::snprintf(e2, sizeof(e2), "qs_batch_create: state %d gate %zu: %s", s, i, err);
                    return set_error(QS_EINVAL, e2);
                }
                if (adj[i].op == OP_SIDE) {  // both sides in the sweep (the sweep never skips a side)
                    double Ud[8];
                    dagger8(gs[i].U, Ud);
                    plan_gate(n, dtype, gs[i].target, gs[i].ctrl_mask, gs[i].ctrl_vals, Ud, QS_GATE_U, OP_DIAG, &adj[i],
                              err, sizeof(err));
                }
                if (gs[i].kind == QS_GATE_RY || gs[i].kind == QS_GATE_RZ) {
                    dus[i] = kMarker;
                    slots[i] = gs[i].param;
                }
            }
            // forward program: two consecutive rotations on the same qubit with the same controls
            // (RY then RZ in the ansatz) become one general gate whose matrix the kernel forms
            // per state at staging (u = R2 R1); the sweep keeps every gate for its gradients
            std::vector<GatePlan> fwdm;
            std::vector<std::pair<int, int>> srcm;  // merged plan -> (first gate, second gate or -1)
            for (size_t i = 0; i < gc; ++i) {
                const bool rot = gs[i].kind == QS_GATE_RY || gs[i].kind == QS_GATE_RZ;
                if (rot && i + 1 < gc && (gs[i + 1].kind == QS_GATE_RY || gs[i + 1].kind == QS_GATE_RZ) &&
                    gs[i + 1].target == gs[i].target && gs[i + 1].ctrl_mask == gs[i].ctrl_mask &&
                    gs[i + 1].ctrl_vals == gs[i].ctrl_vals) {
                    static const double kGeneral[8] = {0.5, 0.1, 0.3, 0.0, 0.2, 0.0, 0.4, -0.2};  // structure only
                    GatePlan m;
                    if (!plan_gate(n, dtype, gs[i].target, gs[i].ctrl_mask, gs[i].ctrl_vals, kGeneral, QS_GATE_U, OP_GEN,
                                   &m, err, sizeof(err)))
                        return set_error(QS_EINVAL, err);
                    fwdm.push_back(m);
                    srcm.push_back({(int)i, (int)i + 1});
                    ++i;
                } else {
                    fwdm.push_back(fwd[i]);
                    srcm.push_back({(int)i, -1});
                }
            }
            const bool small = n <= small_bits;
            const int k = small ? n : tile_bits;
            std::vector<int> seqf(fwdm.size()), seq(gc);
            std::iota(seqf.begin(), seqf.end(), 0);
            std::iota(seq.begin(), seq.end(), 0);
            FusedProgram pf, pa;
            // the batch kernel runs kGroupBits-qubit groups forward, kGroupBitsAdjoint in the sweep
            plan_fused(n, dtype, k, seqf, fwdm, nullptr, nullptr, &pf, max_pass_gates, false, kGroupBits);
            std::reverse(seq.begin(), seq.end());
            plan_fused(n, dtype, k, seq, adj, &dus, &slots, &pa, max_pass_gates, false, kGroupBitsAdjoint);
            BatchProg bp{};
            bp.small = small;
            bp.n = n;
            for (int dir = 0; dir < 2; ++dir) {
                FusedProgram &fp = dir ? pa : pf;
                const int base = (int)tgates.size();
                const int gbase = (int)tgroups.size();
                for (TileGroup Gr : fp.groups) {
                    Gr.gate_begin += base;
                    tgroups.push_back(Gr);
                }
                for (size_t gi = 0; gi < fp.gates.size(); ++gi) {
                    RegGate &G = fp.gates[gi];  // rotation fields filled in place (the pass-major path keeps fp)
                    const int first = dir ? fp.gate_src[gi] : srcm[fp.gate_src[gi]].first;
                    const int second = dir ? -1 : srcm[fp.gate_src[gi]].second;
                    const qs_gate &src = gs[first];
                    G.pkind2 = 0;
                    G.pidx2 = 0;
                    if (src.kind == QS_GATE_RY || src.kind == QS_GATE_RZ) {
                        G.pkind = src.kind;
                        G.pidx = src.param;
                        G.slot = dir ? src.param : -1;
                        if (second >= 0) {
                            G.pkind2 = gs[second].kind;
                            G.pidx2 = gs[second].param;
                        }
                    } else {
                        G.slot = -1;
                        G.pkind = 0;
                    }
                    tgates.push_back(G);
                }
                if (dir) bp.adj_begin = (int)passes.size();
                else bp.fwd_begin = (int)passes.size();
                for (TilePass P : fp.passes) {
                    P.gate_begin += base;
                    P.group_begin += gbase;
                    passes.push_back(P);
                }
                if (dir) bp.adj_count = (int)passes.size() - bp.adj_begin;
                else bp.fwd_count = (int)passes.size() - bp.fwd_begin;
            }
            pid = (int)progs.size();
            progs.push_back(bp);
            prog_of.emplace(key, pid);
            host_progs.push_back({std::move(pf), std::move(pa)});
        }
        states[s].n = n;
        states[s].prog = pid;
        states[s].nparam = (int32_t)np;
        states[s].param_off = param_offsets[s];
        max_params = std::max<int>(max_params, (int)np);
        if (n <= small_bits) max_small_n = std::max(max_small_n, n);
        else max_large_n = std::max(max_large_n, n);
    }
    smem_bits = std::max(max_small_n, max_large_n > 0 ? std::min(tile_bits, max_large_n) : 0);
    smem_bits = std::max(smem_bits, 1);
    std::vector<int32_t> order(num_states);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return states[a].n > states[b].n; });

    const size_t smem = batch_smem_bytes(dtype, smem_bits, max_params);
    if (smem > 227 * 1024) return set_error(QS_EINVAL, "qs_batch_create: shared memory per CTA would exceed 227 KB");
    const int grid = batch_grid(dtype, smem);
    if (grid <= 0) return set_error(QS_ECUDA, "qs_batch_create: no resident CTA for this shared memory size");

    qs_batch *b = new (std::nothrow) qs_batch();
    if (!b) return set_error(QS_ENOMEM, "qs_batch_create: host allocation failed");
    b->dtype = dtype;
    b->num_states = num_states;
    b->num_params = param_offsets[num_states];
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    b->grid = grid;
    b->smem = smem;
    b->small_bits = small_bits;
    b->tile_bits = tile_bits;
    b->max_pass_gates = max_pass_gates;
    qs_status st;
    if ((st = upload(states, &b->d_states)) != QS_OK || (st = upload(order, &b->d_order)) != QS_OK ||
        (st = upload(progs, &b->d_progs)) != QS_OK || (st = upload(passes, &b->d_passes)) != QS_OK ||
        (st = upload(tgates, &b->d_gates)) != QS_OK || (st = upload(tgroups, &b->d_groups)) != QS_OK) {
        free_batch(b);
        return st;
    }
    const uint64_t ws_stride = max_large_n > 0 ? (1ull << max_large_n) : 0;
    if (ws_stride) {
        const size_t bytes = (size_t)grid * 2 * ws_stride * es;
        cudaError_t e = cudaMalloc(&b->workspace, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->workspace = nullptr;
            free_batch(b);
            return set_error(QS_ENOMEM, "qs_batch_create: cannot allocate the large-state workspace");
        }
    }
    if (cudaMalloc(&b->queue, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        b->queue = nullptr;
        free_batch(b);
        return set_error(QS_ENOMEM, "qs_batch_create: cannot allocate the work queue");
    }
    // the pass-major path's programs (states above small_bits), compiled on first use
    {
        std::vector<int> jp_of(progs.size(), -1);
        for (int o = 0; o < num_states; ++o) {
            const int s = order[o];
            if (states[s].n <= small_bits) {
                b->small_order.push_back(s);
                continue;
            }
            const int pid = states[s].prog;
            if (jp_of[pid] < 0) {
                jp_of[pid] = (int)b->jprogs.size();
                b->jprogs.emplace_back();
                BatchJitProg &jp = b->jprogs.back();
                jp.n = states[s].n;
                jp.nparam = states[s].nparam;
                jp.pf = host_progs[pid].first;
                jp.pa = host_progs[pid].second;
            }
            b->jprogs[jp_of[pid]].states.push_back(s);
        }
        b->param_off_host.assign(param_offsets, param_offsets + num_states + 1);
    }
    BatchArgs &a = b->args;
    a.states = static_cast<const BatchState *>(b->d_states);
    a.order = static_cast<const int32_t *>(b->d_order);
    a.progs = static_cast<const BatchProg *>(b->d_progs);
    a.passes = static_cast<const TilePass *>(b->d_passes);
    a.gates = static_cast<const RegGate *>(b->d_gates);
    a.groups = static_cast<const TileGroup *>(b->d_groups);
    a.workspace = b->workspace;
    a.ws_stride = ws_stride;
    a.queue = b->queue;
    a.num_states = num_states;
    a.smem_bits = smem_bits;
    a.max_params = max_params;
    *out = b;
    return QS_OK;
}

qs_status qs_batch_run(qs_batch *b, const double *theta, double *energy, double *grad, int flags) {
    if (!b || b->magic != kBatchMagic) return set_error(QS_EINVAL, "qs_batch_run: batch is NULL or not valid");
    if (!theta || !energy || (b->num_params > 0 && !grad))
        return set_error(QS_EINVAL, "qs_batch_run: theta, energy and grad must be device pointers");
    if (flags & ~(QS_FLAG_GRAPH | QS_FLAG_JIT)) return set_error(QS_EINVAL, "qs_batch_run: unknown flags");
    BatchArgs a = b->args;
    a.theta = theta;
    a.energy = energy;
    a.grad = grad;
    const bool jit = (flags & QS_FLAG_JIT) != 0;
    if (jit) {
        qs_status st = ensure_jit(b);
        if (st != QS_OK) return st;
    }
    auto enqueue = [&](cudaStream_t st) -> cudaError_t {
        if (jit) return enqueue_jit(b, a, st);
        cudaError_t e1 = cudaMemsetAsync(b->queue, 0, sizeof(int), st);
        return e1 == cudaSuccess ? launch_batch(b->dtype, a, b->grid, b->smem, st) : e1;
    };
    cudaError_t e;
    if (!(flags & QS_FLAG_GRAPH)) {
        e = enqueue(b->stream);
        return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_batch_run launch");
    }
    if (!b->exec || b->g_theta != theta || b->g_energy != energy || b->g_grad != grad || b->g_flags != flags) {
        if (b->exec) {
            cudaStreamSynchronize(b->stream);
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        if (!b->capture_stream) {
            e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "qs_batch_run: capture stream");
        }
        e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "qs_batch_run: begin capture");
        cudaError_t e2 = enqueue(b->capture_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->capture_stream, &graph);
        if (e2 != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e2 != cudaSuccess ? e2 : e, "qs_batch_run: capture");
        }
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(e, "qs_batch_run: instantiate");
        }
        b->g_theta = theta;
        b->g_energy = energy;
        b->g_grad = grad;
        b->g_flags = flags;
    }
    e = cudaGraphLaunch(b->exec, b->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_batch_run: graph launch");
}

qs_status qs_batch_info(const qs_batch *b, int *grid, int *small_bits, int *tile_bits, int *max_pass_gates,
                        size_t *smem_bytes, size_t *workspace_bytes) {
    if (!b || b->magic != kBatchMagic) return set_error(QS_EINVAL, "qs_batch_info: batch is NULL or not valid");
    if (grid) *grid = b->grid;
    if (small_bits) *small_bits = b->small_bits;
    if (tile_bits) *tile_bits = b->tile_bits;
    if (max_pass_gates) *max_pass_gates = b->max_pass_gates;
    if (smem_bytes) *smem_bytes = b->smem;
    if (workspace_bytes) *workspace_bytes = b->args.ws_stride * 2 * (size_t)b->grid * elem_bytes(b->dtype);
    return QS_OK;
}

qs_status qs_batch_bytes(const qs_batch *b, double *algorithmic_bytes) {
    if (!b || b->magic != kBatchMagic) return set_error(QS_EINVAL, "qs_batch_bytes: batch is NULL or not valid");
    if (!algorithmic_bytes) return set_error(QS_EINVAL, "qs_batch_bytes: output is NULL");
    // states in shared memory move nothing through HBM; a larger state: |0...0> written, every
    // forward pass reads and writes the tiles its gates select, lambda = O psi reads psi and
    // writes lambda, every sweep pass reads and writes the selected tiles of psi and lambda
    double total = 0.0;
    const double es = (double)elem_bytes(b->dtype);
    for (const BatchJitProg &jp : b->jprogs) {
        const double state = std::ldexp(es, jp.n);
        double per = 3.0 * state;
        for (size_t i = 0; i < jp.pf.passes.size(); ++i) per += 2.0 * state * pass_touched_fraction(jp.pf, (int)i);
        for (size_t i = 0; i < jp.pa.passes.size(); ++i) per += 4.0 * state * pass_touched_fraction(jp.pa, (int)i);
        total += per * (double)jp.states.size();
    }
    *algorithmic_bytes = total;
    return QS_OK;
}

qs_status qs_batch_free(qs_batch *b) {
    if (!b) return QS_OK;
    if (b->magic != kBatchMagic) return set_error(QS_EINVAL, "qs_batch_free: batch is not valid");
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    cudaGetLastError();
    return QS_OK;
}

}  // extern "C"
