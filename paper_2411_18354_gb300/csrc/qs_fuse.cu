// qs_fuse.cu -- host planner that groups consecutive gates into fused tile passes.
//
// A pass keeps the lowest b qubits local (b = 4 for complex64, 3 for complex128, so that tile
// rows are 128 bytes of contiguous memory) and takes a run of consecutive gates whose targets
// fit in k local qubits. A gate's controls need not be local: non-local controls become the
// gate's tile predicate. Costs are in units of one full read + write of the state: a separate
// launch of a gate costs the fraction of 64-byte DRAM units it touches; a pass costs the
// fraction of tiles it touches (union bound over its gates' tile predicates) plus a per-gate
// compute cost inside the tile (measured: about 0.15 for complex64, whose gates are
// memory-bound; complex128 arithmetic gates are FP64-bound alone or in a pass, so there mostly
// exchanges join passes). A run of diagonal gates can also go to one k_diag_run launch (up to
// 64 gates; an uncontrolled gate just before the run can lead it), which costs one read +
// write of the chunks the run can change. The gate sequence is cut into single launches,
// passes and diagonal runs of least total modelled cost (dynamic programming over where each
// segment ends); where every gate must go into a pass, each pass takes as many gates as fit.
// The local set is finally padded with the lowest free qubits up to k.
#include <algorithm>
#include <cstdio>
#include <iterator>
#include <cstring>
#include <vector>

#include "k_tile.cuh"
#include "qs_fuse.cuh"

#ifndef QS_FOLD_EXCHANGES
#define QS_FOLD_EXCHANGES 1
#endif

namespace qs {

static int popc(uint64_t v) { return __builtin_popcountll(v); }

// Fraction of the state a separate k_gate launch moves, counted in 64-byte DRAM units:
// controls on the qubits inside one unit do not reduce it.
// Every launch also pays ~2 us of fixed latency (start and drain, back to back in a graph): in
// units of one state read + write at ~6 TB/s it decides small states (one pass for a whole
// state that fits a tile) and hardly matters from n ~ 24 on.
double launch_latency_cost(int n, int dtype) {
    return 2e-6 / (std::ldexp(2.0 * (dtype == QS_C64 ? 8.0 : 16.0), n) / 6.0e12);
}

double single_launch_cost(const GatePlan &p, int dtype) {
    const int unit_bits = dtype == QS_C64 ? 3 : 2;
    const uint64_t high = p.ctrl_mask & ~((1ull << unit_bits) - 1ull);
    return std::ldexp(1.0, -popc(high));
}

// A gate of a pass in local coordinates (before grouping).
struct LocalGate {
    int t;                 // local target position
    uint32_t cm, cv;       // local controls (local index bits) and their values
    uint64_t hmask, hvals; // non-local controls
    int op, side;
    double U[8];
};

static LocalGate make_local_gate(const GatePlan &p, uint64_t Lmask, const int *local_of) {
    LocalGate g;
    std::memset(&g, 0, sizeof(g));
    g.t = local_of[p.t];
    uint64_t lc = p.ctrl_mask & Lmask;
    while (lc) {
        const int q = __builtin_ctzll(lc);
        lc &= lc - 1;
        g.cm |= 1u << local_of[q];
        if ((p.ctrl_vals >> q) & 1ull) g.cv |= 1u << local_of[q];
    }
    g.hmask = p.ctrl_mask & ~Lmask;
    g.hvals = p.ctrl_vals & g.hmask;
    g.op = p.op;
    g.side = p.side;
    std::memcpy(g.U, p.U, sizeof(g.U));
    return g;
}

// ---------------------------------------------------------------------------------------------
// Gate order
// ---------------------------------------------------------------------------------------------
// A circuit may run in any order that keeps every pair of gates that might not commute in its
// given order. Sufficient for two gates to commute: each qubit they share is, in both of them,
// a control or a qubit of a diagonal gate. In the computational basis of the shared qubits both
// are then block diagonal, and the blocks act on disjoint qubits. (The rule is structural: it
// holds for every value of a rotation angle, since a rotation's kind fixes which qubits it is
// diagonal on.) Per qubit this gives the dependencies: a gate that is not diagonal on the
// qubit follows the last such gate and every gate that used the qubit since; any other use
// follows the last gate that is not diagonal on it.
struct OrderItem {
    int t;        // target position; -1: the gate changes nothing (no dependencies)
    uint64_t q;   // positions the gate uses (target and controls)
    uint64_t nd;  // positions on which it is not diagonal (its target, unless it is diagonal)
    bool param;   // counts against the parameter limit of a block
};

// List scheduling into blocks of at most K target positions (always those in `forced`),
// max_items items and max_param parameterised items. A block takes every item that is ready
// (all its predecessors placed) and has its target in the block, repeatedly; when none is
// left it adds the position whose closure (the items adding it would make takeable, directly
// or through the items they release) is largest, ties to the position whose closure holds the
// earliest item, until the block is full or nothing more can join. Items keep their given
// order as the priority. Returns the items in execution order.
static std::vector<int> block_schedule(const std::vector<OrderItem> &it, int npos, int K, uint64_t forced,
                                       int max_items, int max_param) {
    const int N = (int)it.size();
    std::vector<std::vector<int>> succ(N);
    std::vector<int> indeg(N, 0), stamp(N, -1), last_nd(npos, -1);
    std::vector<std::vector<int>> since(npos);
    for (int i = 0; i < N; ++i) {
        auto dep = [&](int d) {
            if (d >= 0 && stamp[d] != i) {
                stamp[d] = i;
                succ[d].push_back(i);
                ++indeg[i];
            }
        };
        for (uint64_t m = it[i].q; m; m &= m - 1) {
            const int b = __builtin_ctzll(m);
            dep(last_nd[b]);
            if ((it[i].nd >> b) & 1ull)
                for (int d : since[b]) dep(d);
        }
        for (uint64_t m = it[i].q; m; m &= m - 1) {
            const int b = __builtin_ctzll(m);
            if ((it[i].nd >> b) & 1ull) {
                last_nd[b] = i;
                since[b].clear();
            } else {
                since[b].push_back(i);
            }
        }
    }
    auto fits = [&](int i, uint64_t S) { return it[i].t < 0 || ((S >> it[i].t) & 1ull); };
    std::vector<int> ready;  // sorted ascending (priority = given order)
    for (int i = 0; i < N; ++i)
        if (indeg[i] == 0) ready.push_back(i);
    std::vector<int> order, released, dec(N, 0), touched, stack;
    order.reserve(N);
    while (!ready.empty()) {
        uint64_t S = forced;
        int count = 0, np = 0;
        while (true) {
            // take every ready item that fits, until none is left (taking releases others)
            bool progress = true;
            while (progress && count < max_items) {
                progress = false;
                released.clear();
                std::vector<int> keep;
                keep.reserve(ready.size());
                for (int i : ready) {
                    if (count < max_items && fits(i, S) && !(it[i].param && np >= max_param)) {
                        order.push_back(i);
                        ++count;
                        np += it[i].param;
                        for (int s : succ[i])
                            if (--indeg[s] == 0) released.push_back(s);
                        progress = true;
                    } else {
                        keep.push_back(i);
                    }
                }
                std::sort(released.begin(), released.end());
                ready.clear();
                std::merge(keep.begin(), keep.end(), released.begin(), released.end(), std::back_inserter(ready));
            }
            if (count >= max_items || popc(S) >= K) break;
            uint64_t cand = 0;
            for (int i : ready)
                if (it[i].t >= 0 && !((S >> it[i].t) & 1ull)) cand |= 1ull << it[i].t;
            int best = -1, best_got = 0, best_first = N;
            for (uint64_t m = cand; m; m &= m - 1) {
                const int b = __builtin_ctzll(m);
                const uint64_t S2 = S | (1ull << b);
                int got = 0, gp = np, first = N;
                stack.clear();
                for (int i : ready)
                    if (fits(i, S2)) stack.push_back(i);
                while (!stack.empty() && count + got < max_items) {
                    const int i = stack.back();
                    stack.pop_back();
                    if (it[i].param && gp >= max_param) continue;
                    ++got;
                    gp += it[i].param;
                    first = std::min(first, i);
                    for (int s : succ[i]) {
                        if (dec[s]++ == 0) touched.push_back(s);
                        if (dec[s] == indeg[s] && fits(s, S2)) stack.push_back(s);
                    }
                }
                for (int s : touched) dec[s] = 0;
                touched.clear();
                if (got > best_got || (got == best_got && got > 0 && first < best_first)) {
                    best = b;
                    best_got = got;
                    best_first = first;
                }
            }
            if (best < 0) break;
            S |= 1ull << best;
        }
        if (count == 0) {  // nothing could join (limits below one item): place the first alone
            const int i = ready.front();
            ready.erase(ready.begin());
            order.push_back(i);
            released.clear();
            for (int s : succ[i])
                if (--indeg[s] == 0) released.push_back(s);
            std::sort(released.begin(), released.end());
            std::vector<int> merged;
            std::merge(ready.begin(), ready.end(), released.begin(), released.end(), std::back_inserter(merged));
            ready.swap(merged);
        }
    }
    return order;
}

// Choose the group qubits Q (r of them, containing the targets S): the rows of a warp vary
// the lowest local qubits outside Q, and for shared-memory accesses without bank conflicts
// the lowest `sw` of those must land on distinct low bits after the swizzle (qubit b lands on
// b mod sw). Pads S with the lowest positions that keep that property, else with the best
// found.
static uint32_t choose_group(uint32_t S, int k, int r, int sw) {
    auto score = [&](uint32_t Q) {
        int seen = 0, distinct = 0, taken = 0;
        for (int b = 0; b < k && taken < sw; ++b) {
            if ((Q >> b) & 1u) continue;
            ++taken;
            const int res = b % sw;
            if (!((seen >> res) & 1)) {
                seen |= 1 << res;
                ++distinct;
            }
        }
        return (taken - distinct);  // colliding lanes; 0 = conflict-free
    };
    const int need = r - __builtin_popcount(S);
    if (need <= 0) return S;
    std::vector<int> free_pos;
    for (int b = 0; b < k; ++b)
        if (!((S >> b) & 1u)) free_pos.push_back(b);
    uint32_t best = 0;
    int best_score = 1 << 30;
    // combinations of `need` free positions, lexicographic (lowest first)
    std::vector<int> idx(need);
    for (int i = 0; i < need; ++i) idx[i] = i;
    const int m = (int)free_pos.size();
    while (true) {
        uint32_t Q = S;
        for (int i = 0; i < need; ++i) Q |= 1u << free_pos[idx[i]];
        const int sc = score(Q);
        if (sc < best_score) {
            best_score = sc;
            best = Q;
            if (sc == 0) break;
        }
        int i = need - 1;
        while (i >= 0 && idx[i] == m - need + i) --i;
        if (i < 0) break;
        ++idx[i];
        for (int j = i + 1; j < need; ++j) idx[j] = idx[j - 1] + 1;
    }
    return best;
}

// Split a pass's gates into register groups and append them to the program.
// Register groups a pass's gates form in this order: runs of consecutive gates with at most r
// distinct targets.
static int count_groups(const std::vector<LocalGate> &lg, int r) {
    int groups = 0;
    size_t i = 0;
    while (i < lg.size()) {
        uint32_t S = 0;
        while (i < lg.size() && popc(S | (1u << lg[i].t)) <= r) S |= 1u << lg[i++].t;
        ++groups;
    }
    return groups;
}

// The pass's gates in an order of fewer register groups where the gate order allows it (the
// commutation rule of block_schedule on the local positions: non-local controls are controls
// of every gate that has them, so they never order two gates).
static void order_for_groups(std::vector<LocalGate> &lg, std::vector<int> &slots, std::vector<const double *> &ds,
                             std::vector<int> &src, int k, int r) {
    if (lg.size() < 3) return;
    uint32_t targets = 0;
    for (const LocalGate &g : lg) targets |= 1u << g.t;
    const int in_order = count_groups(lg, r);
    if (in_order <= (popc(targets) + r - 1) / r) return;  // no order needs fewer groups
    std::vector<OrderItem> items(lg.size());
    for (size_t i = 0; i < lg.size(); ++i) {
        const LocalGate &g = lg[i];
        const bool diag = g.op == OP_DIAG || g.op == OP_SIDE;
        items[i] = {g.t, (1ull << g.t) | (uint64_t)g.cm, diag ? 0ull : (1ull << g.t), false};
    }
    const std::vector<int> ord = block_schedule(items, k, r, 0, (int)lg.size(), (int)lg.size());
    std::vector<LocalGate> lg2(lg.size());
    for (size_t i = 0; i < ord.size(); ++i) lg2[i] = lg[ord[i]];
    if (count_groups(lg2, r) >= in_order) return;
    std::vector<int> slots2(lg.size()), src2(lg.size());
    std::vector<const double *> ds2(lg.size());
    for (size_t i = 0; i < ord.size(); ++i) {
        slots2[i] = slots[ord[i]];
        src2[i] = src[ord[i]];
        ds2[i] = ds[ord[i]];
    }
    lg.swap(lg2);
    slots.swap(slots2);
    src.swap(src2);
    ds.swap(ds2);
}

static void add_groups(std::vector<LocalGate> lg, std::vector<int> slots, std::vector<const double *> ds,
                       std::vector<int> src, int k, int dtype, int group_bits, FusedProgram *prog, TilePass *P) {
    const int r = std::min(group_bits, k);
    const int sw = dtype == QS_C64 ? 4 : 3;
    order_for_groups(lg, slots, ds, src, k, r);
    prog->order.insert(prog->order.end(), src.begin(), src.end());  // the executed order
    P->group_begin = (int)prog->groups.size();
    P->gate_begin = (int)prog->gates.size();
    bool folded = false;
    size_t i = 0;
    while (i < lg.size()) {
        uint32_t S = 0;
        size_t j = i;
        while (j < lg.size()) {
            const uint32_t S2 = S | (1u << lg[j].t);
            if (__builtin_popcount(S2) > r) break;
            S = S2;
            ++j;
        }
        const uint32_t Q = choose_group(S, k, r, sw);
        TileGroup Gr;
        std::memset(&Gr, 0, sizeof(Gr));
        Gr.r = (uint8_t)r;
        int pos[kGroupBits], m = 0, place[kTileMaxBits];
        for (int b = 0; b < k; ++b) {
            place[b] = -1;
            if ((Q >> b) & 1u) {
                place[b] = m;
                pos[m++] = b;
                Gr.q[m - 1] = (uint8_t)b;
            }
        }
        IndexMap map;
        build_map(k, pos, m, 0, &map);
        Gr.nrseg = (uint8_t)map.nseg;
        for (int s = 0; s < map.nseg; ++s) {
            Gr.rmask[s] = (uint32_t)map.mask[s];
            Gr.rshift[s] = (uint8_t)map.shift[s];
        }
        Gr.gate_begin = (int)prog->gates.size();
        for (int q = 0; q < kGroupBits; ++q) Gr.qsw[q] = q < m ? tile_swizzle(1u << Gr.q[q], sw) : 0u;
        std::vector<RegGate> rg;
        std::vector<int> rsrc;
        for (size_t g = i; g < j; ++g) {
            const LocalGate &L = lg[g];
            RegGate R;
            std::memset(&R, 0, sizeof(R));
            R.p = (uint8_t)place[L.t];
            for (int b = 0; b < k; ++b) {
                if (!((L.cm >> b) & 1u)) continue;
                const int val = (L.cv >> b) & 1u;
                if (place[b] >= 0) {
                    R.cqm |= (uint8_t)(1u << place[b]);
                    R.cqv |= (uint8_t)(val << place[b]);
                } else {
                    R.crm |= 1u << b;
                    R.crv |= (uint32_t)val << b;
                }
            }
            R.hmask = L.hmask;
            R.hvals = L.hvals;
            R.op = L.op;
            R.side = L.side;
            R.slot = slots[g];
            std::memcpy(R.U, L.U, sizeof(R.U));
            for (int q = 0; q < 8; ++q) R.Uf[q] = (float)R.U[q];
            if (ds[g]) {
                std::memcpy(R.D, ds[g], sizeof(R.D));
                for (int q = 0; q < 8; ++q) R.Df[q] = (float)R.D[q];
            }
            rg.push_back(R);
            rsrc.push_back(src[g]);
        }
        // leading and trailing exchanges with all controls in the group: a permutation of the
        // 2^m elements, applied by the row copies (gather / scatter offsets) instead of gates
        auto foldable = [&](const RegGate &R) {
            return QS_FOLD_EXCHANGES && m == r && m == group_bits && R.op == OP_SWAP && R.crm == 0 && R.hmask == 0 &&
                   R.slot < 0;
        };
        size_t lead = 0, trail = 0;
        while (lead < rg.size() && foldable(rg[lead])) ++lead;
        while (trail < rg.size() - lead && foldable(rg[rg.size() - 1 - trail])) ++trail;
        auto apply_x = [](const RegGate &R, uint32_t x) {
            return ((x & R.cqm) == R.cqv) ? (x ^ (1u << R.p)) : x;
        };
        auto offset = [&](uint32_t x) {
            uint32_t o = 0;
            for (int q = 0; q < m; ++q)
                if ((x >> q) & 1u) o ^= Gr.qsw[q];
            return (uint16_t)o;
        };
        const uint32_t E = 1u << m;
        if (lead > 0) {  // element e of the row receives the amplitude that the exchanges move to e
            Gr.has_g = 1;
            for (uint32_t x = 0; x < E; ++x) {
                uint32_t y = x;
                for (size_t g = 0; g < lead; ++g) y = apply_x(rg[g], y);
                Gr.gperm[y] = offset(x);
            }
        }
        if (trail > 0) {  // element e goes where the exchanges move it
            Gr.has_s = 1;
            for (uint32_t x = 0; x < E; ++x) {
                uint32_t y = x;
                for (size_t g = rg.size() - trail; g < rg.size(); ++g) y = apply_x(rg[g], y);
                Gr.sperm[x] = offset(y);
            }
        }
        for (size_t g = lead; g < rg.size() - trail; ++g) {
            prog->gates.push_back(rg[g]);
            prog->gate_src.push_back(rsrc[g]);
        }
        Gr.gate_count = (int)prog->gates.size() - Gr.gate_begin;
        for (int g = Gr.gate_begin; g < Gr.gate_begin + Gr.gate_count; ++g) Gr.hctrl |= prog->gates[g].hmask != 0;
        P->hctrl |= Gr.hctrl;
        folded |= Gr.has_g || Gr.has_s;
        prog->groups.push_back(Gr);
        i = j;
    }
    // folded exchanges act on every tile: the pass may then skip no tile
    if (folded) P->hctrl = 0;
    P->group_count = (int)prog->groups.size() - P->group_begin;
    P->gate_count = (int)prog->gates.size() - P->gate_begin;
}

static void make_pass(int n, uint64_t Lmask, TilePass *P) {
    std::memset(P, 0, sizeof(*P));
    P->n = n;
    P->k = popc(Lmask);
    int local = 0, nr = 0;
    for (int q = 0; q < n; ++q) {
        if (!((Lmask >> q) & 1ull)) continue;
        if (nr > 0 && P->run_dst[nr - 1] + P->run_len[nr - 1] == q) {
            P->run_len[nr - 1]++;
        } else {
            P->run_src[nr] = (uint8_t)local;
            P->run_dst[nr] = (uint8_t)q;
            P->run_len[nr] = 1;
            ++nr;
        }
        ++local;
    }
    P->nruns = nr;
    int pos[64];
    int m = 0;
    for (int q = 0; q < n; ++q)
        if ((Lmask >> q) & 1ull) pos[m++] = q;
    IndexMap map;
    build_map(n, pos, m, 0, &map);
    P->tnseg = map.nseg;
    for (int s = 0; s < map.nseg; ++s) {
        P->tmask[s] = map.mask[s];
        P->tshift[s] = map.shift[s];
    }
    P->ntiles = 1ull << (n - P->k);
}

// Compute cost a gate adds inside a pass, in units of one state read + write. complex64,
// measured at n = 24 (2^12-amplitude tiles, one state read + write = 45 us): 8-13 us per gate
// whatever its kind (general 11.3, real 9.1, exchange 8.2 unless folded into a register
// group's gather / scatter, diagonal about as much: the interpreter's per-gate work, not the
// arithmetic, sets it), also for gates whose non-local controls select only some tiles;
// 0.15 fits the measured plans best. complex128 gates are FP64-bound alone and inside a pass
// alike (a general 2x2 costs ~3 units either way), so only exchanges (no arithmetic, ~0.33)
// gain from a pass.
static double pass_gate_cost(int dtype, const GatePlan &p, bool jit) {
    if (dtype == QS_C64 && !jit) return 0.15;
    if (dtype == QS_C64) {
        // passes compiled for their shape (QS_FLAG_JIT), measured at n = 24 in units of one
        // state read + write (45 us): general 2x2 5.8 us, real 2.8, exchange 1.8, diagonal and
        // one-sided less; a gate computes only the pairs its controls select (in-row controls
        // skip the arithmetic, row predicates most of it)
        double c = p.op == OP_GEN ? 0.13 : p.op == OP_REAL ? 0.065 : p.op == OP_SWAP ? 0.04 : 0.035;
        return c * std::max(std::ldexp(1.0, -popc(p.ctrl_mask)), 0.125);
    }
    return p.op == OP_SWAP ? 0.33 : 3.0;
}

// Compute cost of one diagonal gate inside a k_diag_run launch (its factor is formed once per
// chunk of 8 amplitudes, or once per warp): small against the launch's state read + write.
static double diag_run_gate_cost(int dtype) { return dtype == QS_C64 ? 0.005 : 0.02; }

enum { SEG_SINGLE, SEG_PASS, SEG_DIAG, SEG_LEAD_DIAG, SEG_NONE };

// A cut of the gate sequence into segments: [i, cut[i]) of kind kind[i], from i = 0 on, and
// the modelled cost of the whole.
struct Segments {
    bool done = false;
    double cost = 0.0;
    std::vector<size_t> cut;
    std::vector<char> kind;
};

// The planner proper, gates in the order seq gives: cuts the sequence (into `sg`, unless it is
// already cut) and, with `prog`, emits the program.
static void plan_in_order(int n, int dtype, int k, const std::vector<int> &seq, const std::vector<GatePlan> &plans,
                          const std::vector<const double *> *dus, const std::vector<int> *gslots, FusedProgram *prog,
                          int max_gates, bool allow_single, int group_bits, bool jit, Segments *sg) {
    if (prog) {
        prog->order.clear();
        prog->ops.clear();
        prog->passes.clear();
        prog->gates.clear();
        prog->groups.clear();
        prog->gate_src.clear();
        prog->druns.clear();
        prog->dgates.clear();
        prog->model_cost = 0.0;
    }
    max_gates = std::max(1, std::min(max_gates, kPassMaxGates));
    // k >= b0 + 1 so that any single target fits next to the b0 low qubits (n permitting)
    const int b0 = dtype == QS_C64 ? 4 : 3;
    k = std::min(std::min(std::max(k, b0 + 1), kTileMaxBits), n);
    const int b = std::min(k, b0);
    const uint64_t low = (b >= 64) ? ~0ull : ((1ull << b) - 1ull);
    const bool adjoint = dus != nullptr;
    const bool diag_runs = !adjoint && allow_single && n >= kDiagChunkBits;
    auto is_param = [&](int g) { return adjoint && (*dus)[g] != nullptr; };
    const size_t N = seq.size();
    // per position: target bit (0: changes nothing), controls, parameter, per-gate pass cost
    std::vector<uint64_t> tbit_of(N), ctrl_of(N);
    std::vector<char> param_of(N);
    std::vector<double> cost_of(N);
    for (size_t j = 0; j < N; ++j) {
        const GatePlan &p = plans[seq[j]];
        const bool param = is_param(seq[j]);
        const bool real = p.units != 0 || param;
        tbit_of[j] = real ? (1ull << p.t) : 0ull;
        ctrl_of[j] = p.ctrl_mask;
        param_of[j] = param;
        cost_of[j] = real ? pass_gate_cost(dtype, p, jit) * (param && jit ? 1.5 : 1.0) : 0.0;
    }
    // Take gates seq[i], seq[i + 1], ... (before `end`) into one pass while its targets fit in
    // k local qubits and the gate and parameter limits allow; visit(j, frac, compute, real)
    // after gate j joined: frac = fraction of tiles touched (union bound over the gates' tile
    // predicates), compute = summed per-gate cost, real = non-identity gates so far.
    auto extend = [&](size_t i0, size_t end, auto &&visit) {
        uint64_t L = low;
        double frac = 0.0, compute = 0.0;
        int nparam = 0, real = 0, count = 0;
        const size_t stop = std::min(end, i0 + (size_t)max_gates);
        for (size_t j = i0; j < stop; ++j) {
            if (tbit_of[j]) {
                const uint64_t L2 = L | tbit_of[j];
                if (L2 != L && popc(L2) > k) break;
                if (param_of[j] && nparam >= kTileMaxParam) break;
                if (frac < 1.0) frac = std::min(1.0, frac + std::ldexp(1.0, -popc(ctrl_of[j] & ~L2)));
                compute += cost_of[j];
                L = L2;
                nparam += param_of[j];
                ++real;
            }
            ++count;
            visit(j, frac, compute, real);
        }
    };
    // One pass of gates seq[a, b) (identities skipped), its local set padded with the lowest
    // free qubits.
    auto emit_pass = [&](size_t a, size_t b) {
        uint64_t L = low;
        for (size_t j = a; j < b; ++j)
            if (plans[seq[j]].units != 0 || is_param(seq[j])) L |= 1ull << plans[seq[j]].t;
        for (int q = 0; q < n && popc(L) < k; ++q) L |= 1ull << q;
        int local_of[64];
        for (int q = 0, l = 0; q < n; ++q) local_of[q] = ((L >> q) & 1ull) ? l++ : -1;
        TilePass P;
        make_pass(n, L, &P);
        std::vector<LocalGate> lg;
        std::vector<int> slots, src;
        std::vector<const double *> ds;
        for (size_t j = a; j < b; ++j) {
            const int mbr = seq[j];
            if (plans[mbr].units == 0 && !is_param(mbr)) continue;
            LocalGate g = make_local_gate(plans[mbr], L, local_of);
            const double *d = nullptr;
            int slot = -1;
            if (is_param(mbr)) {
                if (g.op != OP_GEN && g.op != OP_DIAG && g.op != OP_REAL) g.op = OP_GEN;
                d = (*dus)[mbr];
                slot = P.nparam;
                P.param_gslot[P.nparam++] = (*gslots)[mbr];
            }
            lg.push_back(g);
            slots.push_back(slot);
            ds.push_back(d);
            src.push_back(mbr);
        }
        add_groups(lg, slots, ds, src, P.k, dtype, group_bits > 0 ? group_bits : (adjoint ? kGroupBitsAdjoint : kGroupBits),
                   prog, &P);
        prog->ops.push_back({(int)prog->passes.size(), -1});
        prog->passes.push_back(P);
    };
    auto is_diag = [&](int g) { return plans[g].op == OP_DIAG || plans[g].op == OP_SIDE; };
    // Diagonal gates seq[a, b) (identities skipped) in k_diag_run launches of at most
    // kDiagMaxGates gates; lead >= 0: that uncontrolled gate goes first in the first launch.
    auto emit_diag = [&](size_t a, size_t b, int lead) {
        std::vector<DiagGate> run;
        if (lead >= 0) prog->order.push_back(lead);
        for (size_t q = a; q < b; ++q) {
            const GatePlan &p = plans[seq[q]];
            if (p.units == 0) continue;
            prog->order.push_back(seq[q]);
            DiagGate dg;
            make_diag_gate(p, &dg);
            run.push_back(dg);
        }
        for (size_t q0 = 0; q0 < run.size(); q0 += kDiagMaxGates) {
            const size_t q1 = std::min(run.size(), q0 + kDiagMaxGates);
            DiagRun r;
            r.begin = (int)prog->dgates.size();
            r.count = (int)(q1 - q0);
            const int lt = (q0 == 0 && lead >= 0) ? plans[lead].t : -1;
            r.nc = assign_diag_classes(run.data() + q0, r.count, n, lt);
            if (lt >= 0) std::memcpy(r.nc.lu, plans[lead].Ufull, sizeof(r.nc.lu));
            prog->dgates.insert(prog->dgates.end(), run.begin() + q0, run.begin() + q1);
            prog->ops.push_back({-1, -1, (int)prog->druns.size()});
            prog->druns.push_back(r);
        }
    };
    // emit the program of a cut sequence
    auto emit_all = [&](const Segments &S) {
        prog->model_cost = S.cost;
        for (size_t i = 0; i < N; i = S.cut[i]) {
            switch (S.kind[i]) {
            case SEG_PASS:
                emit_pass(i, S.cut[i]);
                break;
            case SEG_DIAG:
                emit_diag(i, S.cut[i], -1);
                break;
            case SEG_LEAD_DIAG:
                emit_diag(i + 1, S.cut[i], seq[i]);
                break;
            case SEG_SINGLE:
                if (plans[seq[i]].units != 0 || is_param(seq[i])) {
                    prog->ops.push_back({-1, seq[i]});
                    prog->order.push_back(seq[i]);
                }
                break;
            default:
                break;
            }
        }
    };
    if (sg->done) {
        if (prog) emit_all(*sg);
        return;
    }
    sg->cut.assign(N + 1, N);
    sg->kind.assign(N + 1, SEG_NONE);
    sg->cost = 0.0;
    if (!allow_single) {  // every gate goes into a pass: each pass takes as many as fit
        size_t i = 0;
        while (i < N) {
            size_t e = i;
            double cost = 0.0;
            int nreal = 0;
            extend(i, N, [&](size_t j, double frac, double compute, int real) {
                e = j;
                cost = frac + compute;
                nreal = real;
            });
            sg->cut[i] = e + 1;
            if (nreal > 0) {  // identity gates alone need no pass
                sg->kind[i] = SEG_PASS;
                sg->cost += cost;
            }
            i = e + 1;
        }
        sg->done = true;
        if (prog) emit_all(*sg);
        return;
    }
    // Least modelled cost of gates [j, N): best[j]. The first segment is [j, cut[j]) of kind
    // kind[j]: a single launch, a tile pass, a diagonal run, or an uncontrolled gate leading a
    // diagonal run. A pass may end wherever its targets still fit; a diagonal run of up to
    // kDiagMaxGates gates costs one read + write of the chunks it can change (all of them with
    // a leading gate; else those whose bits >= 3 match the controls every gate of the run
    // shares).
    const double launch_cost = launch_latency_cost(n, dtype);
    std::vector<double> best(N + 1, 0.0);
    std::vector<size_t> &cut = sg->cut;
    std::vector<char> &kind = sg->kind;
    const uint64_t chunk_low = (1ull << kDiagChunkBits) - 1ull;
    // fraction of the state a diagonal run over seq[a, e] changes (no leading gate)
    auto diag_span = [&](size_t a, size_t end, bool lead, auto &&visit) {
        uint64_t fm = ~0ull, fv = 0;
        bool first = true;
        int real = 0;
        for (size_t e = a; e < end; ++e) {
            const int g = seq[e];
            const GatePlan &p = plans[g];
            if (p.units != 0) {
                if (!is_diag(g) || real >= kDiagMaxGates) break;
                if (first) {
                    fm = p.ctrl_mask & ~chunk_low;
                    fv = p.ctrl_vals & fm;
                    first = false;
                } else {
                    fm &= p.ctrl_mask & ~((p.ctrl_vals ^ fv) | chunk_low);
                    fv &= fm;
                }
                ++real;
            }
            const double frac = lead ? 1.0 : std::ldexp(1.0, -std::min(popc(fm), kDiagMaxFixed));
            visit(e, frac, real);
        }
    };
    for (size_t j = N; j-- > 0;) {
        const int g0 = seq[j];
        const GatePlan &p0 = plans[g0];
        const double alone = (p0.units == 0 && !is_param(g0)) ? 0.0 : single_launch_cost(p0, dtype) + launch_cost;
        double bv = alone + best[j + 1];
        size_t bc = j + 1;
        char bk = SEG_SINGLE;
        extend(j, N, [&](size_t e, double frac, double compute, int real) {
            if (real < 2) return;
            const double v = launch_cost + frac + compute + best[e + 1];
            if (v < bv - 1e-9) {
                bv = v;
                bc = e + 1;
                bk = SEG_PASS;
            }
        });
        if (diag_runs && p0.units != 0 && is_diag(g0)) {
            diag_span(j, N, false, [&](size_t e, double frac, int real) {
                if (real < 2) return;
                const double v = launch_cost + frac + real * diag_run_gate_cost(dtype) + best[e + 1];
                if (v < bv - 1e-9) {
                    bv = v;
                    bc = e + 1;
                    bk = SEG_DIAG;
                }
            });
        }
        if (diag_runs && n >= kDiagChunkBits + 1 && p0.units != 0 && p0.ctrl_mask == 0 && p0.op != OP_SWAP &&
            !is_diag(g0) && j + 1 < N) {
            diag_span(j + 1, N, true, [&](size_t e, double frac, int real) {
                if (real < 1) return;
                const double v = launch_cost + frac + real * diag_run_gate_cost(dtype) + best[e + 1];
                if (v < bv - 1e-9) {
                    bv = v;
                    bc = e + 1;
                    bk = SEG_LEAD_DIAG;
                }
            });
        }
        best[j] = bv;
        cut[j] = bc;
        kind[j] = bk;
    }
    sg->cost = best[0];
    sg->done = true;
    if (prog) emit_all(*sg);
}

bool plan_fused(int n, int dtype, int k, const std::vector<int> &seq, const std::vector<GatePlan> &plans,
                const std::vector<const double *> *dus, const std::vector<int> *gslots, FusedProgram *prog,
                int max_gates, bool allow_single, int group_bits, bool jit) {
    // The gates in the given order and in the order block_schedule gives for passes of k local
    // qubits (the same limits as plan_in_order's passes): both are cut, and the program of the
    // one of lower modelled cost is emitted.
    Segments s1;
    const int N = (int)seq.size();
    if (N < 3) {
        plan_in_order(n, dtype, k, seq, plans, dus, gslots, prog, max_gates, allow_single, group_bits, jit, &s1);
        return true;
    }
    plan_in_order(n, dtype, k, seq, plans, dus, gslots, nullptr, max_gates, allow_single, group_bits, jit, &s1);
    const int b0 = dtype == QS_C64 ? 4 : 3;
    const int kk = std::min(std::min(std::max(k, b0 + 1), kTileMaxBits), n);
    const int b = std::min(kk, b0);
    const uint64_t low = (1ull << b) - 1ull;
    const int mg = std::max(1, std::min(max_gates, kPassMaxGates));
    std::vector<OrderItem> items(N);
    for (int i = 0; i < N; ++i) {
        const int g = seq[i];
        const GatePlan &p = plans[g];
        const bool param = dus != nullptr && (*dus)[g] != nullptr;
        if (p.units == 0 && !param) {
            items[i] = {-1, 0ull, 0ull, false};
            continue;
        }
        const bool diag = p.op == OP_DIAG || p.op == OP_SIDE;
        items[i] = {p.t, (1ull << p.t) | p.ctrl_mask, diag ? 0ull : (1ull << p.t), param};
    }
    const std::vector<int> ord = block_schedule(items, n, kk, low, mg, dus ? kTileMaxParam : N);
    bool same = true;
    for (int i = 0; i < N && same; ++i) same = ord[i] == i;
    if (!same) {
        std::vector<int> seq2(N);
        for (int i = 0; i < N; ++i) seq2[i] = seq[ord[i]];
        Segments s2;
        plan_in_order(n, dtype, k, seq2, plans, dus, gslots, nullptr, max_gates, allow_single, group_bits, jit, &s2);
        if (s2.cost < s1.cost - 1e-9) {
            plan_in_order(n, dtype, k, seq2, plans, dus, gslots, prog, max_gates, allow_single, group_bits, jit, &s2);
            return true;
        }
    }
    plan_in_order(n, dtype, k, seq, plans, dus, gslots, prog, max_gates, allow_single, group_bits, jit, &s1);
    return true;
}

// Fraction of the assignments of the non-local bits that satisfy at least one of the terms
// (mask, vals): split on one bit at a time (Shannon expansion), dropping terms a shorter one
// subsumes. Exact unless more than `budget` nodes are visited; then the union bound.
static double union_fraction(std::vector<std::pair<uint64_t, uint64_t>> terms, long *budget) {
    if (terms.empty()) return 0.0;
    for (auto &t : terms)
        if (t.first == 0) return 1.0;
    if (--*budget < 0) {
        double u = 0.0;
        for (auto &t : terms) u += std::ldexp(1.0, -popc(t.first));
        return std::min(1.0, u);
    }
    // drop duplicates and subsumed terms (t1's literals a subset of t2's: t2 adds nothing)
    std::vector<std::pair<uint64_t, uint64_t>> keep;
    for (size_t i = 0; i < terms.size(); ++i) {
        bool drop = false;
        for (size_t j = 0; j < terms.size() && !drop; ++j) {
            if (i == j) continue;
            const auto &a = terms[j], &b = terms[i];
            const bool subset = (a.first & ~b.first) == 0 && (b.second & a.first) == a.second;
            if (subset && (a.first != b.first || j < i)) drop = true;
        }
        if (!drop) keep.push_back(terms[i]);
    }
    const uint64_t bit = keep[0].first & (~keep[0].first + 1);
    std::vector<std::pair<uint64_t, uint64_t>> t0, t1;
    for (auto &t : keep) {
        if (!(t.first & bit)) {
            t0.push_back(t);
            t1.push_back(t);
        } else if (t.second & bit) {
            t1.push_back({t.first & ~bit, t.second & ~bit});
        } else {
            t0.push_back({t.first & ~bit, t.second & ~bit});
        }
    }
    return 0.5 * (union_fraction(std::move(t0), budget) + union_fraction(std::move(t1), budget));
}

double pass_touched_fraction(const FusedProgram &prog, int pass) {
    const TilePass &P = prog.passes[pass];
    if (!P.hctrl) return 1.0;
    std::vector<std::pair<uint64_t, uint64_t>> terms;
    for (int g = P.gate_begin; g < P.gate_begin + P.gate_count; ++g)
        terms.push_back({prog.gates[g].hmask, prog.gates[g].hvals});
    long budget = 200000;
    return union_fraction(std::move(terms), &budget);
}

static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

static size_t dgate_offset(const FusedProgram &p) {
    return align16(p.groups.size() * sizeof(TileGroup)) + align16(p.gates.size() * sizeof(RegGate));
}

size_t program_table_bytes(const FusedProgram &p) { return dgate_offset(p) + p.dgates.size() * sizeof(DiagGate); }

void pack_program_table(const FusedProgram &p, void *host_dst) {
    char *d = static_cast<char *>(host_dst);
    if (!p.groups.empty()) std::memcpy(d, p.groups.data(), p.groups.size() * sizeof(TileGroup));
    if (!p.gates.empty())
        std::memcpy(d + align16(p.groups.size() * sizeof(TileGroup)), p.gates.data(), p.gates.size() * sizeof(RegGate));
    if (!p.dgates.empty()) std::memcpy(d + dgate_offset(p), p.dgates.data(), p.dgates.size() * sizeof(DiagGate));
}

const DiagGate *table_dgates(const FusedProgram &p, const void *dev_base) {
    return reinterpret_cast<const DiagGate *>(static_cast<const char *>(dev_base) + dgate_offset(p));
}

const TileGroup *table_groups(const FusedProgram &, const void *dev_base) {
    return static_cast<const TileGroup *>(dev_base);
}

const RegGate *table_gates(const FusedProgram &p, const void *dev_base) {
    return reinterpret_cast<const RegGate *>(static_cast<const char *>(dev_base) +
                                             align16(p.groups.size() * sizeof(TileGroup)));
}

}  // namespace qs
