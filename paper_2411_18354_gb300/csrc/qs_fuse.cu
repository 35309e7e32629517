// qs_fuse.cu -- host planner that groups consecutive gates into fused tile passes.
//
// Greedy, in execution order: a pass starts with the lowest b qubits local (b = 4 for
// complex64, 3 for complex128, so that tile rows are 128 or 128 bytes of contiguous memory)
// and takes the following gates while their targets fit in k local qubits. A gate's controls
// need not be local: non-local controls become the gate's tile predicate. A gate joins only if
// the pass's estimated traffic grows by less than the gate's own traffic as a separate
// launch (fraction of tiles touched, union bound over the gates' tile predicates, against the
// fraction of 64-byte DRAM units a separate launch touches). Runs of one gate stay separate
// launches. The local set is finally padded with the lowest free qubits up to k.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "k_tile.cuh"
#include "qs_fuse.cuh"

namespace qs {

static int popc(uint64_t v) { return __builtin_popcountll(v); }

// Fraction of the state a separate k_gate launch moves, counted in 64-byte DRAM units:
// controls on the qubits inside one unit do not reduce it.
static double single_fraction(const GatePlan &p, int dtype) {
    const int unit_bits = dtype == QS_C64 ? 3 : 2;
    const uint64_t high = p.ctrl_mask & ~((1ull << unit_bits) - 1ull);
    return std::ldexp(1.0, -popc(high));
}

static void make_tile_gate(const GatePlan &p, uint64_t Lmask, int k, const int *local_of, TileGate *G) {
    std::memset(G, 0, sizeof(*G));
    const int t_loc = local_of[p.t];
    uint32_t cm = 0, cv = 0;
    uint64_t lc = p.ctrl_mask & Lmask;
    while (lc) {
        const int q = __builtin_ctzll(lc);
        lc &= lc - 1;
        cm |= 1u << local_of[q];
        if ((p.ctrl_vals >> q) & 1ull) cv |= 1u << local_of[q];
    }
    int pos[kTileMaxBits];
    int m = 0;
    uint32_t all = cm | (1u << t_loc);
    while (all) {
        pos[m++] = __builtin_ctz(all);
        all &= all - 1;
    }
    IndexMap map;
    build_map(k, pos, m, cv, &map);
    G->nseg = (uint8_t)map.nseg;
    for (int s = 0; s < map.nseg; ++s) {
        G->mask[s] = (uint32_t)map.mask[s];
        G->shift[s] = (uint8_t)map.shift[s];
    }
    G->ins = cv;
    G->tbit = 1u << t_loc;
    G->log_pairs = (uint32_t)(k - m);
    G->hmask = p.ctrl_mask & ~Lmask;
    G->hvals = p.ctrl_vals & G->hmask;
    G->op = p.op;
    G->side = p.side;
    G->slot = -1;
    std::memcpy(G->U, p.U, sizeof(G->U));
    for (int i = 0; i < 8; ++i) G->Uf[i] = (float)p.U[i];
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

bool plan_fused(int n, int dtype, int k, const std::vector<int> &seq, const std::vector<GatePlan> &plans,
                const std::vector<const double *> *dus, const std::vector<int> *gslots, FusedProgram *prog,
                int max_gates, bool allow_single) {
    prog->ops.clear();
    prog->passes.clear();
    prog->gates.clear();
    prog->gate_src.clear();
    max_gates = std::max(1, std::min(max_gates, kTileMaxGates));
    // k >= b0 + 1 so that any single target fits next to the b0 low qubits (n permitting)
    const int b0 = dtype == QS_C64 ? 4 : 3;
    k = std::min(std::min(std::max(k, b0 + 1), kTileMaxBits), n);
    const int b = std::min(k, b0);
    const uint64_t low = (b >= 64) ? ~0ull : ((1ull << b) - 1ull);
    const bool adjoint = dus != nullptr;
    size_t i = 0;
    while (i < seq.size()) {
        uint64_t L = low;
        double frac = 0.0;
        int nparam = 0;
        std::vector<int> members;
        size_t j = i;
        while (j < seq.size() && (int)members.size() < max_gates) {
            const GatePlan &p = plans[seq[j]];
            const bool param = adjoint && (*dus)[seq[j]] != nullptr;
            if (p.units == 0 && !param) {  // identity: nothing to apply
                members.push_back(-1 - seq[j]);
                ++j;
                continue;
            }
            const uint64_t L2 = L | (1ull << p.t);
            if (popc(L2) > k) break;
            if (param && nparam >= kTileMaxParam) break;
            const double f = std::ldexp(1.0, -popc(p.ctrl_mask & ~L2));
            const double frac2 = std::min(1.0, frac + f);
            int real = 0;
            for (int mbr : members) real += mbr >= 0;
            if (real > 0 && frac2 > frac + single_fraction(p, dtype)) break;
            frac = frac2;
            L = L2;
            members.push_back(seq[j]);
            nparam += param;
            ++j;
        }
        int real = 0;
        for (int mbr : members) real += mbr >= 0;
        if (real == 0) {  // only identity gates (j > i here: the first real gate always fits)
            i = std::max(j, i + 1);
            continue;
        }
        if (real < 2 && allow_single) {  // not worth a pass: the first gate runs alone
            const int g = seq[i];
            const bool param = adjoint && (*dus)[g] != nullptr;
            if (plans[g].units != 0 || param) prog->ops.push_back({-1, g});
            ++i;
            continue;
        }
        // pad the local set with the lowest free qubits
        for (int q = 0; q < n && popc(L) < k; ++q) L |= 1ull << q;
        int local_of[64];
        for (int q = 0, l = 0; q < n; ++q) local_of[q] = ((L >> q) & 1ull) ? l++ : -1;
        TilePass P;
        make_pass(n, L, &P);
        P.gate_begin = (int)prog->gates.size();
        for (int mbr : members) {
            if (mbr < 0) continue;
            TileGate G;
            make_tile_gate(plans[mbr], L, P.k, local_of, &G);
            if (adjoint && (*dus)[mbr]) {
                if (G.op != OP_GEN && G.op != OP_DIAG && G.op != OP_REAL) G.op = OP_GEN;
                std::memcpy(G.D, (*dus)[mbr], sizeof(G.D));
                for (int q = 0; q < 8; ++q) G.Df[q] = (float)G.D[q];
                G.slot = P.nparam;
                P.param_gslot[P.nparam++] = (*gslots)[mbr];
            }
            prog->gates.push_back(G);
            prog->gate_src.push_back(mbr);
        }
        P.gate_count = (int)prog->gates.size() - P.gate_begin;
        prog->ops.push_back({(int)prog->passes.size(), -1});
        prog->passes.push_back(P);
        i = j;
    }
    return true;
}

}  // namespace qs
