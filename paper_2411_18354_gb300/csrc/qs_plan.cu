// qs_plan.cu -- host-side gate planning (argument checks, sorted insertion positions,
// operation class and unit layout) and the launch entry points used by the C interface.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "qs_internal.cuh"

namespace qs {

cudaError_t launch_gate_c64(void *psi, const GatePlan &p, bool masked, uint64_t cmask,
                            uint64_t cvals, cudaStream_t st);
cudaError_t launch_gate_c128(void *psi, const GatePlan &p, bool masked, uint64_t cmask,
                             uint64_t cvals, cudaStream_t st);

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    static std::atomic<int> sms_of[64];  // per device, 0 = not read yet (thread-safe)
    if (dev < 0 || dev >= 64) dev = 0;
    int sms = sms_of[dev].load(std::memory_order_relaxed);
    if (sms == 0) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        sms_of[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

static int ctz64(uint64_t v) { return __builtin_ctzll(v); }

// Counter -> index map for the inserted positions pos[0..m-1] (ascending) with inserted
// values `ins`. Segment s collects the free bits between pos[s-1] and pos[s]; each of
// them comes from the counter bit s places lower (Eq. 4 applied for every inserted
// position in ascending order, Section III-B).
void build_map(int n, const int *pos, int m, uint64_t ins, IndexMap *map) {
    std::memset(map, 0, sizeof(*map));
    map->ins = ins;
    int ns = 0;
    for (int s = 0; s <= m; ++s) {
        const int lo = (s == 0) ? 0 : pos[s - 1] + 1;
        const int hi = (s == m) ? n : pos[s];
        if (hi <= lo) continue;
        const uint64_t upto_hi = (hi >= 64) ? ~0ull : ((1ull << hi) - 1ull);
        const uint64_t below_lo = (1ull << lo) - 1ull;
        map->mask[ns] = upto_hi & ~below_lo;
        map->shift[ns] = s;
        ++ns;
    }
    map->nseg = ns;
}

static bool finite8(const double *U) {
    for (int i = 0; i < 8; ++i)
        if (!std::isfinite(U[i])) return false;
    return true;
}

static bool is_one(const double *z) { return z[0] == 1.0 && z[1] == 0.0; }
static bool is_zero(const double *z) { return z[0] == 0.0 && z[1] == 0.0; }

bool plan_gate(int n, int dtype, int target, uint64_t ctrl_mask, uint64_t ctrl_vals,
               const double U[8], int kind, int force_op, GatePlan *p, char *err, size_t errlen) {
    if (n < 1 || n > kMaxQubits) {
        std::snprintf(err, errlen, "n=%d out of range [1, %d]", n, kMaxQubits);
        return false;
    }
    if (target < 0 || target >= n) {
        std::snprintf(err, errlen, "target %d out of range [0, %d)", target, n);
        return false;
    }
    const uint64_t tbit = 1ull << target;
    const uint64_t valid = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
    if (ctrl_mask & ~valid) {
        std::snprintf(err, errlen, "ctrl_mask 0x%llx has qubits >= n=%d", (unsigned long long)ctrl_mask, n);
        return false;
    }
    if (ctrl_mask & tbit) {
        std::snprintf(err, errlen, "ctrl_mask 0x%llx contains the target %d", (unsigned long long)ctrl_mask, target);
        return false;
    }
    if (ctrl_vals & ~ctrl_mask) {
        std::snprintf(err, errlen, "ctrl_vals 0x%llx has bits outside ctrl_mask 0x%llx",
                      (unsigned long long)ctrl_vals, (unsigned long long)ctrl_mask);
        return false;
    }
    std::memset(p, 0, sizeof(*p));
    p->n = n;
    p->t = target;
    p->tbit = tbit;
    p->c = __builtin_popcountll(ctrl_mask);
    p->ctrl_mask = ctrl_mask;
    p->ctrl_vals = ctrl_vals;
    if (kind == QS_GATE_X) {
        p->Ufull[2] = 1.0;
        p->Ufull[4] = 1.0;
    } else if (U) {
        std::memcpy(p->Ufull, U, sizeof(p->Ufull));
    }

    // Operation class from the exact structure of U (exact zeros and ones only).
    if (force_op >= 0) {
        if (kind != QS_GATE_U || !U || !finite8(U)) {
            std::snprintf(err, errlen, "gate matrix missing or not finite");
            return false;
        }
        std::memcpy(p->U, U, sizeof(p->U));
        p->op = force_op;
    } else if (kind == QS_GATE_X) {
        p->op = OP_SWAP;
    } else if (kind == QS_GATE_U) {
        if (!U || !finite8(U)) {
            std::snprintf(err, errlen, "gate matrix missing or not finite");
            return false;
        }
        std::memcpy(p->U, U, sizeof(p->U));
        const double *a = U, *b = U + 2, *c = U + 4, *d = U + 6;
        if (is_zero(b) && is_zero(c)) {
            if (is_one(a) && is_one(d)) {
                p->op = OP_DIAG;
                p->units = 0;  // identity: nothing to do
                p->map.nseg = 0;
                return true;
            } else if (is_one(a)) {
                p->op = OP_SIDE;
                p->side = 1;
                p->U[0] = d[0];
                p->U[1] = d[1];
            } else if (is_one(d)) {
                p->op = OP_SIDE;
                p->side = 0;
                p->U[0] = a[0];
                p->U[1] = a[1];
            } else {
                p->op = OP_DIAG;
            }
        } else if (is_zero(a) && is_zero(d) && is_one(b) && is_one(c)) {
            p->op = OP_SWAP;
        } else if (U[1] == 0.0 && U[3] == 0.0 && U[5] == 0.0 && U[7] == 0.0) {
            p->op = OP_REAL;
        } else {
            p->op = OP_GEN;
        }
    } else {
        std::snprintf(err, errlen, "gate kind %d needs a parameter (use qs_apply_circuit)", kind);
        return false;
    }

    // Fixed point: one update form for every matrix (exchanges stay exchanges, an exact move
    // that gives the same integers as the general form of [[0, 1], [1, 0]]; the identity, left
    // out above, leaves every integer unchanged under the general form too).
    if (dtype == QS_Q30 && p->op != OP_SWAP) p->op = OP_GEN;

    // Inserted positions: the target (value 0) and the controls (their values), ascending.
    int pos[64];
    int m = 0;
    uint64_t all = ctrl_mask | tbit;
    while (all) {
        pos[m++] = ctz64(all);
        all &= all - 1;
    }
    const int free_bits = n - m;
    build_map(n, pos, m, ctrl_vals, &p->map);

    // Unit layout: one 16-byte vector per side where the lowest free bits allow (complex64: 2
    // amplitudes, complex128: 1; with t = 0 one vector holds the pair). Consecutive threads take
    // consecutive units, so each warp-wide load or store covers 512 contiguous bytes per side;
    // units of two adjacent vectors per side made every warp instruction stride over memory and
    // capped an in-place update at ~88 % of a copy's bandwidth (measured on GB300: 5.8-5.9
    // against 6.3-6.7 TB/s for the uncontrolled update at n = 30).
    const bool c64 = dtype == QS_C64 || dtype == QS_Q30;  // 8-byte amplitudes
    if (target == 0 && p->op != OP_SIDE) {
        p->layout = LAY_ADJ;
        p->r = 0;
    } else {
        p->layout = LAY_SPLIT;
        int r = c64 ? 1 : 0;
        r = std::min(r, pos[0]);
        r = std::min(r, free_bits);
        p->r = std::max(r, 0);
    }
    p->units = 1ull << (free_bits - p->r);
    return true;
}

void plan_masked(const GatePlan &compact, GatePlan *out) {
    *out = compact;
    int pos[1] = {compact.t};
    build_map(compact.n, pos, 1, 0, &out->map);
    out->op = OP_GEN;
    out->units = 1ull << (compact.n - 1 - compact.r);
}

cudaError_t launch_gate(int dtype, void *psi, const GatePlan &p, cudaStream_t st) {
    if (dtype == QS_Q30) return launch_gate_q30(psi, p, false, 0, 0, st);
    return dtype == QS_C64 ? launch_gate_c64(psi, p, false, 0, 0, st)
                           : launch_gate_c128(psi, p, false, 0, 0, st);
}

cudaError_t launch_gate_masked(int dtype, void *psi, const GatePlan &p, uint64_t ctrl_mask,
                               uint64_t ctrl_vals, cudaStream_t st) {
    if (dtype == QS_Q30) return launch_gate_q30(psi, p, true, ctrl_mask, ctrl_vals, st);
    return dtype == QS_C64 ? launch_gate_c64(psi, p, true, ctrl_mask, ctrl_vals, st)
                           : launch_gate_c128(psi, p, true, ctrl_mask, ctrl_vals, st);
}

}  // namespace qs
