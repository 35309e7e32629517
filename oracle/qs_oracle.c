/*
 * qs_oracle.c -- CPU reference oracle for the controlled single-qubit gate update.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or includes this
 * file; only the test suite, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header or constant with the CUDA path.
 *
 * Everything here is plain, slow and written to be checked against the paper by eye:
 * double precision, one loop over all 2^n amplitude indices, the control test done per
 * index exactly as the paper's baseline kernel does it (Fig. "sim_baseline_kernel",
 * Section III-A), no blocking, no vectorisation, no reordering of the arithmetic.
 *
 * State layout: psi[2*k] = Re C_k, psi[2*k+1] = Im C_k for k in [0, 2^n). Qubit t = 0 is
 * the least significant bit of k (Section III).
 *
 * Matrix layout: U[0..7] = (re a, im a, re b, im b, re c, im c, re d, im d) for the gate
 * G = [a b; c d] of Section III, Eq. 2.
 *
 * Parallelism: the gate loops carry an OpenMP "parallel for"; every index k with bit t
 * clear owns the pair (k, k + 2^t) alone, so the iterations are independent (Section III:
 * the iterations of one gate can run in parallel). Reductions are sequential so that
 * their rounding order is fixed.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

/* ---------------------------------------------------------------------------------- */
/* Index helpers (Section III-B)                                                        */
/* ---------------------------------------------------------------------------------- */

/* ithCleared(i, t): index of the first element of pair i for target t, i.e. i with a 0
 * inserted at bit position t. The paper takes this helper from QCGPU without writing it
 * out; the second pair element is this value + 2^t (Section III-A pseudocode), which
 * fixes the reading: bits below t stay, bits from t upwards move up by one. */
uint64_t oracle_ith_cleared(uint64_t i, int t)
{
    uint64_t low = i & ((1ull << t) - 1ull);
    uint64_t high = i >> t;
    return (high << (t + 1)) | low;
}

/* Eq. 3 (adjusted control) and Eq. 4 (iterative map), in the paper's order: starting from
 * a reduced iteration index i_r of I_r = [0, 2^(n-1-n_c)), map through the controls taken
 * in ascending order c_0 < c_1 < ... (Section III-B requires this order) to a global
 * iteration index i_g in I_g = [0, 2^(n-1)). `controls` must hold n_c qubit indices,
 * none equal to t. The formula uses integer floor division and the skip interval
 * 2^(c_adj) exactly as Eq. 4 states. */
uint64_t oracle_eq4_map(uint64_t i_r, int t, const int *controls, int n_c)
{
    uint64_t i = i_r;
    for (int k = 0; k < n_c; ++k) {
        int c = controls[k];
        int c_adj = (c > t) ? c - 1 : c;          /* Eq. 3 */
        uint64_t skip = 1ull << c_adj;             /* skip interval 2^(c_adj) */
        i = i + (i / skip + 1ull) * skip;          /* Eq. 4 */
    }
    return i;
}

/* ---------------------------------------------------------------------------------- */
/* Gate application (Section III, Eq. 2; controls per Section III-B)                   */
/* ---------------------------------------------------------------------------------- */

/* Apply G = [a b; c d] to target t with controls: for every amplitude index k whose bit t
 * is 0 and whose bits under ctrl_mask equal ctrl_vals,
 *     C'_k       = a C_k + b C_{k+2^t}
 *     C'_{k+2^t} = c C_k + d C_{k+2^t}.
 * A control on |1> (Section III-B) is a mask bit with the same bit set in ctrl_vals; a
 * control on |0> (Fig. 1, right) is a mask bit with that bit clear in ctrl_vals. Both
 * elements of a pair differ only in bit t, so testing k alone decides the pair
 * (Section III-B). */
void oracle_apply_gate(double *psi, int n, int t, uint64_t ctrl_mask, uint64_t ctrl_vals,
                       const double *U)
{
    const int64_t N = (int64_t)1 << n;
    const uint64_t stride = 1ull << t;
    const double ar = U[0], ai = U[1], br = U[2], bi = U[3];
    const double cr = U[4], ci = U[5], dr = U[6], di = U[7];
#pragma omp parallel for schedule(static)
    for (int64_t kk = 0; kk < N; ++kk) {
        uint64_t k = (uint64_t)kk;
        if (k & stride) continue;                       /* k is the first element     */
        if ((k & ctrl_mask) != ctrl_vals) continue;     /* control check (baseline)   */
        uint64_t k2 = k + stride;                        /* second element: k + 2^t    */
        double xr = psi[2 * k], xi = psi[2 * k + 1];
        double yr = psi[2 * k2], yi = psi[2 * k2 + 1];
        /* a x + b y */
        psi[2 * k]      = (ar * xr - ai * xi) + (br * yr - bi * yi);
        psi[2 * k + 1]  = (ar * xi + ai * xr) + (br * yi + bi * yr);
        /* c x + d y */
        psi[2 * k2]     = (cr * xr - ci * xi) + (dr * yr - di * yi);
        psi[2 * k2 + 1] = (cr * xi + ci * xr) + (dr * yi + di * yr);
    }
}

/* The X gate of Section II-A "flips a qubit ... by swapping of the qubit's probability
 * amplitudes": for every selected pair, exchange C_k and C_{k+2^t}. No arithmetic, so the
 * result is bit-exact. With controls this is CNOT / Toffoli (Fig. 1, left). */
void oracle_apply_x(double *psi, int n, int t, uint64_t ctrl_mask, uint64_t ctrl_vals)
{
    const int64_t N = (int64_t)1 << n;
    const uint64_t stride = 1ull << t;
#pragma omp parallel for schedule(static)
    for (int64_t kk = 0; kk < N; ++kk) {
        uint64_t k = (uint64_t)kk;
        if (k & stride) continue;
        if ((k & ctrl_mask) != ctrl_vals) continue;
        uint64_t k2 = k + stride;
        double xr = psi[2 * k], xi = psi[2 * k + 1];
        psi[2 * k] = psi[2 * k2];
        psi[2 * k + 1] = psi[2 * k2 + 1];
        psi[2 * k2] = xr;
        psi[2 * k2 + 1] = xi;
    }
}

/* Output amplitude `k` of one gate, from the two input amplitudes of its pair. Used to
 * check sampled outputs of a single gate on states too large to update on the host. */
void oracle_gate_output(uint64_t k, int t, uint64_t ctrl_mask, uint64_t ctrl_vals,
                        const double *U, const double *in_k, const double *in_partner,
                        double *out)
{
    const uint64_t stride = 1ull << t;
    uint64_t k0 = k & ~stride;                          /* first element of k's pair */
    if ((k0 & ctrl_mask) != ctrl_vals) {                /* pair not selected         */
        out[0] = in_k[0];
        out[1] = in_k[1];
        return;
    }
    const double *x = (k & stride) ? in_partner : in_k;  /* C_{k0}       */
    const double *y = (k & stride) ? in_k : in_partner;  /* C_{k0+2^t}   */
    const double *r = (k & stride) ? U + 4 : U;          /* row [c d] or [a b] */
    out[0] = (r[0] * x[0] - r[1] * x[1]) + (r[2] * y[0] - r[3] * y[1]);
    out[1] = (r[0] * x[1] + r[1] * x[0]) + (r[2] * y[1] + r[3] * y[0]);
}

/* ---------------------------------------------------------------------------------- */
/* Reductions (sequential double-precision sums over k = 0 .. 2^n - 1)                  */
/* ---------------------------------------------------------------------------------- */

/* sum_k |C_k|^2 (Section II, Eq. 1: the squared moduli of the amplitudes sum to 1). */
double oracle_norm2(const double *psi, int n)
{
    const uint64_t N = 1ull << n;
    double s = 0.0;
    for (uint64_t k = 0; k < N; ++k)
        s += psi[2 * k] * psi[2 * k] + psi[2 * k + 1] * psi[2 * k + 1];
    return s;
}

/* <Z_i> = sum_k |C_k|^2 (1 - 2 bit_i(k)) for every qubit i: Z is +1 on |0> and -1 on
 * |1> of qubit i, and qubit i is bit i of k. */
void oracle_expect_z(const double *psi, int n, double *out)
{
    const uint64_t N = 1ull << n;
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    for (uint64_t k = 0; k < N; ++k) {
        double p = psi[2 * k] * psi[2 * k] + psi[2 * k + 1] * psi[2 * k + 1];
        for (int i = 0; i < n; ++i) {
            if ((k >> i) & 1ull) out[i] -= p;
            else out[i] += p;
        }
    }
}

/* Re <a|b> = sum_k Re(conj(a_k) b_k). */
double oracle_inner_re(const double *a, const double *b, int n)
{
    const uint64_t N = 1ull << n;
    double s = 0.0;
    for (uint64_t k = 0; k < N; ++k)
        s += a[2 * k] * b[2 * k] + a[2 * k + 1] * b[2 * k + 1];
    return s;
}

/* Number of OpenMP threads the gate loops use (1 when built without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------- */
/* Fixed-point amplitudes (Q1.30), the paper's conclusion's future-work format          */
/* ---------------------------------------------------------------------------------- */

/* The paper names fixed-point amplitudes as future work without a format; the format taken
 * here (written down with the library): each real and imaginary part is a signed 32-bit
 * integer v meaning v / 2^30. */

/* A real number in Q1.30: v * 2^30 rounded to the nearest integer, halves away from zero,
 * then clamped to [-2^31, 2^31 - 1]. */
int32_t oracle_quantize_q30(double v)
{
    double s = v * 1073741824.0;
    double r = (s >= 0.0) ? floor(s + 0.5) : -floor(-s + 0.5);
    if (r > 2147483647.0) r = 2147483647.0;
    if (r < -2147483648.0) r = -2147483648.0;
    return (int32_t)r;
}

/* One output component from its exact 64-bit sum S (a sum of products of Q1.30 values, i.e.
 * of value * 2^60): floor((S + 2^29) / 2^30), the nearest integer with halves rounded toward
 * +infinity, clamped to the int32 range. */
static int32_t q30_round(long long S)
{
    long long r = S + (1ll << 29);
    /* floor division by 2^30 (an arithmetic right shift, written out for negative values) */
    long long q = (r >= 0) ? (r / 1073741824ll) : -((-r + 1073741823ll) / 1073741824ll);
    if (q > 2147483647ll) q = 2147483647ll;
    if (q < -2147483648ll) q = -2147483648ll;
    return (int32_t)q;
}

/* Eq. 2 in Q1.30 for every selected pair (the same loop and control test as
 * oracle_apply_gate): C'_k = a C_k + b C_{k+2^t}, C'_{k+2^t} = c C_k + d C_{k+2^t}, each
 * component's four products summed exactly in 64 bits and rounded once by q30_round.
 * psi[2k], psi[2k+1] = Re, Im of C_k; U[0..7] = a, b, c, d as (re, im), in Q1.30. */
void oracle_apply_gate_q30(int32_t *psi, int n, int t, uint64_t ctrl_mask, uint64_t ctrl_vals, const int32_t *U)
{
    const int64_t N = (int64_t)1 << n;
    const uint64_t stride = 1ull << t;
    const long long ar = U[0], ai = U[1], br = U[2], bi = U[3];
    const long long cr = U[4], ci = U[5], dr = U[6], di = U[7];
#pragma omp parallel for schedule(static)
    for (int64_t kk = 0; kk < N; ++kk) {
        uint64_t k = (uint64_t)kk;
        if (k & stride) continue;
        if ((k & ctrl_mask) != ctrl_vals) continue;
        uint64_t k2 = k + stride;
        long long xr = psi[2 * k], xi = psi[2 * k + 1];
        long long yr = psi[2 * k2], yi = psi[2 * k2 + 1];
        psi[2 * k]      = q30_round(ar * xr - ai * xi + br * yr - bi * yi);
        psi[2 * k + 1]  = q30_round(ar * xi + ai * xr + br * yi + bi * yr);
        psi[2 * k2]     = q30_round(cr * xr - ci * xi + dr * yr - di * yi);
        psi[2 * k2 + 1] = q30_round(cr * xi + ci * xr + dr * yi + di * yr);
    }
}

/* Output amplitude k of one Q1.30 gate from its pair's inputs (sampled checks). */
void oracle_gate_output_q30(uint64_t k, int t, uint64_t ctrl_mask, uint64_t ctrl_vals, const int32_t *U,
                            const int32_t *in_k, const int32_t *in_partner, int32_t *out)
{
    const uint64_t stride = 1ull << t;
    uint64_t k0 = k & ~stride;
    if ((k0 & ctrl_mask) != ctrl_vals) {
        out[0] = in_k[0];
        out[1] = in_k[1];
        return;
    }
    const int32_t *x = (k & stride) ? in_partner : in_k;
    const int32_t *y = (k & stride) ? in_k : in_partner;
    const int32_t *r = (k & stride) ? U + 4 : U;
    out[0] = q30_round((long long)r[0] * x[0] - (long long)r[1] * x[1] + (long long)r[2] * y[0] - (long long)r[3] * y[1]);
    out[1] = q30_round((long long)r[0] * x[1] + (long long)r[1] * x[0] + (long long)r[2] * y[1] + (long long)r[3] * y[0]);
}

/* <Z_i> of a Q1.30 state: |C_k|^2 = (re^2 + im^2) / 2^60, summed sequentially in double. */
void oracle_expect_z_q30(const int32_t *psi, int n, double *out)
{
    const uint64_t N = 1ull << n;
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    for (uint64_t k = 0; k < N; ++k) {
        long long re = psi[2 * k], im = psi[2 * k + 1];
        double p = (double)(re * re + im * im) * 8.673617379884035e-19; /* 2^-60 */
        for (int i = 0; i < n; ++i) {
            if ((k >> i) & 1ull) out[i] -= p;
            else out[i] += p;
        }
    }
}
