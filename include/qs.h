/*
 * qs.h -- C interface of libqs, a state-vector kernel library for sm_103a (GB300).
 *
 * The library applies single-qubit 2x2 gates with any number of control qubits to a
 * vector of 2^n complex amplitudes held in GPU memory, scheduling only the 2^(n-1-c)
 * amplitude pairs whose control bits are satisfied (arXiv 2411.18354, Section III-B:
 * "reduced iteration index set", Eqs. 3-4). Each pair index is formed on the device by
 * inserting the target bit (value 0) and the control bits (their required values) into a
 * compact counter, the bit-level form of Eq. 4 followed by ithCleared.
 *
 * Conventions shared by every call:
 *  - Amplitude k of an n-qubit state is stored at element k; qubit 0 is the least
 *    significant bit of k (Section III). Elements are interleaved (re, im): complex64 =
 *    2 x float32 (8 bytes), complex128 = 2 x float64 (16 bytes).
 *  - A gate matrix U[8] is G = [a b; c d] of Section III, Eq. 2, row-major, each entry as
 *    (re, im) doubles: {re a, im a, re b, im b, re c, im c, re d, im d}. For complex64
 *    states the entries are rounded to float32 once per call.
 *  - Controls: bit q of ctrl_mask marks qubit q as a control; the gate acts on pairs whose
 *    index bits under ctrl_mask equal ctrl_vals (bit set = control on |1>, Section III-B;
 *    bit clear = control on |0>, Fig. 1 right). ctrl_vals must not have bits outside
 *    ctrl_mask, and ctrl_mask must not contain the target or qubits >= n.
 *  - Every call returns a qs_status. On an error nothing has been launched and
 *    qs_last_error() holds a message for the calling thread. Calls never throw.
 *  - Work is enqueued asynchronously on the state's CUDA stream (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream) unless a call says it synchronises.
 *  - Device pointers are plain CUDA device addresses on the device that is current when
 *    the state is created; the caller keeps that device current for later calls.
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum qs_status {
    QS_OK = 0,
    QS_EINVAL = 1,        /* bad argument: nothing was launched                     */
    QS_ENOMEM = 2,        /* device allocation failed                               */
    QS_ECUDA = 3,         /* a CUDA runtime call failed (message has the CUDA text)  */
    QS_ETIMEOUT = 4,      /* a bounded device-side wait gave up (status word set)    */
    QS_EUNSUPPORTED = 5   /* valid request this build does not handle               */
} qs_status;

/* Amplitude formats. QS_C64: complex float32 (8 bytes); QS_C128: complex float64 (16 bytes);
 * QS_Q30: fixed point, each real and imaginary part a signed 32-bit integer v meaning
 * v / 2^30 (Q1.30, 8 bytes per amplitude, interleaved (re, im)). For QS_Q30 the gate matrix is
 * rounded once to Q1.30 (nearest, halves away from zero, clamped to int32) and each output
 * component of a selected pair is the exact 64-bit sum of its four products rounded to the
 * nearest Q1.30 value with halves toward +infinity (floor((S + 2^29) / 2^30)), clamped to
 * int32: results are exact integer arithmetic and reproducible bit for bit. Valid for
 * components and matrix entries of magnitude <= 1 (normalised states, unitary gates), where
 * no 64-bit sum can overflow. QS_Q30 supports single gates, the masked comparator, unfused
 * circuits (also as graphs), <Z_i> and host copies; fused passes, gradients and batches
 * return QS_EUNSUPPORTED. (The paper's conclusion names fixed-point amplitudes as future work
 * without a format; this one is the library's choice.) */
typedef enum qs_dtype { QS_C64 = 0, QS_C128 = 1, QS_Q30 = 2 } qs_dtype;

/* Gate kinds of qs_gate.kind. */
enum {
    QS_GATE_U = 0,   /* general 2x2 matrix in U                                     */
    QS_GATE_X = 1,   /* exchange the two amplitudes of each selected pair (X, CNOT,
                        Toffoli; Section II-A: X swaps the amplitudes). Bit-exact.  */
    QS_GATE_RY = 2,  /* RY(theta[param]) = exp(-i theta Y/2) = [[cos, -sin],[sin, cos]]
                        of theta/2; U ignored                                       */
    QS_GATE_RZ = 3   /* RZ(theta[param]) = exp(-i theta Z/2) =
                        diag(e^{-i theta/2}, e^{+i theta/2}); U ignored              */
};

/* Flags of qs_apply_circuit / qs_adjoint_grad / qs_batch_create. */
enum {
    QS_FLAG_FUSE = 1,        /* group runs of low-target gates into one tile pass      */
    QS_FLAG_GRAPH = 2,       /* launch the whole sequence as one CUDA graph            */
    QS_FLAG_OUT_DEVICE = 4,  /* energy / grad / expectation outputs are device pointers */
    QS_FLAG_MASKED = 8,      /* qs_apply_circuit: baseline schedule (comparator only)   */
    QS_FLAG_JIT = 16,        /* with QS_FLAG_FUSE: tile passes as kernels compiled for
                                their exact shape (see qs_circuit_compile)             */
    QS_FLAG_ADJOINT = 32     /* qs_circuit_schedule: the launches of qs_adjoint_grad   */
};

/* One gate (96 bytes, naturally aligned). Section III-A: target t, controls, matrix. */
typedef struct qs_gate {
    int32_t target;      /* target qubit t, 0 <= t < n                              */
    int32_t kind;        /* QS_GATE_*                                              */
    uint64_t ctrl_mask;  /* control qubits                                          */
    uint64_t ctrl_vals;  /* required values of the control qubits                   */
    int32_t param;       /* RY/RZ: index into theta; ignored for other kinds        */
    int32_t reserved;    /* must be 0                                               */
    double U[8];         /* QS_GATE_U: row-major [a b; c d], (re, im) interleaved   */
} qs_gate;

typedef struct qs_state qs_state;  /* opaque */

/* Message of the last failing call on this thread ("" if none). Valid until the next
 * failing call on the same thread. */
const char *qs_last_error(void);

/* Number of SMs / library build string, for diagnostics. Never fails. */
const char *qs_build_info(void);

/* ------------------------------------------------------------------------------------ */
/* State vectors (Section III: 2^n complex numbers in device memory)                     */
/* ------------------------------------------------------------------------------------ */

/* Allocate a state of n qubits (1 <= n <= 40) owned by the library, initialised to
 * |0...0> (amplitude 0 = 1) on `stream`. EINVAL for n out of range or a bad dtype;
 * ENOMEM if cudaMalloc fails. *out receives the handle. */
qs_status qs_state_alloc(int n, qs_dtype dtype, void *stream, qs_state **out);

/* Wrap caller-owned device memory of `bytes` bytes as an n-qubit state (contents are
 * left as they are). The library never frees it. EINVAL if bytes < 2^n * element size or
 * dev_ptr is not 256-byte aligned. */
qs_status qs_state_wrap(void *dev_ptr, size_t bytes, int n, qs_dtype dtype, void *stream,
                        qs_state **out);

/* Release the handle, its library-owned buffers and, for qs_state_alloc states, the
 * amplitude buffer. Synchronises the state's stream first. NULL is accepted. */
qs_status qs_state_free(qs_state *s);

/* Query n, dtype and the amplitude buffer's device address (any pointer may be NULL). */
qs_status qs_state_info(const qs_state *s, int *n, qs_dtype *dtype, void **dev_ptr);

/* Change the stream later calls enqueue on. */
qs_status qs_state_set_stream(qs_state *s, void *stream);

/* Set the state to the basis state |k> (k < 2^n). Asynchronous. */
qs_status qs_state_set_basis(qs_state *s, uint64_t k);

/* Copy all 2^n amplitudes to / from host memory (`bytes` must equal 2^n * element
 * size). Synchronous: returns after the copy has finished. */
qs_status qs_state_copy_to_host(const qs_state *s, void *dst, size_t bytes);
qs_status qs_state_copy_from_host(qs_state *s, const void *src, size_t bytes);

/* The same copies enqueued on the state's stream, in order with its gates; they return at
 * once. The host buffer must stay valid and untouched until the stream reaches the copy (see
 * qs_state_synchronize); with page-locked host memory the copy runs asynchronously and overlaps
 * work on other streams, with pageable memory the CUDA runtime may stage it synchronously. */
qs_status qs_state_copy_to_host_async(const qs_state *s, void *dst, size_t bytes);
qs_status qs_state_copy_from_host_async(qs_state *s, const void *src, size_t bytes);

/* Wait until everything enqueued on the state's stream has finished. */
qs_status qs_state_synchronize(const qs_state *s);

/* ------------------------------------------------------------------------------------ */
/* Gates (Section III, Eq. 2 on the reduced iteration set of Section III-B)             */
/* ------------------------------------------------------------------------------------ */

/* Apply G = U to `target` on the pairs selected by (ctrl_mask, ctrl_vals); 2^(n-1-c)
 * pairs are scheduled, c = popcount(ctrl_mask). U is not checked for unitarity. EINVAL if
 * target is out of range, the mask holds the target or bits >= n, ctrl_vals has bits
 * outside the mask, or U holds a NaN/Inf. Exact structure in U is used: [[0,1],[1,0]]
 * runs the exchange path (bit-exact), b = c = 0 runs a diagonal path, and a diagonal with
 * a == 1 (or d == 1) touches only the amplitudes it changes. */
qs_status qs_apply_gate(qs_state *s, int target, uint64_t ctrl_mask, uint64_t ctrl_vals,
                        const double U[8]);

/* Exchange the amplitudes of each selected pair (X / CNOT / Toffoli): bit-exact. */
qs_status qs_apply_x(qs_state *s, int target, uint64_t ctrl_mask, uint64_t ctrl_vals);

/* Comparator for the paper's baseline scheduling (Section III-A pseudocode): launches
 * all 2^(n-1) pair iterations and skips those whose controls fail. Same result as
 * qs_apply_gate; exists to measure the difference. */
qs_status qs_apply_gate_masked(qs_state *s, int target, uint64_t ctrl_mask,
                               uint64_t ctrl_vals, const double U[8]);

/* Apply `count` gates in order (gates run serially, Section III). RY/RZ gates read
 * theta[param] (theta may be NULL when no gate is parameterised; n_theta is its length).
 * All gates are validated before anything is launched. flags: QS_FLAG_FUSE runs runs of
 * consecutive gates whose targets fit in one shared-memory tile in one HBM round trip (a tile
 * pass; controls outside the tile select the tiles a gate changes) and runs of diagonal
 * gates in one pass each, as qs_circuit_schedule plans them. Such a plan may apply gates that
 * commute in another order than the given one (qs_circuit_order returns it): two gates keep
 * their order unless every qubit they share is, in both, a control or a qubit of a diagonal
 * gate. QS_FLAG_GRAPH records the
 * launches into a CUDA graph and launches it. Each state keeps up to 16 recorded graphs; a
 * call whose gate records, theta, flags, state buffer and tile size equal a recorded graph's
 * byte for byte replays it without validating or planning again (the hash that finds the
 * candidate is always confirmed by comparing the stored bytes).
 * Fused plans (of this call and of qs_adjoint_grad) are kept process-wide, the last 8: a call
 * with the same n, precision, flags, tile sizes and gate records whose gates keep their
 * structure for the new theta (the same operation class per gate: an angle that makes a
 * rotation the identity changes it) reuses the plan with its own matrices instead of planning
 * again; plans with diagonal-run passes or more than 65536 gates are not kept.
 * QS_FLAG_MASKED runs every gate with the baseline schedule of Section III-A instead (all
 * 2^(n-1) pair iterations, controls tested per pair, the general 2x2 update), the
 * comparator of qs_apply_gate_masked for whole circuits; QS_EINVAL with QS_FLAG_FUSE. */
qs_status qs_apply_circuit(qs_state *s, const qs_gate *gates, size_t count,
                           const double *theta, size_t n_theta, int flags);

/* The launch schedule qs_apply_circuit would use for `count` gates on an n-qubit state of
 * precision `dtype` with `flags`, computed on the host: no state, device or CUDA call is
 * needed. With QS_FLAG_ADJOINT: the schedule of qs_adjoint_grad with the other flags (forward
 * program, energy and lambda, reverse sweep over psi and lambda: a sweep launch moves both
 * vectors, so it counts twice in algorithmic_bytes and model_cost). Gates and flags are validated as by qs_apply_circuit (QS_EINVAL, nothing filled).
 * With QS_FLAG_FUSE this is the fusion planner's result (gate fusion is the optimisation
 * the paper's conclusion proposes): the gates, after same-target merging, cut into single
 * launches, tile passes and diagonal runs of least modelled cost. model_cost is that cost
 * in units of one read + write of the whole state (the planner's estimate, not a
 * measurement): per launch the fraction of the state it moves, the per-gate work inside a
 * pass, and ~2 us of launch latency; without QS_FLAG_FUSE the fraction is each gate's own
 * (1 per gate with QS_FLAG_MASKED). pass_gates does not count exchanges folded into a
 * register group's row copies. */
typedef struct {
    int32_t launches;      /* kernel launches */
    int32_t single_gates;  /* launches of one gate */
    int32_t tile_passes;   /* fused passes over shared-memory tiles */
    int32_t diag_runs;     /* passes that apply a run of diagonal gates */
    int32_t gates;         /* gates after same-target merging (identities included) */
    int32_t pass_gates;    /* gates applied inside tile passes */
    double model_cost;
    double algorithmic_bytes; /* bytes the launches must read + write: per single gate its
                                 selected amplitudes (2 * 2^(n-c) * s), per tile pass the
                                 tiles one of its gates selects (2 * fraction * 2^n * s),
                                 per diagonal run the chunks it can change */
    double algorithmic_flops; /* floating-point operations of the gate updates, in the state's
                                 precision: per selected pair 28 for a general 2x2 (16
                                 multiplications, 12 additions), 12 for a real or a diagonal
                                 matrix, 6 for a one-sided phase, 0 for an exchange; with
                                 QS_FLAG_ADJOINT also the sweep's un-apply of each gate on psi
                                 and on lambda, 8 per pair for each parameterised gate's
                                 derivative product Im <lambda|P psi> / 2 (P = Y or Z), and 8
                                 per amplitude for the energy and lambda = O psi. The same with
                                 and without QS_FLAG_FUSE (the circuit's arithmetic, not a
                                 kernel's). */
} qs_schedule;

qs_status qs_circuit_schedule(int n, qs_dtype dtype, const qs_gate *gates, size_t count,
                              const double *theta, size_t n_theta, int flags,
                              qs_schedule *out);

/* The order in which the plan of qs_circuit_schedule (same arguments) applies the gates:
 * order[0..count-1] receives a permutation of 0..count-1, gate indices as given, first
 * applied first; with QS_FLAG_ADJOINT the order of the reverse sweep (first un-applied
 * first). Host only, like qs_circuit_schedule. With QS_FLAG_FUSE the planner may apply gates
 * that commute in another order than the given one (Section III applies them serially; any
 * order that keeps each pair of gates that might not commute gives the same state): it
 * fills each tile pass with every gate whose predecessors have run and whose target is
 * local, adding the local qubit that releases the most gates, and keeps that order where its
 * modelled cost is lower. Gates merged with their same-target neighbours stay consecutive;
 * gates that change nothing (identity matrices) come last. Without QS_FLAG_FUSE the order is
 * the given one (reversed for the sweep). Errors as qs_circuit_schedule; order must hold
 * `count` entries (QS_EINVAL if NULL with count > 0). */
qs_status qs_circuit_order(int n, qs_dtype dtype, const qs_gate *gates, size_t count,
                           const double *theta, size_t n_theta, int flags, int32_t *order);

/* Measured FMA rate of the current device in the arithmetic of `dtype` (QS_C64: float32,
 * QS_C128: float64), in flop/s (2 per FMA): one launch of independent FMA chains on every SM
 * for `iters` iterations (1 .. 2^24), timed with CUDA events on `stream`; synchronises the
 * stream. It is the denominator of the arithmetic rooflines (the complex128 path runs on the
 * FP64 pipe). Not part of the paper's method. */
qs_status qs_measure_fma_peak(qs_dtype dtype, int iters, void *stream, double *flops_per_s);

/* Debug build (the library compiled with QS_DEBUG_CHECKS, libqs_debug.so): the gate,
 * sweep, tile-pass, diagonal-run and compiled single-state pass kernels check every global
 * access against a state of n_amps amplitudes (0: no check) and, when `counts` (device,
 * count_n uint32 entries) is given, count the writes of each amplitude with atomics. An access
 * outside the state is not made; the status word records it (bit 0) with one failing index.
 * qs_debug_configure synchronises the device, sets the checks and clears the status;
 * qs_debug_status synchronises and reads it. In the release build both return
 * QS_EUNSUPPORTED and qs_debug_build() returns 0. Not part of the paper's method. */
int qs_debug_build(void);
qs_status qs_debug_configure(uint64_t n_amps, unsigned int *counts, uint64_t count_n);
qs_status qs_debug_status(unsigned int *status, uint64_t *first_bad);

/* Compile the tile-pass kernels that qs_apply_circuit (adjoint = 0) or qs_adjoint_grad
 * (adjoint = 1: the forward and the reverse-sweep programs) would launch for these gates with
 * QS_FLAG_FUSE | QS_FLAG_JIT, without running anything; needs no device or state.
 * With QS_FLAG_JIT a fused pass is not interpreted gate by gate: the library writes the CUDA
 * source of one kernel for the pass's exact shape (its tile map, register groups, and every
 * gate's operation, target and controls as constants; the matrices stay kernel parameters),
 * compiles it for sm_103a with NVRTC and caches it for the life of the process by its source
 * text. Circuits with the same structure (e.g. the layers of a parameterised ansatz at other
 * angles) reuse the compiled kernels; the first call that needs a new shape compiles it,
 * which takes a fraction of a second to seconds. This call moves that cost out of the timed
 * or latency-critical path. With the environment variable QS_JIT_CACHE_DIR set to a writable
 * directory (created if its parent exists), every compiled kernel is also kept there (one file per kernel: its full source and
 * cubin, keyed by a hash of the source, the compile options and the NVRTC version; used only
 * when the stored source equals the wanted one), so that later processes load instead of
 * compiling. *compile_seconds (may be NULL) receives the compile (or load) time of this
 * call (0 when everything was cached), *passes (may be NULL) the number of tile passes.
 * QS_EINVAL for invalid gates (as qs_apply_circuit), QS_ECUDA if compilation fails. */
qs_status qs_circuit_compile(int n, qs_dtype dtype, const qs_gate *gates, size_t count,
                             const double *theta, size_t n_theta, int flags, int adjoint,
                             double *compile_seconds, int *passes);

/* Tile size of the fused passes (QS_FLAG_FUSE) for one precision, forward (adjoint = 0) or
 * adjoint sweep (adjoint = 1): `bits` local qubits per shared-memory tile, or 0 for the
 * library default (complex64: 12, and 11 for a sweep compiled with QS_FLAG_JIT; complex128:
 * 11 forward, 10 adjoint). Valid: 5 up to the
 * largest tile whose block fits one SM's shared memory (complex64 14 forward / 13 adjoint,
 * complex128 13 / 12); EINVAL otherwise. Process-wide; normally set from the autotuner's
 * cache. The QS_TILE_BITS environment variable overrides it (capped at that largest tile). */
qs_status qs_set_tile_bits(qs_dtype dtype, int adjoint, int bits);
/* The tile size the next fused call without QS_FLAG_JIT will use. */
int qs_get_tile_bits(qs_dtype dtype, int adjoint);

/* DRAM fetch size of the L2 (the context limit cudaLimitMaxL2FetchGranularity of this
 * process) that qs_state_alloc / qs_state_wrap set on their device: 32 (default), 64 or 128
 * bytes, or 0 to leave the context's limit alone. A gate whose controls sit on low qubits
 * selects runs of 8-64 bytes (every other run of 2^p amplitudes, p the lowest inserted
 * bit); with a 128-byte fetch each run costs a whole 128-byte DRAM block. The limit
 * belongs to the process's context and ends with it; it applies to every kernel of the
 * process on that device. The QS_L2_FETCH_BYTES environment variable sets the initial
 * value. EINVAL for any other value; takes effect at the next state on a device. */
qs_status qs_set_l2_fetch_bytes(int bytes);
int qs_get_l2_fetch_bytes(void);

/* ------------------------------------------------------------------------------------ */
/* Reductions (double-precision accumulation on the device)                             */
/* ------------------------------------------------------------------------------------ */

/* out[i] = <Z_i> = sum_k |psi_k|^2 (1 - 2 bit_i(k)) for i = 0..n-1, and, if out_norm2 is
 * not NULL, *out_norm2 = sum_k |psi_k|^2 -- all in one pass over the state. Complex64
 * states sum |psi_k|^2 in float32 within a tile of 8192 amplitudes, with a compensated
 * (Kahan) float32 running sum over a block's tiles and float64 across blocks; complex128
 * states sum in float64 throughout. Deterministic (fixed summation order).
 * With QS_FLAG_OUT_DEVICE in flags, out / out_norm2 are device pointers and the call is
 * asynchronous; otherwise they are host pointers and the call synchronises the stream. */
qs_status qs_expect_z(const qs_state *s, double *out, double *out_norm2, int flags);

/* Same results as qs_expect_z, for callers that cannot allocate device memory: code whose
 * device memory belongs to another allocator (a framework pool or a fixed arena), code on a
 * latency budget that cannot afford a cudaMalloc, code that must not run out of memory in
 * the middle of a job. No device or host memory is allocated by this call. (The paper has
 * no counterpart; this is an interface addition.)
 *  - psi: device pointer to 2^n amplitudes of `dtype` (16-byte aligned), read only.
 *  - out_z (n doubles) / out_norm2 (1 double): device pointers, either may be NULL (not both).
 *  - psi, out_z and out_norm2 must be device (or managed) memory of the current device:
 *    host memory or another device's memory is rejected with QS_EINVAL before any launch.
 *  - Enqueued on `stream`; returns without waiting.
 *  - The per-block partial sums go to one fixed device array inside the library
 *    (1024 * 41 doubles = 335,872 bytes per device, held until the process exits), which
 *    covers every n <= 40; larger requests are rejected with QS_EINVAL.
 *  - The first call on a device looks up that array's device address (a runtime query,
 *    done once per device with the device current); make that first call before any
 *    stream capture. The address is kept for the life of the process: after a
 *    cudaDeviceReset of that device, do not call this entry point again in the process.
 *  - All calls on a device share the array. Calls that may run at the same time on the GPU
 *    (other streams, other host threads) overwrite each other's partial sums: serialise
 *    them. Nothing needs clearing between calls: each call writes every slot it reads. */
qs_status qs_expect_z_noalloc(const void *psi, int n, qs_dtype dtype, void *stream, double *out_z,
                              double *out_norm2);

/* ------------------------------------------------------------------------------------ */
/* Adjoint gradient (reverse sweep that un-applies gates; no checkpoints)               */
/* ------------------------------------------------------------------------------------ */

/* For E(theta) = <psi|O|psi>, O = sum_i Z_i, psi = C(theta)|psi_in>: on entry the state
 * holds psi_in; the call applies the circuit, writes E to *energy and dE/dtheta[p] to
 * grad[p] for p < n_theta (parameters that drive no gate get 0), running the reverse
 * sweep psi <- U_g^dagger psi, lambda <- U_g^dagger lambda with
 * grad += 2 Re <lambda| dU_g/dtheta psi> for every RY/RZ gate. On return the state holds
 * psi_in recomputed by the sweep (up to rounding). A second vector (lambda) is allocated
 * on first use and kept with the state. Inner products accumulate in float64.
 * QS_FLAG_FUSE groups low-target gates into tile passes (and may apply commuting gates in
 * another order, forward and in the sweep; see qs_circuit_order); QS_FLAG_OUT_DEVICE makes
 * energy and grad device pointers (asynchronous); otherwise host pointers (synchronous).
 * Fused plans are kept as for qs_apply_circuit. */
qs_status qs_adjoint_grad(qs_state *s, const qs_gate *gates, size_t count,
                          const double *theta, size_t n_theta, double *energy,
                          double *grad, int flags);

/* ------------------------------------------------------------------------------------ */
/* Batched forward energy + adjoint gradient (one persistent launch in a CUDA graph)     */
/* ------------------------------------------------------------------------------------ */

typedef struct qs_batch qs_batch;  /* opaque */

/* Plan a batch of independent states. State s has n_qubits[s] qubits (1..30), starts from
 * |0...0>, runs gates[gate_offsets[s] .. gate_offsets[s+1]) (qs_gate records; RY/RZ
 * parameter indices are relative to the state), and owns the parameters
 * theta[param_offsets[s] .. param_offsets[s+1]) (at most 4096 per state). Both offset arrays
 * have num_states + 1 entries and start at 0. The observable is sum_i Z_i for every state.
 * Tuning (0 = library default): small_bits — states with n <= small_bits stay in shared memory
 * for the whole computation; tile_bits (5..14) — local qubits of the tile passes of larger
 * states; max_pass_gates — gates per tile pass (fusion depth). All arguments are host
 * memory and copied; everything is validated before any device work. Allocates the device
 * descriptors and, for states above small_bits, a per-CTA workspace of two vectors of the
 * largest such state. ENOMEM / EINVAL / ECUDA on failure. */
qs_status qs_batch_create(int num_states, const int *n_qubits, const qs_gate *gates,
                          const uint64_t *gate_offsets, const uint64_t *param_offsets, qs_dtype dtype,
                          int small_bits, int tile_bits, int max_pass_gates, void *stream,
                          qs_batch **out);

/* Run the batch: theta (device, param_offsets[num_states] doubles) -> energy[s] (device,
 * num_states doubles) and grad (device, param_offsets[num_states] doubles), all in float64.
 * One persistent kernel: each CTA takes states from a device work queue (largest first;
 * nothing waits on anything, so no bounded wait is needed). With QS_FLAG_GRAPH the queue
 * reset and the kernel are recorded once into a CUDA graph (re-recorded when the three
 * pointers change) and launched as a graph; otherwise they are launched directly.
 * Asynchronous on the batch's stream. */
qs_status qs_batch_run(qs_batch *b, const double *theta, double *energy, double *grad, int flags);

/* Chosen launch configuration and memory of a batch (any pointer may be NULL). */
qs_status qs_batch_info(const qs_batch *b, int *grid, int *small_bits, int *tile_bits,
                        int *max_pass_gates, size_t *smem_bytes, size_t *workspace_bytes);

/* Bytes one run of the batch must move through device memory (its states above small_bits:
 * |0...0> written, each forward pass reading and writing the tiles its gates select, lambda =
 * O psi, each sweep pass reading and writing the selected tiles of psi and lambda; states in
 * shared memory move none): the numerator of the batch's roofline. Host only. */
qs_status qs_batch_bytes(const qs_batch *b, double *algorithmic_bytes);

/* Release a batch (synchronises its stream first). NULL is accepted. */
qs_status qs_batch_free(qs_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* QS_H */
