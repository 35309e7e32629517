"""Seeded synthetic inputs for the controlled-gate state-vector path.

This module only draws random numbers and lays them out: gate lists (targets, control
sets, 2x2 matrices, parameter indices) and start states. It applies no gate, computes no
amplitude update and holds none of the method's arithmetic, so both the CUDA library and
the CPU oracle can take its output as their common input.

Gate records use ``GATE_DTYPE``, a numpy structured dtype whose layout is the C struct
``qs_gate`` (96 bytes): target, kind, ctrl_mask, ctrl_vals, param, reserved, U[8] with U
the row-major 2x2 matrix [a b; c d] as interleaved (re, im) doubles (Section III, Eq. 2
names the entries a, b, c, d). Qubit 0 is the least significant bit of an amplitude index
(Section III).

Readings of the workload descriptions (stated here because the source text leaves them
open):
- "Haar-random 2x2 unitary (QR of a complex Gaussian)": Q from the QR factorisation of a
  2x2 matrix of i.i.d. standard complex Gaussians, with each column rescaled by the phase
  of the matching diagonal entry of R (Mezzadri's correction; without it the
  distribution is not Haar).
- "0-k controls drawn uniformly from the other qubits": the count c is uniform on
  {0..k}, then c distinct qubits are drawn uniformly from the n-1 non-target qubits, all
  controls on |1> (ctrl_vals == ctrl_mask).
- Permutation gates "X/CNOT/Toffoli making up 25%": each gate is a permutation gate with
  probability 0.25, uniform over {X, CNOT, Toffoli} on distinct random qubits.
- Hardware-efficient ansatz: per layer RY(theta) then RZ(theta) on every qubit (separate
  parameters), then CNOT(i -> i+1) for i = 0..n-2 (an open ladder), from |0...0>.
- R_m (QFT, Section IV-A) is not defined in the text: R_m = diag(1, exp(2 pi i / 2^m)).
- Seeds: numpy ``default_rng(seed)``; seed = workload index 0..4; state s of the batch
  uses seed 4_000_000 + s.
"""
from __future__ import annotations

import numpy as np

# Gate kinds (same values as the QS_GATE_* constants of the C interface).
KIND_U = 0   # general 2x2 matrix in U
KIND_X = 1   # permutation: exchange the two amplitudes of each selected pair
KIND_RY = 2  # RY(theta[param]) = exp(-i theta Y / 2)
KIND_RZ = 3  # RZ(theta[param]) = exp(-i theta Z / 2)

GATE_DTYPE = np.dtype(
    [
        ("target", "<i4"),
        ("kind", "<i4"),
        ("ctrl_mask", "<u8"),
        ("ctrl_vals", "<u8"),
        ("param", "<i4"),
        ("reserved", "<i4"),
        ("U", "<f8", (8,)),
    ],
    align=True,
)
assert GATE_DTYPE.itemsize == 96

# Hadamard and Pauli-X as written in Section II-A.
H_MATRIX = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / np.sqrt(2.0)
X_MATRIX = np.array([[0.0, 1.0], [1.0, 0.0]], dtype=np.complex128)

SWEEP_TARGETS = (0, 15, 29)


def pack_u(u2: np.ndarray) -> np.ndarray:
    """Row-major 2x2 complex matrix -> 8 interleaved doubles [re a, im a, re b, ...]."""
    u2 = np.asarray(u2, dtype=np.complex128).reshape(2, 2)
    out = np.empty(8, dtype=np.float64)
    out[0::2] = u2.reshape(-1).real
    out[1::2] = u2.reshape(-1).imag
    return out


def unpack_u(u8: np.ndarray) -> np.ndarray:
    u8 = np.asarray(u8, dtype=np.float64)
    return (u8[0::2] + 1j * u8[1::2]).reshape(2, 2)


def make_gate(target: int, u2=None, controls=(), vals=None, kind: int = KIND_U, param: int = -1):
    """One gate record. ``controls`` are qubit indices; ``vals`` the required bit values
    (default: all 1)."""
    g = np.zeros((), dtype=GATE_DTYPE)
    mask = 0
    v = 0
    controls = list(controls)
    if vals is None:
        vals = [1] * len(controls)
    for q, b in zip(controls, vals):
        mask |= 1 << int(q)
        if b:
            v |= 1 << int(q)
    g["target"] = int(target)
    g["kind"] = int(kind)
    g["ctrl_mask"] = mask
    g["ctrl_vals"] = v
    g["param"] = int(param)
    if u2 is not None:
        g["U"] = pack_u(u2)
    elif kind == KIND_X:
        g["U"] = pack_u(X_MATRIX)
    return g


def gate_list(gates) -> np.ndarray:
    arr = np.zeros(len(gates), dtype=GATE_DTYPE)
    for i, g in enumerate(gates):
        arr[i] = g
    return arr


def haar_2x2(rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(2) by QR of a complex Gaussian matrix with Mezzadri's phase fix."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return q * ph[None, :]


def random_controls(rng: np.random.Generator, n: int, target: int, c: int):
    others = np.array([q for q in range(n) if q != target], dtype=np.int64)
    if c == 0:
        return []
    return sorted(int(q) for q in rng.choice(others, size=c, replace=False))


def random_gate(rng: np.random.Generator, n: int, cmax: int):
    t = int(rng.integers(0, n))
    c = int(rng.integers(0, min(cmax, n - 1) + 1))
    ctrls = random_controls(rng, n, t, c)
    return make_gate(t, haar_2x2(rng), ctrls)


def random_circuit(n: int, count: int, cmax: int, seed: int, hadamard_prefix: bool = False,
                   perm_fraction: float = 0.0) -> np.ndarray:
    """``count`` random gates on ``n`` qubits: Haar 2x2 with 0..cmax controls on |1>; with
    probability ``perm_fraction`` a gate is instead X, CNOT or Toffoli on random qubits."""
    rng = np.random.default_rng(seed)
    gates = []
    if hadamard_prefix:
        gates.extend(make_gate(q, H_MATRIX) for q in range(n))
    for _ in range(count):
        if perm_fraction > 0.0 and rng.random() < perm_fraction:
            nc = int(rng.integers(0, min(2, n - 1) + 1))  # X, CNOT or Toffoli
            qs = [int(q) for q in rng.choice(n, size=nc + 1, replace=False)]
            gates.append(make_gate(qs[0], None, sorted(qs[1:]), kind=KIND_X))
        else:
            gates.append(random_gate(rng, n, cmax))
    return gate_list(gates)


def small_exact_circuit(seed: int = 0) -> np.ndarray:
    """12 qubits: H on every qubit, then 200 Haar gates with 0-3 controls (seed 0)."""
    return random_circuit(12, 200, 3, seed, hadamard_prefix=True)


def scale_circuit(n: int = 30, count: int = 1000, seed: int = 1) -> np.ndarray:
    """The 1000-gate random circuit at scale: 0-8 controls."""
    return random_circuit(n, count, 8, seed)


def precision_circuit(n: int = 32, count: int = 2000, seed: int = 2) -> np.ndarray:
    """2000 gates: Haar with 0-6 controls, 25 % permutation gates."""
    return random_circuit(n, count, 6, seed, perm_fraction=0.25)


def sweep_gates(n: int = 30, cmax: int = 8, targets=SWEEP_TARGETS, sets: int = 8, seed: int = 1):
    """Single-gate sweep: for every control count c = 0..cmax and target in ``targets``,
    ``sets`` seeded random control sets, each with its own Haar matrix.

    Returns a dict (c, t) -> gate array of length ``sets``."""
    rng = np.random.default_rng(seed)
    out = {}
    for c in range(cmax + 1):
        for t in targets:
            gl = []
            for _ in range(sets):
                ctrls = random_controls(rng, n, t, c)
                gl.append(make_gate(t, haar_2x2(rng), ctrls))
            out[(c, t)] = gate_list(gl)
    return out


def hea_circuit(n: int, layers: int) -> np.ndarray:
    """Hardware-efficient ansatz: per layer RY then RZ on every qubit, then a CNOT ladder
    i -> i+1. Parameter p indexes theta; 2*n*layers parameters in gate order."""
    gates = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            gates.append(make_gate(q, None, (), kind=KIND_RY, param=p))
            p += 1
            gates.append(make_gate(q, None, (), kind=KIND_RZ, param=p))
            p += 1
        for q in range(n - 1):
            gates.append(make_gate(q + 1, None, (q,), kind=KIND_X))
    return gate_list(gates)


def hea_params(n: int, layers: int, seed: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 2.0 * np.pi, size=2 * n * layers)


def batch_workload(num_states: int = 4096, nmin: int = 10, nmax: int = 20, layers: int = 8,
                   seed: int = 4):
    """Batch of independent ansatz states: qubit counts uniform on nmin..nmax (seed 4),
    parameters of state s drawn from seed 4_000_000 + s."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=num_states).astype(np.int32)
    thetas = [hea_params(int(n), layers, seed=4_000_000 + s) for s, n in enumerate(ns)]
    return ns, thetas


def phase_rm(m: int) -> np.ndarray:
    """R_m = diag(1, exp(2 pi i / 2^m)). The text uses R_m in its QFT circuit without
    defining it; this is the usual QFT phase gate."""
    return np.diag([1.0 + 0.0j, np.exp(2j * np.pi / float(1 << m))])


def qft_circuit(n: int) -> np.ndarray:
    """The QFT staircase of Section IV-A (Fig. qft_circuit) for n qubits, as drawn: for
    j = 0..n-1, H on q_j, then R_m on q_j controlled by q_(j+m-1) for m = 2..n-j. No final
    swaps. n + n(n-1)/2 gates (435 at n = 29)."""
    gates = []
    for j in range(n):
        gates.append(make_gate(j, H_MATRIX))
        for m in range(2, n - j + 1):
            gates.append(make_gate(j, phase_rm(m), (j + m - 1,)))
    return gate_list(gates)


def streaming_circuit(n: int, reverse: bool = False) -> np.ndarray:
    """The streaming circuit of Section IV-C (Fig. streaming_circ): X on x_q controlled by
    x_0..x_(q-1) on |1>, for q = 0..n-1 in drawn order (``reverse`` runs q = n-1..0). Gate q
    has q controls, so the last one has n-1."""
    order = range(n - 1, -1, -1) if reverse else range(n)
    return gate_list([make_gate(q, None, tuple(range(q)), kind=KIND_X) for q in order])


def random_state(n: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Normalised complex Gaussian state of 2^n amplitudes, rounded to ``dtype``."""
    rng = np.random.default_rng(seed)
    N = 1 << n
    if dtype == np.complex64:
        v = np.empty(N, dtype=np.complex64)
        f = v.view(np.float32)
        chunk = 1 << 24
        s = 0.0
        for i in range(0, 2 * N, chunk):
            blk = rng.standard_normal(min(chunk, 2 * N - i), dtype=np.float32)
            f[i:i + blk.size] = blk
            s += float(np.dot(blk.astype(np.float64), blk.astype(np.float64)))
        f *= np.float32(1.0 / np.sqrt(s))
        return v
    v = rng.standard_normal(2 * N).view(np.complex128)
    v /= np.sqrt(np.vdot(v, v).real)
    return v.astype(dtype, copy=False)


def basis_state(n: int, k: int, dtype=np.complex128) -> np.ndarray:
    v = np.zeros(1 << n, dtype=dtype)
    v[k] = 1.0
    return v
