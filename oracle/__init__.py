"""CPU reference oracle for the controlled single-qubit gate path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg are the only users. The product library never imports this package, and
this package imports nothing from the product library.

Pieces and the passages they follow:
- ``apply_gate`` / ``apply_x``: Section III, Eq. 2 with the per-index control test of the
  baseline kernel (Section III-A), written in plain C (``qs_oracle.c``), double precision.
- ``gate_output``: the same update for one output amplitude (sampled checks at full size).
- ``ith_cleared`` / ``eq4_map``: Section III-B, Eqs. 3 and 4, the paper's reduced-to-global
  iteration map, used by the pins that fix the index arithmetic.
- ``expect_z`` / ``norm2`` / ``inner_re``: sequential double sums over all amplitudes.
- ``ry`` / ``rz``: the rotation matrices exp(-i theta Y/2), exp(-i theta Z/2) (standard
  definitions; the paper has no parameterised gates).
- ``energy`` / ``param_shift_grad`` / ``fd_grad``: E = <psi|sum_i Z_i|psi>; its gradient by
  the two-term parameter-shift rule (exact for RY/RZ, Mitarai et al. 2018; Schuld et al.
  2019) and by central finite differences.
- ``quantize_q30`` / ``apply_gate_q30`` / ``run_circuit_q30`` / ``gate_output_q30`` /
  ``expect_z_q30``: fixed-point amplitudes (the paper's conclusion names them as future work;
  the format is this library's choice): Q1.30 integers, Eq. 2 in exact 64-bit integer
  products, one rounding per output component (nearest, halves toward +infinity), clamped.

Parity: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import numpy as np

from .build import build as _build, LIB_PATH

_lib = None
_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)

KIND_U, KIND_X, KIND_RY, KIND_RZ = 0, 1, 2, 3


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            _build()
        L = ctypes.CDLL(LIB_PATH)
        L.oracle_ith_cleared.restype = _u64
        L.oracle_ith_cleared.argtypes = [_u64, ctypes.c_int]
        L.oracle_eq4_map.restype = _u64
        L.oracle_eq4_map.argtypes = [_u64, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        L.oracle_apply_gate.restype = None
        L.oracle_apply_gate.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _u64, _u64, _dp]
        L.oracle_apply_x.restype = None
        L.oracle_apply_x.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _u64, _u64]
        L.oracle_gate_output.restype = None
        L.oracle_gate_output.argtypes = [_u64, ctypes.c_int, _u64, _u64, _dp, _dp, _dp, _dp]
        L.oracle_norm2.restype = ctypes.c_double
        L.oracle_norm2.argtypes = [_dp, ctypes.c_int]
        L.oracle_expect_z.restype = None
        L.oracle_expect_z.argtypes = [_dp, ctypes.c_int, _dp]
        L.oracle_inner_re.restype = ctypes.c_double
        L.oracle_inner_re.argtypes = [_dp, _dp, ctypes.c_int]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        _ip = ctypes.POINTER(ctypes.c_int32)
        L.oracle_quantize_q30.restype = ctypes.c_int32
        L.oracle_quantize_q30.argtypes = [ctypes.c_double]
        L.oracle_apply_gate_q30.restype = None
        L.oracle_apply_gate_q30.argtypes = [_ip, ctypes.c_int, ctypes.c_int, _u64, _u64, _ip]
        L.oracle_gate_output_q30.restype = None
        L.oracle_gate_output_q30.argtypes = [_u64, ctypes.c_int, _u64, _u64, _ip, _ip, _ip, _ip]
        L.oracle_expect_z_q30.restype = None
        L.oracle_expect_z_q30.argtypes = [_ip, ctypes.c_int, _dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _check_state(psi: np.ndarray, n: int):
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.size != (1 << n):
        raise ValueError("oracle state must be a contiguous complex128 array of 2^n amplitudes")


def _check_gate(n: int, t: int, ctrl_mask: int, ctrl_vals: int):
    if not (0 <= t < n) or ctrl_mask >> n or (ctrl_mask >> t) & 1 or ctrl_vals & ~ctrl_mask:
        raise ValueError(f"invalid gate for n={n}: t={t}, mask={ctrl_mask:#x}, vals={ctrl_vals:#x}")


def _u8(U) -> np.ndarray:
    U = np.asarray(U)
    if U.dtype == np.complex128 or U.shape == (2, 2):
        U = np.asarray(U, dtype=np.complex128).reshape(4)
        out = np.empty(8)
        out[0::2] = U.real
        out[1::2] = U.imag
        return out
    return np.ascontiguousarray(U, dtype=np.float64).reshape(8)


def num_threads() -> int:
    return lib().oracle_num_threads()


def ith_cleared(i: int, t: int) -> int:
    return int(lib().oracle_ith_cleared(i, t))


def eq4_map(i_r: int, t: int, controls) -> int:
    c = (ctypes.c_int * max(1, len(controls)))(*controls)
    return int(lib().oracle_eq4_map(i_r, t, c, len(controls)))


def apply_gate(psi: np.ndarray, n: int, t: int, ctrl_mask: int, ctrl_vals: int, U) -> None:
    """In place: Eq. 2 on the pairs of target t whose bits under ctrl_mask equal ctrl_vals."""
    _check_state(psi, n)
    _check_gate(n, t, ctrl_mask, ctrl_vals)
    u = _u8(U)
    lib().oracle_apply_gate(_ptr(psi.view(np.float64)), n, t, ctrl_mask, ctrl_vals, _ptr(u))


def apply_x(psi: np.ndarray, n: int, t: int, ctrl_mask: int = 0, ctrl_vals: int = 0) -> None:
    """In place: exchange the amplitudes of every selected pair (X, CNOT, Toffoli)."""
    _check_state(psi, n)
    _check_gate(n, t, ctrl_mask, ctrl_vals)
    lib().oracle_apply_x(_ptr(psi.view(np.float64)), n, t, ctrl_mask, ctrl_vals)


def gate_output(k: int, t: int, ctrl_mask: int, ctrl_vals: int, U, in_k: complex,
                in_partner: complex) -> complex:
    """Output amplitude k of one gate, given input amplitudes C_k and C_{k xor 2^t}."""
    a = np.array([in_k.real, in_k.imag])
    b = np.array([in_partner.real, in_partner.imag])
    o = np.empty(2)
    u = _u8(U)
    lib().oracle_gate_output(k, t, ctrl_mask, ctrl_vals, _ptr(u), _ptr(a), _ptr(b), _ptr(o))
    return complex(o[0], o[1])


def norm2(psi: np.ndarray, n: int) -> float:
    _check_state(psi, n)
    return float(lib().oracle_norm2(_ptr(psi.view(np.float64)), n))


def expect_z(psi: np.ndarray, n: int) -> np.ndarray:
    _check_state(psi, n)
    out = np.empty(n)
    lib().oracle_expect_z(_ptr(psi.view(np.float64)), n, _ptr(out))
    return out


def inner_re(a: np.ndarray, b: np.ndarray, n: int) -> float:
    _check_state(a, n)
    _check_state(b, n)
    return float(lib().oracle_inner_re(_ptr(a.view(np.float64)), _ptr(b.view(np.float64)), n))


def ry(theta: float) -> np.ndarray:
    """RY(theta) = exp(-i theta Y / 2) = [[cos, -sin], [sin, cos]] of theta/2."""
    c, s = np.cos(theta / 2.0), np.sin(theta / 2.0)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(theta: float) -> np.ndarray:
    """RZ(theta) = exp(-i theta Z / 2) = diag(e^{-i theta/2}, e^{+i theta/2})."""
    return np.array([[np.exp(-0.5j * theta), 0.0], [0.0, np.exp(0.5j * theta)]], dtype=np.complex128)


def gate_matrix(g, theta=None) -> np.ndarray:
    """2x2 matrix of one gate record (a ``GATE_DTYPE`` element)."""
    kind = int(g["kind"])
    if kind == KIND_RY:
        return ry(float(theta[int(g["param"])]))
    if kind == KIND_RZ:
        return rz(float(theta[int(g["param"])]))
    if kind == KIND_X:
        return np.array([[0.0, 1.0], [1.0, 0.0]], dtype=np.complex128)
    u = np.asarray(g["U"], dtype=np.float64)
    return (u[0::2] + 1j * u[1::2]).reshape(2, 2)


def run_circuit(psi: np.ndarray, n: int, gates, theta=None) -> np.ndarray:
    """Apply the gate records in order (serially, Section III-A), in place; returns psi."""
    for g in gates:
        t = int(g["target"])
        m = int(g["ctrl_mask"])
        v = int(g["ctrl_vals"])
        if int(g["kind"]) == KIND_X:
            apply_x(psi, n, t, m, v)
        else:
            apply_gate(psi, n, t, m, v, gate_matrix(g, theta))
    return psi


def energy(n: int, gates, theta, psi0=None) -> float:
    """E(theta) = <psi|sum_i Z_i|psi> with psi = circuit(theta)|psi0> (psi0 = |0...0>)."""
    if psi0 is None:
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1.0
    else:
        psi = np.array(psi0, dtype=np.complex128, copy=True)
    run_circuit(psi, n, gates, theta)
    return float(np.sum(expect_z(psi, n)))


def param_shift_grad(n: int, gates, theta, psi0=None) -> np.ndarray:
    """dE/dtheta_p = [E(theta_p + pi/2) - E(theta_p - pi/2)] / 2, exact for uncontrolled RY/RZ
    gates (generator with eigenvalues +-1/2) when each parameter drives one gate. A controlled
    rotation's generator also has eigenvalue 0, where the two-term rule does not hold: such
    circuits are rejected (use fd_grad)."""
    for g in gates:
        if int(g["kind"]) in (KIND_RY, KIND_RZ) and int(g["ctrl_mask"]) != 0:
            raise ValueError("param_shift_grad: the two-term shift rule needs uncontrolled rotations")
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros_like(theta)
    for p in range(theta.size):
        tp = theta.copy()
        tp[p] += np.pi / 2
        tm = theta.copy()
        tm[p] -= np.pi / 2
        g[p] = 0.5 * (energy(n, gates, tp, psi0) - energy(n, gates, tm, psi0))
    return g


def fd_grad(n: int, gates, theta, h: float = 1e-4, psi0=None) -> np.ndarray:
    """Central finite differences [E(theta_p + h) - E(theta_p - h)] / (2h), error O(h^2)."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros_like(theta)
    for p in range(theta.size):
        tp = theta.copy()
        tp[p] += h
        tm = theta.copy()
        tm[p] -= h
        g[p] = (energy(n, gates, tp, psi0) - energy(n, gates, tm, psi0)) / (2.0 * h)
    return g


# ---------------------------------------------------------------------------------------
# Fixed-point amplitudes (Q1.30): int32 (re, im) pairs, value = integer / 2^30
# ---------------------------------------------------------------------------------------

Q30_ONE = 1 << 30


def quantize_q30(v: float) -> int:
    """Q1.30 integer of a real number: nearest, halves away from zero, clamped to int32."""
    return int(lib().oracle_quantize_q30(float(v)))


def q30_matrix(U) -> np.ndarray:
    """A 2x2 complex matrix (or 8 interleaved doubles) as 8 Q1.30 integers."""
    u = _u8(U)
    return np.array([quantize_q30(x) for x in u], dtype=np.int32)


def _check_q30(psi: np.ndarray, n: int):
    if psi.dtype != np.int32 or not psi.flags.c_contiguous or psi.shape != (1 << n, 2):
        raise ValueError("Q1.30 oracle state must be a contiguous int32 array of shape (2^n, 2)")


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def apply_gate_q30(psi: np.ndarray, n: int, t: int, ctrl_mask: int, ctrl_vals: int, U) -> None:
    """In place: Eq. 2 in Q1.30 on the selected pairs (U quantised with quantize_q30)."""
    _check_q30(psi, n)
    _check_gate(n, t, ctrl_mask, ctrl_vals)
    uq = q30_matrix(U)
    lib().oracle_apply_gate_q30(_iptr(psi), n, t, ctrl_mask, ctrl_vals, _iptr(uq))


def run_circuit_q30(psi: np.ndarray, n: int, gates, theta=None) -> np.ndarray:
    """Apply the gate records in order to a Q1.30 state (X gates as their exact matrix)."""
    for g in gates:
        apply_gate_q30(psi, n, int(g["target"]), int(g["ctrl_mask"]), int(g["ctrl_vals"]), gate_matrix(g, theta))
    return psi


def gate_output_q30(k: int, t: int, ctrl_mask: int, ctrl_vals: int, U, in_k, in_partner) -> tuple:
    uq = q30_matrix(U)
    a = np.ascontiguousarray(in_k, dtype=np.int32)
    b = np.ascontiguousarray(in_partner, dtype=np.int32)
    o = np.empty(2, dtype=np.int32)
    lib().oracle_gate_output_q30(k, t, ctrl_mask, ctrl_vals, _iptr(uq), _iptr(a), _iptr(b), _iptr(o))
    return int(o[0]), int(o[1])


def expect_z_q30(psi: np.ndarray, n: int) -> np.ndarray:
    _check_q30(psi, n)
    out = np.empty(n)
    lib().oracle_expect_z_q30(_iptr(psi), n, _ptr(out))
    return out


def to_q30(psi: np.ndarray) -> np.ndarray:
    """A complex vector as Q1.30 integers (each part quantised)."""
    psi = np.asarray(psi, dtype=np.complex128)
    out = np.empty((psi.size, 2), dtype=np.int32)
    lib_q = lib().oracle_quantize_q30
    for k, z in enumerate(psi):
        out[k, 0] = lib_q(float(z.real))
        out[k, 1] = lib_q(float(z.imag))
    return out
