"""Pins for the CPU oracle: each check fixes the oracle to something other than itself
(values the paper prints, closed forms, textbook special cases, invariants, brute force on
tiny inputs), so that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------------------
# Index map: Section III-B, Eqs. 3-4
# --------------------------------------------------------------------------------------

def test_worked_example_eq4():
    """The paper's worked example (3 qubits, t = 1) after Eq. 4."""
    g = _load("worked_example_eq4.json")
    t = g["t"]
    for case in g["cases"]:
        ctrls = case["controls"]
        adj = [c - 1 if c > t else c for c in ctrls]
        assert adj == case["adjusted"]
        got = [oracle.eq4_map(i, t, ctrls) for i in case["I_r"]]
        assert got == case["I_g"], case


def _masked_pairs(n, t, ctrls):
    """Brute force: first pair elements k (bit t clear) whose control bits are all 1."""
    out = []
    for k in range(1 << n):
        if (k >> t) & 1:
            continue
        if all((k >> c) & 1 for c in ctrls):
            out.append(k)
    return out


def test_eq4_matches_masked_enumeration_exhaustive():
    """For n <= 7, every target and every ascending control subset, ithCleared(Eq. 4 map of
    I_r) enumerates exactly the masked pairs of the baseline kernel, in increasing order."""
    for n in range(1, 8):
        for t in range(n):
            others = [q for q in range(n) if q != t]
            for nc in range(len(others) + 1):
                for ctrls in itertools.combinations(others, nc):
                    size = 1 << (n - 1 - nc)
                    got = [oracle.ith_cleared(oracle.eq4_map(i, t, list(ctrls)), t)
                           for i in range(size)]
                    assert got == _masked_pairs(n, t, ctrls), (n, t, ctrls)


def test_eq4_needs_ascending_controls():
    """Section III-B: the map only works with controls in ascending order; in descending
    order it fails for some cases."""
    bad = 0
    n = 5
    for t in range(n):
        others = [q for q in range(n) if q != t]
        for ctrls in itertools.combinations(others, 2):
            desc = list(reversed(ctrls))
            got = [oracle.ith_cleared(oracle.eq4_map(i, t, desc), t)
                   for i in range(1 << (n - 3))]
            if sorted(got) != _masked_pairs(n, t, ctrls):
                bad += 1
    assert bad > 0


def test_ith_cleared_pairs():
    """ithCleared(i, t) and ithCleared(i, t) + 2^t partition all indices into the pairs of
    target t (Section III: pairs are 2^t apart)."""
    for n in range(1, 9):
        for t in range(n):
            firsts = [oracle.ith_cleared(i, t) for i in range(1 << (n - 1))]
            seconds = [k + (1 << t) for k in firsts]
            assert sorted(firsts + seconds) == list(range(1 << n))
            assert all(((k >> t) & 1) == 0 for k in firsts)


# --------------------------------------------------------------------------------------
# Gate update: Section III, Eq. 2, against a dense Kronecker brute force
# --------------------------------------------------------------------------------------

def _kron_all(ops):
    """ops[q] is the 2x2 operator on qubit q; qubit n-1 is the leftmost factor."""
    M = np.array([[1.0 + 0j]])
    for op in reversed(ops):
        M = np.kron(M, op)
    return M


def dense_controlled(n, t, ctrls, vals, U):
    """Dense 2^n x 2^n matrix: (I - P) + P (U on t), P the projector onto the control
    pattern (|v_q><v_q| on every control q, identity elsewhere)."""
    I2 = np.eye(2, dtype=np.complex128)
    P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
    P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)
    proj = [I2] * n
    for q, v in zip(ctrls, vals):
        proj[q] = P1 if v else P0
    P = _kron_all(proj)
    uops = [I2] * n
    uops[t] = np.asarray(U, dtype=np.complex128)
    Ut = _kron_all(uops)
    return np.eye(1 << n, dtype=np.complex128) - P + P @ Ut


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_apply_gate_matches_dense_kronecker(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(6 if n < 10 else 3):
        t = int(rng.integers(0, n))
        others = [q for q in range(n) if q != t]
        nc = int(rng.integers(0, len(others) + 1)) if others else 0
        ctrls = sorted(rng.choice(others, size=nc, replace=False).tolist()) if nc else []
        vals = [int(b) for b in rng.integers(0, 2, size=nc)]
        U = W.haar_2x2(rng) * (1.0 + 0.5 * rng.random())  # not unitary: no symmetry to hide behind
        U[0, 1] += 0.3j  # break U == U^T
        psi = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n))
        want = dense_controlled(n, t, ctrls, vals, U) @ psi
        got = psi.copy()
        mask = sum(1 << c for c in ctrls)
        v = sum(1 << c for c, b in zip(ctrls, vals) if b)
        oracle.apply_gate(got, n, t, mask, v, U)
        assert np.max(np.abs(got - want)) < 1e-12


def test_gate_output_matches_apply_gate():
    rng = np.random.default_rng(7)
    n = 9
    for _ in range(10):
        g = W.random_gate(rng, n, 4)
        U = W.unpack_u(g["U"])
        psi = W.random_state(n, int(rng.integers(1 << 30)))
        ref = psi.copy()
        oracle.apply_gate(ref, n, int(g["target"]), int(g["ctrl_mask"]), int(g["ctrl_vals"]), U)
        t = int(g["target"])
        for k in rng.integers(0, 1 << n, size=40):
            k = int(k)
            o = oracle.gate_output(k, t, int(g["ctrl_mask"]), int(g["ctrl_vals"]), U,
                                   psi[k], psi[k ^ (1 << t)])
            assert o == ref[k]


# --------------------------------------------------------------------------------------
# Section II-A gate definitions, Fig. 1, truth tables
# --------------------------------------------------------------------------------------

def test_x_and_h_actions():
    g = _load("section2_gates.json")
    for vin, vout in zip(g["X_action"]["in"], g["X_action"]["out"]):
        psi = np.array(vin, dtype=np.complex128)
        oracle.apply_x(psi, 1, 0)
        assert np.array_equal(psi, np.array(vout, dtype=np.complex128))
        psi = np.array(vin, dtype=np.complex128)
        oracle.apply_gate(psi, 1, 0, 0, 0, W.X_MATRIX)
        assert np.array_equal(psi, np.array(vout, dtype=np.complex128))
    for vin, vout in zip(g["H_action"]["in"], g["H_action"]["out_times_sqrt2"]):
        psi = np.array(vin, dtype=np.complex128)
        oracle.apply_gate(psi, 1, 0, 0, 0, W.H_MATRIX)
        assert np.allclose(psi * np.sqrt(2.0), vout, atol=1e-15, rtol=0)


def test_cnot_truth_table_fig1():
    g = _load("section2_gates.json")["cnot_fig1_left"]["map"]
    for kin, kout in g.items():
        kin, kout = int(kin), int(kout)
        psi = W.basis_state(2, kin)
        oracle.apply_x(psi, 2, 0, 0b10, 0b10)
        assert np.array_equal(psi, W.basis_state(2, kout))


@pytest.mark.parametrize("n", [3, 4, 6])
def test_toffoli_and_x_truth_tables(n):
    """X flips bit t; CNOT flips t iff the control is 1; Toffoli iff both controls are 1
    (also with negative controls: flip iff the control bits equal ctrl_vals)."""
    for t in range(n):
        others = [q for q in range(n) if q != t]
        for nc in range(3):
            for ctrls in itertools.combinations(others, nc):
                for vals in itertools.product([0, 1], repeat=nc):
                    mask = sum(1 << c for c in ctrls)
                    v = sum(1 << c for c, b in zip(ctrls, vals) if b)
                    for k in range(1 << n):
                        psi = W.basis_state(n, k)
                        oracle.apply_x(psi, n, t, mask, v)
                        expect = k ^ (1 << t) if (k & mask) == v else k
                        assert psi[expect] == 1.0 and np.count_nonzero(psi) == 1


def test_negative_control_identity_fig1():
    """Fig. 1 (right): G with a negative control on q1 == X(q1); C-G; X(q1)."""
    rng = np.random.default_rng(11)
    n = 5
    for _ in range(10):
        t, c = [int(q) for q in rng.choice(n, size=2, replace=False)]
        U = W.haar_2x2(rng)
        psi = W.random_state(n, int(rng.integers(1 << 30)))
        a = psi.copy()
        oracle.apply_gate(a, n, t, 1 << c, 0, U)          # control on |0>
        b = psi.copy()
        oracle.apply_x(b, n, c)
        oracle.apply_gate(b, n, t, 1 << c, 1 << c, U)     # control on |1>
        oracle.apply_x(b, n, c)
        assert np.max(np.abs(a - b)) < 1e-15


def _bit_reverse(x, n):
    x = np.asarray(x, dtype=np.int64)
    r = np.zeros_like(x)
    for i in range(n):
        r |= ((x >> i) & 1) << (n - 1 - i)
    return r


def test_qft_generator_matches_figure():
    """The QFT generator at n = 5 reproduces Fig. qft_circuit gate for gate; R_m is
    diag(1, exp(2 pi i / 2^m)) and H is the Section II-A Hadamard."""
    fig = _load("qft_circuit_5q.json")
    gates = W.qft_circuit(fig["n"])
    assert len(gates) == len(fig["gates"]) == 15
    for g, f in zip(gates, fig["gates"]):
        assert int(g["target"]) == f["target"]
        m = sum(1 << c for c in f["controls"])
        assert int(g["ctrl_mask"]) == m and int(g["ctrl_vals"]) == m
        want = W.H_MATRIX if f["gate"] == "H" else np.diag([1.0, np.exp(2j * np.pi / 2 ** f["m"])])
        assert np.array_equal(W.unpack_u(g["U"]), want)
    assert len(W.qft_circuit(29)) == 29 + 29 * 28 // 2


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_qft_circuit_is_bit_reversed_dft(n):
    """The drawn QFT circuit (q0 processed first, no swaps, q0 the least significant bit)
    maps psi to out[y] = 2^(-n/2) sum_x psi[x] exp(2 pi i rev(x) y / 2^n), rev the n-bit
    reversal: the textbook QFT with the input read in reversed bit order. Checked against
    numpy's inverse FFT."""
    N = 1 << n
    psi = W.random_state(n, 100 + n)
    out = psi.copy()
    for g in W.qft_circuit(n):
        oracle.apply_gate(out, n, int(g["target"]), int(g["ctrl_mask"]), int(g["ctrl_vals"]),
                          W.unpack_u(g["U"]))
    a = np.empty(N, dtype=np.complex128)
    a[_bit_reverse(np.arange(N), n)] = psi
    want = np.sqrt(N) * np.fft.ifft(a)
    assert np.max(np.abs(out - want)) < 1e-13
    # basis input |x>: every amplitude has modulus 2^(-n/2) and phase 2 pi rev(x) y / 2^n
    x = (0x2D5 * n + 3) % N
    out = W.basis_state(n, x)
    for g in W.qft_circuit(n):
        oracle.apply_gate(out, n, int(g["target"]), int(g["ctrl_mask"]), int(g["ctrl_vals"]),
                          W.unpack_u(g["U"]))
    y = np.arange(N)
    ph = 2.0 * np.pi * ((int(_bit_reverse(x, n)) * y) % N) / N
    assert np.max(np.abs(out - np.exp(1j * ph) / np.sqrt(N))) < 1e-13


@pytest.mark.parametrize("n", [2, 3, 4, 7, 10])
def test_streaming_circuit_closed_form(n):
    """Fig. streaming_circ, read with x0 as the least significant bit, maps |k> to
    |k - 1 mod 2^n>; in reverse gate order it maps |k> to |k + 1 mod 2^n>."""
    fig = _load("streaming_circuit_4q.json")
    assert [g["target"] for g in fig["gates"]] == [0, 1, 2, 3]
    gen = W.streaming_circuit(fig["n"])
    for g, f in zip(gen, fig["gates"]):
        m = sum(1 << c for c in f["controls"])
        assert int(g["target"]) == f["target"] and int(g["kind"]) == W.KIND_X
        assert int(g["ctrl_mask"]) == m and int(g["ctrl_vals"]) == m
    assert [int(g["target"]) for g in W.streaming_circuit(n, reverse=True)] == list(range(n - 1, -1, -1))
    gates = [(q, list(range(q))) for q in range(n)]
    for order, step in ((gates, -1), (list(reversed(gates)), +1)):
        for k in range(1 << n):
            psi = W.basis_state(n, k)
            for t, ctrls in order:
                m = sum(1 << c for c in ctrls)
                oracle.apply_x(psi, n, t, m, m)
            assert psi[(k + step) % (1 << n)] == 1.0


# --------------------------------------------------------------------------------------
# Invariants and closed forms
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_hadamard_on_all_qubits_is_uniform(n):
    psi = W.basis_state(n, 0)
    for q in range(n):
        oracle.apply_gate(psi, n, q, 0, 0, W.H_MATRIX)
    assert np.max(np.abs(psi - 2.0 ** (-n / 2.0))) < 1e-15


def test_unitary_roundtrip_and_norm():
    """A random circuit followed by its inverse (reversed order, U^dagger) returns the
    input; every unitary gate preserves the norm."""
    n = 10
    gates = W.random_circuit(n, 60, 5, seed=5)
    psi0 = W.random_state(n, 55)
    psi = psi0.copy()
    for g in gates:
        oracle.apply_gate(psi, n, int(g["target"]), int(g["ctrl_mask"]), int(g["ctrl_vals"]),
                          W.unpack_u(g["U"]))
        assert abs(oracle.norm2(psi, n) - 1.0) < 1e-13
    for g in gates[::-1]:
        oracle.apply_gate(psi, n, int(g["target"]), int(g["ctrl_mask"]), int(g["ctrl_vals"]),
                          W.unpack_u(g["U"]).conj().T)
    assert np.max(np.abs(psi - psi0)) < 1e-13


def test_expect_z_closed_forms():
    n = 6
    for k in [0, 1, 5, 37, 63]:
        z = oracle.expect_z(W.basis_state(n, k), n)
        assert np.array_equal(z, np.array([1.0 - 2.0 * ((k >> i) & 1) for i in range(n)]))
    # H on qubit i from |0>: <Z_i> = 0, others 1.  RY(theta) on qubit i: <Z_i> = cos(theta).
    for i in range(n):
        psi = W.basis_state(n, 0)
        oracle.apply_gate(psi, n, i, 0, 0, W.H_MATRIX)
        z = oracle.expect_z(psi, n)
        assert abs(z[i]) < 1e-15 and np.max(np.abs(np.delete(z, i) - 1.0)) < 1e-15
        th = 0.3 + i
        psi = W.basis_state(n, 0)
        oracle.apply_gate(psi, n, i, 0, 0, oracle.ry(th))
        assert abs(oracle.expect_z(psi, n)[i] - np.cos(th)) < 1e-15
    psi = W.random_state(n, 3)
    assert abs(oracle.norm2(psi, n) - 1.0) < 1e-14
    assert abs(oracle.inner_re(psi, psi, n) - 1.0) < 1e-14


def test_inner_re_pins():
    """Re <a|b> = sum over amplitudes of Re(conj(a_k) b_k): basis states are orthonormal, purely
    imaginary amplitudes count like real ones (a dropped or sign-flipped imaginary term fails),
    a relative phase gives its cosine, and the polarisation identity
    Re <a|b> = (|a + b|^2 - |a - b|^2) / 4 holds with the oracle's own norm2 (pinned above)."""
    n = 5
    for j in (0, 7, 31):
        for k in (0, 7, 31):
            assert oracle.inner_re(W.basis_state(n, j), W.basis_state(n, k), n) == (1.0 if j == k else 0.0)
    a = 1j * W.basis_state(n, 9)
    assert oracle.inner_re(a, a, n) == 1.0
    for al, be in ((0.3, 1.1), (2.0, -0.7), (0.0, np.pi)):
        x = np.exp(1j * al) * W.basis_state(n, 4)
        y = np.exp(1j * be) * W.basis_state(n, 4)
        assert abs(oracle.inner_re(x, y, n) - np.cos(be - al)) < 1e-15
    rng = np.random.default_rng(8)
    for _ in range(5):
        u = rng.normal(size=2**n) + 1j * rng.normal(size=2**n)
        v = rng.normal(size=2**n) + 1j * rng.normal(size=2**n)
        pol = (oracle.norm2(u + v, n) - oracle.norm2(u - v, n)) / 4.0
        assert abs(oracle.inner_re(u, v, n) - pol) < 1e-12 * (1.0 + abs(pol))


def test_rotation_definitions():
    """RY(theta) = exp(-i theta Y/2), RZ(theta) = exp(-i theta Z/2): compare with the matrix
    exponential series of the Pauli generators."""
    Y = np.array([[0, -1j], [1j, 0]])
    Z = np.diag([1.0, -1.0]).astype(np.complex128)
    for th in [0.0, 0.4, 2.5, -1.1]:
        for gen, fn in ((Y, oracle.ry), (Z, oracle.rz)):
            A = -0.5j * th * gen
            E = np.eye(2, dtype=np.complex128)
            term = np.eye(2, dtype=np.complex128)
            for k in range(1, 30):
                term = term @ A / k
                E = E + term
            assert np.max(np.abs(E - fn(th))) < 1e-14


def test_param_shift_closed_forms():
    """Product ansatz (RY then RZ per qubit, no entangler): E = sum_q cos(theta_y,q), so
    dE/dtheta_y = -sin(theta_y) and dE/dtheta_z = 0. Two qubits RY(a) on q0, CNOT(0->1),
    RY(b) on q1: E = cos a + cos a cos b."""
    n = 3
    gates = W.gate_list([g for q in range(n) for g in (
        W.make_gate(q, None, (), kind=W.KIND_RY, param=2 * q),
        W.make_gate(q, None, (), kind=W.KIND_RZ, param=2 * q + 1))])
    th = np.array([0.3, 1.0, 2.0, -0.4, 4.0, 0.7])
    assert abs(oracle.energy(n, gates, th) - np.sum(np.cos(th[0::2]))) < 1e-14
    g = oracle.param_shift_grad(n, gates, th)
    want = np.zeros_like(th)
    want[0::2] = -np.sin(th[0::2])
    assert np.max(np.abs(g - want)) < 1e-14

    gates2 = W.gate_list([W.make_gate(0, None, (), kind=W.KIND_RY, param=0),
                          W.make_gate(1, None, (0,), kind=W.KIND_X),
                          W.make_gate(1, None, (), kind=W.KIND_RY, param=1)])
    a, b = 0.9, -2.2
    assert abs(oracle.energy(2, gates2, [a, b]) - (np.cos(a) + np.cos(a) * np.cos(b))) < 1e-14
    g2 = oracle.param_shift_grad(2, gates2, [a, b])
    assert np.max(np.abs(g2 - [-np.sin(a) * (1 + np.cos(b)), -np.cos(a) * np.sin(b)])) < 1e-14


def test_param_shift_matches_finite_differences_on_ansatz():
    n, layers = 5, 2
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    ps = oracle.param_shift_grad(n, gates, th)
    fd = oracle.fd_grad(n, gates, th, h=1e-4)
    assert np.max(np.abs(ps - fd)) < 1e-7


def test_parameter_shift_rejects_controlled_rotations():
    """The two-term shift rule holds for generators with eigenvalues +-1/2 only; a controlled
    rotation's generator also has 0, so the oracle refuses rather than return a wrong value,
    and its finite differences show the difference."""
    n = 3
    gl = [W.make_gate(q, None, (), kind=W.KIND_RY, param=q) for q in range(n)]
    gl.append(W.make_gate(0, None, (2,), kind=W.KIND_RZ, param=3))  # RZ on q0, control q2
    gl += [W.make_gate(q, None, (), kind=W.KIND_RY, param=4 + q) for q in range(n)]
    gates = W.gate_list(gl)
    th = np.array([0.7, 1.1, 0.4, 1.9, 0.5, 0.8, 1.2])
    with pytest.raises(ValueError):
        oracle.param_shift_grad(n, gates, th)
    fd = oracle.fd_grad(n, gates, th)
    tp, tm = th.copy(), th.copy()
    tp[3] += np.pi / 2
    tm[3] -= np.pi / 2
    two_term = 0.5 * (oracle.energy(n, gates, tp) - oracle.energy(n, gates, tm))
    assert abs(two_term - fd[3]) > 1e-2  # 0.220 against 0.159


# ---------------------------------------------------------------------------------------
# Fixed-point amplitudes (Q1.30): the format's rounding rules, exactness of exchanges, the
# index arithmetic (dense brute force), and agreement with the float64 oracle within the
# rounding the format implies
# ---------------------------------------------------------------------------------------

def test_q30_quantisation_rule():
    """Matrix entries: nearest Q1.30 integer, halves away from zero, clamped to int32."""
    q = oracle.quantize_q30
    assert q(0.5) == 1 << 29 and q(-0.5) == -(1 << 29) and q(1.0) == 1 << 30
    assert q(2.0 ** -31) == 1 and q(-(2.0 ** -31)) == -1          # exactly half a step: away from 0
    assert q(3 * 2.0 ** -32) == 1 and q(2.0 ** -32) == 0          # 0.75 and 0.25 of a step
    assert q(1 / np.sqrt(2)) == 759250125                         # 759250124.9919... rounds up
    assert q(2.5) == 2 ** 31 - 1 and q(-3.0) == -(2 ** 31)        # clamped


def test_q30_rounding_of_the_update():
    """One output component is floor((S + 2^29) / 2^30) of its exact 64-bit sum S, clamped:
    ties go toward +infinity, and the sum of two full-scale terms saturates."""
    one = 1 << 30
    # n = 1, target 0, U = [[a, 0], [0, 1]]: x' = round(a x)
    for a_raw, x_raw, want in ((1, 1 << 29, 1),      # S = 2^29: exactly half -> up to 1
                               (1, -(1 << 29), 0),   # S = -2^29: half -> up to 0
                               (3, 1 << 29, 2),      # S = 1.5 * 2^30 -> 2
                               (-3, 1 << 29, -1),    # S = -1.5 * 2^30 -> -1
                               (1, (1 << 29) - 1, 0)):
        psi = np.zeros((2, 2), dtype=np.int32)
        psi[0, 0] = x_raw
        U = np.zeros(8)
        U[0] = a_raw / one
        U[6] = 1.0
        oracle.apply_gate_q30(psi, 1, 0, 0, 0, U)
        assert psi[0, 0] == want, (a_raw, x_raw, psi[0, 0])
    psi = np.full((2, 2), 0, dtype=np.int32)
    psi[0, 0] = psi[1, 0] = one
    oracle.apply_gate_q30(psi, 1, 0, 0, 0, np.array([[1.0, 1.0], [1.0, -1.0]]))  # x + y = 2 saturates
    assert psi[0, 0] == 2 ** 31 - 1 and psi[1, 0] == 0


def test_q30_exchanges_and_hadamard_exact_values():
    """X on Q1.30 amplitudes moves the integers unchanged (Section II-A, bit-exact); H on
    |0> gives round(2^30 * q(1/sqrt 2) / 2^30) = q(1/sqrt 2) on both amplitudes."""
    rng = np.random.default_rng(3)
    n = 5
    psi = rng.integers(-(1 << 30), 1 << 30, size=(1 << n, 2)).astype(np.int32)
    ref = psi.copy()
    oracle.apply_gate_q30(psi, n, 2, 0b1001, 0b0001, W.X_MATRIX)
    for k in range(1 << n):
        if (k & 0b1001) == 0b0001:
            assert np.array_equal(psi[k], ref[k ^ 0b100])
        else:
            assert np.array_equal(psi[k], ref[k])
    psi = np.zeros((2, 2), dtype=np.int32)
    psi[0, 0] = 1 << 30
    oracle.apply_gate_q30(psi, 1, 0, 0, 0, W.H_MATRIX)
    assert psi[0, 0] == 759250125 and psi[1, 0] == 759250125 and psi[0, 1] == 0 and psi[1, 1] == 0


def _dense_q30(n, t, mask, vals, Uq, psi):
    """Brute force: the full 2^n x 2^n integer matrix of the gate (P_sat (x) U + rest (x) I,
    entries as Q1.30 integers), each output component's exact sum rounded by the format's
    rule."""
    N = 1 << n
    u = [(int(Uq[2 * i]), int(Uq[2 * i + 1])) for i in range(4)]  # a, b, c, d
    M = {}  # (row, column) -> complex integer entry as (re, im)
    for k in range(N):
        if (k & mask) != vals:
            M[(k, k)] = (1 << 30, 0)
            continue
        bit = (k >> t) & 1
        k0 = k & ~(1 << t)
        M[(k, k0)] = u[0] if bit == 0 else u[2]
        M[(k, k0 | (1 << t))] = u[1] if bit == 0 else u[3]
    out = np.zeros((N, 2), dtype=np.int64)
    for k in range(N):
        sr = si = 0
        for j in range(N):
            mr, mi = M.get((k, j), (0, 0))
            xr, xi = int(psi[j, 0]), int(psi[j, 1])
            sr += mr * xr - mi * xi
            si += mr * xi + mi * xr
        for c, S in ((0, sr), (1, si)):
            r = (S + (1 << 29)) >> 30  # Python's >> floors
            out[k, c] = max(-(2 ** 31), min(2 ** 31 - 1, r))
    return out.astype(np.int32)


def test_q30_gate_against_dense_brute_force():
    """Every target, control subset and control value at n <= 4: the Q1.30 gate equals the
    dense integer matrix product with the same rounding, bit for bit."""
    rng = np.random.default_rng(30)
    for n in (1, 2, 3, 4):
        for t in range(n):
            others = [q for q in range(n) if q != t]
            for m in range(1 << len(others)):
                mask = sum(1 << others[i] for i in range(len(others)) if (m >> i) & 1)
                vals = mask & int(rng.integers(0, 1 << n))
                U = W.haar_2x2(rng)
                psi = rng.integers(-(1 << 29), 1 << 29, size=(1 << n, 2)).astype(np.int32)
                want = _dense_q30(n, t, mask, vals, oracle.q30_matrix(U), psi)
                got = psi.copy()
                oracle.apply_gate_q30(got, n, t, mask, vals, U)
                assert np.array_equal(got, want), (n, t, mask, vals)


def test_q30_circuit_tracks_float64_within_rounding():
    """A random 200-gate circuit (0-3 controls) on a random normalised 8-qubit state: the
    Q1.30 result differs from the float64 oracle by at most the format's rounding: per gate
    each output component gains <= 2^-31 from its rounding plus <= 4 * 2^-31 from the
    quantised matrix (entries within 2^-31, |inputs| <= 1), so 200 gates stay below
    1000 * 2^-31 = 4.7e-7; and <Z_i> of the Q1.30 state equals the float64 <Z_i> of its
    dequantised vector."""
    n = 8
    gates = W.random_circuit(n, 200, 3, seed=31)
    psi0 = W.random_state(n, 32)
    ref = psi0.copy()
    oracle.run_circuit(ref, n, gates)
    q = oracle.to_q30(psi0)
    oracle.run_circuit_q30(q, n, gates)
    deq = (q[:, 0].astype(np.float64) + 1j * q[:, 1].astype(np.float64)) / (1 << 30)
    assert np.max(np.abs(deq - ref)) <= 1000 * 2.0 ** -31
    assert np.max(np.abs(oracle.expect_z_q30(q, n) - oracle.expect_z(deq.astype(np.complex128), n))) <= 1e-12


def test_q30_gate_output_matches_whole_vector_update():
    """The one-amplitude Q1.30 update (used by sampled checks at full size) equals the whole
    vector update element by element, for targets and controls of both polarities."""
    rng = np.random.default_rng(33)
    n = 7
    for t, mask, vals in ((0, 0, 0), (6, 0b11, 0b01), (3, 0b1000001, 0b1000000), (2, 0b10, 0)):
        psi = rng.integers(-(1 << 30), 1 << 30, size=(1 << n, 2)).astype(np.int32)
        U = W.haar_2x2(rng)
        ref = psi.copy()
        oracle.apply_gate_q30(ref, n, t, mask, vals, U)
        for k in range(1 << n):
            got = oracle.gate_output_q30(k, t, mask, vals, U, psi[k], psi[k ^ (1 << t)])
            assert got == (int(ref[k, 0]), int(ref[k, 1])), (t, mask, k)
