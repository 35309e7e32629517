"""GPU parity: the CUDA gate path (through the C-ABI) against the CPU oracle."""
import itertools

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import (ATOL_CIRCUIT, NP, RTOL_GATE, c128_of, oracle_outputs, prepare_product, product_amp,
                         random_state, rotations, sample_indices)

pytestmark = pytest.mark.gpu

DTYPES = ["c64", "c128"]


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


def _run_gpu(qs, n, dtype, psi0, gates, mode="gate", theta=None):
    st = qs.State(n, dtype)
    try:
        st.from_numpy(psi0)
        if mode == "gate":
            for g in gates:
                if int(g["kind"]) == W.KIND_X:
                    st.apply_x(int(g["target"]), int(g["ctrl_mask"]), int(g["ctrl_vals"]))
                else:
                    st.apply_gate(int(g["target"]), W.unpack_u(g["U"]), int(g["ctrl_mask"]), int(g["ctrl_vals"]))
        elif mode == "circuit":
            st.apply_circuit(gates, theta)
        elif mode == "graph":
            st.apply_circuit(gates, theta, flags=qs.QS_FLAG_GRAPH)
        return st.to_numpy()
    finally:
        st.close()


def _run_oracle(n, psi0, gates, theta=None):
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates, theta)
    return ref


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", ["gate", "circuit", "graph"])
def test_small_exact_circuit(qs, dtype, mode):
    """n = 12 from |0>: H on every qubit, then 200 Haar gates with 0-3 controls."""
    n = 12
    gates = W.small_exact_circuit(0)
    psi0 = W.basis_state(n, 0, NP[dtype])
    got = _run_gpu(qs, n, dtype, psi0, gates, mode)
    ref = _run_oracle(n, psi0, gates)
    err = np.max(np.abs(c128_of(got) - ref))
    assert err <= ATOL_CIRCUIT[dtype], err


@pytest.mark.parametrize("dtype", DTYPES)
def test_random_single_gates_fuzz(qs, dtype):
    """Random (t, controls, control values, matrix) for n = 1..16, one gate at a time."""
    rng = np.random.default_rng(1234)
    for n in range(1, 17):
        for trial in range(6):
            t = int(rng.integers(0, n))
            others = [q for q in range(n) if q != t]
            c = int(rng.integers(0, len(others) + 1)) if others else 0
            ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
            vals = [int(b) for b in rng.integers(0, 2, size=c)]
            U = W.haar_2x2(rng)
            g = W.gate_list([W.make_gate(t, U, ctrls, vals)])
            psi0 = random_state(n, dtype, 1000 * n + trial)
            got = c128_of(_run_gpu(qs, n, dtype, psi0, g))
            ref = _run_oracle(n, psi0, g)
            scale = np.max(np.abs(c128_of(psi0)))
            assert np.max(np.abs(got - ref)) <= 4 * RTOL_GATE[dtype] * scale, (n, t, ctrls, vals)


def _layout_cases(n):
    """(t, controls) pairs that reach every unit layout: t = 0 with the next inserted bit at
    1, 2 and higher; t > 0 with the lowest inserted bit at 0, 1, 2 and higher; all qubits
    but one as controls; controls next to the target."""
    cases = [(0, []), (0, [1]), (0, [2]), (0, [3, 5]), (1, []), (2, []), (5, []), (n - 1, []),
             (3, [0]), (3, [1]), (3, [2]), (4, [2, 3]), (4, [3, 5]), (2, [0, 1]), (n - 1, [0, n - 2]),
             (n - 1, list(range(n - 1))), (0, list(range(1, n))), (n // 2, [q for q in range(n) if q != n // 2])]
    return cases


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [7, 13, 18])
def test_every_layout_and_op(qs, dtype, n):
    rng = np.random.default_rng(n)
    Us = {
        "general": W.haar_2x2(rng),
        "diag": np.diag(np.exp(1j * rng.uniform(0, 6, 2))),
        "phase_hi": np.diag([1.0, np.exp(0.7j)]),
        "phase_lo": np.diag([np.exp(-0.3j), 1.0]),
        "xmatrix": W.X_MATRIX,
        "identity": np.eye(2),
    }
    for (t, ctrls), (name, U) in itertools.product(_layout_cases(n), Us.items()):
        for vals in ([1] * len(ctrls), [int(b) for b in rng.integers(0, 2, size=len(ctrls))]):
            g = W.gate_list([W.make_gate(t, U, ctrls, vals)])
            psi0 = random_state(n, dtype, 77)
            got = c128_of(_run_gpu(qs, n, dtype, psi0, g))
            ref = _run_oracle(n, psi0, g)
            scale = np.max(np.abs(c128_of(psi0)))
            assert np.max(np.abs(got - ref)) <= 4 * RTOL_GATE[dtype] * scale, (n, t, ctrls, vals, name)


@pytest.mark.parametrize("dtype", DTYPES)
def test_permutation_gates_bit_exact(qs, dtype):
    """X / CNOT / Toffoli (and X given as a matrix) move amplitudes without arithmetic:
    the result equals the oracle's exchange bit for bit."""
    for n in (1, 2, 5, 11, 15):
        rng = np.random.default_rng(n)
        gl = []
        for _ in range(40):
            nc = int(rng.integers(0, min(2, n - 1) + 1))
            qs_ = [int(q) for q in rng.choice(n, size=nc + 1, replace=False)]
            vals = [int(b) for b in rng.integers(0, 2, size=nc)]
            gl.append(W.make_gate(qs_[0], None, sorted(qs_[1:]), vals, kind=W.KIND_X))
        gates = W.gate_list(gl)
        psi0 = random_state(n, dtype, 5)
        got = _run_gpu(qs, n, dtype, psi0, gates)
        ref = _run_oracle(n, psi0, gates).astype(NP[dtype])
        assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))
        # the same gates given as explicit X matrices take the exchange path too
        gm = gates.copy()
        gm["kind"] = W.KIND_U
        got2 = _run_gpu(qs, n, dtype, psi0, gm)
        assert np.array_equal(got2.view(np.uint8), ref.view(np.uint8))


@pytest.mark.parametrize("dtype", DTYPES)
def test_masked_comparator_matches(qs, dtype):
    """The baseline schedule (all 2^(n-1) pairs, controls tested per pair) gives the same
    amplitudes as the reduced schedule, bit for bit, and matches the oracle."""
    n = 14
    rng = np.random.default_rng(9)
    for t, ctrls in _layout_cases(n):
        vals = [int(b) for b in rng.integers(0, 2, size=len(ctrls))]
        m = sum(1 << c for c in ctrls)
        v = sum(1 << c for c, b in zip(ctrls, vals) if b)
        U = W.haar_2x2(rng)
        psi0 = random_state(n, dtype, 3)
        a = qs.State(n, dtype)
        b = qs.State(n, dtype)
        try:
            a.from_numpy(psi0)
            b.from_numpy(psi0)
            a.apply_gate(t, U, m, v)
            b.apply_gate_masked(t, U, m, v)
            ga, gb = a.to_numpy(), b.to_numpy()
        finally:
            a.close()
            b.close()
        assert np.array_equal(ga.view(np.uint8), gb.view(np.uint8)), (t, ctrls)
        ref = c128_of(psi0).copy()
        oracle.apply_gate(ref, n, t, m, v, U)
        assert np.max(np.abs(c128_of(ga) - ref)) <= 4 * RTOL_GATE[dtype] * np.max(np.abs(psi0))


@pytest.mark.parametrize("dtype", DTYPES)
def test_circuit_at_twenty_qubits(qs, dtype):
    """1000 random gates with 0-8 controls at n = 20 (the scale circuit's recipe): full
    vector against the oracle, and the norm stays within 1e-5 of 1."""
    n = 20
    gates = W.random_circuit(n, 1000, 8, seed=1)
    psi0 = random_state(n, dtype, 21)
    got = c128_of(_run_gpu(qs, n, dtype, psi0, gates, "circuit"))
    ref = _run_oracle(n, psi0, gates)
    assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype]
    assert abs(np.vdot(got, got).real - np.vdot(ref, ref).real) <= 1e-5


def test_streaming_circuit_on_gpu(qs):
    """Fig. streaming_circ at n = 13: |k> -> |k - 1 mod 2^n>, bit-exact."""
    n = 13
    gates = W.gate_list([W.make_gate(q, None, list(range(q)), kind=W.KIND_X) for q in range(n)])
    psi0 = random_state(n, "c64", 8)
    got = _run_gpu(qs, n, "c64", psi0, gates, "circuit")
    assert np.array_equal(got, np.roll(psi0, -1))


@pytest.mark.parametrize("dtype", DTYPES)
def test_full_size_sweep_sampled(qs, dtype):
    """The single-gate sweep at its full size (n = 30, c = 0..8, targets 0/15/29) in the
    launch configuration the benchmark times: the input is a product state whose amplitudes
    have a closed form; every output sampled is checked against the oracle's one-amplitude
    update from the input values at k and k ^ 2^t."""
    import torch

    n = 30
    al, be = rotations(n, 30)
    buf = torch.empty(1 << n, dtype=torch.complex64 if dtype == "c64" else torch.complex128, device="cuda")
    st = qs.State.wrap(buf, n)
    try:
        prepare_product(st, al, be)
        torch.cuda.synchronize()
        ks = sample_indices(n, 1 << 14, 1)
        kt = torch.from_numpy(ks.astype(np.int64)).cuda()
        inp = buf.clone()
        got_in = buf[kt].cpu().numpy().astype(np.complex128)
        want_in = product_amp(ks, al, be)
        scale = np.abs(want_in)
        assert np.all(np.abs(got_in - want_in) <= (60 * RTOL_GATE[dtype] + 1e-15) * (scale + 1e-30) + 1e-300)
        sweep = W.sweep_gates(n, 8, W.SWEEP_TARGETS, sets=1, seed=1)
        for (c, t), gl in sweep.items():
            g = gl[0]
            m, v = int(g["ctrl_mask"]), int(g["ctrl_vals"])
            U = W.unpack_u(g["U"])
            buf.copy_(inp)
            st.apply_gate(t, U, m, v)
            kp = torch.from_numpy((ks ^ np.uint64(1 << t)).astype(np.int64)).cuda()
            xin = inp[kt].cpu().numpy()
            pin = inp[kp].cpu().numpy()
            out = buf[kt].cpu().numpy().astype(np.complex128)
            want = oracle_outputs(ks, t, m, v, U, xin.astype(np.complex128), pin.astype(np.complex128))
            tol = 4 * RTOL_GATE[dtype] * (np.abs(xin) + np.abs(pin)) + 1e-300
            assert np.all(np.abs(out - want) <= tol), (c, t)
            assert np.max(np.abs(out - want)) <= ATOL_CIRCUIT[dtype]
    finally:
        st.close()
        del buf
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tile_bits", [2, 5, 9, 12])
def test_fused_circuits_match_oracle(qs, dtype, tile_bits, monkeypatch):
    """QS_FLAG_FUSE (and FUSE | GRAPH): runs of gates grouped into shared-memory tile passes
    give the oracle's state, for several tile sizes, random controls (also negative, also
    on non-local qubits), diagonal / one-sided / exchange gates and tile predicates."""
    monkeypatch.setenv("QS_TILE_BITS", str(tile_bits))
    rng = np.random.default_rng(tile_bits)
    for n in (3, 9, 14, 17):
        gl = []
        for i in range(120):
            t = int(rng.integers(0, n))
            others = [q for q in range(n) if q != t]
            c = int(rng.integers(0, min(3, n - 1) + 1))
            ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
            vals = [int(b) for b in rng.integers(0, 2, size=c)]
            r = rng.random()
            if r < 0.15:
                gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_X))
            elif r < 0.3:
                gl.append(W.make_gate(t, np.diag(np.exp(1j * rng.uniform(0, 6, 2))), ctrls, vals))
            elif r < 0.4:
                gl.append(W.make_gate(t, np.diag([1.0, np.exp(0.3j)]), ctrls, vals))
            else:
                gl.append(W.make_gate(t, W.haar_2x2(rng), ctrls, vals))
        gates = W.gate_list(gl)
        psi0 = random_state(n, dtype, n)
        ref = _run_oracle(n, psi0, gates)
        for flags in (qs.QS_FLAG_FUSE, qs.QS_FLAG_FUSE | qs.QS_FLAG_GRAPH):
            st = qs.State(n, dtype)
            try:
                st.from_numpy(psi0)
                st.apply_circuit(gates, flags=flags)
                got = c128_of(st.to_numpy())
            finally:
                st.close()
            assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype], (n, flags)


@pytest.mark.parametrize("dtype", DTYPES)
def test_fused_ansatz_matches_unfused(qs, dtype):
    """The differentiation ansatz (n = 20, 4 layers) fused and unfused, against the oracle."""
    n, layers = 20, 4
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    psi0 = W.basis_state(n, 0, NP[dtype])
    ref = _run_oracle(n, psi0, gates, th)
    for flags in (0, qs.QS_FLAG_FUSE):
        st = qs.State(n, dtype)
        try:
            st.apply_circuit(gates, th, flags=flags)
            got = c128_of(st.to_numpy())
        finally:
            st.close()
        assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype], flags


def test_async_host_copies_on_two_streams(qs):
    """qs_state_copy_from_host_async / _to_host_async / qs_state_synchronize: two states on two
    streams each upload a page-locked input, apply gates and download, overlapped; the results
    equal the synchronous path and the oracle. Wrong sizes are rejected before any copy."""
    import torch

    n = 16
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    states = [qs.State(n, "c64", stream=int(s.cuda_stream)) for s in streams]
    try:
        hosts = [torch.empty(1 << n, dtype=torch.complex64).pin_memory() for _ in range(2)]
        hnp = [h.numpy() for h in hosts]
        psis = [random_state(n, "c64", 60 + i) for i in range(2)]
        gates = [W.random_circuit(n, 40, 3, seed=61 + i) for i in range(2)]
        for i in range(2):
            hnp[i][:] = psis[i]
        for i in range(2):
            qs.qs_state_copy_from_host_async(states[i].h, hnp[i])
            states[i].apply_circuit(gates[i])
            qs.qs_state_copy_to_host_async(states[i].h, hnp[i])
        for i in range(2):
            qs.qs_state_synchronize(states[i].h)
        for i in range(2):
            ref = c128_of(psis[i]).copy()
            oracle.run_circuit(ref, n, gates[i])
            assert np.max(np.abs(c128_of(hnp[i]) - ref)) <= ATOL_CIRCUIT["c64"]
            assert np.array_equal(hnp[i], states[i].to_numpy())
        with pytest.raises(qs.QsError):
            qs.qs_state_copy_from_host_async(states[0].h, hnp[0][:100])
        with pytest.raises(qs.QsError):
            qs.qs_state_copy_to_host_async(states[0].h, np.empty(3, dtype=np.complex64))
    finally:
        for s in states:
            s.close()


def test_allocation_failure_is_reported_and_recoverable(qs):
    """A state larger than the device (n = 40, complex128: 17.6 TB) fails with QS_ENOMEM and
    leaves the library usable."""
    with pytest.raises(qs.QsError) as e:
        qs.qs_state_alloc(40, qs.QS_C128)
    assert e.value.status == qs._lib.QS_ENOMEM
    with qs.State(10, "c64") as st:
        st.apply_gate(0, W.H_MATRIX)
        z, nrm = st.expect_z()
    assert abs(nrm - 1.0) < 1e-6 and abs(z[0]) < 1e-6
