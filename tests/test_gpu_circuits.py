"""GPU parity on the paper's circuit families (Section IV: QFT, streaming), the precision
circuit (n = 32, complex64 against complex128) and the 32/64-bit index boundary."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import ATOL_CIRCUIT, NP, RTOL_GATE, c128_of, oracle_outputs, prepare_product, random_state, \
    rotations, sample_indices

pytestmark = pytest.mark.gpu

DTYPES = ["c64", "c128"]
MODES = ["gate", "circuit", "fuse", "masked", "masked_circuit"]
# QFT output on a basis input: every amplitude has modulus 2^(-n/2). Relative error bound of
# the whole 435-gate circuit: each gate adds at most ~3u (u = 2^-24 / 2^-53) to the error
# norm and unitary gates do not grow it, so 435 * 3u = 8e-5 (c64) / 1.5e-13 (c128); the
# assertions allow a factor of ~4 over that.
QFT_RTOL = {"c64": 3e-4, "c128": 1e-12}


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


def _apply(qs, st, gates, mode):
    if mode == "circuit":
        st.apply_circuit(gates)
    elif mode == "fuse":
        st.apply_circuit(gates, flags=qs.QS_FLAG_FUSE)
    elif mode == "masked_circuit":
        st.apply_circuit(gates, flags=qs.QS_FLAG_MASKED | qs.QS_FLAG_GRAPH)
    else:
        for g in gates:
            t, m, v = int(g["target"]), int(g["ctrl_mask"]), int(g["ctrl_vals"])
            if mode == "masked":
                st.apply_gate_masked(t, W.unpack_u(g["U"]), m, v)
            elif int(g["kind"]) == W.KIND_X:
                st.apply_x(t, m, v)
            else:
                st.apply_gate(t, W.unpack_u(g["U"]), m, v)


def _bit_reverse(x: int, n: int) -> int:
    return int(format(x, f"0{n}b")[::-1], 2)


def _qft_basis_amplitudes(x: int, n: int, ys: np.ndarray) -> np.ndarray:
    """QFT circuit as drawn applied to |x>: amplitude y is exp(2 pi i rev(x) y / 2^n) 2^(-n/2)
    (pinned against the oracle and numpy's FFT on the CPU)."""
    N = 1 << n
    r = _bit_reverse(x, n)
    ph = np.array([(r * int(y)) % N for y in ys], dtype=np.float64) * (2.0 * np.pi / N)
    return np.exp(1j * ph) / np.sqrt(N)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
def test_qft_matches_oracle(qs, dtype, mode):
    """QFT (Fig. qft_circuit pattern) at n = 14 from a random state, every schedule."""
    n = 14
    gates = W.qft_circuit(n)
    psi0 = random_state(n, dtype, 140)
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates)
    with qs.State(n, dtype) as st:
        st.from_numpy(psi0)
        _apply(qs, st, gates, mode)
        got = c128_of(st.to_numpy())
    assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("reverse", [False, True])
def test_streaming_matches_oracle_bit_exact(qs, dtype, mode, reverse):
    """Streaming circuit (Fig. streaming_circ) at n = 15: gates with 0..14 controls; the result
    equals the oracle's bit for bit and is the closed-form shift by -1 (drawn order) / +1."""
    n = 15
    gates = W.streaming_circuit(n, reverse)
    psi0 = random_state(n, dtype, 150)
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates)
    with qs.State(n, dtype) as st:
        st.from_numpy(psi0)
        _apply(qs, st, gates, mode)
        got = st.to_numpy()
    assert np.array_equal(got, ref.astype(NP[dtype]))
    assert np.array_equal(got, np.roll(psi0, 1 if reverse else -1))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", ["circuit", "fuse"])
def test_qft29_basis_closed_form(qs, dtype, mode):
    """QFT29 (the paper's 29-qubit QFT, 435 gates) on a basis state: 2^14 sampled amplitudes
    against the closed form, and the modulus of every amplitude (whole vector, on the
    device) equal to 2^(-n/2)."""
    import torch

    n = 29
    x = 0x0A5C3E71 & ((1 << n) - 1)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    buf = torch.empty(1 << n, dtype=tdt, device="cuda")
    st = qs.State.wrap(buf, n)
    try:
        st.set_basis(x)
        _apply(qs, st, W.qft_circuit(n), mode)
        torch.cuda.synchronize()
        ys = sample_indices(n, 1 << 14, 29)
        got = buf[torch.from_numpy(ys.astype(np.int64)).cuda()].cpu().numpy().astype(np.complex128)
        want = _qft_basis_amplitudes(x, n, ys)
        scale = 2.0 ** (-n / 2.0)
        assert np.max(np.abs(got - want)) <= QFT_RTOL[dtype] * scale
        mod_err = 0.0
        for i in range(0, 1 << n, 1 << 26):
            blk = buf[i:i + (1 << 26)].abs().double() * (2.0 ** (n / 2.0))
            mod_err = max(mod_err, float((blk - 1.0).abs().max()))
        assert mod_err <= 2 * QFT_RTOL[dtype]
    finally:
        st.close()
        del buf
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", ["circuit", "fuse", "masked_circuit"])
def test_stream29_whole_vector_shift(qs, dtype, mode):
    """Streaming circuit at n = 29 (the paper's Stream29, gates with up to 28 controls) on a
    product state with distinct amplitudes: the whole output vector is the input shifted by
    one index, bit for bit (compared on the device)."""
    import torch

    n = 29
    al, be = rotations(n, 290)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    buf = torch.empty(1 << n, dtype=tdt, device="cuda")
    st = qs.State.wrap(buf, n)
    try:
        prepare_product(st, al, be)
        torch.cuda.synchronize()
        inp = buf.clone()
        _apply(qs, st, W.streaming_circuit(n), mode)
        torch.cuda.synchronize()
        assert torch.equal(buf[:-1], inp[1:])
        assert torch.equal(buf[-1:], inp[:1])
        del inp
    finally:
        st.close()
        del buf
        torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [32, 33])
def test_index_width_boundary_sampled(qs, n):
    """n = 32 (the last size with 32-bit device indices) and n = 33 (64-bit indices,
    68.7 GB complex64): single gates with targets and controls on the lowest and highest
    qubits, sampled outputs against the oracle's one-amplitude update; then the streaming
    circuit fused and unfused, sampled outputs against the inputs one index up."""
    import torch

    al, be = rotations(n, n)
    buf = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    st = qs.State.wrap(buf, n)
    inp = None
    try:
        prepare_product(st, al, be)
        torch.cuda.synchronize()
        inp = buf.clone()
        ks = sample_indices(n, 1 << 13, n)
        kt = torch.from_numpy(ks.astype(np.int64)).cuda()
        xin = inp[kt].cpu().numpy().astype(np.complex128)
        rng = np.random.default_rng(n)
        cases = [(0, 0, ()), (n - 1, 0, ()), (n - 1, 1, (0,)), (0, 1, (n - 1,)), (n // 2, 3, (1, n - 2, n - 1)),
                 (n - 1, 8, (0, 2, 5, 9, 14, 20, 27, n - 2)), (3, 5, (0, 1, 2, n - 2, n - 1))]
        for t, c, ctrls in cases:
            vals = [int(b) for b in rng.integers(0, 2, size=c)]
            g = W.make_gate(t, W.haar_2x2(rng), ctrls, vals)
            m, v, U = int(g["ctrl_mask"]), int(g["ctrl_vals"]), W.unpack_u(g["U"])
            buf.copy_(inp)
            st.apply_gate(t, U, m, v)
            kp = torch.from_numpy((ks ^ np.uint64(1 << t)).astype(np.int64)).cuda()
            pin = inp[kp].cpu().numpy().astype(np.complex128)
            out = buf[kt].cpu().numpy().astype(np.complex128)
            want = oracle_outputs(ks, t, m, v, U, xin, pin)
            assert np.all(np.abs(out - want) <= 4 * RTOL_GATE["c64"] * (np.abs(xin) + np.abs(pin)) + 1e-300), (t, c)
        N = np.uint64(1 << n)
        kup = torch.from_numpy(((ks + np.uint64(1)) % N).astype(np.int64)).cuda()
        want = inp[kup].cpu().numpy()
        for flags in (0, qs.QS_FLAG_FUSE):
            buf.copy_(inp)
            st.apply_circuit(W.streaming_circuit(n), flags=flags)
            assert np.array_equal(buf[kt].cpu().numpy(), want), flags
    finally:
        st.close()
        del buf, inp
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", DTYPES)
def test_precision_recipe_against_oracle(qs, dtype):
    """The precision circuit's recipe (2000 gates, 0-6 controls, 25 % X / CNOT / Toffoli) at
    n = 20: whole vector against the oracle, plain and fused."""
    n = 20
    gates = W.precision_circuit(n, 2000, seed=2)
    psi0 = random_state(n, dtype, 220)
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates)
    for mode in ("circuit", "fuse"):
        with qs.State(n, dtype) as st:
            st.from_numpy(psi0)
            _apply(qs, st, gates, mode)
            got = c128_of(st.to_numpy())
        assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype], mode


def test_precision_circuit_n32(qs):
    """The precision circuit at full size: n = 32 from H on every qubit, 2000 gates, run in
    complex128 (68.7 GB) and complex64 (34.4 GB, plain and fused) on the device. complex64
    against complex128: max-abs amplitude error <= 3e-5, norm drift <= 1e-5, and every
    <Z_i> within 2 ||psi64 - psi128|| (+ the float64 sums' rounding) of the complex128 one;
    complex128 keeps its norm to 1e-11."""
    import torch

    n = 32
    gates = W.precision_circuit(n, 2000, seed=2)
    prefix = W.gate_list([W.make_gate(q, W.H_MATRIX) for q in range(n)])
    b128 = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    b64 = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    s128 = qs.State.wrap(b128, n)
    s64 = qs.State.wrap(b64, n)
    try:
        s128.set_basis(0)
        s128.apply_circuit(prefix)
        s128.apply_circuit(gates)
        z128, nrm128 = s128.expect_z()
        assert abs(nrm128 - 1.0) <= 1e-11
        for flags in (0, qs.QS_FLAG_FUSE):
            s64.set_basis(0)
            s64.apply_circuit(prefix, flags=flags)
            s64.apply_circuit(gates, flags=flags)
            z64, nrm64 = s64.expect_z()
            torch.cuda.synchronize()
            err = 0.0
            d2 = 0.0
            for i in range(0, 1 << n, 1 << 26):
                d = b64[i:i + (1 << 26)].to(torch.complex128) - b128[i:i + (1 << 26)]
                err = max(err, float(d.abs().max()))
                d2 += float((d.abs() ** 2).sum())
            assert err <= 3e-5, (flags, err)
            assert abs(nrm64 - 1.0) <= 1e-5, (flags, nrm64)
            assert np.max(np.abs(np.asarray(z64) - np.asarray(z128))) <= 2.0 * np.sqrt(d2) + 1e-9, flags
    finally:
        s128.close()
        s64.close()
        del b128, b64
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", ["circuit", "fuse"])
def test_runs_on_one_target_match_oracle(qs, dtype, mode):
    """Forward application multiplies runs of consecutive gates with the same target and
    controls into one matrix: runs of 2-5 gates (Haar, parameterised RY / RZ, exchanges, with
    and without controls) against the oracle applying every gate; runs of exchanges alone stay
    bit-exact (X X X = X, X X = identity)."""
    n = 13
    rng = np.random.default_rng(77)
    gl = []
    theta = rng.uniform(0, 6.3, size=64)
    p = 0
    for r in range(40):
        t = int(rng.integers(0, n))
        others = [q for q in range(n) if q != t]
        c = int(rng.integers(0, 3))
        ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
        vals = [int(b) for b in rng.integers(0, 2, size=c)]
        for _ in range(int(rng.integers(2, 6))):
            u = rng.random()
            if u < 0.3:
                gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_X))
            elif u < 0.5 and p < 64:
                gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_RY if u < 0.4 else W.KIND_RZ, param=p))
                p += 1
            else:
                gl.append(W.make_gate(t, W.haar_2x2(rng), ctrls, vals))
    gates = W.gate_list(gl)
    psi0 = random_state(n, dtype, 78)
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates, theta)
    with qs.State(n, dtype) as st:
        st.from_numpy(psi0)
        st.apply_circuit(gates, theta, flags=qs.QS_FLAG_FUSE if mode == "fuse" else 0)
        got = c128_of(st.to_numpy())
    assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype]
    # exchanges only: runs of 1-4 X gates on one target, bit-exact
    xs = []
    for r in range(30):
        t = int(rng.integers(0, n))
        m = [q for q in range(n) if q != t][: int(rng.integers(0, 3))]
        xs += [W.make_gate(t, None, m, kind=W.KIND_X)] * int(rng.integers(1, 5))
    xs = W.gate_list(xs)
    ref = psi0.copy().astype(np.complex128)
    oracle.run_circuit(ref, n, xs)
    with qs.State(n, dtype) as st:
        st.from_numpy(psi0)
        st.apply_circuit(xs, flags=qs.QS_FLAG_FUSE if mode == "fuse" else 0)
        got = st.to_numpy()
    assert np.array_equal(got, ref.astype(NP[dtype]))


def _diag_gate(rng, n, t, ctrls, vals):
    u = rng.random()
    if u < 0.35:   # one-sided: phase on the |1> side (R_m, S, T, CZ-like)
        D = np.diag([1.0, np.exp(1j * rng.uniform(0, 6.3))])
    elif u < 0.5:  # one-sided on the |0> side
        D = np.diag([np.exp(1j * rng.uniform(0, 6.3)), 1.0])
    elif u < 0.6:  # identity (drops out)
        D = np.eye(2)
    elif u < 0.9:  # general diagonal phase
        D = np.diag(np.exp(1j * rng.uniform(0, 6.3, 2)))
    else:          # non-unit modulus (the library does not require unitarity)
        D = np.diag(rng.uniform(0.97, 1.03, 2) * np.exp(1j * rng.uniform(0, 6.3, 2)))
    return W.make_gate(t, D, ctrls, vals)


@pytest.mark.parametrize("dtype", DTYPES)
def test_diagonal_runs_match_oracle(qs, dtype):
    """Fused programs put runs of diagonal gates into diagonal-run passes (k_diag): targets and
    controls on the lowest three qubits (inside a chunk) and above, control values 0 and 1,
    one-sided / general / identity diagonals, runs longer than one launch (64 gates), mixed
    with non-diagonal gates; n = 3..16 against the oracle."""
    rng = np.random.default_rng(314)
    for n in (3, 4, 5, 9, 16):
        gl = []
        for blk in range(6):
            for _ in range(int(rng.integers(1, 4))):
                gl.append(W.make_gate(int(rng.integers(0, n)), W.haar_2x2(rng)))
            for _ in range(int(rng.choice([3, 4, 9, 70]))):
                t = int(rng.integers(0, n))
                others = [q for q in range(n) if q != t]
                c = int(rng.integers(0, min(3, n - 1) + 1))
                ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
                vals = [int(b) for b in rng.integers(0, 2, size=c)]
                gl.append(_diag_gate(rng, n, t, ctrls, vals))
        if n >= 8:  # runs whose gates all need one bit value: skipped by the compact counter
            for _ in range(2):
                common = int(rng.integers(3, n))
                cv = int(rng.integers(0, 2))
                for _ in range(10):
                    t = int(rng.choice([q for q in range(n) if q != common]))
                    others = [q for q in range(n) if q not in (t, common)]
                    extra = sorted(int(q) for q in rng.choice(others, size=int(rng.integers(0, 3)), replace=False))
                    ctrls = sorted(extra + [common])
                    vals = [cv if q == common else int(rng.integers(0, 2)) for q in ctrls]
                    gl.append(_diag_gate(rng, n, t, ctrls, vals))
                t = int(rng.integers(3, n))  # one-sided gates sharing a target: bit t = 1 needed
                for _ in range(10):
                    others = [q for q in range(n) if q != t]
                    ctrls = sorted(int(q) for q in rng.choice(others, size=int(rng.integers(0, 3)), replace=False))
                    gl.append(W.make_gate(t, np.diag([1.0, np.exp(1j * rng.uniform(0, 6.3))]), ctrls))
                gl.append(W.make_gate(int(rng.integers(0, n)), W.haar_2x2(rng)))
        if n >= 9:  # runs sharing one low target, controls on qubits >= 8 (warp-level classes)
            for t in (0, 2, 5):
                for _ in range(12):
                    c = int(rng.integers(0, min(3, n - 8) + 1))
                    ctrls = sorted(int(q) for q in rng.choice(range(8, n), size=c, replace=False)) if c else []
                    vals = [int(b) for b in rng.integers(0, 2, size=c)]
                    gl.append(_diag_gate(rng, n, t, ctrls, vals))
                gl.append(W.make_gate(int(rng.integers(0, n)), W.haar_2x2(rng)))
        gates = W.gate_list(gl)
        psi0 = random_state(n, dtype, 300 + n)
        ref = c128_of(psi0).copy()
        oracle.run_circuit(ref, n, gates)
        for flags in (qs.QS_FLAG_FUSE, qs.QS_FLAG_FUSE | qs.QS_FLAG_GRAPH):
            with qs.State(n, dtype) as st:
                st.from_numpy(psi0)
                st.apply_circuit(gates, flags=flags)
                got = c128_of(st.to_numpy())
            assert np.max(np.abs(got - ref)) <= 4 * ATOL_CIRCUIT[dtype] * max(1.0, np.max(np.abs(ref))), (n, flags)


@pytest.mark.parametrize("dtype", DTYPES)
def test_short_diagonal_runs_match_oracle(qs, dtype, monkeypatch):
    """Runs of only 2 or 3 diagonal gates, after an uncontrolled gate (which can lead the run)
    or after a doubly controlled X (which cannot): the planner gives them diagonal-run passes
    (checked on its schedule; complex64 with 2^6-amplitude tiles, so that tile passes cannot
    hold a block) and the result matches the oracle, n = 20."""
    if dtype == "c64":
        monkeypatch.setenv("QS_TILE_BITS", "6")
    n = 20
    rng = np.random.default_rng(77)
    gl = []
    for blk in range(16):
        if blk % 2:
            t = int(rng.integers(0, n))
            c = sorted(int(q) for q in rng.choice([q for q in range(n) if q != t], size=2, replace=False))
            gl.append(W.make_gate(t, None, c, kind=W.KIND_X))
        else:
            gl.append(W.make_gate(int(rng.integers(0, n)), W.haar_2x2(rng)))
        for _ in range(2 + blk % 3 // 2):
            t = int(rng.integers(0, n))
            others = [q for q in range(n) if q != t]
            c = int(rng.integers(0, 3))
            ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
            vals = [int(b) for b in rng.integers(0, 2, size=c)]
            gl.append(_diag_gate(rng, n, t, ctrls, vals))
    gates = W.gate_list(gl)
    sched = qs.circuit_schedule(n, gates, dtype=dtype)
    assert sched["diag_runs"] >= 3, sched
    psi0 = random_state(n, dtype, 77)
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates)
    for flags in (qs.QS_FLAG_FUSE, qs.QS_FLAG_FUSE | qs.QS_FLAG_GRAPH):
        with qs.State(n, dtype) as st:
            st.from_numpy(psi0)
            st.apply_circuit(gates, flags=flags)
            got = c128_of(st.to_numpy())
        assert np.max(np.abs(got - ref)) <= 4 * ATOL_CIRCUIT[dtype] * max(1.0, np.max(np.abs(ref))), flags


@pytest.mark.parametrize("dtype", DTYPES)
def test_fused_programs_at_the_smallest_sizes(qs, dtype):
    """n = 1..5 with QS_FLAG_FUSE: diagonal runs (only from n = 3: one 8-amplitude chunk),
    leading gates on every target (chunk pairs from n = 4), exchanges and general gates,
    against the oracle; an empty circuit changes nothing."""
    rng = np.random.default_rng(5)
    for n in range(1, 6):
        gl = []
        for blk in range(5):
            gl.append(W.make_gate(int(rng.integers(0, n)), W.haar_2x2(rng)))
            for _ in range(int(rng.integers(3, 8))):
                t = int(rng.integers(0, n))
                others = [q for q in range(n) if q != t]
                c = int(rng.integers(0, len(others) + 1)) if others else 0
                ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
                vals = [int(b) for b in rng.integers(0, 2, size=c)]
                gl.append(_diag_gate(rng, n, t, ctrls, vals))
            gl.append(W.make_gate(int(rng.integers(0, n)), None, (), kind=W.KIND_X))
        gates = W.gate_list(gl)
        psi0 = random_state(n, dtype, 500 + n)
        ref = c128_of(psi0).copy()
        oracle.run_circuit(ref, n, gates)
        with qs.State(n, dtype) as st:
            st.from_numpy(psi0)
            st.apply_circuit(gates, flags=qs.QS_FLAG_FUSE)
            got = c128_of(st.to_numpy())
            st.from_numpy(psi0)
            st.apply_circuit(W.gate_list([]), flags=qs.QS_FLAG_FUSE)
            assert np.array_equal(st.to_numpy(), psi0.astype(NP[dtype]))
        assert np.max(np.abs(got - ref)) <= 4 * ATOL_CIRCUIT[dtype] * max(1.0, np.max(np.abs(ref))), n


def test_complex128_passes_of_exchanges(qs):
    """complex128 fused programs: arithmetic gates run alone (FP64-bound either way), runs of
    exchanges go into tile passes, also behind an arithmetic first gate; against the oracle
    (exchange-only runs bit for bit)."""
    rng = np.random.default_rng(128)
    n = 14
    gl = []
    for blk in range(6):
        gl.append(W.make_gate(int(rng.integers(0, 6)), W.haar_2x2(rng)))
        for _ in range(20):
            t = int(rng.integers(0, 8))
            c = [q for q in range(n) if q != t][int(rng.integers(0, n - 1))]
            gl.append(W.make_gate(t, None, (c,) if rng.random() < 0.5 else (), kind=W.KIND_X))
    gates = W.gate_list(gl)
    psi0 = random_state(n, "c128", 129)
    ref = psi0.copy()
    oracle.run_circuit(ref, n, gates)
    with qs.State(n, "c128") as st:
        st.from_numpy(psi0)
        st.apply_circuit(gates, flags=qs.QS_FLAG_FUSE)
        got = st.to_numpy()
    assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT["c128"]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tile_bits", [6, 9])
def test_folded_exchanges_with_tile_predicates(qs, dtype, tile_bits, monkeypatch):
    """CNOT ladders inside register groups are folded into the row copies; the same passes
    hold gates whose controls are not local (tiles they skip): every tile must still see the
    folded exchanges. Forward against the oracle, gradient against its finite differences
    (h = 1e-4, error O(h^2)), n = 15."""
    monkeypatch.setenv("QS_TILE_BITS", str(tile_bits))
    n, layers = 15, 3
    rng = np.random.default_rng(tile_bits)
    gl = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            gl.append(W.make_gate(q, None, (), kind=W.KIND_RY, param=p))
            p += 1
        for q in range(n - 1):
            gl.append(W.make_gate(q + 1, None, (q,), kind=W.KIND_X))
        for _ in range(4):  # controlled rotations with a far, non-local control
            t = int(rng.integers(0, 4))
            gl.append(W.make_gate(t, None, (n - 1 - int(rng.integers(0, 3)),), kind=W.KIND_RZ, param=p))
            p += 1
        for q in range(n - 2, -1, -1):
            gl.append(W.make_gate(q + 1, None, (q,), kind=W.KIND_X))
    gates = W.gate_list(gl)
    th = rng.uniform(0, 6.3, size=p)
    psi0 = W.basis_state(n, 0, NP[dtype])
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates, th)
    with qs.State(n, dtype) as st:
        st.apply_circuit(gates, th, flags=qs.QS_FLAG_FUSE)
        got = c128_of(st.to_numpy())
    assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype]
    fd = oracle.fd_grad(n, gates, th)  # controlled rotations: no two-term shift rule
    with qs.State(n, dtype) as st:
        e, g = st.adjoint_grad(gates, th, qs.QS_FLAG_FUSE)
    assert np.max(np.abs(g - fd)) <= (1e-4 if dtype == "c64" else 1e-6)
