"""Tile passes compiled for their exact shape (QS_FLAG_JIT): the same fused programs as the
interpreted passes, against the oracle (forward) and against parameter shift / finite
differences (adjoint sweep)."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import ATOL_CIRCUIT, NP, c128_of, random_state

pytestmark = pytest.mark.gpu

DTYPES = ["c64", "c128"]


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


def _random_gates(rng, n, count, cmax=3):
    gl = []
    for _ in range(count):
        t = int(rng.integers(0, n))
        others = [q for q in range(n) if q != t]
        c = int(rng.integers(0, min(cmax, n - 1) + 1))
        ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
        vals = [int(b) for b in rng.integers(0, 2, size=c)]
        r = rng.random()
        if r < 0.15:
            gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_X))
        elif r < 0.3:
            gl.append(W.make_gate(t, np.diag(np.exp(1j * rng.uniform(0, 6, 2))), ctrls, vals))
        elif r < 0.4:
            gl.append(W.make_gate(t, np.diag([1.0, np.exp(0.3j)]), ctrls, vals))
        elif r < 0.5:
            th = rng.uniform(0, 6)
            gl.append(W.make_gate(t, np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]]), ctrls, vals))
        else:
            gl.append(W.make_gate(t, W.haar_2x2(rng), ctrls, vals))
    return W.gate_list(gl)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tile_bits", [2, 5, 9, 12])
def test_jit_fused_circuits_match_oracle(qs, dtype, tile_bits, monkeypatch):
    """Random circuits (controls also negative and non-local; general, real, diagonal,
    one-sided and exchange gates) with QS_FLAG_FUSE | QS_FLAG_JIT, plain and recorded into a
    graph, several tile sizes, n = 3..17, against the oracle; the interpreted passes give the
    same state within rounding."""
    monkeypatch.setenv("QS_TILE_BITS", str(tile_bits))
    rng = np.random.default_rng(100 + tile_bits)
    for n in (3, 9, 14, 17):
        gates = _random_gates(rng, n, 120)
        psi0 = random_state(n, dtype, n)
        ref = c128_of(psi0).copy()
        oracle.run_circuit(ref, n, gates)
        outs = {}
        for flags in (qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT | qs.QS_FLAG_GRAPH,
                      qs.QS_FLAG_FUSE):
            with qs.State(n, dtype) as st:
                st.from_numpy(psi0)
                st.apply_circuit(gates, flags=flags)
                outs[flags] = c128_of(st.to_numpy())
            assert np.max(np.abs(outs[flags] - ref)) <= ATOL_CIRCUIT[dtype], (n, flags)
        jit, interp = outs[qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT], outs[qs.QS_FLAG_FUSE]
        assert np.max(np.abs(jit - interp)) <= ATOL_CIRCUIT[dtype], n


@pytest.mark.parametrize("dtype", DTYPES)
def test_jit_exchanges_bit_exact(qs, dtype):
    """Exchange-only circuits (X / CNOT / Toffoli, folded into row copies or not) stay bit-exact
    in shape-compiled passes."""
    rng = np.random.default_rng(7)
    n = 15
    gl = []
    for _ in range(200):
        t = int(rng.integers(0, n))
        others = [q for q in range(n) if q != t]
        c = int(rng.integers(0, 3))
        ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
        gl.append(W.make_gate(t, None, ctrls, [int(b) for b in rng.integers(0, 2, size=c)], kind=W.KIND_X))
    gates = W.gate_list(gl)
    psi0 = random_state(n, dtype, 8)
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates)
    with qs.State(n, dtype) as st:
        st.from_numpy(psi0)
        st.apply_circuit(gates, flags=qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)
        got = st.to_numpy()
    assert np.array_equal(got, ref.astype(NP[dtype]))


@pytest.mark.parametrize("dtype", DTYPES)
def test_jit_ansatz_and_qft(qs, dtype):
    """The differentiation ansatz (n = 20, 4 layers; merged rotations and folded CNOT ladders)
    and the QFT (n = 16) fused with compiled passes, against the oracle."""
    n, layers = 20, 4
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    ref = W.basis_state(n, 0)
    oracle.run_circuit(ref, n, gates, th)
    with qs.State(n, dtype) as st:
        st.apply_circuit(gates, th, flags=qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)
        got = c128_of(st.to_numpy())
    assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype]
    n = 16
    q = W.qft_circuit(n)
    psi0 = random_state(n, dtype, 16)
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, q)
    with qs.State(n, dtype) as st:
        st.from_numpy(psi0)
        st.apply_circuit(q, flags=qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)
        got = c128_of(st.to_numpy())
    assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype]


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-10), ("c64", 1e-4)])
def test_jit_adjoint_hea_against_parameter_shift(qs, dtype, tol):
    """Fused gradient with compiled forward and sweep passes, n = 10, 20 layers, against the
    oracle's parameter shift; the sweep returns the start state."""
    n, layers = 10, 20
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    with qs.State(n, dtype) as st:
        e, g = st.adjoint_grad(gates, th, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)
        back = c128_of(st.to_numpy())
    ps = oracle.param_shift_grad(n, gates, th)
    assert abs(e - oracle.energy(n, gates, th)) <= tol
    assert np.max(np.abs(g - ps)) <= tol
    assert abs(back[0] - 1.0) <= (1e-10 if dtype == "c128" else 1e-4)


@pytest.mark.parametrize("tile_bits", [3, 6])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-6), ("c64", 1e-4)])
def test_jit_adjoint_controlled_rotations(qs, dtype, tol, tile_bits, monkeypatch):
    """Controlled (also negatively) RY / RZ with shared parameters, exchanges and Haar gates
    from a random start state, compiled sweep passes, against central finite differences of
    the oracle energy; parameters that drive no gate get 0."""
    monkeypatch.setenv("QS_TILE_BITS", str(tile_bits))
    n = 8
    rng = np.random.default_rng(23)
    gl = []
    for _ in range(70):
        t = int(rng.integers(0, n))
        others = [q for q in range(n) if q != t]
        c = int(rng.integers(0, 3))
        ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
        vals = [int(b) for b in rng.integers(0, 2, size=c)]
        r = rng.random()
        if r < 0.35:
            gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_RY, param=int(rng.integers(0, 12))))
        elif r < 0.7:
            gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_RZ, param=int(rng.integers(0, 12))))
        elif r < 0.85:
            gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_X))
        else:
            gl.append(W.make_gate(t, W.haar_2x2(rng), ctrls, vals))
    gates = W.gate_list(gl)
    th = rng.uniform(0, 2 * np.pi, size=14)
    psi0 = W.random_state(n, 99, dtype=NP[dtype])
    with qs.State(n, dtype) as st:
        st.from_numpy(psi0)
        e, g = st.adjoint_grad(gates, th, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)
    fd = oracle.fd_grad(n, gates, th, h=1e-4, psi0=psi0.astype(np.complex128))
    assert np.max(np.abs(g - fd)) <= tol
    assert g[12] == 0.0 and g[13] == 0.0
    assert abs(e - oracle.energy(n, gates, th, psi0.astype(np.complex128))) <= tol


@pytest.mark.parametrize("dtype,tile_bits", [("c64", 13), ("c128", 12), ("c64", 11)])
def test_jit_many_tiles_per_block(qs, dtype, tile_bits, monkeypatch):
    """n = 22 with tiles large enough that a block holds one tile buffer only (complex64 2^13,
    complex128 2^12 amplitudes) and small enough that every block processes several tiles;
    2^11 complex64 tiles are double-buffered with the same property. Random circuit with
    non-local controls (tiles skipped) against the oracle."""
    monkeypatch.setenv("QS_TILE_BITS", str(tile_bits))
    n = 22
    rng = np.random.default_rng(220 + tile_bits)
    gates = _random_gates(rng, n, 150, cmax=2)
    psi0 = random_state(n, dtype, 22)
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates)
    with qs.State(n, dtype) as st:
        st.from_numpy(psi0)
        st.apply_circuit(gates, flags=qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)
        got = c128_of(st.to_numpy())
    assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype]


@pytest.mark.parametrize("dtype,tile_bits", [("c64", 12), ("c128", 10)])
def test_jit_adjoint_many_tiles_per_block(qs, dtype, tile_bits, monkeypatch):
    """Sweep passes with several tiles per block, n = 21: psi and lambda tiles of 2^12
    complex64 amplitudes (one buffer per block) and of 2^10 complex128 amplitudes (two
    buffers): energy against the oracle, gradient against the interpreted passes and against
    central finite differences of the oracle energy for a few parameters."""
    monkeypatch.setenv("QS_TILE_BITS", str(tile_bits))
    n, layers = 21, 2
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=21)
    with qs.State(n, dtype) as st:
        e, g = st.adjoint_grad(gates, th, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)
        st.set_basis(0)
        e2, g2 = st.adjoint_grad(gates, th, qs.QS_FLAG_FUSE)
    tol = 1e-4 if dtype == "c64" else 1e-9
    assert abs(e - oracle.energy(n, gates, th)) <= tol
    assert np.max(np.abs(g - g2)) <= tol
    h = 1e-4
    for p in (0, 17, 2 * n * layers - 1):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (oracle.energy(n, gates, tp) - oracle.energy(n, gates, tm)) / (2 * h)
        assert abs(g[p] - fd) <= (1e-4 if dtype == "c64" else 1e-6), p


@pytest.mark.parametrize("jit", [False, True])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-6), ("c64", 1e-4)])
def test_reordered_plans_match_oracle(qs, dtype, tol, jit, monkeypatch):
    """Plans that apply commuting gates out of the given order (tile passes of 2^7 amplitudes:
    the ansatz's layers interleave across passes): checked to be reordered on the host, then the
    forward state against the oracle's in-order run and the gradient (its sweep in its own
    order) against the oracle's finite differences, interpreted and compiled passes."""
    monkeypatch.setenv("QS_TILE_BITS", "7")
    n, layers = 12, 6
    gl = list(W.hea_circuit(n, layers))
    npar = 2 * n * layers
    for q in range(0, n - 2, 3):  # controlled phases and controlled rotations between layers
        gl.append(W.make_gate(q + 2, np.diag([1.0, np.exp(0.7j)]), [q], [1]))
        gl.append(W.make_gate(q + 1, None, [q + 2], [0], kind=W.KIND_RY, param=npar))
        npar += 1
    tail = W.hea_circuit(n, 2)
    tail["param"] += npar
    gates = W.gate_list(gl + list(tail))
    th = np.random.default_rng(9).uniform(0.0, 2.0 * np.pi, size=npar + 4 * n)
    flags = qs.QS_FLAG_FUSE | (qs.QS_FLAG_JIT if jit else 0)
    order = qs.circuit_order(n, gates, th, flags, dtype=dtype)
    assert (order != np.arange(len(gates))).any()
    ref = W.basis_state(n, 0)
    oracle.run_circuit(ref, n, gates, th)
    with qs.State(n, dtype) as st:
        st.apply_circuit(gates, th, flags=flags)
        got = c128_of(st.to_numpy())
        assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype]
        st.set_basis(0)
        e, g = st.adjoint_grad(gates, th, flags)
    assert abs(e - oracle.energy(n, gates, th)) <= tol
    assert np.max(np.abs(g - oracle.fd_grad(n, gates, th))) <= tol


@pytest.mark.parametrize("jit", [False, True])
def test_kept_plans_take_new_angles(qs, jit):
    """qs_apply_circuit keeps fused plans by structure: the same circuit with new angles (plain
    and recorded into graphs), another circuit in between and an angle of 0 (a rotation
    becomes the identity: planned again) all match the oracle."""
    flags = qs.QS_FLAG_FUSE | (qs.QS_FLAG_JIT if jit else 0)
    n, layers = 14, 5
    gates = W.hea_circuit(n, layers)
    rng = np.random.default_rng(31)
    thetas = [rng.uniform(0.1, 6.2, 2 * n * layers) for _ in range(3)]
    zero = thetas[1].copy()
    zero[[2, 9]] = 0.0
    other = _random_gates(rng, n, 80)
    psi0 = random_state(n, "c128", 7)
    with qs.State(n, "c128") as st:
        for th, extra in ((thetas[0], 0), (thetas[1], qs.QS_FLAG_GRAPH), (None, 0), (thetas[2], 0), (zero, 0),
                          (thetas[0], qs.QS_FLAG_GRAPH)):
            st.from_numpy(psi0)
            g, t = (other, None) if th is None else (gates, th)
            st.apply_circuit(g, t, flags=flags | extra)
            ref = psi0.copy()
            oracle.run_circuit(ref, n, g, t)
            assert np.max(np.abs(st.to_numpy() - ref)) <= ATOL_CIRCUIT["c128"]


def test_kernels_loaded_from_disk_match_oracle(tmp_path):
    """QS_JIT_CACHE_DIR: a process that loads the compiled passes from the directory (written by
    an earlier process) runs them correctly: both processes' states against the oracle."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out_files = [tmp_path / "psi0.npy", tmp_path / "psi1.npy"]
    code = ("import sys, numpy as np\n"
            "import paper_2411_18354_gb300 as qs, workloads as W\n"
            "n = 14\n"
            "g = W.hea_circuit(n, 4)\n"
            "th = W.hea_params(n, 4, seed=2)\n"
            "with qs.State(n, 'c128') as st:\n"
            "    st.apply_circuit(g, th, flags=qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)\n"
            "    np.save(sys.argv[1], st.to_numpy())\n")
    env = dict(os.environ, QS_JIT_CACHE_DIR=str(tmp_path / "kernels"), PYTHONPATH=root)
    n = 14
    ref = W.basis_state(n, 0)
    oracle.run_circuit(ref, n, W.hea_circuit(n, 4), W.hea_params(n, 4, seed=2))
    for f in out_files:
        r = subprocess.run([sys.executable, "-c", code, str(f)], env=env, capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stderr
        assert np.max(np.abs(np.load(f) - ref)) <= ATOL_CIRCUIT["c128"]
    assert list((tmp_path / "kernels").glob("qs_jit_*.bin"))
