"""GPU tests of interface paths: stream changes, the CUDA-graph cache beyond its capacity,
the smallest states for reductions and gradients, parameterised gates in every schedule."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import ATOL_CIRCUIT, c128_of, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


def test_set_stream_moves_the_work(qs):
    """Gates enqueued after qs_state_set_stream run on the new stream, in order with work the
    caller puts there."""
    import torch

    n = 14
    psi0 = random_state(n, "c64", 11)
    gates = W.random_circuit(n, 60, 4, seed=12)
    s = torch.cuda.Stream()
    with qs.State(n, "c64") as st:
        st.from_numpy(psi0)
        st.set_stream(int(s.cuda_stream))
        st.apply_circuit(gates, flags=qs.QS_FLAG_FUSE)
        s.synchronize()
        got = c128_of(st.to_numpy())
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates)
    assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT["c64"]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_graph_cache_beyond_capacity(qs, dtype):
    """20 different circuits launched with QS_FLAG_GRAPH on one state (the cache keeps 16 and
    drops the oldest), then the first ones again: every result against the oracle."""
    n = 10
    circuits = [W.random_circuit(n, 15, 3, seed=200 + i) for i in range(20)]
    ref = W.basis_state(n, 0)
    with qs.State(n, dtype) as st:
        for i in list(range(20)) + [0, 1, 2]:
            flags = qs.QS_FLAG_GRAPH | (qs.QS_FLAG_FUSE if i % 2 else 0)
            st.apply_circuit(circuits[i], flags=flags)
            oracle.run_circuit(ref, n, circuits[i])
            got = c128_of(st.to_numpy())
            assert np.max(np.abs(got - ref)) <= 4 * ATOL_CIRCUIT[dtype], i


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-5), ("c128", 1e-12)])
def test_smallest_states(qs, dtype, tol):
    """n = 1, 2, 3: <Z_i> and the norm against the oracle; the adjoint gradient of a small
    parameterised circuit against parameter shift, fused and not."""
    for n in (1, 2, 3):
        psi0 = random_state(n, dtype, 30 + n)
        with qs.State(n, dtype) as st:
            st.from_numpy(psi0)
            z, nrm = st.expect_z()
        ref = c128_of(psi0)
        assert np.max(np.abs(z - oracle.expect_z(ref, n))) <= tol
        assert abs(nrm - oracle.norm2(ref, n)) <= tol
        gl = []
        for q in range(n):
            gl.append(W.make_gate(q, None, (), kind=W.KIND_RY, param=2 * q))
            gl.append(W.make_gate(q, None, (), kind=W.KIND_RZ, param=2 * q + 1))
        for q in range(n - 1):
            gl.append(W.make_gate(q + 1, None, (q,), kind=W.KIND_X))
        gates = W.gate_list(gl)
        th = np.random.default_rng(n).uniform(0, 6.3, size=2 * n)
        ps = oracle.param_shift_grad(n, gates, th)
        for flags in (0, qs.QS_FLAG_FUSE):
            with qs.State(n, dtype) as st:
                e, g = st.adjoint_grad(gates, th, flags)
            assert abs(e - oracle.energy(n, gates, th)) <= 10 * tol
            assert np.max(np.abs(g - ps)) <= 10 * tol, (n, flags)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_parameterised_gates_in_every_schedule(qs, dtype):
    """RY / RZ gates (controlled and not) read theta in the reduced, graph, fused and masked
    schedules alike."""
    n = 11
    rng = np.random.default_rng(7)
    gl = []
    for i in range(80):
        t = int(rng.integers(0, n))
        others = [q for q in range(n) if q != t]
        c = int(rng.integers(0, 3))
        ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
        kind = W.KIND_RY if i % 3 == 0 else (W.KIND_RZ if i % 3 == 1 else W.KIND_U)
        if kind == W.KIND_U:
            gl.append(W.make_gate(t, W.haar_2x2(rng), ctrls))
        else:
            gl.append(W.make_gate(t, None, ctrls, kind=kind, param=i))
    gates = W.gate_list(gl)
    th = rng.uniform(0, 6.3, size=80)
    psi0 = random_state(n, dtype, 8)
    ref = c128_of(psi0).copy()
    oracle.run_circuit(ref, n, gates, th)
    for flags in (0, qs.QS_FLAG_GRAPH, qs.QS_FLAG_FUSE, qs.QS_FLAG_MASKED, qs.QS_FLAG_MASKED | qs.QS_FLAG_GRAPH):
        with qs.State(n, dtype) as st:
            st.from_numpy(psi0)
            st.apply_circuit(gates, th, flags)
            got = c128_of(st.to_numpy())
        assert np.max(np.abs(got - ref)) <= ATOL_CIRCUIT[dtype], flags


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_graph_cache_key_collision(qs, dtype, monkeypatch):
    """QS_TEST_GRAPH_KEY forces every recorded graph onto one hash value: a second circuit
    whose hash collides with a recorded one must not replay that graph but be validated,
    planned and recorded itself (the cache compares the stored key bytes). Then both
    circuits are replayed again; every result against the oracle. A circuit that differs
    only in theta, or only in its gate count (a prefix), collides the same way."""
    monkeypatch.setenv("QS_TEST_GRAPH_KEY", "0x5eed")
    n = 11
    a = W.random_circuit(n, 40, 3, seed=901)
    b = W.random_circuit(n, 40, 3, seed=902)
    prefix = a[:25]
    rng = np.random.default_rng(903)
    rot = W.gate_list([W.make_gate(q, None, (), kind=W.KIND_RY, param=q) for q in range(n)])
    th1 = rng.uniform(0, 6.3, size=n)
    th2 = th1.copy()
    th2[3] += 0.5
    for flags in (qs.QS_FLAG_GRAPH, qs.QS_FLAG_GRAPH | qs.QS_FLAG_FUSE):
        ref = W.basis_state(n, 0)
        with qs.State(n, dtype) as st:
            for gates, th in ((a, None), (b, None), (prefix, None), (rot, th1), (rot, th2), (a, None), (b, None),
                              (rot, th1)):
                st.apply_circuit(gates, th, flags=flags)
                oracle.run_circuit(ref, n, gates, th)
                got = c128_of(st.to_numpy())
                assert np.max(np.abs(got - ref)) <= 4 * ATOL_CIRCUIT[dtype], flags
