"""Host tests of the launch planner through qs_circuit_schedule (no device needed): argument
checks, the unfused and masked schedules, and properties of the fused plan (tile passes,
runs of diagonal gates, the modelled cost never above launching every gate alone)."""
import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


def test_schedule_validates_arguments(qs):
    g = W.random_circuit(8, 10, 2, seed=1)
    for bad in (
        dict(n=0, dtype="c64", flags=qs.QS_FLAG_FUSE),
        dict(n=41, dtype="c64", flags=qs.QS_FLAG_FUSE),
        dict(n=8, dtype="c64", flags=qs.QS_FLAG_FUSE | qs.QS_FLAG_MASKED),
        dict(n=8, dtype="c64", flags=64),
    ):
        with pytest.raises(qs.QsError):
            qs.circuit_schedule(bad["n"], g, flags=bad["flags"], dtype=bad["dtype"])
    with pytest.raises(qs.QsError):  # target 9 on 8 qubits
        qs.circuit_schedule(8, W.gate_list([W.make_gate(9, W.H_MATRIX, ())]))
    with pytest.raises(qs.QsError):  # parameterised gate without theta
        qs.circuit_schedule(8, W.gate_list([W.make_gate(0, None, (), kind=W.KIND_RY, param=0)]))


def test_unfused_and_masked_schedules_launch_every_gate(qs):
    n = 12
    gl = [W.make_gate(q, W.H_MATRIX, ()) for q in range(n)]
    gl += [W.make_gate(q + 1, None, (q,), kind=W.KIND_X) for q in range(n - 1)]
    g = W.gate_list(gl)
    s = qs.circuit_schedule(n, g, flags=0)
    assert s["launches"] == s["single_gates"] == s["gates"] == len(gl)
    assert s["tile_passes"] == 0 and s["diag_runs"] == 0
    # H: whole state; CNOT with a control on qubit >= 3: half of it (64-byte units, complex64);
    # each launch also ~2 us of latency against the state's read + write at 6 TB/s
    lat = 2e-6 / (2 * 8 * 2**n / 6e12)
    assert s["model_cost"] == pytest.approx(n + sum(0.5 if q >= 3 else 1.0 for q in range(n - 1)) + len(gl) * lat)
    m = qs.circuit_schedule(n, g, flags=qs.QS_FLAG_MASKED)
    assert m["launches"] == len(gl) and m["model_cost"] == pytest.approx(len(gl) * (1 + lat))


def test_same_target_gates_merge_before_planning(qs):
    """RY then RZ on one qubit (same controls) becomes one gate."""
    n = 6
    gl = []
    for q in range(n):
        gl.append(W.make_gate(q, None, (), kind=W.KIND_RY, param=2 * q))
        gl.append(W.make_gate(q, None, (), kind=W.KIND_RZ, param=2 * q + 1))
    th = np.linspace(0.1, 1.2, 2 * n)
    assert qs.circuit_schedule(n, W.gate_list(gl), th, flags=0)["gates"] == n


def test_state_within_one_tile_is_one_pass(qs):
    """A circuit on n <= tile bits: one tile pass holds the whole state."""
    n = 10
    s = qs.circuit_schedule(n, W.qft_circuit(n))
    assert s == {**s, "launches": 1, "tile_passes": 1, "single_gates": 0, "diag_runs": 0}
    assert s["pass_gates"] == n + n * (n - 1) // 2


def test_ansatz_ladder_goes_into_passes(qs):
    """Hardware-efficient ansatz at n = 24: every CNOT of the ladder runs inside a tile pass
    (five passes per layer), none as a launch of its own."""
    n, layers = 24, 20
    s = qs.circuit_schedule(n, W.hea_circuit(n, layers), W.hea_params(n, layers, seed=3))
    assert s["single_gates"] <= 1
    assert s["tile_passes"] == 5 * layers
    assert s["model_cost"] < 0.5 * qs.circuit_schedule(n, W.hea_circuit(n, layers), W.hea_params(n, layers, seed=3),
                                                        flags=0)["model_cost"]


def test_qft_phases_go_to_diagonal_runs(qs):
    """QFT on 29 qubits: each Hadamard leads the run of controlled phases aimed at its qubit in
    one diagonal-run pass (the last qubits, whose runs are short, share a tile pass); no gate
    runs alone and no launch is spent on fewer gates than before diagonal runs existed."""
    n = 29
    s = qs.circuit_schedule(n, W.qft_circuit(n))
    assert s["single_gates"] == 0
    assert s["diag_runs"] >= 20 and s["launches"] < n
    assert s["model_cost"] < 0.2 * qs.circuit_schedule(n, W.qft_circuit(n), flags=0)["model_cost"]


def test_diagonal_gates_go_to_diagonal_runs(qs):
    """A run of diagonal gates on many qubits (targets too many for one tile) is applied by
    diagonal-run passes of at most 64 gates each."""
    n = 26
    rng = np.random.default_rng(5)
    gl = []
    for i in range(150):
        t = int(rng.integers(0, n))
        c = [int(q) for q in rng.choice([q for q in range(n) if q != t], size=int(rng.integers(0, 3)), replace=False)]
        ph = np.exp(1j * rng.uniform(0, 6.28))
        gl.append(W.make_gate(t, np.array([[1, 0], [0, ph]]), sorted(c)))
    s = qs.circuit_schedule(n, W.gate_list(gl))
    assert s["diag_runs"] == 3 and s["launches"] == 3


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_fused_cost_never_above_unfused(qs, dtype):
    """Launching every gate alone is one of the plans the planner weighs, so its modelled cost
    is never higher."""
    for seed in range(6):
        n = 14 + seed
        g = W.random_circuit(n, 120, 4, seed=seed)
        f = qs.circuit_schedule(n, g, dtype=dtype)
        u = qs.circuit_schedule(n, g, flags=0, dtype=dtype)
        assert f["model_cost"] <= u["model_cost"] + 1e-9
        assert f["gates"] == u["gates"]


def test_complex128_arithmetic_gates_stay_out_of_passes(qs):
    """complex128 gates are FP64-bound alone or in a pass: only exchanges are fused."""
    n = 20
    rng = np.random.default_rng(9)
    gl = [W.make_gate(int(rng.integers(0, n)), W.haar_2x2(rng), ()) for _ in range(30)]
    s = qs.circuit_schedule(n, W.gate_list(gl), dtype="c128")
    assert s["tile_passes"] == 0 and s["launches"] == s["gates"]


def test_identity_gates_launch_nothing(qs):
    """Exact identities (U = I, controlled or not, and RZ(0)) need no launch, fused or not; they
    do not split a pass either."""
    n = 16
    gl = [W.make_gate(q, np.eye(2), ([q + 1] if q < n - 1 else [])) for q in range(n)]
    gl.append(W.make_gate(3, None, (), kind=W.KIND_RZ, param=0))
    th = np.zeros(1)
    for flags in (0, qs.QS_FLAG_FUSE):
        s = qs.circuit_schedule(n, W.gate_list(gl), th, flags=flags)
        assert s["launches"] == 0, (flags, s)
    mixed = [W.make_gate(0, W.H_MATRIX, ()), W.make_gate(5, np.eye(2), ()), W.make_gate(1, W.H_MATRIX, ())]
    s = qs.circuit_schedule(20, W.gate_list(mixed))
    assert s["launches"] == 1 and s["tile_passes"] == 1, s


def test_schedule_validates_theta(qs):
    """Parameter indices past theta and non-finite angles are rejected as by qs_apply_circuit;
    RY(0) is an exact identity and needs no launch."""
    g = W.gate_list([W.make_gate(0, None, (), kind=W.KIND_RY, param=3)])
    with pytest.raises(qs.QsError):
        qs.circuit_schedule(4, g, np.zeros(2))
    with pytest.raises(qs.QsError):
        qs.circuit_schedule(4, g, np.array([0.0, 0.0, 0.0, np.nan]))
    assert qs.circuit_schedule(4, g, np.zeros(4))["launches"] == 0
    assert qs.circuit_schedule(4, g, np.full(4, 0.3))["launches"] == 1


def test_circuit_compile_caches_by_shape(qs):
    """qs_circuit_compile generates and compiles the shape-specialised pass kernels on the
    host (NVRTC, no device): a second call with the same structure at other angles is served
    from the cache (no compile time); invalid gates are rejected as by qs_apply_circuit."""
    import numpy as np
    import workloads as W

    q = qs
    n, layers = 12, 2
    g = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    r1 = q.qs_circuit_compile(n, q.QS_C64, g, th)
    assert r1["passes"] > 0
    r2 = q.qs_circuit_compile(n, q.QS_C64, g, th + 0.5)
    assert r2["passes"] == r1["passes"] and r2["compile_seconds"] == 0.0
    ra = q.qs_circuit_compile(n, q.QS_C128, g, th, adjoint=True)
    assert ra["passes"] > 0
    bad = g.copy()
    bad[0]["target"] = n
    with pytest.raises(q.QsError):
        q.qs_circuit_compile(n, q.QS_C64, bad, th)
