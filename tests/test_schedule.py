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
    """Hardware-efficient ansatz at n = 24: every CNOT of the ladder runs inside a tile pass,
    none as a launch of its own; passes take gates of several layers (the circuit's own order
    needs five per layer)."""
    n, layers = 24, 20
    s = qs.circuit_schedule(n, W.hea_circuit(n, layers), W.hea_params(n, layers, seed=3))
    assert s["single_gates"] <= 1
    assert s["tile_passes"] <= 2 * layers
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


def _mixed_circuit(n: int, count: int, seed: int):
    """Gates of every structure the order rule distinguishes: general, real (RY), diagonal
    (RZ, two-sided and one-sided phases), exchanges; 0-3 controls with random values."""
    rng = np.random.default_rng(seed)
    gl, p = [], 0
    for _ in range(count):
        t = int(rng.integers(n))
        c = int(rng.integers(0, 4))
        ctrls = W.random_controls(rng, n, t, c)
        vals = [int(v) for v in rng.integers(0, 2, size=len(ctrls))]
        kind = int(rng.integers(6))
        if kind == 0:
            gl.append(W.make_gate(t, W.haar_2x2(rng), ctrls, vals))
        elif kind == 1:
            gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_X))
        elif kind == 2:
            ph = np.exp(1j * rng.uniform(0, 2 * np.pi, 2))
            gl.append(W.make_gate(t, np.diag(ph), ctrls, vals))
        elif kind == 3:
            gl.append(W.make_gate(t, np.diag([1.0, np.exp(1j * rng.uniform(0, 2 * np.pi))]), ctrls, vals))
        else:
            gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_RY if kind == 4 else W.KIND_RZ, param=p))
            p += 1
    return W.gate_list(gl), rng.uniform(-np.pi, np.pi, max(p, 1))


@pytest.fixture(params=[5, 7])
def small_tiles(qs, request):
    """Tiles of 2^5 or 2^7 amplitudes (forward and sweep), so that circuits on a few qubits need
    many passes and the planner reorders; the defaults are restored afterwards."""
    for adj in (0, 1):
        qs.qs_set_tile_bits(qs.QS_C64, adj, request.param)
    yield
    for adj in (0, 1):
        qs.qs_set_tile_bits(qs.QS_C64, adj, 0)


def _run(oracle, n, gates, theta, psi0):
    return oracle.run_circuit(psi0.copy(), n, gates, theta)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_fused_order_applies_the_same_circuit(qs, small_tiles, seed):
    """The order qs_circuit_order reports for a fused plan (gates that commute moved, Section
    III applies the circuit serially) gives the state of the given order: the oracle runs both."""
    import oracle

    n = 10
    gates, theta = _mixed_circuit(n, 160, seed)
    psi0 = W.random_state(n, seed + 100)
    ref = _run(oracle, n, gates, theta, psi0)
    for flags in (qs.QS_FLAG_FUSE, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT):
        order = qs.circuit_order(n, gates, theta, flags)
        assert sorted(order.tolist()) == list(range(len(gates)))
        got = _run(oracle, n, gates[order], theta, psi0)
        assert np.max(np.abs(got - ref)) < 1e-12
    sweep = qs.circuit_order(n, gates, theta, qs.QS_FLAG_FUSE | qs.QS_FLAG_ADJOINT)
    assert sorted(sweep.tolist()) == list(range(len(gates)))
    got = _run(oracle, n, gates[sweep[::-1]], theta, psi0)  # the sweep un-applies in this order
    assert np.max(np.abs(got - ref)) < 1e-12


def test_fused_order_check_detects_a_wrong_order(qs, small_tiles):
    """The comparison above is sensitive: swapping two neighbouring gates that do not commute
    (the same target, general matrices) changes the oracle's state."""
    import oracle

    n = 10
    gates, theta = _mixed_circuit(n, 160, 7)
    psi0 = W.random_state(n, 107)
    ref = _run(oracle, n, gates, theta, psi0)
    order = qs.circuit_order(n, gates, theta, qs.QS_FLAG_FUSE)
    for i in range(len(order) - 1):
        a, b = gates[order[i]], gates[order[i + 1]]
        if a["target"] == b["target"] and a["kind"] == W.KIND_U and b["kind"] == W.KIND_U and \
                np.abs(a["U"][2:6]).sum() > 1e-3 and np.abs(b["U"][2:6]).sum() > 1e-3:
            bad = order.copy()
            bad[i], bad[i + 1] = bad[i + 1], bad[i]
            assert np.max(np.abs(_run(oracle, n, gates[bad], theta, psi0) - ref)) > 1e-6
            return
    pytest.skip("no adjacent pair of general gates on one target in this order")


def test_fused_order_fills_passes_across_layers(qs):
    """Hardware-efficient ansatz (RY, RZ per qubit, CNOT ladder): its gates commute enough
    that a tile pass takes gates of several layers, so the fused plan needs far fewer passes
    than the 5 per layer of the circuit's own order (n = 24, 12-qubit tiles, 4 always local)."""
    n, layers = 24, 20
    g = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    for flags in (qs.QS_FLAG_FUSE, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT):
        s = qs.circuit_schedule(n, g, th, flags)
        assert s["tile_passes"] <= 2 * layers
        order = qs.circuit_order(n, g, th, flags)
        assert (order != np.arange(len(g))).any()
    s = qs.circuit_schedule(n, g, th, qs.QS_FLAG_FUSE | qs.QS_FLAG_ADJOINT)
    assert s["tile_passes"] + s["single_gates"] <= 3 * layers + 4  # forward + sweep, was 5 + 5 per layer


def test_compiled_kernels_kept_on_disk(qs, tmp_path):
    """QS_JIT_CACHE_DIR: a second process loads the compiled pass kernels from the directory
    instead of compiling them (host only: compilation needs no device); a file whose stored
    source differs from the wanted kernel is not used but compiled again and rewritten."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import paper_2411_18354_gb300 as qs, workloads as W\n"
            "g = W.hea_circuit(12, 3)\n"
            "th = W.hea_params(12, 3, seed=1)\n"
            "print(qs.qs_circuit_compile(12, qs.QS_C64, g, th)['compile_seconds'])\n")
    env = dict(os.environ, QS_JIT_CACHE_DIR=str(tmp_path), PYTHONPATH=root)

    def run():
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stderr
        return float(out.stdout.strip().splitlines()[-1])

    first = run()
    files = sorted(tmp_path.glob("qs_jit_*.bin"))
    assert files and first > 0.05
    assert run() < first / 5  # loaded, not compiled
    for f in files:  # another source under the same name: ignored
        f.write_bytes(b"QSJITC1\n" + (5).to_bytes(8, "little") + b"other" + b"\0" * 64)
    assert run() > first / 5  # compiled again
    assert all(f.read_bytes().count(b"qs_pass") > 0 for f in files)  # and rewritten
    assert run() < first / 5


def test_order_validates_arguments(qs):
    """qs_circuit_order rejects what qs_circuit_schedule rejects, and a NULL output, before
    planning; without QS_FLAG_FUSE the order is the given one (reversed for the sweep)."""
    import ctypes

    g = W.random_circuit(8, 10, 2, seed=1)
    with pytest.raises(qs.QsError):
        qs.circuit_order(8, W.gate_list([W.make_gate(9, W.H_MATRIX, ())]))
    with pytest.raises(qs.QsError):
        qs.circuit_order(8, g, flags=qs.QS_FLAG_FUSE | qs.QS_FLAG_MASKED)
    with pytest.raises(qs.QsError):
        qs.circuit_order(0, g)
    gp = g.ctypes.data_as(ctypes.c_void_p)
    assert qs._lib.lib().qs_circuit_order(8, qs.QS_C64, gp, g.size, None, 0, qs.QS_FLAG_FUSE, None) != 0
    assert (qs.circuit_order(8, g, flags=0) == np.arange(g.size)).all()
    assert (qs.circuit_order(8, g, flags=qs.QS_FLAG_ADJOINT) == np.arange(g.size)[::-1]).all()
