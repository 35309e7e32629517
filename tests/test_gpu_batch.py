"""GPU parity of the batched persistent kernel (forward energy + adjoint gradient of many
states in one launch) against the CPU oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-4, "c128": 1e-9}


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


def _run_batch(qs, ns, circuits, nparams, thetas, dtype, flags=None, **tune):
    import torch

    b = qs.Batch(ns, circuits, nparams, dtype, **tune)
    try:
        th = torch.tensor(np.concatenate(thetas) if thetas else np.zeros(0), dtype=torch.float64, device="cuda")
        en = torch.full((len(ns),), float("nan"), dtype=torch.float64, device="cuda")
        gr = torch.full((max(1, b.num_params),), float("nan"), dtype=torch.float64, device="cuda")
        b.run(th, en, gr, qs.QS_FLAG_GRAPH if flags is None else flags)
        torch.cuda.synchronize()
        info = b.info()
    finally:
        b.close()
    e = en.cpu().numpy()
    g = gr.cpu().numpy()[: int(np.sum(nparams))]
    offs = np.concatenate([[0], np.cumsum(nparams)]).astype(int)
    return e, [g[offs[s]:offs[s + 1]] for s in range(len(ns))], info


@pytest.mark.parametrize("jit", [False, True])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("tune", [{}, {"small_bits": 5, "tile_bits": 5, "max_pass_gates": 3},
                                  {"small_bits": 5, "tile_bits": 7, "max_pass_gates": 64}])
def test_batch_ansatz_against_parameter_shift(qs, dtype, tune, jit):
    """States of 2..9 qubits running the ansatz (2 layers) with their own parameters: energies
    and gradients against the oracle's parameter-shift rule. The second and third tunings
    force the large-state path for n > 5 (tile passes through global memory; with
    QS_FLAG_JIT the pass-major path: every pass compiled for its shape and run over all
    states of one size at once)."""
    rng = np.random.default_rng(44)
    ns = [int(v) for v in rng.integers(2, 10, size=14)]
    circuits = [W.hea_circuit(n, 2) for n in ns]
    nparams = [4 * n for n in ns]
    thetas = [rng.uniform(0, 2 * np.pi, size=p) for p in nparams]
    flags = qs.QS_FLAG_GRAPH | (qs.QS_FLAG_JIT if jit else 0)
    e, g, _ = _run_batch(qs, ns, circuits, nparams, thetas, dtype, flags=flags, **tune)
    for s, n in enumerate(ns):
        assert abs(e[s] - oracle.energy(n, circuits[s], thetas[s])) <= TOL[dtype], s
        ps = oracle.param_shift_grad(n, circuits[s], thetas[s])
        assert np.max(np.abs(g[s] - ps)) <= TOL[dtype], s


def _random_param_circuit(rng, n, nparam, count):
    gl = []
    for _ in range(count):
        t = int(rng.integers(0, n))
        others = [q for q in range(n) if q != t]
        c = int(rng.integers(0, min(2, n - 1) + 1))
        ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
        vals = [int(b) for b in rng.integers(0, 2, size=c)]
        r = rng.random()
        if r < 0.3:
            gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_RY, param=int(rng.integers(0, nparam))))
        elif r < 0.6:
            gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_RZ, param=int(rng.integers(0, nparam))))
        elif r < 0.75:
            gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_X))
        elif r < 0.85:
            gl.append(W.make_gate(t, np.diag([1.0, np.exp(0.4j)]), ctrls, vals))
        else:
            gl.append(W.make_gate(t, W.haar_2x2(rng), ctrls, vals))
    return W.gate_list(gl)


@pytest.mark.parametrize("jit", [False, True])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("tune", [{}, {"small_bits": 4, "tile_bits": 5, "max_pass_gates": 5}])
def test_batch_random_circuits_against_finite_differences(qs, dtype, tune, jit):
    """Random controlled (also negatively controlled) RY/RZ with shared parameters, fixed
    Haar / phase / X gates, per-state gate lists: against oracle central differences (also
    with two states sharing one gate list, which the pass-major path runs together)."""
    rng = np.random.default_rng(7)
    ns = [3, 6, 8, 9, 7, 5, 8]
    nparams = [5, 6, 3, 7, 4, 2, 3]
    circuits = [_random_param_circuit(rng, n, p, 40) for n, p in zip(ns[:-1], nparams[:-1])]
    circuits.append(circuits[2])
    thetas = [rng.uniform(0, 2 * np.pi, size=p) for p in nparams]
    flags = qs.QS_FLAG_GRAPH | (qs.QS_FLAG_JIT if jit else 0)
    e, g, _ = _run_batch(qs, ns, circuits, nparams, thetas, dtype, flags=flags, **tune)
    tol = 1e-4 if dtype == "c64" else 1e-6
    for s, n in enumerate(ns):
        assert abs(e[s] - oracle.energy(n, circuits[s], thetas[s])) <= tol
        fd = oracle.fd_grad(n, circuits[s], thetas[s], h=1e-4)
        assert np.max(np.abs(g[s] - fd)) <= tol, s


def test_batch_graph_and_direct_launch_agree(qs):
    rng = np.random.default_rng(3)
    ns = [int(v) for v in rng.integers(4, 15, size=40)]
    circuits = [W.hea_circuit(n, 3) for n in ns]
    nparams = [6 * n for n in ns]
    thetas = [rng.uniform(0, 2 * np.pi, size=p) for p in nparams]
    e1, g1, _ = _run_batch(qs, ns, circuits, nparams, thetas, "c64", flags=qs.QS_FLAG_GRAPH)
    e2, g2, _ = _run_batch(qs, ns, circuits, nparams, thetas, "c64", flags=0)
    assert np.array_equal(e1, e2)
    for a, b in zip(g1, g2):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("jit", [False, True])
def test_batch_full_workload_sampled(qs, jit):
    """The batching workload at full size: 4096 states, n uniform in 10..20, 8 layers of the
    ansatz, complex64, interpreted and pass-major (QS_FLAG_JIT). Sampled states are checked
    against the oracle: parameter shift for two n = 10 states, central differences on two
    parameters of one n = 20 state."""
    ns, thetas = W.batch_workload(4096, 10, 20, 8, seed=4)
    ns = [int(v) for v in ns]
    circ = {n: W.hea_circuit(n, 8) for n in set(ns)}
    circuits = [circ[n] for n in ns]
    nparams = [16 * n for n in ns]
    e, g, info = _run_batch(qs, ns, circuits, nparams, thetas, "c64",
                            flags=qs.QS_FLAG_GRAPH | (qs.QS_FLAG_JIT if jit else 0))
    assert np.all(np.isfinite(e))
    small = [s for s, n in enumerate(ns) if n == 10][:2]
    for s in small:
        assert abs(e[s] - oracle.energy(10, circuits[s], thetas[s])) <= 1e-4
        assert np.max(np.abs(g[s] - oracle.param_shift_grad(10, circuits[s], thetas[s]))) <= 1e-4
    big = [s for s, n in enumerate(ns) if n == 20][0]
    assert abs(e[big] - oracle.energy(20, circuits[big], thetas[big])) <= 1e-4
    for p in (3, 250):
        tp, tm = thetas[big].copy(), thetas[big].copy()
        tp[p] += 1e-4
        tm[p] -= 1e-4
        fd = (oracle.energy(20, circuits[big], tp) - oracle.energy(20, circuits[big], tm)) / 2e-4
        assert abs(g[big][p] - fd) <= 1e-4


def test_batch_rejects_bad_input(qs):
    with pytest.raises(qs.QsError):
        qs.Batch([5, 31], [W.hea_circuit(5, 1), W.hea_circuit(5, 1)], [10, 10], "c64")  # n > 30
    with pytest.raises(qs.QsError):
        qs.Batch([5], [W.hea_circuit(5, 1)], [3], "c64")  # parameter index beyond the state's parameters
    with pytest.raises(qs.QsError):
        qs.Batch([5], [W.hea_circuit(5, 1)], [10], "c64", tile_bits=4)


def test_batch_jit_matches_interpreted(qs):
    """The pass-major path and the persistent kernel agree on a 40-state batch of 4..14
    qubits (3 layers), directly launched and as a graph."""
    rng = np.random.default_rng(3)
    ns = [int(v) for v in rng.integers(4, 15, size=40)]
    circuits = [W.hea_circuit(n, 3) for n in ns]
    nparams = [6 * n for n in ns]
    thetas = [rng.uniform(0, 2 * np.pi, size=p) for p in nparams]
    tune = {"small_bits": 8, "tile_bits": 8}
    e1, g1, _ = _run_batch(qs, ns, circuits, nparams, thetas, "c64", flags=qs.QS_FLAG_GRAPH, **tune)
    for flags in (qs.QS_FLAG_JIT, qs.QS_FLAG_JIT | qs.QS_FLAG_GRAPH):
        e2, g2, _ = _run_batch(qs, ns, circuits, nparams, thetas, "c64", flags=flags, **tune)
        assert np.max(np.abs(e1 - e2)) <= 1e-5
        for a, b in zip(g1, g2):
            assert np.max(np.abs(a - b)) <= 1e-4
