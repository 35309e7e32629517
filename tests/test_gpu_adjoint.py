"""GPU parity of the adjoint gradient: against the oracle's parameter-shift and
finite-difference gradients, and properties that hold at any size."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


def _adjoint(qs, n, dtype, gates, theta, psi0=None, flags=0):
    st = qs.State(n, dtype)
    try:
        if psi0 is not None:
            st.from_numpy(psi0)
        e, g = st.adjoint_grad(gates, theta, flags)
        back = st.to_numpy()
    finally:
        st.close()
    return e, g, back


@pytest.mark.parametrize("fuse", [0, 1])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-10), ("c64", 1e-4)])
def test_hea_n10_against_parameter_shift(qs, dtype, tol, fuse):
    """Hardware-efficient ansatz, n = 10, 20 layers (400 parameters) against the oracle's
    parameter-shift gradient; complex64 within the stated 1e-4 gradient error."""
    n, layers = 10, 20
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    e, g, back = _adjoint(qs, n, dtype, gates, th, flags=qs.QS_FLAG_FUSE if fuse else 0)
    ps = oracle.param_shift_grad(n, gates, th)
    e_ref = oracle.energy(n, gates, th)
    assert abs(e - e_ref) <= tol
    assert np.max(np.abs(g - ps)) <= tol
    # the sweep un-applies every gate: the state is back to |0...0>
    back = back.astype(np.complex128)
    assert abs(back[0] - 1.0) <= (1e-10 if dtype == "c128" else 1e-4)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-10), ("c64", 1e-4)])
def test_diagonal_layers_against_parameter_shift(qs, dtype, tol):
    """Layers of RY on every qubit, then RZ on every qubit and a CZ ladder (runs of diagonal
    gates, which the fused forward pass applies as diagonal-run passes, the Hadamard-free RY
    before them as a leading gate), n = 9, 6 layers, against parameter shift."""
    n, layers = 9, 6
    gl = []
    p = 0
    cz = np.diag([1.0, -1.0])
    for _ in range(layers):
        for q in range(n):
            gl.append(W.make_gate(q, None, (), kind=W.KIND_RY, param=p))
            p += 1
        for q in range(n):
            gl.append(W.make_gate(q, None, (), kind=W.KIND_RZ, param=p))
            p += 1
        for q in range(n - 1):
            gl.append(W.make_gate(q + 1, cz, (q,)))
    gates = W.gate_list(gl)
    th = np.random.default_rng(91).uniform(0, 2 * np.pi, size=p)
    ps = oracle.param_shift_grad(n, gates, th)
    e_ref = oracle.energy(n, gates, th)
    for flags in (qs.QS_FLAG_FUSE, 0):
        e, g, _ = _adjoint(qs, n, dtype, gates, th, flags=flags)
        assert abs(e - e_ref) <= tol, flags
        assert np.max(np.abs(g - ps)) <= tol, flags


@pytest.mark.parametrize("tile_bits", [None, 3, 6])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-6), ("c64", 1e-4)])
def test_controlled_rotations_against_finite_differences(qs, dtype, tol, tile_bits, monkeypatch):
    """Random circuit with controlled (also negatively controlled) RY/RZ, shared parameters
    and fixed Haar gates, from a random start state, against central finite differences of
    the oracle energy (h = 1e-4: truncation error O(h^2))."""
    n = 7
    rng = np.random.default_rng(17)
    gl = []
    for i in range(60):
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
    th = rng.uniform(0, 2 * np.pi, size=14)  # parameters 12, 13 drive no gate
    psi0 = W.random_state(n, 99, dtype=np.complex64 if dtype == "c64" else np.complex128)
    flags = 0
    if tile_bits is not None:
        monkeypatch.setenv("QS_TILE_BITS", str(tile_bits))
        flags = qs.QS_FLAG_FUSE
    e, g, _ = _adjoint(qs, n, dtype, gates, th, psi0, flags=flags)
    fd = oracle.fd_grad(n, gates, th, h=1e-4, psi0=psi0.astype(np.complex128))
    assert np.max(np.abs(g - fd)) <= tol
    assert g[12] == 0.0 and g[13] == 0.0
    assert abs(e - oracle.energy(n, gates, th, psi0.astype(np.complex128))) <= tol


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_hea_n18_sampled_finite_differences(qs, dtype):
    """n = 18, 20 layers: a few gradient entries against oracle finite differences."""
    n, layers = 18, 20
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    e, g, _ = _adjoint(qs, n, dtype, gates, th)
    h = 1e-4
    for p in (0, 37, 401, 2 * n * layers - 1 - n):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (oracle.energy(n, gates, tp) - oracle.energy(n, gates, tm)) / (2 * h)
        assert abs(g[p] - fd) <= (1e-6 if dtype == "c128" else 1e-4), p


def test_hea_n24_properties(qs):
    """The differentiation workload (n = 24, 20 layers, 960 parameters):
    - the last layer's RZ angles do not change any Z probability (only a basis permutation
      follows them), so their gradient entries are 0 up to rounding;
    - the energy equals sum_i <Z_i> of the forward-only circuit;
    - complex64 and complex128 gradients agree within 1e-4."""
    n, layers = 24, 20
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    e64, g64, _ = _adjoint(qs, n, "c64", gates, th)
    e128, g128, back = _adjoint(qs, n, "c128", gates, th)
    e64f, g64f, _ = _adjoint(qs, n, "c64", gates, th, flags=qs.QS_FLAG_FUSE)
    e128f, g128f, _ = _adjoint(qs, n, "c128", gates, th, flags=qs.QS_FLAG_FUSE)
    assert np.max(np.abs(g128f - g128)) <= 1e-10 and abs(e128f - e128) <= 1e-10
    assert np.max(np.abs(g64f - g128)) <= 1e-4
    last_rz = [2 * n * (layers - 1) + 2 * q + 1 for q in range(n)]
    assert np.max(np.abs(g128[last_rz])) <= 1e-12
    assert np.max(np.abs(g64[last_rz])) <= 1e-5
    assert np.max(np.abs(g64 - g128)) <= 1e-4
    st = qs.State(n, "c128")
    try:
        st.apply_circuit(gates, th)
        z, _ = st.expect_z()
    finally:
        st.close()
    assert abs(e128 - z.sum()) <= 1e-10
    assert abs(back[0] - 1.0) <= 1e-10


def test_device_outputs_and_autograd(qs):
    import torch

    from paper_2411_18354_gb300.autograd import AdjointEnergy

    n, layers = 8, 3
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=5)
    st = qs.State(n, "c128")
    try:
        e_host, g_host = st.adjoint_grad(gates, th)
        st.set_basis(0)
        de = torch.zeros(1, dtype=torch.float64, device="cuda")
        dg = torch.zeros(th.size, dtype=torch.float64, device="cuda")
        qs.qs_adjoint_grad(st.h, gates, th, qs.QS_FLAG_OUT_DEVICE, de.data_ptr(), dg.data_ptr())
        torch.cuda.synchronize()
    finally:
        st.close()
    assert de.item() == e_host
    assert np.array_equal(dg.cpu().numpy(), g_host)
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    E = AdjointEnergy.apply(theta, n, gates, "c128")
    E.backward()
    assert abs(E.item() - e_host) <= 1e-12
    assert np.max(np.abs(theta.grad.cpu().numpy() - g_host)) <= 1e-12


def test_autograd_reuses_its_state_across_steps(qs):
    """Several optimisation steps through AdjointEnergy (compiled passes): each step's energy
    and gradient match the oracle's parameter shift, the working state is created once, and a
    step after an update starts again from |0...0> (no drift from the previous step)."""
    import torch

    from paper_2411_18354_gb300 import autograd as ag

    n, layers = 7, 2
    gates = W.hea_circuit(n, layers)
    theta = torch.tensor(W.hea_params(n, layers, seed=9), dtype=torch.float64, device="cuda", requires_grad=True)
    before = len(ag._STATES)
    for step in range(3):
        theta.grad = None
        E = ag.AdjointEnergy.apply(theta, n, gates, "c64", qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)
        E.backward()
        th = theta.detach().cpu().numpy()
        assert abs(E.item() - oracle.energy(n, gates, th)) <= 1e-5, step
        assert np.max(np.abs(theta.grad.cpu().numpy() - oracle.param_shift_grad(n, gates, th))) <= 1e-4, step
        with torch.no_grad():
            theta -= 0.1 * theta.grad
    assert len(ag._STATES) <= before + 1


@pytest.mark.parametrize("flags_name", ["fuse", "fuse_jit"])
def test_plan_cache_new_angles_and_structure_changes(qs, flags_name):
    """Repeated gradients of one circuit with new angles reuse the kept plan with the new
    matrices: every call matches the oracle's parameter shift, also after another circuit was
    differentiated in between and when an angle of 0 turns a rotation into the identity (its
    structure changes, so the call plans again)."""
    flags = qs.QS_FLAG_FUSE | (qs.QS_FLAG_JIT if flags_name == "fuse_jit" else 0)
    n, layers = 10, 6
    gates = W.hea_circuit(n, layers)
    other = W.hea_circuit(n, 2)
    rng = np.random.default_rng(21)
    thetas = [rng.uniform(0.1, 6.2, 2 * n * layers) for _ in range(3)]
    zero = thetas[0].copy()
    zero[[0, 5, 17]] = 0.0  # RY(0), RZ(0), RZ(0): identities
    with qs.State(n, "c128") as st:
        for th in (thetas[0], thetas[1], None, thetas[2], zero, thetas[0]):
            st.set_basis(0)
            if th is None:
                t2 = rng.uniform(0.1, 6.2, 2 * n * 2)
                e, g = st.adjoint_grad(other, t2, flags)
                assert np.max(np.abs(g - oracle.param_shift_grad(n, other, t2))) <= 1e-10
                continue
            e, g = st.adjoint_grad(gates, th, flags)
            assert abs(e - oracle.energy(n, gates, th)) <= 1e-10
            assert np.max(np.abs(g - oracle.param_shift_grad(n, gates, th))) <= 1e-10
