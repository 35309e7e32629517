"""Fixed-point amplitudes (QS_Q30, Q1.30 integers) on the GPU, bit for bit against the Q1.30
oracle: single gates of every kind with controls of both polarities at n = 1..16, whole
circuits (one launch per gate, as a graph, the masked comparator), the paper's QFT and
streaming circuits, sampled outputs at n = 30, <Z_i>, and the calls that are not built for
the format."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import prepare_product, rotations, sample_indices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


def _random_q30_state(n, seed):
    return oracle.to_q30(W.random_state(n, seed))


def test_q30_single_gates_bit_exact(qs):
    rng = np.random.default_rng(300)
    for n in range(1, 17):
        psi0 = _random_q30_state(n, n)
        ref = psi0.copy()
        with qs.State(n, "q30") as st:
            st.from_numpy(psi0)
            for _ in range(10):
                t = int(rng.integers(0, n))
                others = [q for q in range(n) if q != t]
                c = int(rng.integers(0, min(4, n - 1) + 1))
                ctrls = [int(q) for q in rng.choice(others, size=c, replace=False)] if c else []
                mask = sum(1 << q for q in ctrls)
                vals = int(rng.integers(0, 1 << 16)) & mask
                kind = int(rng.integers(0, 5))
                if kind == 0:
                    st.apply_x(t, mask, vals)
                    oracle.apply_gate_q30(ref, n, t, mask, vals, W.X_MATRIX)
                else:
                    U = [W.haar_2x2(rng), np.diag(np.exp(1j * rng.uniform(0, 6, 2))),
                         np.diag([1.0, np.exp(0.7j)]), np.array([[0.6, -0.8], [0.8, 0.6]])][kind - 1]
                    st.apply_gate(t, U, mask, vals)
                    oracle.apply_gate_q30(ref, n, t, mask, vals, U)
            got = st.to_numpy()
        assert np.array_equal(got, ref), n


@pytest.mark.parametrize("mode", ["circuit", "graph", "masked", "masked_graph"])
def test_q30_circuits_bit_exact(qs, mode):
    """A 300-gate random circuit (0-3 controls, 25 % X / CNOT / Toffoli) at n = 14, the QFT
    (n = 12) and the streaming circuit (n = 13): every schedule equals the oracle bit for bit."""
    flags = {"circuit": 0, "graph": qs.QS_FLAG_GRAPH, "masked": qs.QS_FLAG_MASKED,
             "masked_graph": qs.QS_FLAG_MASKED | qs.QS_FLAG_GRAPH}[mode]
    for n, gates in ((14, W.random_circuit(14, 300, 3, seed=301, perm_fraction=0.25)), (12, W.qft_circuit(12)),
                     (13, W.streaming_circuit(13))):
        psi0 = _random_q30_state(n, 302 + n)
        ref = psi0.copy()
        oracle.run_circuit_q30(ref, n, gates)
        with qs.State(n, "q30") as st:
            st.from_numpy(psi0)
            st.apply_circuit(gates, flags=flags)
            got = st.to_numpy()
        assert np.array_equal(got, ref), (n, mode)


def test_q30_expect_z_and_basis(qs):
    """<Z_i> and the squared norm of Q1.30 states against the oracle's (float64 sums of the
    exact integer squares), n = 1..18; |0...0> is the integer 2^30."""
    for n in (1, 2, 5, 11, 12, 13, 18):
        psi0 = _random_q30_state(n, 700 + n)
        with qs.State(n, "q30") as st:
            st.from_numpy(psi0)
            z, nrm = st.expect_z()
            st.set_basis(3 % (1 << n))
            b = st.to_numpy()
        zr = oracle.expect_z_q30(psi0, n)
        assert np.max(np.abs(z - zr)) <= 1e-12, n
        p = (psi0[:, 0].astype(np.float64) ** 2 + psi0[:, 1].astype(np.float64) ** 2) / 2.0 ** 60
        assert abs(nrm - p.sum()) <= 1e-12
        want = np.zeros((1 << n, 2), dtype=np.int32)
        want[3 % (1 << n), 0] = 1 << 30
        assert np.array_equal(b, want)


def test_q30_full_size_sampled(qs):
    """n = 30 (8.6 GB of Q1.30 integers): a product state prepared on the device, then single
    gates with targets and controls on the lowest and highest qubits; 2^13 sampled outputs of
    each gate equal the oracle's one-amplitude update bit for bit."""
    import torch

    n = 30
    al, be = rotations(n, 30)
    buf = torch.empty((1 << n, 2), dtype=torch.int32, device="cuda")
    st = qs.State.wrap_q30(buf, n)
    try:
        prepare_product(st, al, be)
        inp = buf.clone()
        ks = sample_indices(n, 1 << 13, 31)
        kt = torch.from_numpy(ks.astype(np.int64)).cuda()
        xin = inp[kt].cpu().numpy()
        rng = np.random.default_rng(3030)
        for t, ctrls in ((0, ()), (n - 1, ()), (n - 1, (0,)), (0, (n - 1,)), (15, (1, 2, 27, 28)), (3, (0, 1, 2, 29))):
            vals = int(rng.integers(0, 1 << 30)) & sum(1 << q for q in ctrls)
            mask = sum(1 << q for q in ctrls)
            U = W.haar_2x2(rng)
            buf.copy_(inp)
            st.apply_gate(t, U, mask, vals)
            out = buf[kt].cpu().numpy()
            kp = torch.from_numpy((ks ^ np.uint64(1 << t)).astype(np.int64)).cuda()
            pin = inp[kp].cpu().numpy()
            want = np.array([oracle.gate_output_q30(int(k), t, mask, vals, U, xin[i], pin[i]) for i, k in enumerate(ks)],
                            dtype=np.int32)
            assert np.array_equal(out, want), (t, ctrls)
    finally:
        st.close()
        del buf
        torch.cuda.empty_cache()


def test_q30_unsupported_calls(qs):
    with qs.State(6, "q30") as st:
        g = W.hea_circuit(6, 1)
        th = W.hea_params(6, 1, seed=1)
        for flags in (qs.QS_FLAG_FUSE, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT):
            with pytest.raises(qs.QsError) as e:
                st.apply_circuit(g, th, flags)
            assert e.value.status == qs._lib.QS_EUNSUPPORTED
        with pytest.raises(qs.QsError) as e:
            st.adjoint_grad(g, th)
        assert e.value.status == qs._lib.QS_EUNSUPPORTED
    with pytest.raises(qs.QsError):
        qs.Batch([5], [W.hea_circuit(5, 1)], [10], "q30")
