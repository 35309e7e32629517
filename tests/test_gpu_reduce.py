"""GPU parity of the one-pass <Z_i> / norm reduction against the oracle and closed forms."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import c128_of, prepare_product, random_state, rotations

pytestmark = pytest.mark.gpu

# complex64: |psi|^2 summed in float32 over at most 32 terms per thread and a 32-lane tree
# per warp, float64 above: relative error below (32 + 5) * 2^-24 ~ 2.2e-6 of the total.
TOL = {"c64": 5e-6, "c128": 1e-13}


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 2, 5, 11, 12, 13, 14, 17, 21])
def test_expect_z_random_states(qs, dtype, n):
    psi = random_state(n, dtype, 40 + n)
    st = qs.State(n, dtype)
    try:
        st.from_numpy(psi)
        z, nrm = st.expect_z()
    finally:
        st.close()
    ref = c128_of(psi)
    zr = oracle.expect_z(ref, n)
    nr = oracle.norm2(ref, n)
    assert np.max(np.abs(z - zr)) <= TOL[dtype]
    assert abs(nrm - nr) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_expect_z_basis_states_exact(qs, dtype):
    """|k>: <Z_i> = 1 - 2 bit_i(k) exactly, norm exactly 1."""
    for n in (3, 12, 13, 16):
        for k in (0, 1, (1 << n) - 1, 0x5A5A & ((1 << n) - 1)):
            st = qs.State(n, dtype)
            try:
                st.set_basis(k)
                z, nrm = st.expect_z()
            finally:
                st.close()
            assert np.array_equal(z, np.array([1.0 - 2.0 * ((k >> i) & 1) for i in range(n)]))
            assert nrm == 1.0


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_expect_z_full_size_product_state(qs, dtype):
    """n = 30: for prod_q RZ(beta_q) RY(alpha_q)|0>, <Z_q> = cos(alpha_q) and the norm is 1
    (closed forms at any size); tolerance adds the 60 preparation gates' rounding."""
    n = 30
    al, be = rotations(n, 31)
    st = qs.State(n, dtype)
    try:
        prepare_product(st, al, be)
        z, nrm = st.expect_z()
    finally:
        st.close()
    tol = 2e-5 if dtype == "c64" else 1e-12
    assert np.max(np.abs(z - np.cos(al))) <= tol
    assert abs(nrm - 1.0) <= tol


def test_expect_z_device_outputs(qs):
    import torch

    n = 15
    psi = random_state(n, "c64", 3)
    st = qs.State(n, "c64")
    try:
        st.from_numpy(psi)
        dz = torch.zeros(n, dtype=torch.float64, device="cuda")
        dn = torch.zeros(1, dtype=torch.float64, device="cuda")
        qs.qs_expect_z(st.h, qs.QS_FLAG_OUT_DEVICE, dz.data_ptr(), dn.data_ptr())
        torch.cuda.synchronize()
        z, nrm = st.expect_z()
    finally:
        st.close()
    assert np.array_equal(dz.cpu().numpy(), z)
    assert dn.item() == nrm
