"""qs_expect_z_noalloc: the <Z_i> / norm reduction that allocates nothing.

Some callers cannot allocate device memory at the moment they need a reduction: their
memory belongs to another allocator, or they run on a latency budget that a cudaMalloc
would break. This entry point takes the state as a raw device pointer, writes its results
to caller-provided device memory, and keeps its partial sums in one fixed array inside the
library. These tests call it through the C interface twice in a row and compare each result
with the allocating entry point, qs_expect_z, within the tolerances of the reduction tests.
The file is named so that pytest collects it last; it also runs on its own in a fresh process.
"""
import numpy as np
import pytest

from gpu_helpers import random_state

pytestmark = pytest.mark.gpu

TOL = {"c64": 5e-6, "c128": 1e-13}


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [3, 12, 13, 20, 24])
def test_noalloc_matches_allocating_entry_point(qs, dtype, n):
    import torch

    psi = random_state(n, dtype, 500 + n)
    st = qs.State(n, dtype)
    try:
        st.from_numpy(psi)
        z_ref, nrm_ref = st.expect_z()  # allocating entry point, host outputs
        stream = torch.cuda.current_stream().cuda_stream
        dt = qs.QS_C64 if dtype == "c64" else qs.QS_C128
        for call in range(2):  # the shared scratch keeps the previous call's contents
            dz = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            dn = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            qs.qs_expect_z_noalloc(st.device_ptr, n, dt, stream, dz.data_ptr(), dn.data_ptr())
            torch.cuda.synchronize()
            z = dz.cpu().numpy()
            nrm = dn.item()
            assert np.max(np.abs(z - z_ref)) <= TOL[dtype], (call, z, z_ref)
            assert abs(nrm - nrm_ref) <= TOL[dtype], call
    finally:
        st.close()


def test_noalloc_rejects_bad_arguments(qs):
    import torch

    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(qs.QsError):
        qs.qs_expect_z_noalloc(0, 10, qs.QS_C64, 0, d.data_ptr(), 0)  # NULL state
    with pytest.raises(qs.QsError) as e:
        qs.qs_expect_z_noalloc(d.data_ptr(), 41, qs.QS_C64, 0, d.data_ptr(), 0)  # beyond the maximum
    assert "out of range" in str(e.value)
    with pytest.raises(qs.QsError):
        qs.qs_expect_z_noalloc(d.data_ptr(), 2, qs.QS_C64, 0, 0, 0)  # no output
    # host buffers are rejected on the host, before any launch (a kernel given one would fault)
    host_out = np.zeros(4, dtype=np.float64)
    with pytest.raises(qs.QsError) as e:
        qs.qs_expect_z_noalloc(d.data_ptr(), 2, qs.QS_C64, 0, host_out.ctypes.data, 0)
    assert "device" in str(e.value)
    host_psi = np.zeros(8, dtype=np.complex64)
    with pytest.raises(qs.QsError):
        qs.qs_expect_z_noalloc(host_psi.ctypes.data, 3, qs.QS_C64, 0, d.data_ptr(), 0)
    pinned = torch.zeros(4, dtype=torch.float64).pin_memory()
    with pytest.raises(qs.QsError):
        qs.qs_expect_z_noalloc(d.data_ptr(), 2, qs.QS_C64, 0, 0, pinned.data_ptr())
    # the entry point still works after the rejections
    z = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    psi = torch.zeros(4, dtype=torch.complex64, device="cuda")
    psi[0] = 1.0
    qs.qs_expect_z_noalloc(psi.data_ptr(), 2, qs.QS_C64, torch.cuda.current_stream().cuda_stream, z.data_ptr(), 0)
    torch.cuda.synchronize()
    assert z.cpu().tolist() == [1.0, 1.0]
