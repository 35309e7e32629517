"""``torch.autograd.Function`` over the library's adjoint gradient.

``AdjointEnergy.apply(theta, n, gates, dtype)`` returns E(theta) = <psi|sum_i Z_i|psi> for
psi = C(theta)|0...0> as a 0-d float64 tensor; its backward multiplies the incoming
gradient by dE/dtheta, which the forward call already computed with one reverse sweep
(qs_adjoint_grad). theta lives on the GPU; energy and gradient are written straight into
torch device tensors (QS_FLAG_OUT_DEVICE), on torch's current stream. The working state of each
(n, dtype, device) is created once and reused by later calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from ._lib import QS_FLAG_OUT_DEVICE


_STATES = {}  # (n, dtype, device index) -> State reused by every call (its lambda vector too)


def _state(n: int, dtype: str, device: torch.device):
    """The working state of (n, dtype) on `device`, created on first use and kept: a training
    loop then allocates nothing per step (qs_adjoint_grad keeps its lambda vector and scratch
    with the state)."""
    from . import State

    key = (int(n), str(dtype), device.index if device.index is not None else torch.cuda.current_device())
    st = _STATES.get(key)
    if st is None:
        with torch.cuda.device(key[2]):
            st = State(n, dtype)
        _STATES[key] = st
    return st


class AdjointEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, n: int, gates, dtype: str = "c64", flags: int = 0):
        # the gate matrices are built on the host from theta: this copy is the call's only
        # host round trip; energy and gradient are written to device tensors on torch's current
        # stream without waiting
        th = theta.detach().to("cpu", torch.float64).numpy()
        st = _state(n, dtype, theta.device)
        _lib.qs_state_set_stream(st.h, int(torch.cuda.current_stream(theta.device).cuda_stream))
        st.set_basis(0)
        energy = torch.empty((), dtype=torch.float64, device=theta.device)
        grad = torch.empty(th.size, dtype=torch.float64, device=theta.device)
        _lib.qs_adjoint_grad(st.h, gates, th, flags | QS_FLAG_OUT_DEVICE, energy.data_ptr(), grad.data_ptr())
        ctx.save_for_backward(grad)
        return energy

    @staticmethod
    def backward(ctx, g_out):
        (grad,) = ctx.saved_tensors
        return (g_out * grad).to(grad.dtype), None, None, None, None


def energy_and_grad(theta, n: int, gates, dtype: str = "c64"):
    """Convenience: numpy in, (E, dE/dtheta) numpy out."""
    from . import State

    with State(n, dtype) as st:
        return _lib.qs_adjoint_grad(st.h, gates, np.asarray(theta, dtype=np.float64))
