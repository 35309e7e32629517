"""``torch.autograd.Function`` over the library's adjoint gradient.

``AdjointEnergy.apply(theta, n, gates, dtype)`` returns E(theta) = <psi|sum_i Z_i|psi> for
psi = C(theta)|0...0> as a 0-d float64 tensor; its backward multiplies the incoming
gradient by dE/dtheta, which the forward call already computed with one reverse sweep
(qs_adjoint_grad). theta lives on the GPU; energy and gradient are written straight into
torch device tensors (QS_FLAG_OUT_DEVICE), on torch's current stream.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from ._lib import QS_FLAG_OUT_DEVICE


class AdjointEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, n: int, gates, dtype: str = "c64", flags: int = 0):
        from . import State

        th = theta.detach().to("cpu", torch.float64).numpy()  # gate matrices are built on the host
        st = State(n, dtype)
        try:
            energy = torch.empty((), dtype=torch.float64, device=theta.device)
            grad = torch.empty(th.size, dtype=torch.float64, device=theta.device)
            _lib.qs_adjoint_grad(st.h, gates, th, flags | QS_FLAG_OUT_DEVICE, energy.data_ptr(), grad.data_ptr())
            torch.cuda.current_stream().synchronize()
        finally:
            st.close()
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
