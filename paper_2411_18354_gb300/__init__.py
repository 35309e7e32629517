"""GB300 (sm_103a) state-vector kernels for controlled single-qubit gates.

A gate on target t with c controls is applied by scheduling only the 2^(n-1-c) amplitude
pairs whose controls hold, each pair index built by inserting the target and control bits
into a compact counter (arXiv 2411.18354, Section III-B, Eqs. 3-4). Everything runs in the
CUDA library ``libqs.so`` behind the C interface of ``include/qs.h``; this package is its
ctypes binding (``_lib``: same names as the C calls), a small ``State`` wrapper, and a
``torch.autograd.Function`` over the adjoint gradient. PyTorch is used only for streams and
device memory.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401  (re-exported C-ABI names)
    QS_C64, QS_C128, QS_Q30, QS_FLAG_ADJOINT, QS_FLAG_FUSE, QS_FLAG_GRAPH, QS_FLAG_JIT, QS_FLAG_MASKED, QS_FLAG_OUT_DEVICE, QS_GATE_U,
    QS_GATE_X, QS_GATE_RY, QS_GATE_RZ, QsError, qs_adjoint_grad, qs_apply_circuit, qs_apply_gate, qs_circuit_compile, qs_circuit_order,
    qs_circuit_schedule,
    qs_apply_gate_masked, qs_apply_x, qs_build_info, qs_expect_z, qs_expect_z_noalloc, qs_last_error,
    qs_measure_fma_peak, qs_debug_build, qs_debug_configure, qs_debug_status,
    qs_state_alloc, qs_batch_bytes, qs_batch_create, qs_batch_free, qs_batch_info, qs_batch_run, qs_get_l2_fetch_bytes, qs_get_tile_bits,
    qs_set_l2_fetch_bytes, qs_set_tile_bits,
    qs_state_copy_from_host, qs_state_copy_from_host_async, qs_state_copy_to_host, qs_state_copy_to_host_async,
    qs_state_free, qs_state_info, qs_state_set_basis, qs_state_set_stream, qs_state_synchronize, qs_state_wrap,
)
from .gates import GATE_DTYPE, as_gate_array  # noqa: F401

_DT = {"c64": QS_C64, "complex64": QS_C64, "c128": QS_C128, "complex128": QS_C128, "q30": QS_Q30}
_NP = {QS_C64: np.complex64, QS_C128: np.complex128}  # QS_Q30: int32 array of shape (2^n, 2)


def circuit_schedule(n: int, gates, theta=None, flags: int = QS_FLAG_FUSE, dtype="c64") -> dict:
    """Launch schedule of ``State(n, dtype).apply_circuit(gates, theta, flags)``: launches,
    single gates, tile passes, diagonal runs and the planner's modelled cost (host only)."""
    return qs_circuit_schedule(n, _DT[dtype], gates, theta, flags)


def circuit_order(n: int, gates, theta=None, flags: int = QS_FLAG_FUSE, dtype="c64") -> np.ndarray:
    """Gate indices in the order that schedule applies them (first applied first; with
    QS_FLAG_ADJOINT the reverse sweep's order); host only."""
    return qs_circuit_order(n, _DT[dtype], gates, theta, flags)


def _current_stream() -> int:
    import torch

    return int(torch.cuda.current_stream().cuda_stream)


class State:
    """An n-qubit state vector on the current CUDA device (owned by libqs unless wrapped)."""

    def __init__(self, n: int, dtype="c64", stream: int | None = None, _handle: int | None = None):
        self.dtype = _DT[dtype] if isinstance(dtype, str) else int(dtype)
        self.n = int(n)
        if _handle is not None:
            self.h = _handle
        else:
            self.h = qs_state_alloc(self.n, self.dtype, _current_stream() if stream is None else stream)

    @classmethod
    def wrap(cls, tensor, n: int, stream: int | None = None) -> "State":
        """Use a contiguous torch complex64/complex128 CUDA tensor of 2^n elements as the state."""
        import torch

        dt = QS_C64 if tensor.dtype == torch.complex64 else QS_C128 if tensor.dtype == torch.complex128 else None
        if dt is None or not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("need a contiguous complex64/complex128 CUDA tensor")
        h = qs_state_wrap(tensor.data_ptr(), tensor.numel() * tensor.element_size(), n, dt,
                          _current_stream() if stream is None else stream)
        st = cls(n, dt, _handle=h)
        st._tensor = tensor  # keep the memory alive
        return st

    @classmethod
    def wrap_q30(cls, tensor, n: int, stream: int | None = None) -> "State":
        """Use a contiguous torch int32 CUDA tensor of shape (2^n, 2) as a QS_Q30 state."""
        import torch

        if tensor.dtype != torch.int32 or not tensor.is_cuda or not tensor.is_contiguous() or \
                tuple(tensor.shape) != (1 << n, 2):
            raise ValueError("need a contiguous int32 CUDA tensor of shape (2^n, 2)")
        h = qs_state_wrap(tensor.data_ptr(), tensor.numel() * tensor.element_size(), n, QS_Q30,
                          _current_stream() if stream is None else stream)
        st = cls(n, QS_Q30, _handle=h)
        st._tensor = tensor
        return st

    def close(self):
        if getattr(self, "h", None):
            qs_state_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def device_ptr(self) -> int:
        return qs_state_info(self.h)[2]

    def set_basis(self, k: int = 0):
        qs_state_set_basis(self.h, k)

    def set_stream(self, stream: int):
        qs_state_set_stream(self.h, stream)

    def apply_gate(self, target: int, U, ctrl_mask: int = 0, ctrl_vals: int | None = None):
        qs_apply_gate(self.h, target, ctrl_mask, ctrl_mask if ctrl_vals is None else ctrl_vals, U)

    def apply_x(self, target: int, ctrl_mask: int = 0, ctrl_vals: int | None = None):
        qs_apply_x(self.h, target, ctrl_mask, ctrl_mask if ctrl_vals is None else ctrl_vals)

    def apply_gate_masked(self, target: int, U, ctrl_mask: int = 0, ctrl_vals: int | None = None):
        qs_apply_gate_masked(self.h, target, ctrl_mask, ctrl_mask if ctrl_vals is None else ctrl_vals, U)

    def apply_circuit(self, gates, theta=None, flags: int = 0):
        qs_apply_circuit(self.h, gates, theta, flags)

    def expect_z(self):
        return qs_expect_z(self.h)

    def adjoint_grad(self, gates, theta, flags: int = 0):
        return qs_adjoint_grad(self.h, gates, theta, flags)

    def to_numpy(self) -> np.ndarray:
        """The amplitudes: complex64 / complex128, or for QS_Q30 the Q1.30 integers as an int32
        array of shape (2^n, 2) (real, imaginary)."""
        if self.dtype == QS_Q30:
            out = np.empty((1 << self.n, 2), dtype=np.int32)
        else:
            out = np.empty(1 << self.n, dtype=_NP[self.dtype])
        qs_state_copy_to_host(self.h, out)
        return out

    def from_numpy(self, a: np.ndarray):
        if self.dtype == QS_Q30:
            a = np.ascontiguousarray(a, dtype=np.int32)
            if a.shape != (1 << self.n, 2):
                raise ValueError("a QS_Q30 state takes an int32 array of shape (2^n, 2)")
        else:
            a = np.ascontiguousarray(a, dtype=_NP[self.dtype])
            if a.size != (1 << self.n):
                raise ValueError("wrong number of amplitudes")
        qs_state_copy_from_host(self.h, a)


class Batch:
    """Many independent states (own qubit count, gate list and parameters) whose energies
    <sum_i Z_i> and adjoint gradients are computed by one persistent, graph-launched kernel."""

    def __init__(self, n_qubits, circuits, n_params, dtype="c64", small_bits=0, tile_bits=0, max_pass_gates=0,
                 stream: int | None = None):
        import numpy as _np

        self.dtype = _DT[dtype] if isinstance(dtype, str) else int(dtype)
        self.n_qubits = _np.asarray(n_qubits, dtype=_np.int32)
        gl = [as_gate_array(c) for c in circuits]
        self.gate_offsets = _np.concatenate([[0], _np.cumsum([len(g) for g in gl])]).astype(_np.uint64)
        self.param_offsets = _np.concatenate([[0], _np.cumsum(n_params)]).astype(_np.uint64)
        gates = _np.concatenate(gl) if gl else _np.zeros(0, dtype=GATE_DTYPE)
        self.h = qs_batch_create(self.n_qubits, gates, self.gate_offsets, self.param_offsets, self.dtype,
                                 small_bits, tile_bits, max_pass_gates,
                                 _current_stream() if stream is None else stream)

    @property
    def num_params(self) -> int:
        return int(self.param_offsets[-1])

    def info(self) -> dict:
        return qs_batch_info(self.h)

    def algorithmic_bytes(self) -> float:
        return qs_batch_bytes(self.h)

    def run(self, theta, energy, grad, flags: int = QS_FLAG_GRAPH):
        """theta / energy / grad: torch float64 CUDA tensors (or device addresses)."""
        addr = lambda t: t if isinstance(t, int) else t.data_ptr()  # noqa: E731
        qs_batch_run(self.h, addr(theta), addr(energy), addr(grad), flags)

    def close(self):
        if getattr(self, "h", None):
            qs_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build(force: bool = False, debug: bool = False) -> str:
    from .build import build as _b

    return _b(force=force, debug=debug)
