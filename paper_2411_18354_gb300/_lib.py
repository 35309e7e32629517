"""ctypes binding of libqs (``include/qs.h``): argument marshalling only.

Every function here has the name of the C entry point it calls, converts Python/numpy
arguments to the C types, and raises ``QsError`` when the call returns a status other than
QS_OK. No step of the computation runs in Python: if the shared library is missing, loading
fails with an error instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import DEBUG_LIB_PATH, LIB_PATH

QS_OK, QS_EINVAL, QS_ENOMEM, QS_ECUDA, QS_ETIMEOUT, QS_EUNSUPPORTED = range(6)
QS_C64, QS_C128, QS_Q30 = 0, 1, 2
QS_GATE_U, QS_GATE_X, QS_GATE_RY, QS_GATE_RZ = 0, 1, 2, 3
QS_FLAG_FUSE, QS_FLAG_GRAPH, QS_FLAG_OUT_DEVICE, QS_FLAG_MASKED, QS_FLAG_JIT, QS_FLAG_ADJOINT = 1, 2, 4, 8, 16, 32

STATUS_NAMES = {0: "QS_OK", 1: "QS_EINVAL", 2: "QS_ENOMEM", 3: "QS_ECUDA", 4: "QS_ETIMEOUT", 5: "QS_EUNSUPPORTED"}


class QsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_c_state_p = ctypes.c_void_p
_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p

# (name, restype, argtypes) for every function declared in include/qs.h
_SIGNATURES = [
    ("qs_last_error", ctypes.c_char_p, []),
    ("qs_build_info", ctypes.c_char_p, []),
    ("qs_state_alloc", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_c_state_p)]),
    ("qs_state_wrap", ctypes.c_int, [_vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_c_state_p)]),
    ("qs_state_free", ctypes.c_int, [_c_state_p]),
    ("qs_state_info", ctypes.c_int, [_c_state_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(_vp)]),
    ("qs_state_set_stream", ctypes.c_int, [_c_state_p, _vp]),
    ("qs_state_set_basis", ctypes.c_int, [_c_state_p, _u64]),
    ("qs_state_copy_to_host", ctypes.c_int, [_c_state_p, _vp, ctypes.c_size_t]),
    ("qs_state_copy_from_host", ctypes.c_int, [_c_state_p, _vp, ctypes.c_size_t]),
    ("qs_state_copy_to_host_async", ctypes.c_int, [_c_state_p, _vp, ctypes.c_size_t]),
    ("qs_state_copy_from_host_async", ctypes.c_int, [_c_state_p, _vp, ctypes.c_size_t]),
    ("qs_state_synchronize", ctypes.c_int, [_c_state_p]),
    ("qs_apply_gate", ctypes.c_int, [_c_state_p, ctypes.c_int, _u64, _u64, _dp]),
    ("qs_apply_x", ctypes.c_int, [_c_state_p, ctypes.c_int, _u64, _u64]),
    ("qs_apply_gate_masked", ctypes.c_int, [_c_state_p, ctypes.c_int, _u64, _u64, _dp]),
    ("qs_apply_circuit", ctypes.c_int, [_c_state_p, _vp, ctypes.c_size_t, _dp, ctypes.c_size_t, ctypes.c_int]),
    ("qs_circuit_schedule", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _dp, ctypes.c_size_t,
                                           ctypes.c_int, _vp]),
    ("qs_circuit_order", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _dp, ctypes.c_size_t,
                                        ctypes.c_int, _vp]),
    ("qs_circuit_compile", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _dp, ctypes.c_size_t,
                                          ctypes.c_int, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int)]),
    ("qs_measure_fma_peak", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _dp]),
    ("qs_debug_build", ctypes.c_int, []),
    ("qs_debug_configure", ctypes.c_int, [_u64, _vp, _u64]),
    ("qs_debug_status", ctypes.c_int, [ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(_u64)]),
    ("qs_expect_z", ctypes.c_int, [_c_state_p, _dp, _dp, ctypes.c_int]),
    ("qs_expect_z_noalloc", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _dp, _dp]),
    ("qs_adjoint_grad", ctypes.c_int, [_c_state_p, _vp, ctypes.c_size_t, _dp, ctypes.c_size_t, _dp, _dp, ctypes.c_int]),
    ("qs_batch_create", ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    ("qs_batch_run", ctypes.c_int, [_vp, _dp, _dp, _dp, ctypes.c_int]),
    ("qs_batch_info", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    ("qs_batch_bytes", ctypes.c_int, [_vp, _dp]),
    ("qs_batch_free", ctypes.c_int, [_vp]),
    ("qs_set_tile_bits", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("qs_get_tile_bits", ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    ("qs_set_l2_fetch_bytes", ctypes.c_int, [ctypes.c_int]),
    ("qs_get_l2_fetch_bytes", ctypes.c_int, []),
]

_lib = None


def lib_path() -> str:
    """libqs.so, or its debug build when QS_LIB_VARIANT=debug."""
    return DEBUG_LIB_PATH if os.environ.get("QS_LIB_VARIANT") == "debug" else LIB_PATH


def lib():
    """Load libqs.so (built in-tree by ``paper_2411_18354_gb300.build``)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise ImportError(f"{os.path.basename(path)} not found at {path}: build it with "
                              f"paper_2411_18354_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return [name for name, _, _ in _SIGNATURES]


def _check(status: int):
    if status != QS_OK:
        raise QsError(status, lib().qs_last_error().decode(errors="replace"))


def _dptr(a):
    if a is None:
        return None
    return ctypes.cast(ctypes.c_void_p(int(a)), _dp) if isinstance(a, int) else a.ctypes.data_as(_dp)


def _u8(U) -> np.ndarray:
    U = np.asarray(U)
    if np.iscomplexobj(U) or U.shape == (2, 2):
        U = np.asarray(U, dtype=np.complex128).reshape(4)
        out = np.empty(8)
        out[0::2] = U.real
        out[1::2] = U.imag
        return out
    return np.ascontiguousarray(U, dtype=np.float64).reshape(8)


def qs_last_error() -> str:
    return lib().qs_last_error().decode(errors="replace")


def qs_build_info() -> str:
    return lib().qs_build_info().decode(errors="replace")


def qs_state_alloc(n: int, dtype: int, stream: int = 0) -> int:
    h = _c_state_p()
    _check(lib().qs_state_alloc(n, dtype, _vp(stream or None), ctypes.byref(h)))
    return h.value


def qs_state_wrap(dev_ptr: int, nbytes: int, n: int, dtype: int, stream: int = 0) -> int:
    h = _c_state_p()
    _check(lib().qs_state_wrap(_vp(dev_ptr), nbytes, n, dtype, _vp(stream or None), ctypes.byref(h)))
    return h.value


def qs_state_free(h: int) -> None:
    _check(lib().qs_state_free(_c_state_p(h)))


def qs_state_info(h: int):
    n = ctypes.c_int()
    dt = ctypes.c_int()
    p = _vp()
    _check(lib().qs_state_info(_c_state_p(h), ctypes.byref(n), ctypes.byref(dt), ctypes.byref(p)))
    return n.value, dt.value, p.value


def qs_state_set_stream(h: int, stream: int) -> None:
    _check(lib().qs_state_set_stream(_c_state_p(h), _vp(stream or None)))


def qs_state_set_basis(h: int, k: int) -> None:
    _check(lib().qs_state_set_basis(_c_state_p(h), k))


def qs_state_copy_to_host(h: int, dst: np.ndarray) -> None:
    if not dst.flags.c_contiguous:
        raise ValueError("dst must be contiguous")
    _check(lib().qs_state_copy_to_host(_c_state_p(h), _vp(dst.ctypes.data), dst.nbytes))


def qs_state_copy_from_host(h: int, src: np.ndarray) -> None:
    src = np.ascontiguousarray(src)
    _check(lib().qs_state_copy_from_host(_c_state_p(h), _vp(src.ctypes.data), src.nbytes))


def qs_state_copy_to_host_async(h: int, dst: np.ndarray) -> None:
    """Enqueue the copy on the state's stream; dst (contiguous, page-locked for overlap) must
    stay alive and untouched until qs_state_synchronize."""
    if not dst.flags.c_contiguous:
        raise ValueError("dst must be contiguous")
    _check(lib().qs_state_copy_to_host_async(_c_state_p(h), _vp(dst.ctypes.data), dst.nbytes))


def qs_state_copy_from_host_async(h: int, src: np.ndarray) -> None:
    """Enqueue the copy on the state's stream; src must be contiguous (no temporary copy is
    made) and stay alive and unchanged until qs_state_synchronize."""
    if not src.flags.c_contiguous:
        raise ValueError("src must be contiguous")
    _check(lib().qs_state_copy_from_host_async(_c_state_p(h), _vp(src.ctypes.data), src.nbytes))


def qs_state_synchronize(h: int) -> None:
    _check(lib().qs_state_synchronize(_c_state_p(h)))


def qs_apply_gate(h: int, target: int, ctrl_mask: int, ctrl_vals: int, U) -> None:
    u = _u8(U)
    _check(lib().qs_apply_gate(_c_state_p(h), target, ctrl_mask, ctrl_vals, u.ctypes.data_as(_dp)))


def qs_apply_x(h: int, target: int, ctrl_mask: int = 0, ctrl_vals: int = 0) -> None:
    _check(lib().qs_apply_x(_c_state_p(h), target, ctrl_mask, ctrl_vals))


def qs_apply_gate_masked(h: int, target: int, ctrl_mask: int, ctrl_vals: int, U) -> None:
    u = _u8(U)
    _check(lib().qs_apply_gate_masked(_c_state_p(h), target, ctrl_mask, ctrl_vals, u.ctypes.data_as(_dp)))


def _gates_arg(gates):
    from .gates import as_gate_array

    g = as_gate_array(gates)
    return g, _vp(g.ctypes.data) if g.size else None


def _theta_arg(theta):
    if theta is None:
        return None, None, 0
    t = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    return t, t.ctypes.data_as(_dp), t.size


def qs_apply_circuit(h: int, gates, theta=None, flags: int = 0) -> None:
    g, gp = _gates_arg(gates)
    t, tp, nt = _theta_arg(theta)
    _check(lib().qs_apply_circuit(_c_state_p(h), gp, g.size, tp, nt, flags))


class QsSchedule(ctypes.Structure):
    """``qs_schedule`` of include/qs.h."""

    _fields_ = [("launches", ctypes.c_int32), ("single_gates", ctypes.c_int32), ("tile_passes", ctypes.c_int32),
                ("diag_runs", ctypes.c_int32), ("gates", ctypes.c_int32), ("pass_gates", ctypes.c_int32),
                ("model_cost", ctypes.c_double), ("algorithmic_bytes", ctypes.c_double),
                ("algorithmic_flops", ctypes.c_double)]


def qs_circuit_schedule(n: int, dtype: int, gates, theta=None, flags: int = 0) -> dict:
    """The launch schedule qs_apply_circuit would use (host only, no device needed)."""
    g, gp = _gates_arg(gates)
    t, tp, nt = _theta_arg(theta)
    out = QsSchedule()
    _check(lib().qs_circuit_schedule(n, dtype, gp, g.size, tp, nt, flags, _vp(ctypes.addressof(out))))
    return {name: getattr(out, name) for name, _ in QsSchedule._fields_}


def qs_circuit_order(n: int, dtype: int, gates, theta=None, flags: int = 0):
    """The order (gate indices, first applied first) in which the plan of qs_circuit_schedule
    applies the gates; with QS_FLAG_ADJOINT the reverse sweep's order (host only)."""
    import numpy as np

    g, gp = _gates_arg(gates)
    t, tp, nt = _theta_arg(theta)
    out = np.zeros(max(1, g.size), dtype=np.int32)
    _check(lib().qs_circuit_order(n, dtype, gp, g.size, tp, nt, flags, _vp(out.ctypes.data)))
    return out[: g.size].copy()


def qs_circuit_compile(n: int, dtype: int, gates, theta=None, flags: int = QS_FLAG_FUSE | QS_FLAG_JIT,
                       adjoint: bool = False) -> dict:
    """Compile the shape-specialised tile-pass kernels of a fused circuit (or of its gradient's
    forward and sweep programs) without running them; no device needed."""
    g, gp = _gates_arg(gates)
    t, tp, nt = _theta_arg(theta)
    secs = ctypes.c_double(0.0)
    passes = ctypes.c_int(0)
    _check(lib().qs_circuit_compile(n, dtype, gp, g.size, tp, nt, flags, 1 if adjoint else 0, ctypes.byref(secs),
                                    ctypes.byref(passes)))
    return {"compile_seconds": secs.value, "passes": passes.value}


def qs_debug_build() -> bool:
    return bool(lib().qs_debug_build())


def qs_debug_configure(n_amps: int, counts_dev: int = 0, count_n: int = 0) -> None:
    """Debug build: check accesses against n_amps amplitudes (0: off) and count writes per
    amplitude into the device array counts_dev (uint32, count_n entries; 0: off)."""
    _check(lib().qs_debug_configure(n_amps, _vp(counts_dev or None), count_n))


def qs_debug_status():
    """Debug build: (status word, an index that failed the bounds check)."""
    st = ctypes.c_uint(0)
    bad = _u64(0)
    _check(lib().qs_debug_status(ctypes.byref(st), ctypes.byref(bad)))
    return st.value, bad.value


def qs_measure_fma_peak(dtype: int, iters: int = 1 << 16, stream: int = 0) -> float:
    """Measured FMA rate (flop/s) of the current device in the arithmetic of ``dtype``."""
    out = ctypes.c_double(0.0)
    _check(lib().qs_measure_fma_peak(dtype, iters, _vp(stream or None), ctypes.byref(out)))
    return out.value


def qs_expect_z(h: int, flags: int = 0, out=None, out_norm2=None):
    """Host outputs (default): returns (z[n] numpy array, norm2). With QS_FLAG_OUT_DEVICE,
    ``out`` / ``out_norm2`` are device addresses (ints) and nothing is returned."""
    if flags & QS_FLAG_OUT_DEVICE:
        _check(lib().qs_expect_z(_c_state_p(h), _dptr(out), _dptr(out_norm2), flags))
        return None
    n, _, _ = qs_state_info(h)
    z = np.empty(n)
    nrm = np.empty(1)
    _check(lib().qs_expect_z(_c_state_p(h), z.ctypes.data_as(_dp), nrm.ctypes.data_as(_dp), flags))
    return z, float(nrm[0])


def qs_expect_z_noalloc(psi_dev: int, n: int, dtype: int, stream: int, out_z_dev: int, out_norm2_dev: int) -> None:
    """<Z_i> and the squared norm of the 2^n amplitudes at device address ``psi_dev``, written
    to device addresses (ints; 0 = not wanted), without allocating anything (see qs.h)."""
    _check(lib().qs_expect_z_noalloc(_vp(psi_dev), n, dtype, _vp(stream or None),
                                     _dptr(out_z_dev) if out_z_dev else None,
                                     _dptr(out_norm2_dev) if out_norm2_dev else None))


def qs_adjoint_grad(h: int, gates, theta, flags: int = 0, energy_out=None, grad_out=None):
    """Host outputs (default): returns (energy, grad numpy array). With QS_FLAG_OUT_DEVICE,
    ``energy_out`` / ``grad_out`` are device addresses (ints) and nothing is returned."""
    g, gp = _gates_arg(gates)
    t, tp, nt = _theta_arg(theta)
    if flags & QS_FLAG_OUT_DEVICE:
        _check(lib().qs_adjoint_grad(_c_state_p(h), gp, g.size, tp, nt, _dptr(energy_out), _dptr(grad_out), flags))
        return None
    e = np.empty(1)
    gr = np.empty(max(nt, 1))
    _check(lib().qs_adjoint_grad(_c_state_p(h), gp, g.size, tp, nt, e.ctypes.data_as(_dp),
                                 gr.ctypes.data_as(_dp), flags))
    return float(e[0]), gr[:nt]


def qs_batch_create(n_qubits, gates, gate_offsets, param_offsets, dtype: int, small_bits: int = 0, tile_bits: int = 0,
                    max_pass_gates: int = 0, stream: int = 0) -> int:
    """Plan a batch (see qs.h). ``gates`` is one concatenated gate array; offsets have
    len(n_qubits) + 1 entries."""
    from .gates import as_gate_array

    nq = np.ascontiguousarray(n_qubits, dtype=np.int32)
    g = as_gate_array(gates)
    go = np.ascontiguousarray(gate_offsets, dtype=np.uint64)
    po = np.ascontiguousarray(param_offsets, dtype=np.uint64)
    if go.size != nq.size + 1 or po.size != nq.size + 1:
        raise ValueError("offset arrays need len(n_qubits) + 1 entries")
    h = _vp()
    _check(lib().qs_batch_create(int(nq.size), _vp(nq.ctypes.data), _vp(g.ctypes.data) if g.size else None,
                                 _vp(go.ctypes.data), _vp(po.ctypes.data), dtype, small_bits, tile_bits,
                                 max_pass_gates, _vp(stream or None), ctypes.byref(h)))
    return h.value


def qs_batch_bytes(b: int) -> float:
    """Algorithmic bytes of one run of the batch (host only)."""
    out = ctypes.c_double(0.0)
    _check(lib().qs_batch_bytes(_vp(b), ctypes.byref(out)))
    return out.value


def qs_batch_run(b: int, theta_dev: int, energy_dev: int, grad_dev: int, flags: int = QS_FLAG_GRAPH) -> None:
    _check(lib().qs_batch_run(_vp(b), _dptr(theta_dev), _dptr(energy_dev), _dptr(grad_dev), flags))


def qs_batch_info(b: int) -> dict:
    grid, sb, tb, mg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    smem, ws = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().qs_batch_info(_vp(b), ctypes.byref(grid), ctypes.byref(sb), ctypes.byref(tb), ctypes.byref(mg),
                               ctypes.byref(smem), ctypes.byref(ws)))
    return {"grid": grid.value, "small_bits": sb.value, "tile_bits": tb.value, "max_pass_gates": mg.value,
            "smem_bytes": smem.value, "workspace_bytes": ws.value}


def qs_batch_free(b: int) -> None:
    _check(lib().qs_batch_free(_vp(b)))


def qs_set_tile_bits(dtype: int, adjoint: int, bits: int) -> None:
    _check(lib().qs_set_tile_bits(dtype, adjoint, bits))


def qs_get_tile_bits(dtype: int, adjoint: int) -> int:
    return int(lib().qs_get_tile_bits(dtype, adjoint))


def qs_set_l2_fetch_bytes(nbytes: int) -> None:
    _check(lib().qs_set_l2_fetch_bytes(nbytes))


def qs_get_l2_fetch_bytes() -> int:
    return int(lib().qs_get_l2_fetch_bytes())
