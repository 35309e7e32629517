"""Gate records in the layout of the C struct ``qs_gate`` (include/qs.h)."""
from __future__ import annotations

import numpy as np

GATE_DTYPE = np.dtype(
    [
        ("target", "<i4"),
        ("kind", "<i4"),
        ("ctrl_mask", "<u8"),
        ("ctrl_vals", "<u8"),
        ("param", "<i4"),
        ("reserved", "<i4"),
        ("U", "<f8", (8,)),
    ],
    align=True,
)
assert GATE_DTYPE.itemsize == 96


def as_gate_array(gates) -> np.ndarray:
    """Contiguous array of ``GATE_DTYPE`` records from any structured array with the same
    field names (or a list of such records)."""
    if isinstance(gates, np.ndarray) and gates.dtype == GATE_DTYPE and gates.flags.c_contiguous:
        return gates
    src = np.asarray(gates)
    if src.dtype.names is None:
        raise TypeError("gates must be a structured array with the qs_gate fields")
    out = np.zeros(src.shape[0] if src.ndim else 1, dtype=GATE_DTYPE)
    for name in GATE_DTYPE.names:
        out[name] = src[name]
    return out
