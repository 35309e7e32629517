"""Shared helpers of the GPU parity tests (input preparation and comparisons only)."""
from __future__ import annotations

import numpy as np

import oracle
import workloads as W

# Per-gate error bounds used by the parity tests, derived from the arithmetic of one
# update x' = a x + b y (four real products, three additions per component, the matrix
# rounded to the state precision once): |x'_gpu - x'_exact| <= k * u * (|a||x| + |b||y|)
# with u = 2^-24 (float32) or 2^-53 (float64) and k ~ 8. With |a|, |b| <= 1 (unitary)
# that is below RTOL * (|x| + |y|).
RTOL_GATE = {"c64": 1e-6, "c128": 1e-14}
# Whole-circuit targets: complex128 max-abs amplitude error <= 1e-12; complex64 <= 3e-5.
ATOL_CIRCUIT = {"c64": 3e-5, "c128": 1e-12}
NP = {"c64": np.complex64, "c128": np.complex128}


def rotations(n: int, seed: int):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.2, np.pi - 0.2, size=n), rng.uniform(-np.pi, np.pi, size=n)


def product_amp(k: np.ndarray, alphas, betas) -> np.ndarray:
    """Amplitudes of prod_q RZ(beta_q) RY(alpha_q)|0>: factor cos(alpha/2) e^{-i beta/2} when
    bit q of k is 0, sin(alpha/2) e^{+i beta/2} when it is 1 (closed form, any n)."""
    k = np.asarray(k, dtype=np.uint64)
    out = np.ones(k.shape, dtype=np.complex128)
    for q, (a, b) in enumerate(zip(alphas, betas)):
        bit = ((k >> np.uint64(q)) & np.uint64(1)).astype(bool)
        f0 = np.cos(a / 2) * np.exp(-0.5j * b)
        f1 = np.sin(a / 2) * np.exp(0.5j * b)
        out *= np.where(bit, f1, f0)
    return out


def prepare_product(st, alphas, betas):
    """|0> then RY(alpha_q), RZ(beta_q) on every qubit, through the library's gate calls."""
    st.set_basis(0)
    for q, (a, b) in enumerate(zip(alphas, betas)):
        st.apply_gate(q, oracle.ry(a))
        st.apply_gate(q, oracle.rz(b))


def sample_indices(n: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    N = 1 << n
    ks = rng.integers(0, N, size=count, dtype=np.uint64)
    edge = np.array([0, 1, N - 1, N - 2, N >> 1, (N >> 1) - 1], dtype=np.uint64)
    return np.unique(np.concatenate([ks, edge[edge < N]]))


def oracle_outputs(ks, t, mask, vals, U, inp_k, inp_p):
    """Expected outputs of one gate at indices ks from the inputs at ks and ks ^ 2^t."""
    out = np.empty(len(ks), dtype=np.complex128)
    for i, k in enumerate(ks):
        out[i] = oracle.gate_output(int(k), t, mask, vals, U, complex(inp_k[i]), complex(inp_p[i]))
    return out


def c128_of(a: np.ndarray) -> np.ndarray:
    return np.asarray(a).astype(np.complex128)


def random_state(n: int, dtype: str, seed: int) -> np.ndarray:
    return W.random_state(n, seed, dtype=NP[dtype])
