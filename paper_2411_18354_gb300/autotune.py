"""Autotuner for the fused tile passes and the batched kernel.

It runs the real workload with each candidate setting, keeps the fastest, applies it, and
caches the choice as JSON keyed by device and workload signature, so that later processes
reuse it without measuring again. Settings:
- fused passes (``qs_apply_circuit`` / ``qs_adjoint_grad`` with QS_FLAG_FUSE): local qubits
  per shared-memory tile, per precision and direction (``qs_set_tile_bits``);
- batch (``qs_batch_create``): ``small_bits`` (states that stay in shared memory),
  ``tile_bits`` (tile passes of larger states) and ``max_pass_gates`` (fusion depth).
Cache file: ``$QS_AUTOTUNE_CACHE`` or ``~/.cache/qs_gb300_autotune.json``.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import _lib

FUSED_CANDIDATES = (10, 11, 12, 13)
BATCH_CANDIDATES = (
    {"small_bits": 12, "tile_bits": 12, "max_pass_gates": 64},
    {"small_bits": 12, "tile_bits": 11, "max_pass_gates": 64},
    {"small_bits": 11, "tile_bits": 11, "max_pass_gates": 64},
    {"small_bits": 13, "tile_bits": 13, "max_pass_gates": 64},
    {"small_bits": 12, "tile_bits": 12, "max_pass_gates": 32},
)


def cache_path() -> str:
    return os.environ.get("QS_AUTOTUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                                "qs_gb300_autotune.json")


def _device_key() -> str:
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.major}{p.minor}|{p.multi_processor_count}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d: dict) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only loses the cache


def _sig(*parts) -> str:
    h = hashlib.sha1()
    for p in parts:
        h.update(p.tobytes() if isinstance(p, np.ndarray) else repr(p).encode())
    return h.hexdigest()[:16]


def _time(fn, reps: int) -> float:
    import torch

    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best


def _dt(dtype) -> int:
    return _lib.QS_C64 if dtype in ("c64", "complex64", _lib.QS_C64) else _lib.QS_C128


def _set_bits(dt: int, adjoint: int, bits: int) -> None:
    """qs_set_tile_bits, falling back to the library default for a value it rejects (one that
    came from the QS_TILE_BITS override, which allows smaller tiles)."""
    try:
        _lib.qs_set_tile_bits(dt, adjoint, bits)
    except _lib.QsError:
        _lib.qs_set_tile_bits(dt, adjoint, 0)


def restore_defaults() -> None:
    """Back to the library's default tile sizes for both precisions and directions (undoes
    every tile size the tuner applied in this process)."""
    for dt in (_lib.QS_C64, _lib.QS_C128):
        for adj in (0, 1):
            _lib.qs_set_tile_bits(dt, adj, 0)


def tune_fused(n: int, dtype: str, gates, theta=None, adjoint: bool = False, candidates=FUSED_CANDIDATES,
               reps: int = 2, use_cache: bool = True, flags: int = 0, apply: bool = True) -> dict:
    """Pick the tile size of the fused passes for this circuit by timing each candidate with
    QS_FLAG_FUSE (| flags, e.g. QS_FLAG_JIT). With apply=True the choice is applied
    process-wide (qs_set_tile_bits); with apply=False the setting in force before the call is
    put back. Candidates the library rejects for the precision and direction are skipped."""
    from . import QS_FLAG_FUSE, State, as_gate_array

    g = as_gate_array(gates)
    dt = _dt(dtype)
    fl = QS_FLAG_FUSE | flags
    key = f"{_device_key()}|fused|{dtype}|{int(adjoint)}|f{fl}|n{n}|{_sig(g['target'], g['ctrl_mask'], g['kind'])}"
    prev = _lib.qs_get_tile_bits(dt, int(adjoint))
    cache = _load() if use_cache else {}
    if key in cache:
        if apply:
            _lib.qs_set_tile_bits(dt, int(adjoint), int(cache[key]["tile_bits"]))
        return dict(cache[key], cached=True)
    results = {}
    try:
        with State(n, dtype) as st:
            for k in candidates:
                try:
                    _lib.qs_set_tile_bits(dt, int(adjoint), k)
                except _lib.QsError:  # a tile whose block does not fit this precision / direction
                    continue
                if adjoint:
                    fn = lambda: (st.set_basis(0), st.adjoint_grad(g, theta, fl))  # noqa: E731
                else:
                    fn = lambda: st.apply_circuit(g, theta, fl)  # noqa: E731
                results[k] = _time(fn, reps)
    finally:
        _set_bits(dt, int(adjoint), prev)
    if not results:
        raise RuntimeError("tune_fused: no candidate tile size is valid for this precision and direction")
    best = min(results, key=results.get)
    if apply:
        _lib.qs_set_tile_bits(dt, int(adjoint), best)
    entry = {"tile_bits": best, "seconds": results[best], "tried": {str(k): v for k, v in results.items()}}
    if use_cache:
        cache = _load()
        cache[key] = entry
        _save(cache)
    return dict(entry, cached=False)


class tuned_tile_bits:
    """Context manager: tune (or take from the cache) and apply the tile size of the fused
    passes for this circuit; on exit the tile size in force before is restored.

        with autotune.tuned_tile_bits(n, "c64", gates, theta) as choice:
            state.apply_circuit(gates, theta, QS_FLAG_FUSE)
    """

    def __init__(self, n, dtype, gates, theta=None, adjoint=False, **kw):
        self.args = (n, dtype, gates, theta, adjoint)
        self.kw = kw
        self.dt = _dt(dtype)
        self.adjoint = int(adjoint)

    def __enter__(self):
        self.prev = _lib.qs_get_tile_bits(self.dt, self.adjoint)
        n, dtype, gates, theta, adjoint = self.args
        return tune_fused(n, dtype, gates, theta, adjoint, apply=True, **self.kw)

    def __exit__(self, *exc):
        _set_bits(self.dt, self.adjoint, self.prev)
        return False


def tune_batch(n_qubits, circuits, n_params, thetas, dtype: str = "c64", candidates=BATCH_CANDIDATES,
               reps: int = 2, use_cache: bool = True) -> dict:
    """Pick (small_bits, tile_bits, max_pass_gates) for a batch by running it."""
    import torch

    from . import QS_FLAG_GRAPH, Batch

    ns = np.asarray(n_qubits, dtype=np.int32)
    key = (f"{_device_key()}|batch|{dtype}|{_sig(np.bincount(ns))}|"
           f"{_sig(np.array([len(c) for c in circuits]), np.asarray(n_params))}")
    cache = _load() if use_cache else {}
    if key in cache:
        return dict(cache[key], cached=True)
    th = torch.tensor(np.concatenate(thetas), dtype=torch.float64, device="cuda")
    en = torch.empty(len(ns), dtype=torch.float64, device="cuda")
    gr = torch.empty(max(1, int(np.sum(n_params))), dtype=torch.float64, device="cuda")
    tried = []
    for cand in candidates:
        try:
            b = Batch(ns, circuits, n_params, dtype, **cand)
        except _lib.QsError:
            continue  # e.g. shared memory too large for this setting
        try:
            t = _time(lambda: b.run(th, en, gr, QS_FLAG_GRAPH), reps)
        finally:
            b.close()
        tried.append((t, cand))
    if not tried:
        raise RuntimeError("no batch setting could be created")
    t, best = min(tried, key=lambda x: x[0])
    entry = dict(best, seconds=t, tried=[dict(c, seconds=s) for s, c in tried])
    if use_cache:
        cache = _load()
        cache[key] = entry
        _save(cache)
    return dict(entry, cached=False)
