"""Runs under the library's debug build (QS_LIB_VARIANT=debug, libqs_debug.so): the gate,
sweep, tile-pass, diagonal-run and compiled pass kernels check every global access against the
state under test and count writes per amplitude (csrc/qs_debug.cuh). Started as a child process
by tests/test_gpu_debug_checks.py (a process loads one variant of the library); exits non-zero
on the first failed check and prints a one-line summary otherwise."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from gpu_helpers import ATOL_CIRCUIT, c128_of, random_state  # noqa: E402


def main():
    import torch

    assert os.environ.get("QS_LIB_VARIANT") == "debug"
    import paper_2411_18354_gb300 as qs

    qs.build(debug=True)
    assert qs.qs_debug_build(), "the debug build was not loaded"
    counts = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    stats = {"gates": 0, "fused_runs": 0, "gradients": 0}

    def arm(n, count=True):
        counts.zero_()
        qs.qs_debug_configure(1 << n, counts.data_ptr() if count else 0, (1 << n) if count else 0)

    def status_ok(what):
        st, bad = qs.qs_debug_status()
        assert st == 0, f"{what}: access outside the state (status {st}, index {bad})"

    # 1. single gates, n = 1..16: every write inside the state, each amplitude written at most
    #    once, and exactly the amplitudes the gate changes written (the reduced iteration set)
    rng = np.random.default_rng(16)
    for dtype in ("c64", "c128"):
        for n in range(1, 17):
            with qs.State(n, dtype) as st:
                st.from_numpy(random_state(n, dtype, n))
                for _ in range(12):
                    t = int(rng.integers(0, n))
                    others = [q for q in range(n) if q != t]
                    c = int(rng.integers(0, min(4, n - 1) + 1))
                    ctrls = [int(q) for q in rng.choice(others, size=c, replace=False)] if c else []
                    mask = sum(1 << q for q in ctrls)
                    vals = int(rng.integers(0, 1 << 16)) & mask
                    kind = int(rng.integers(0, 5))
                    arm(n)
                    if kind == 0:
                        st.apply_x(t, mask, vals)
                        expect = 1 << (n - c)
                    else:
                        U = [W.haar_2x2(rng), np.diag(np.exp(1j * rng.uniform(0, 6, 2))),
                             np.diag([1.0, np.exp(0.7j)]), np.array([[0.6, -0.8], [0.8, 0.6]])][kind - 1]
                        st.apply_gate(t, U, mask, vals)
                        expect = (1 << (n - c)) // (2 if kind == 3 else 1)  # one-sided: one side
                    torch.cuda.synchronize()
                    cs = counts[: 1 << n]
                    status_ok(f"gate n={n} t={t} c={c} kind={kind}")
                    assert int(cs.max()) <= 1, f"an amplitude written twice (n={n}, t={t}, mask={mask:#x})"
                    assert int(cs.sum()) == expect, (n, t, c, kind, int(cs.sum()), expect)
                    stats["gates"] += 1
    # 2. fused programs (interpreted and compiled passes, diagonal runs), several tile sizes:
    #    bounds, and the oracle's result
    for tile_bits in ("5", "9", "12"):
        os.environ["QS_TILE_BITS"] = tile_bits
        for dtype in ("c64", "c128"):
            for n in (3, 9, 14):
                gl = []
                for _ in range(80):
                    t = int(rng.integers(0, n))
                    others = [q for q in range(n) if q != t]
                    c = int(rng.integers(0, min(3, n - 1) + 1))
                    ctrls = sorted(int(q) for q in rng.choice(others, size=c, replace=False)) if c else []
                    vals = [int(b) for b in rng.integers(0, 2, size=c)]
                    r = rng.random()
                    if r < 0.2:
                        gl.append(W.make_gate(t, None, ctrls, vals, kind=W.KIND_X))
                    elif r < 0.5:
                        gl.append(W.make_gate(t, np.diag(np.exp(1j * rng.uniform(0, 6, 2))), ctrls, vals))
                    else:
                        gl.append(W.make_gate(t, W.haar_2x2(rng), ctrls, vals))
                gates = W.gate_list(gl)
                psi0 = random_state(n, dtype, 100 + n)
                ref = c128_of(psi0).copy()
                oracle.run_circuit(ref, n, gates)
                for flags in (qs.QS_FLAG_FUSE, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT):
                    with qs.State(n, dtype) as st:
                        st.from_numpy(psi0)
                        arm(n, count=False)
                        st.apply_circuit(gates, flags=flags)
                        got = c128_of(st.to_numpy())
                    status_ok(f"fused n={n} flags={flags} tile={tile_bits}")
                    assert np.max(np.abs(got - ref)) <= 4 * ATOL_CIRCUIT[dtype], (n, flags, tile_bits)
                    stats["fused_runs"] += 1
    del os.environ["QS_TILE_BITS"]
    # 3. one tile pass over a whole 10-qubit state (tiles of 2^12): each amplitude written once
    n = 10
    gates = W.random_circuit(n, 40, 2, seed=5)
    for flags in (qs.QS_FLAG_FUSE, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT):
        sched = qs.circuit_schedule(n, gates, flags=flags)
        if sched["launches"] != 1 or sched["tile_passes"] != 1:
            continue  # planned otherwise: nothing to count per launch
        with qs.State(n, "c64") as st:
            st.from_numpy(random_state(n, "c64", 3))
            arm(n)
            st.apply_circuit(gates, flags=flags)
            torch.cuda.synchronize()
        status_ok(f"one pass flags={flags}")
        assert int(counts[: 1 << n].min()) == 1 and int(counts[: 1 << n].max()) == 1, flags
    # 4. gradients (unfused sweep steps, interpreted and compiled sweep passes): bounds
    n = 9
    hea = W.hea_circuit(n, 3)
    th = W.hea_params(n, 3, seed=9)
    ps = oracle.param_shift_grad(n, hea, th)
    for dtype in ("c64", "c128"):
        for flags in (0, qs.QS_FLAG_FUSE, qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT):
            with qs.State(n, dtype) as st:
                arm(n, count=False)
                e, g = st.adjoint_grad(hea, th, flags)
            status_ok(f"gradient {dtype} flags={flags}")
            assert np.max(np.abs(g - ps)) <= 1e-4
            stats["gradients"] += 1
    # 5. the checks catch what they are meant to: a state declared half its size makes the
    #    accesses to its upper half fail the check (they are skipped, no memory outside the real
    #    buffer is touched), and applying a gate twice shows counts of 2
    n = 12
    with qs.State(n, "c64") as st:
        counts.zero_()
        qs.qs_debug_configure(1 << (n - 1), 0, 0)
        st.apply_gate(n - 1, W.H_MATRIX)
        stq, bad = qs.qs_debug_status()
        assert stq & 1 and bad >= (1 << (n - 1)), (stq, bad)
        arm(n)
        st.apply_gate(3, W.H_MATRIX)
        st.apply_gate(3, W.H_MATRIX)
        torch.cuda.synchronize()
        assert int(counts[: 1 << n].max()) == 2
    qs.qs_debug_configure(0, 0, 0)
    print(json.dumps({"debug_checks": "ok", **stats}))


if __name__ == "__main__":
    main()
