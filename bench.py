#!/usr/bin/env python
"""Benchmark of the controlled-gate path on GB300.

Workload (the single-gate sweep at scale): an n = 30 complex64 state (8.6 GB, larger than
L2) receives, per step, one Haar-random gate for every control count c = 0..8 and target
t in {0, 15, 29} (27 gates), control sets rotating through 8 seeded sets per (c, t). The
metric is algorithmic gate-apply bandwidth: 2 * 2^(n-c) amplitudes * 8 bytes per gate
(read + write of the selected pairs), summed over the step, divided by the step's device
time. Also reported: the same sweep end to end with host buffers, per-c bandwidth and
fraction of the measured HBM peak, the complex128 sweep against the FP64 ALU bound, and
the adjoint gradient (n = 24 hardware-efficient ansatz, 960 parameters) in complex64 vs
the plain complex128 path.

``--impl reference`` times the CPU oracle (plain loop over all 2^n indices with control
checks) on the host cores instead, on a bounded sample of the same sweep.

Multi-GPU: the path does not shard (every box has one GPU); under torchrun each rank runs
an independent replica and rank 0 reports the aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gate-apply GB/s & % HBM roofline at n=30, c=0..8; adjoint grads/s vs plain"
CMAX = 8
SETS = 8


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--quick", action="store_true", help="headline sweep only (for profiler runs)")
    ap.add_argument("--only", default="",
                    help="comma list: run only these extra measurements after the headline sweep "
                         "(e2e,c128,q30,adjoint,fused,reduce,masked,batch,paper,precision,cpu)")
    ap.add_argument("--ncu-case", type=int, default=None, metavar="C",
                    help="small profiling case: the 3 sweep gates with C controls (set 0) at --n, run twice "
                         "(profile with -s 3 -c 3 to skip the first round)")
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"], help="state precision of --ncu-case")
    ap.add_argument("--ncu-fused", action="store_true",
                    help="small profiling case: 2 layers of the ansatz at n=24, fused forward then fused gradient")
    ap.add_argument("--ncu-reduce", action="store_true",
                    help="small profiling case: <Z_i> + norm of an n=27 state, twice")
    ap.add_argument("--tile-costs", action="store_true",
                    help="per-gate cost of fused tile passes by gate kind (n = 24, 2^12-amplitude tiles)")
    ap.add_argument("--layers", type=int, default=2, help="ansatz layers of the --ncu-fused case")
    ap.add_argument("--ncu-scale", action="store_true",
                    help="profiling case: the 1000-gate scale circuit at n = 30 with compiled passes, twice")
    ap.add_argument("--gate-patterns", action="store_true",
                    help="cold-L2 device time of single sweep gates with c = 6..8 controls at n = 30 (general and "
                         "exchange) against the same control count on the top qubits (contiguous runs)")
    ap.add_argument("--ncu-qft", action="store_true",
                    help="profiling case: the fused QFT (29 qubits, or --n), twice (diagonal-run passes)")
    ap.add_argument("--jit", action="store_true",
                    help="profiling cases --ncu-fused / --ncu-qft: tile passes compiled for their shape (QS_FLAG_JIT), "
                         "compiled before the profiled launches")
    ap.add_argument("--ncu-batch", action="store_true",
                    help="small profiling case: one batch launch of 304 states (n=16, 2 layers of the ansatz)")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# FP64 ALU peak: measured on the device by the library's FMA-rate kernel (qs_measure_fma_peak),
# 2 flops per FMA; NVIDIA's published FP64 figure for GB300 (1.25 TFLOP/s) is context only.
FP64_NOMINAL_TFLOPS = 1.25


def measure_fma_peaks(qs):
    """Measured FMA rates (TFLOP/s) in float64 and float32, best of 3 launches."""
    import torch

    stream = int(torch.cuda.current_stream().cuda_stream)
    out = {}
    for label, dt, iters in (("fp64", qs.QS_C128, 1 << 14), ("fp32", qs.QS_C64, 1 << 16)):
        out[label] = round(max(qs.qs_measure_fma_peak(dt, iters, stream) for _ in range(3)) / 1e12, 3)
    out["how"] = "8 independent FMA chains per thread on every SM, CUDA events, best of 3 (2 flops per FMA)"
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash() -> str:
    h = hashlib.sha1()
    for name in ("k_gate.cuh", "k_gate_dispatch.cuh", "qs_plan.cu", "qs_api.cu"):
        with open(os.path.join(ROOT, "paper_2411_18354_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def profiled_traffic(n: int, dtype: str):
    """DRAM bytes per gate launch from the committed ncu summary of this sweep, if it was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"k_gate_sweep_n{n}_{dtype}_traffic.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch_mean:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


def targets_for(n):
    """Targets 0, 15, 29 at n = 30 (lowest, middle, highest qubit)."""
    return (0, n // 2, n - 1)


def sweep_schedule(n, seed=1):
    import numpy as np

    import workloads as W

    sw = W.sweep_gates(n, CMAX, targets_for(n), sets=SETS, seed=seed)
    sched = []  # per set index: list of (c, t, mask, vals, U8)
    for s in range(SETS):
        row = []
        for t in targets_for(n):
            for c in range(CMAX + 1):
                g = sw[(c, t)][s]
                row.append((c, t, int(g["ctrl_mask"]), int(g["ctrl_vals"]), np.ascontiguousarray(g["U"])))
        sched.append(row)
    return sched


def alg_bytes(n, c, esize):
    return 2 * (1 << (n - c)) * esize


SECTOR_BYTES = 32  # L2 sector = DRAM fetch size the library sets (qs_set_l2_fetch_bytes)


def sector_bytes(n, mask, esize):
    """Bytes of the 32-byte sectors that hold a selected amplitude (read + write): controls
    on the qubits inside one sector (0-1 for complex64, 0 for complex128) do not reduce it."""
    unit_bits = (SECTOR_BYTES // esize).bit_length() - 1
    c_hi = bin(mask >> unit_bits).count("1")
    return 2 * (1 << (n - c_hi)) * esize


def run_sweep(qs, st, n, esize, sched, steps, warmup, per_launch=True):
    """Device-timed sweep steps through qs_apply_gate. Returns per-launch ms and step ms."""
    import torch

    stream = torch.cuda.current_stream()
    apply = qs._lib.qs_apply_gate
    for w in range(warmup):
        for (c, t, m, v, U) in sched[w % SETS]:
            apply(st.h, t, m, v, U)
    torch.cuda.synchronize()
    launches = []  # (c, t, start_event, end_event)
    step_ev = []
    for k in range(steps):
        row = sched[(warmup + k) % SETS]
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for (c, t, m, v, U) in row:
            if per_launch:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                apply(st.h, t, m, v, U)
                e1.record(stream)
                launches.append((c, t, m, e0, e1))
            else:
                apply(st.h, t, m, v, U)
        s1.record(stream)
        step_ev.append((s0, s1))
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    per = [(c, t, a.elapsed_time(b), m) for c, t, m, a, b in launches]
    return step_ms, per


def measure_per_c(qs, st, n, esize, sched, peak, reps=2):
    """Steady-state time per gate for each control count: the 24 sweep gates with c controls
    (8 control sets x 3 targets) back to back, timed as a block after one untimed pass. Each
    gate then pays for its own DRAM traffic (and the write-backs its same-size predecessor
    left in L2), and no gate's footprint comes back within the L2's reach."""
    import torch

    apply = qs._lib.qs_apply_gate
    out = {}
    for c in range(CMAX + 1):
        rows = [r for s in range(SETS) for r in sched[s] if r[0] == c]
        for (_, t, m, v, U) in rows:
            apply(st.h, t, m, v, U)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            for (_, t, m, v, U) in rows:
                apply(st.h, t, m, v, U)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / (reps * len(rows))
        alg = alg_bytes(n, c, esize)
        sect = statistics.mean(sector_bytes(n, m, esize) for (_, _, m, _, _) in rows)
        out[str(c)] = {"ms_per_gate": round(ms, 5), "GBps": round(alg / (ms * 1e-3) / 1e9, 1),
                       "frac": round(alg / (ms * 1e-3) / 1e9 / peak, 3),
                       "frac_sector_adjusted": round(sect / (ms * 1e-3) / 1e9 / peak, 3)}
    return out


def _events_ms(fn, reps):
    """Average device time of fn() over reps runs (CUDA events on the current stream)."""
    import torch

    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure_adjoint(qs, W, peak, reps=3):
    """Differentiation workload: n = 24, 20 layers, 960 parameters. grads/s = parameters /
    time of one full gradient (forward + energy + reverse sweep, host outputs)."""
    import numpy as np
    import torch

    from paper_2411_18354_gb300 import autotune

    n, layers = 24, 20
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    out = {"tile_bits_c64": {}}
    grads = {}
    F, J = qs.QS_FLAG_FUSE, qs.QS_FLAG_JIT
    for label, dtype, flags in (("c64_fused_compiled", "c64", F | J), ("c64_fused", "c64", F), ("c64_unfused", "c64", 0),
                                ("c128_plain", "c128", 0), ("c128_fused", "c128", F)):
        _reset_tile_bits(qs)
        if dtype == "c64" and flags & F:  # tile sizes tuned for this kind of pass (compiled or interpreted)
            tb = [autotune.tune_fused(n, "c64", gates, th, adjoint=adj, use_cache=False, reps=1, flags=flags & J,
                                      candidates=(11, 12, 13))["tile_bits"] for adj in (False, True)]
            out["tile_bits_c64"][label] = {"forward": tb[0], "adjoint": tb[1]}
            if flags & J:
                out["compile_s_c64_compiled"] = _compile(qs, n, gates, th, "c64", adjoint=True)
        st = qs.State(n, dtype)
        try:
            st.adjoint_grad(gates, th, flags)  # warm-up (allocates lambda and scratch)
            ts = []
            for k in range(reps):  # new angles every call, as in a training loop (the last: th)
                st.set_basis(0)
                tk = th + 0.01 * (reps - 1 - k)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                e, g = st.adjoint_grad(gates, tk, flags)
                ts.append(time.perf_counter() - t0)
            grads[label] = g
            out[label] = {"s_per_gradient": round(min(ts), 5), "grads_per_s": round(th.size / min(ts), 1),
                          "energy": e,
                          **program_roofline(qs, n, gates, th, flags | qs.QS_FLAG_ADJOINT, dtype, min(ts) * 1e3, peak)}
        finally:
            st.close()
    for label in ("c64_fused_compiled", "c64_fused", "c64_unfused", "c128_fused"):
        out[f"max_abs_grad_err_{label}_vs_c128"] = float(np.max(np.abs(grads[label] - grads["c128_plain"])))
    out["speedup_c64_fused_vs_c128_plain"] = round(out["c128_plain"]["s_per_gradient"] /
                                                   out["c64_fused_compiled"]["s_per_gradient"], 2)
    out["timing"] = ("wall time of one synchronous qs_adjoint_grad call (host outputs), best of 3 calls with "
                     "different angles (the plan of the circuit kept from the warm-up call, matrices refreshed)")
    _reset_tile_bits(qs)
    out["workload"] = "HEA n=24, 20 layers (RY,RZ per qubit + CNOT ladder), 960 params, observable sum Z_i"
    return out


# Measured FMA rates (TFLOP/s, 2 flops per FMA) of this device, filled in by main before the
# measurements that quote an arithmetic roofline.
FMA_PEAKS = {}


def program_roofline(qs, n, gates, theta, flags, dtype, ms, peak):
    """Both rooflines of the launches qs_apply_circuit (or, with QS_FLAG_ADJOINT,
    qs_adjoint_grad) makes for these flags. Memory: algorithmic bytes (per single gate its
    selected amplitudes, per tile pass the tiles its gates select, per diagonal run the chunks
    it can change; read + write) / time, against the HBM peak. Arithmetic: the circuit's
    algorithmic flops (qs_schedule.algorithmic_flops) / time, against the measured FMA rate of
    the state's precision (which counts an FMA as 2 flops: a multiplication or addition alone
    costs an issue slot for 1, so 1.0 is out of reach for updates with plain multiplies)."""
    sch = qs.circuit_schedule(n, gates, theta, flags=flags & ~qs.QS_FLAG_GRAPH, dtype=dtype)
    gbs = sch["algorithmic_bytes"] / (ms * 1e-3) / 1e9
    out = {"algorithmic_GB": round(sch["algorithmic_bytes"] / 1e9, 3), "achieved_GBps": round(gbs, 1),
           "frac_hbm": round(gbs / peak, 3), "launches": sch["launches"], "tile_passes": sch["tile_passes"]}
    fp = FMA_PEAKS.get("fp32" if dtype == "c64" else "fp64")
    if fp:
        tf = sch["algorithmic_flops"] / (ms * 1e-3) / 1e12
        out.update({"algorithmic_GFLOP": round(sch["algorithmic_flops"] / 1e9, 2), "achieved_TFLOPs": round(tf, 2),
                    "frac_fma_peak": round(tf / fp, 3)})
    return out


def _compile(qs, n, gates, theta, dtype, adjoint=False):
    """Compile the shape-specialised pass kernels ahead of the timed runs; returns seconds."""
    dt = qs.QS_C64 if dtype == "c64" else qs.QS_C128
    return round(qs.qs_circuit_compile(n, dt, gates, theta, adjoint=adjoint)["compile_seconds"], 3)


def _reset_tile_bits(qs):
    """Back to the library's default tile sizes, so that no measurement inherits the tile size
    another one tuned (the autotuner applies its choice process-wide)."""
    from paper_2411_18354_gb300 import autotune

    autotune.restore_defaults()


def measure_fused(qs, W, peak):
    """Fused programs: the 1000-gate scale circuit at n = 30 (complex64) and the ansatz at
    n = 24: one launch per gate, fused with interpreted tile passes, and fused with passes
    compiled for their shape (QS_FLAG_JIT, compiled before timing); gates/s and the
    algorithmic-byte roofline of each schedule. Tile size: library default (2^12 amplitudes)."""
    import torch

    out = {}
    F, G, J = qs.QS_FLAG_FUSE, qs.QS_FLAG_GRAPH, qs.QS_FLAG_JIT
    for name, n, gates, th, reps in (("scale_circuit_n30_c64", 30, W.scale_circuit(30, 1000, seed=1), None, 1),
                                     ("ansatz_n24_c64", 24, W.hea_circuit(24, 20), W.hea_params(24, 20, seed=3), 3)):
        st = qs.State(n, "c64")
        r = {"gates": int(len(gates))}
        try:
            r["compile_s"] = _compile(qs, n, gates, th, "c64")
            for label, flags in (("unfused", G), ("fused_interpreted", F | G), ("fused_compiled", F | G | J)):
                ms = _events_ms(lambda: st.apply_circuit(gates, th, flags), reps)
                r[label] = {"ms": round(ms, 3), "gates_per_s": round(len(gates) / (ms * 1e-3), 1),
                            **program_roofline(qs, n, gates, th, flags, "c64", ms, peak)}
        finally:
            st.close()
            torch.cuda.empty_cache()
        r["speedup_compiled_vs_unfused"] = round(r["unfused"]["ms"] / r["fused_compiled"]["ms"], 2)
        out[name] = r
    return out


def measure_reduce(qs, W, peak):
    """One-pass <Z_i> + norm at n = 30: read bytes / time."""
    import torch

    out = {}
    for dtype, es in (("c64", 8), ("c128", 16)):
        st = qs.State(30, dtype)
        try:
            st.apply_gate(0, W.H_MATRIX)
            dz = torch.empty(30, dtype=torch.float64, device="cuda")
            dn = torch.empty(1, dtype=torch.float64, device="cuda")
            ms = _events_ms(lambda: qs.qs_expect_z(st.h, qs.QS_FLAG_OUT_DEVICE, dz.data_ptr(), dn.data_ptr()), 5)
        finally:
            st.close()
            torch.cuda.empty_cache()
        gbs = (1 << 30) * es / (ms * 1e-3) / 1e9
        out[dtype] = {"ms": round(ms, 4), "GBps": round(gbs, 1), "frac_hbm": round(gbs / peak, 3)}
    return out


def measure_masked(qs, n, sched):
    """The baseline schedule (all 2^(n-1) pairs, controls tested per pair) against the
    reduced schedule, per control count: time ratio masked / reduced."""
    import torch

    st = qs.State(n, "c64")
    out = {}
    try:
        for (c, t, m, v, U) in sched[0]:
            tr = _events_ms(lambda: qs._lib.qs_apply_gate(st.h, t, m, v, U), 2)
            tm = _events_ms(lambda: qs._lib.qs_apply_gate_masked(st.h, t, m, v, U), 2)
            out.setdefault(str(c), []).append(tm / tr)
    finally:
        st.close()
        torch.cuda.empty_cache()
    return {c: round(sum(v) / len(v), 2) for c, v in out.items()}


# Section IV, Tables 2 and 4: whole-circuit times of the 29-qubit QFT and streaming circuits
# (fp32 complex, one OpenCL compute unit) on the paper's GTX Titan Black (GK110B) and Stratix V
# FPGA, baseline (masked) and optimised (reduced iteration set) kernels. Context only.
PAPER_TIMES_S = {
    "qft29": {"gk110b_masked": 9.58, "gk110b_reduced": 9.22, "fpga_masked": 413.83, "fpga_reduced": 251.00},
    "stream29": {"gk110b_masked": 1.73, "gk110b_reduced": 0.95, "fpga_masked": 26.07, "fpga_reduced": 3.78},
}


def measure_paper_circuits(qs, W, peak, reps=3):
    """The paper's 29-qubit QFT (435 gates) and streaming circuit (29 X gates with 0..28
    controls) in complex64, each as one graph launch of the whole circuit through
    qs_apply_circuit: baseline schedule (QS_FLAG_MASKED), reduced iteration set, and fused
    tile passes. Device time per circuit (CUDA events, state 4.3 GB > L2)."""
    import torch

    n = 29
    out = {}
    st = qs.State(n, "c64")
    try:
        for name, gates in (("qft29", W.qft_circuit(n)), ("stream29", W.streaming_circuit(n))):
            r = {"gates": int(len(gates)),
                 "algorithmic_GB": round(sum(2.0 * (1 << (n - bin(int(g["ctrl_mask"])).count("1"))) * 8
                                             for g in gates) / 1e9, 3)}
            r["compile_s"] = _compile(qs, n, gates, None, "c64")
            for label, flags in (("masked", qs.QS_FLAG_MASKED), ("reduced", 0), ("fused", qs.QS_FLAG_FUSE),
                                 ("fused_compiled", qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)):
                st.set_basis(0)
                ms = _events_ms(lambda: st.apply_circuit(gates, flags=flags | qs.QS_FLAG_GRAPH), reps)
                r[f"{label}_ms"] = round(ms, 3)
                if label != "masked":  # the comparator reads the pairs it skips too: no algorithmic roofline
                    rf = program_roofline(qs, n, gates, None, flags, "c64", ms, peak)
                    r[f"{label}_roofline"] = {k: rf[k] for k in ("algorithmic_GB", "achieved_GBps", "frac_hbm",
                                                                 "launches", "achieved_TFLOPs", "frac_fma_peak")
                                              if k in rf}
            r["masked_over_reduced"] = round(r["masked_ms"] / r["reduced_ms"], 2)
            r["paper_s"] = PAPER_TIMES_S[name]
            out[name] = r
    finally:
        st.close()
        torch.cuda.empty_cache()
    out["note"] = ("paper_s: Tables 2 and 4 (GTX Titan Black / Stratix V, one OpenCL compute unit), context only; "
                   "algorithmic_GB counts 2*2^(n-c)*8 bytes per gate; *_roofline: algorithmic bytes of that "
                   "schedule's launches / its time; tile size: library default")
    return out


def measure_precision(qs, W):
    """The precision circuit at full size: n = 32 from H on every qubit, 2000 gates (0-6
    controls, 25 % X / CNOT / Toffoli), complex128 (68.7 GB) and complex64 (34.4 GB, fused) on
    the device; complex64 against complex128: max-abs amplitude error, norm drift, <Z_i>."""
    import numpy as np
    import torch

    n = 32
    gates = W.precision_circuit(n, 2000, seed=2)
    prefix = W.gate_list([W.make_gate(q, W.H_MATRIX) for q in range(n)])
    b128 = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    b64 = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    out = {}
    try:
        s128 = qs.State.wrap(b128, n)
        s64 = qs.State.wrap(b64, n)
        _compile(qs, n, gates, None, "c64")
        for st, label, flags in ((s128, "c128", 0), (s64, "c64_fused", qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)):
            st.set_basis(0)
            st.apply_circuit(prefix, flags=flags & ~qs.QS_FLAG_JIT)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st.apply_circuit(gates, flags=flags)
            torch.cuda.synchronize()
            out[label] = {"s": round(time.perf_counter() - t0, 3)}
        out["c64_fused"]["tile_bits"] = qs.qs_get_tile_bits(qs.QS_C64, 0)  # the library default
        out["c64_fused"]["passes"] = "compiled for their shape (QS_FLAG_JIT), compiled before timing"
        z128, n128 = s128.expect_z()
        z64, n64 = s64.expect_z()
        err = 0.0
        for i in range(0, 1 << n, 1 << 26):
            d = b64[i:i + (1 << 26)].to(torch.complex128) - b128[i:i + (1 << 26)]
            err = max(err, float(d.abs().max()))
        out.update({"max_abs_err_c64_vs_c128": err, "norm_drift_c64": abs(n64 - 1.0), "norm_drift_c128": abs(n128 - 1.0),
                    "max_abs_z_diff": float(np.max(np.abs(np.asarray(z64) - np.asarray(z128)))),
                    "z_c128_first4": [round(float(x), 8) for x in z128[:4]],
                    "workload": "n=32, H on every qubit then 2000 gates (0-6 controls, 25% X/CNOT/Toffoli, seed 2)"})
        s128.close()
        s64.close()
    finally:
        del b128, b64
        torch.cuda.empty_cache()
    return out


def measure_batch(qs, W, peak):
    """Batching workload: 4096 states, n uniform in 10..20, 8 ansatz layers, complex64: one
    graph-launched persistent kernel for energies and gradients; settings from the autotuner."""
    import numpy as np
    import torch

    from paper_2411_18354_gb300 import autotune

    ns, thetas = W.batch_workload(4096, 10, 20, 8, seed=4)
    ns = [int(v) for v in ns]
    circ = {k: W.hea_circuit(k, 8) for k in set(ns)}
    circuits = [circ[k] for k in ns]
    nparams = [16 * k for k in ns]
    cands = ({"small_bits": 12, "tile_bits": 12, "max_pass_gates": 64},
             {"small_bits": 12, "tile_bits": 13, "max_pass_gates": 64},
             {"small_bits": 11, "tile_bits": 12, "max_pass_gates": 64})
    tuned = autotune.tune_batch(ns, circuits, nparams, thetas, "c64", candidates=cands, reps=1, use_cache=False)
    cfg = {k: tuned[k] for k in ("small_bits", "tile_bits", "max_pass_gates")}
    b = qs.Batch(ns, circuits, nparams, "c64", **cfg)
    try:
        th = torch.tensor(np.concatenate(thetas), dtype=torch.float64, device="cuda")
        en = torch.empty(len(ns), dtype=torch.float64, device="cuda")
        gr = torch.empty(b.num_params, dtype=torch.float64, device="cuda")
        ms = _events_ms(lambda: b.run(th, en, gr, qs.QS_FLAG_GRAPH), 2)
        info = b.info()
        bbytes = b.algorithmic_bytes()
    finally:
        b.close()
    out = {"states": len(ns), "ms_per_launch": round(ms, 2), "states_per_s": round(len(ns) / (ms * 1e-3), 1),
           "gradient_entries_per_s": round(sum(nparams) / (ms * 1e-3), 1), "config": cfg,
           "grid": info["grid"], "smem_bytes": info["smem_bytes"],
           "algorithmic_GB": round(bbytes / 1e9, 2), "achieved_GBps": round(bbytes / (ms * 1e-3) / 1e9, 1),
           "frac_hbm": round(bbytes / (ms * 1e-3) / 1e9 / peak, 3),
           "workload": "4096 states, n~U{10..20} (seed 4), HEA 8 layers, energies + adjoint gradients, complex64"}
    # pass-major path: states above small_bits side by side, every pass compiled for its shape and
    # run over all states of one size per launch (first run compiles: untimed)
    best = None
    for jcfg in ({"small_bits": 12, "tile_bits": 12, "max_pass_gates": 64},
                 {"small_bits": 12, "tile_bits": 11, "max_pass_gates": 64}):
        b = qs.Batch(ns, circuits, nparams, "c64", **jcfg)
        try:
            jbytes = b.algorithmic_bytes()
            t0 = time.perf_counter()
            b.run(th, en, gr, qs.QS_FLAG_GRAPH | qs.QS_FLAG_JIT)
            torch.cuda.synchronize()
            first_s = time.perf_counter() - t0
            msj = _events_ms(lambda: b.run(th, en, gr, qs.QS_FLAG_GRAPH | qs.QS_FLAG_JIT), 3)
        finally:
            b.close()
        if best is None or msj < best[0]:
            best = (msj, jcfg, first_s, jbytes)
    msj, jcfg, first_s, jbytes = best
    # the batch's arithmetic: per state that of its circuit's gradient (forward, energy and
    # lambda, sweep), from the planner's schedule of one state of each size
    first = {}
    for i, k in enumerate(ns):
        first.setdefault(k, i)
    flops = sum(ns.count(k) * qs.circuit_schedule(k, circ[k], thetas[first[k]],
                                                   qs.QS_FLAG_FUSE | qs.QS_FLAG_ADJOINT)["algorithmic_flops"]
                for k in first)
    def arith(t_ms):
        if not FMA_PEAKS.get("fp32"):
            return {}
        tf = flops / (t_ms * 1e-3) / 1e12
        return {"algorithmic_GFLOP": round(flops / 1e9, 1), "achieved_TFLOPs": round(tf, 2),
                "frac_fma_peak": round(tf / FMA_PEAKS["fp32"], 3)}

    out.update(arith(ms))
    out["pass_major_compiled"] = {"ms_per_run": round(msj, 2), "states_per_s": round(len(ns) / (msj * 1e-3), 1),
                                  "gradient_entries_per_s": round(sum(nparams) / (msj * 1e-3), 1), "config": jcfg,
                                  "first_run_s_with_compile": round(first_s, 2),
                                  "algorithmic_GB": round(jbytes / 1e9, 2),
                                  "achieved_GBps": round(jbytes / (msj * 1e-3) / 1e9, 1),
                                  "frac_hbm": round(jbytes / (msj * 1e-3) / 1e9 / peak, 3),
                                  "speedup_vs_persistent": round(ms / msj, 2), **arith(msj)}
    return out


def cpu_oracle_sample(n_target: int, sched, max_gates=None):
    """Time the CPU oracle (as it stands) on gates of the sweep; returns throughput in the
    headline unit (algorithmic GB/s at 8 bytes per amplitude) and a description."""
    import numpy as np

    import oracle
    import workloads as W

    oracle.lib()
    n = n_target
    try:
        psi = np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)
    except MemoryError:
        n = 26
        psi = np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)
    row = sched[0] if max_gates is None else sched[0][:max_gates]
    total_bytes = 0
    t0 = time.perf_counter()
    for (c, t, m, v, U) in row:
        oracle.apply_gate(psi, n, t, m, v, U)
        total_bytes += alg_bytes(n, c, 8)
    dt = time.perf_counter() - t0
    return {"value": total_bytes / dt / 1e9, "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{len(row)} sweep gates (c=0..8, t=0/15/29) on an n={n} state, float64 oracle loop over all "
                      f"2^n indices; bytes counted as complex64 algorithmic bytes of the same gates",
            "seconds": dt}


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The maximum of x over all ranks (the timed region of the slowest replica)."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, step_bytes: float, total_ms: float) -> float:
    """Whole-job algorithmic GB/s: every replica moves step_bytes per step; the job takes the
    slowest replica's time."""
    return world * steps * step_bytes / (total_ms * 1e-3) / 1e9


def sweep_config(n, world, gates_per_step):
    """The workload keys of the headline line, shared by both arms."""
    state_gb = (1 << n) * 8 / 1e9
    return {"workload": f"single-gate sweep: n={n} complex64 state, Haar gates with c=0..8 controls on random "
                        f"qubits, targets {'/'.join(str(t) for t in targets_for(n))}, 8 rotating control sets "
                        f"({gates_per_step} gates/step)",
            "n": n, "gates_per_step": gates_per_step, "bytes_counted": "2*2^(n-c)*8 per gate",
            "l2": (f"inputs larger than L2 ({state_gb:.1f} GB state)" if state_gb > 0.13
                   else f"state of {state_gb * 1e3:.1f} MB fits in L2"),
            "parallelism": "replicas" if world > 1 else "1 GPU"}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle on the host cores, same metric/unit/config."""
    if rank != 0:
        return
    sched = sweep_schedule(args.n)
    import numpy as np

    import oracle

    oracle.lib()
    n = args.n
    psi = np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)
    # bounded sample per step: 9 gates (one target, c = 0..8)
    vals = []
    for k in range(args.warmup + args.steps):
        row = sched[k % SETS][9 * (k % 3): 9 * (k % 3) + 9]
        t0 = time.perf_counter()
        byts = 0
        for (c, t, m, v, U) in row:
            oracle.apply_gate(psi, n, t, m, v, U)
            byts += alg_bytes(n, c, 8)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            vals.append((byts, dt))
    tot_b = sum(b for b, _ in vals)
    tot_t = sum(t for _, t in vals)
    value = tot_b / tot_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(vals),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": sweep_config(n, world, len(sched[0])),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"per step 9 of the sweep's gates (one target, c=0..8) on an n={n} float64 "
                                   f"state (uniform superposition), oracle loop over all 2^n indices"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2411_18354_gb300 as qs
    import workloads as W

    qs.build()
    torch.cuda.set_device(local_rank)
    n = args.n
    esize = 8
    sched = sweep_schedule(n)
    st = qs.State(n, "c64")
    # input: uniform superposition (H on every qubit), built by the library
    for q in range(n):
        st.apply_gate(q, W.H_MATRIX)
    torch.cuda.synchronize()
    peak, peak_src = load_peaks()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank)
    clk.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    step_ms, per = run_sweep(qs, st, n, esize, sched, args.steps, args.warmup)
    t_wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    total_ms = max_over_ranks(sum(step_ms), world)
    step_bytes = sum(alg_bytes(n, c, esize) for (c, _, _, _, _) in sched[0])
    value = job_value(world, args.steps, step_bytes, total_ms)

    # per-launch roofline of the gate kernel (algorithmic bytes / CUDA-event launch time)
    launch_bytes = sum(alg_bytes(n, c, esize) for c, _, _, _ in per)
    launch_ms = sum(ms for _, _, ms, _ in per)
    achieved = launch_bytes / (launch_ms * 1e-3) / 1e9
    sect_bytes = sum(sector_bytes(n, m, esize) for _, _, _, m in per)
    per_c = None if args.quick else measure_per_c(qs, st, n, esize, sched, peak)
    traffic = profiled_traffic(n, "c64")

    roof_extra = {}
    if per_c:
        roof_extra = {"per_c_frac": [per_c[str(c)]["frac"] for c in range(CMAX + 1)],
                      "per_c_frac_sector_adjusted": [per_c[str(c)]["frac_sector_adjusted"] for c in range(CMAX + 1)]}
    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 (f32 arithmetic)", "data": "synthetic",
        "config": {**sweep_config(n, world, len(sched[0])),
                   "l2_fetch_bytes": qs.qs_get_l2_fetch_bytes(),
                   "per_c": "steady state: the 24 gates of each c back to back, timed as a block",
                   "sector_adjusted": f"{SECTOR_BYTES}-byte sectors holding a selected amplitude"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_src,
                     "kernel": "k_gate (qs_apply_gate)",
                     "frac_sector_adjusted": round(sect_bytes / (launch_ms * 1e-3) / 1e9 / peak, 4), **roof_extra},
        "per_c": per_c,
        "gpu_launches": len(per),
        "clocks": clocks,
    }

    only = set(x for x in args.only.split(",") if x)
    want = lambda part: not args.quick and (not only or part in only)  # noqa: E731
    if want("e2e"):
        # end to end through the C-ABI with host buffers: every step uploads its input state from
        # page-locked host memory, applies the 27 gates and downloads the result. Three states on
        # three streams rotate, so while one state's gates run, the link carries another's upload
        # and a third's download at once (both directions busy); each step still moves
        # 2 x 8.6 GB.
        st.close()
        torch.cuda.empty_cache()
        nbuf = 3
        streams = [torch.cuda.Stream() for _ in range(nbuf)]
        states = [qs.State(n, "c64", stream=int(sm.cuda_stream)) for sm in streams]
        hosts = [torch.empty(1 << n, dtype=torch.complex64).pin_memory() for _ in range(nbuf)]
        hnps = [h.numpy() for h in hosts]
        for i in range(nbuf):  # inputs: the uniform superposition, written through the library
            for q in range(n):
                states[i].apply_gate(q, W.H_MATRIX)
            qs.qs_state_copy_to_host_async(states[i].h, hnps[i])
            qs.qs_state_synchronize(states[i].h)
        e2e_steps = 18

        phase_ev = []  # per timed step: events before the upload, after it, after the gates, after the download

        def e2e_step(k, record=False):
            i = k % nbuf
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record else None
            if record:
                ev[0].record(streams[i])
            qs.qs_state_copy_from_host_async(states[i].h, hnps[i])
            if record:
                ev[1].record(streams[i])
            for (c, t, m, v, U) in sched[k % SETS]:
                qs._lib.qs_apply_gate(states[i].h, t, m, v, U)
            if record:
                ev[2].record(streams[i])
            qs.qs_state_copy_to_host_async(states[i].h, hnps[i])
            if record:
                ev[3].record(streams[i])
                phase_ev.append(ev)

        for k in range(nbuf):  # warm-up
            e2e_step(k)
        for i in range(nbuf):
            qs.qs_state_synchronize(states[i].h)
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            e2e_step(k, record=True)
        for i in range(nbuf):
            qs.qs_state_synchronize(states[i].h)
        e2e_s = time.perf_counter() - t0
        med = lambda xs: round(sorted(xs)[len(xs) // 2], 2)
        phases = {"h2d_ms": med([e[0].elapsed_time(e[1]) for e in phase_ev]),
                  "gates_ms": med([e[1].elapsed_time(e[2]) for e in phase_ev]),
                  "d2h_ms": med([e[2].elapsed_time(e[3]) for e in phase_ev])}
        result["e2e"] = {"value": round(world * e2e_steps * step_bytes / e2e_s / 1e9, 2), "unit": "GB/s",
                         "h2d_bytes_per_step": int(hnps[0].nbytes), "d2h_bytes_per_step": int(hnps[0].nbytes),
                         "steps": e2e_steps, "pipeline": f"{nbuf} states on {nbuf} streams, async copies from page-locked memory",
                         "median_phase_ms": phases}
        for x in states:
            x.close()
        del hosts, hnps
        st = None

    if st is not None:
        st.close()
    torch.cuda.empty_cache()

    if want("c128") and rank == 0:
        # complex128 sweep (one step): FP64 ALU roofline
        st2 = qs.State(n, "c128")
        for q in range(n):
            st2.apply_gate(q, W.H_MATRIX)
        sm2, per2 = run_sweep(qs, st2, n, 16, sched, 1, 1)
        st2.close()
        torch.cuda.empty_cache()
        b2 = sum(alg_bytes(n, c, 16) for c, _, _, _ in per2)
        ms2 = sum(x for _, _, x, _ in per2)
        pairs = sum(1 << (n - 1 - c) for c, _, _, _ in per2)
        flops = 28.0 * pairs  # general 2x2 complex update: 12 FMA + 4 MUL per pair, FMA = 2 flops
        fp64_instr = 16.0 * pairs  # the FP64 instructions of that update (FMA and MUL issue alike)
        peaks = measure_fma_peaks(qs)
        result["fma_peaks_tflops"] = peaks
        result["c128_sweep"] = {
            "GBps": round(b2 / (ms2 * 1e-3) / 1e9, 1), "frac_hbm": round(b2 / (ms2 * 1e-3) / 1e9 / peak, 3),
            "roofline": {"bound": "alu", "achieved": round(flops / (ms2 * 1e-3) / 1e12, 3),
                         "peak": peaks["fp64"], "unit": "TFLOP/s (FP64)", "peak_source": "measured (qs_measure_fma_peak)",
                         "frac": round(flops / (ms2 * 1e-3) / 1e12 / peaks["fp64"], 3),
                         "nominal_fp64_tflops": FP64_NOMINAL_TFLOPS,
                         # the pipe issues MUL and FMA at one rate: against the measured FMA
                         # instruction rate (peak / 2 flops) the update's 16 instructions per pair
                         "fp64_instr_per_s": round(fp64_instr / (ms2 * 1e-3) / 1e12, 3),
                         "frac_of_fp64_instr_rate": round(fp64_instr / (ms2 * 1e-3) / 1e12 / (peaks["fp64"] / 2), 3)},
        }
    if want("q30") and rank == 0:
        # fixed-point (Q1.30) states: the same sweep, one step, algorithmic bytes at 8 per amplitude
        st3 = qs.State(n, "q30")
        for q in range(n):
            st3.apply_gate(q, W.H_MATRIX)
        sm3, per3 = run_sweep(qs, st3, n, 8, sched, 1, 1)
        st3.close()
        torch.cuda.empty_cache()
        b3 = sum(alg_bytes(n, c, 8) for c, _, _, _ in per3)
        ms3 = sum(x for _, _, x, _ in per3)
        result["q30_sweep"] = {"GBps": round(b3 / (ms3 * 1e-3) / 1e9, 1),
                               "frac_hbm": round(b3 / (ms3 * 1e-3) / 1e9 / peak, 3),
                               "format": "Q1.30 int32 (re, im), exact 64-bit products, one rounding per output"}
    if rank == 0:
        if any(want(p) for p in ("adjoint", "fused", "batch", "paper", "precision")):
            FMA_PEAKS.update(measure_fma_peaks(qs))
            result.setdefault("fma_peaks_tflops", dict(FMA_PEAKS))
        if want("adjoint"):
            result["adjoint"] = measure_adjoint(qs, W, peak)
        if want("fused"):
            result["fused"] = measure_fused(qs, W, peak)
        if want("reduce"):
            result["reduce_expect_z_n30"] = measure_reduce(qs, W, peak)
        if want("masked"):
            result["masked_over_reduced_time_by_c"] = measure_masked(qs, n, sched)
        if want("batch"):
            result["batch"] = measure_batch(qs, W, peak)
        if want("paper"):
            result["paper_circuits"] = measure_paper_circuits(qs, W, peak)
        if want("precision"):
            result["precision_n32"] = measure_precision(qs, W)
        if want("cpu"):
            result["cpu_baseline"] = cpu_oracle_sample(n, sched)

    if rank == 0:
        print(json.dumps(result), flush=True)


def run_ncu_case(args):
    """Profiling case: no timing, no output besides one status line."""
    import torch

    import paper_2411_18354_gb300 as qs

    qs.build()
    rows = [r for r in sweep_schedule(args.n)[0] if r[0] == args.ncu_case]
    st = qs.State(args.n, args.dtype)
    for _ in range(2):
        for (c, t, m, v, U) in rows:
            qs._lib.qs_apply_gate(st.h, t, m, v, U)
    torch.cuda.synchronize()
    st.close()
    print(f"ncu case done: n={args.n} c={args.ncu_case} {args.dtype} targets={[r[1] for r in rows]}")


def run_ncu_fused(args):
    import torch

    import paper_2411_18354_gb300 as qs
    import workloads as W

    qs.build()
    n, layers = 24, args.layers
    g = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    flags = qs.QS_FLAG_FUSE | (qs.QS_FLAG_JIT if args.jit else 0)
    if args.jit:
        _compile(qs, n, g, th, args.dtype, adjoint=True)
    with qs.State(n, args.dtype) as st:
        st.apply_circuit(g, th, flags)
        st.adjoint_grad(g, th, flags)
        torch.cuda.synchronize()
    print("ncu fused case done")


def run_ncu_reduce(args):
    import torch

    import paper_2411_18354_gb300 as qs

    qs.build()
    with qs.State(27, args.dtype) as st:
        st.expect_z()
        st.expect_z()
        torch.cuda.synchronize()
    print("ncu reduce case done")


def run_ncu_batch(args):
    import numpy as np
    import torch

    import paper_2411_18354_gb300 as qs
    import workloads as W

    qs.build()
    ns = [16] * 304
    circ = W.hea_circuit(16, 2)
    th = torch.tensor(np.random.default_rng(1).uniform(0, 6.28, size=304 * 64), dtype=torch.float64, device="cuda")
    b = qs.Batch(ns, [circ] * 304, [64] * 304, "c64", small_bits=12, tile_bits=12)
    en = torch.zeros(304, dtype=torch.float64, device="cuda")
    gr = torch.zeros(304 * 64, dtype=torch.float64, device="cuda")
    b.run(th, en, gr, qs.QS_FLAG_JIT if args.jit else 0)
    torch.cuda.synchronize()
    b.close()
    print("ncu batch case done")


def run_tile_costs(args):
    """Device time of a fused pass of 1, 16 and 64 gates of one kind on local qubits 0..11
    (n = 24, complex64, tiles of 2^12 amplitudes); the slope is the per-gate cost inside a pass."""
    import numpy as np

    os.environ["QS_TILE_BITS"] = "12"
    import paper_2411_18354_gb300 as qs
    import workloads as W

    qs.build()
    n = 24
    rng = np.random.default_rng(0)

    def circ(kind, count):
        gl = []
        for i in range(count):
            t = i % 12
            q = (t // 4) * 4 + ((t % 4) + 1) % 4  # a control in the same 4-qubit group
            if kind == "real":
                th = rng.uniform(0, 6)
                c, s_ = np.cos(th / 2), np.sin(th / 2)
                gl.append(W.make_gate(t, np.array([[c, -s_], [s_, c]])))
            elif kind == "diagonal":
                th = rng.uniform(0, 6)
                gl.append(W.make_gate(t, np.diag([np.exp(-0.5j * th), np.exp(0.5j * th)])))
            elif kind == "general":
                gl.append(W.make_gate(t, W.haar_2x2(rng)))
            elif kind == "exchange":
                gl.append(W.make_gate(t, None, (), kind=W.KIND_X))
            elif kind == "cnot_in_row":
                gl.append(W.make_gate(t, None, (q,), kind=W.KIND_X))
            else:
                gl.append(W.make_gate(t, W.haar_2x2(rng), (q,)))
        return W.gate_list(gl)  # targets cycle over 0..11: neighbours never share one (no merging)

    out = {}
    with qs.State(n, "c64") as st:
        st.apply_gate(0, W.H_MATRIX)
        for label, extra in (("interpreted", 0), ("compiled", qs.QS_FLAG_JIT)):
            res = {}
            for kind in ("real", "diagonal", "general", "exchange", "cnot_in_row", "controlled_general_in_row"):
                t = {}
                for cnt in (1, 16, 64):
                    g = circ(kind, cnt)
                    fl = qs.QS_FLAG_FUSE | qs.QS_FLAG_GRAPH | extra
                    t[cnt] = _events_ms(lambda: st.apply_circuit(g, flags=fl), 10)
                res[kind] = {"pass_us": {str(k): round(v * 1e3, 1) for k, v in t.items()},
                             "us_per_gate": round((t[64] - t[16]) / 48 * 1e3, 2)}
            out[label] = res
    print(json.dumps({"tile_costs_n24_c64": out}), flush=True)


def run_ncu_scale(args):
    """Profiling case: compile, then the 1000-gate scale circuit (n = 30, 0-8 controls) with
    QS_FLAG_FUSE | QS_FLAG_JIT twice; no timing."""
    import torch

    import paper_2411_18354_gb300 as qs
    import workloads as W

    qs.build()
    n = 30
    g = W.scale_circuit(n, 1000, seed=1)
    _compile(qs, n, g, None, "c64")
    with qs.State(n, "c64") as st:
        for _ in range(2):
            st.apply_circuit(g, flags=qs.QS_FLAG_FUSE | qs.QS_FLAG_JIT)
        torch.cuda.synchronize()
    print("ncu scale case done")


def run_gate_patterns(args):
    """Per gate: median device time over 10 launches, each after a read-only pass over a 256 MB
    buffer (the L2 then holds clean lines of that buffer, none of the state); the general 2x2
    and the exchange (same amplitudes moved, no arithmetic) on the sweep's first 12 control
    sets of c = 6, 7, 8, and the same c with the controls on the top qubits."""
    import numpy as np
    import torch

    import paper_2411_18354_gb300 as qs
    import workloads as W

    qs.build()
    n = 30
    peak, _ = load_peaks()
    sched = sweep_schedule(n)
    st = qs.State(n, "c64")
    for q in range(n):
        st.apply_gate(q, W.H_MATRIX)
    flush = torch.empty(1 << 28, dtype=torch.uint8, device="cuda")

    def t_us(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        ev = []
        for _ in range(reps):
            flush.max()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            ev.append((a, b))
        torch.cuda.synchronize()
        return sorted(x.elapsed_time(y) for x, y in ev)[reps // 2] * 1e3

    rng = np.random.default_rng(5)
    out = []
    for c in (6, 7, 8):
        rows = [r for s in range(SETS) for r in sched[s] if r[0] == c][:12]
        alg = alg_bytes(n, c, 8)
        for (_, t, m, v, U) in rows:
            ins = m | (1 << t)
            tg = t_us(lambda: qs._lib.qs_apply_gate(st.h, t, m, v, U))
            tx = t_us(lambda: qs._lib.qs_apply_x(st.h, t, m, v))
            out.append({"c": c, "t": t, "p0": (ins & -ins).bit_length() - 1, "mask": hex(m), "gate_us": round(tg, 2),
                        "exchange_us": round(tx, 2), "frac": round(alg / (tg * 1e-6) / 1e9 / peak, 3),
                        "frac_sector_adjusted": round(sector_bytes(n, m, 8) / (tg * 1e-6) / 1e9 / peak, 3)})
        m = sum(1 << q for q in range(n - c, n))
        t = n - c - 1
        U = W.pack_u(W.haar_2x2(rng))
        tg = t_us(lambda: qs._lib.qs_apply_gate(st.h, t, m, m, U))
        out.append({"c": c, "t": t, "p0": t, "mask": hex(m), "gate_us": round(tg, 2), "contiguous": True,
                    "frac": round(alg / (tg * 1e-6) / 1e9 / peak, 3)})
    st.close()
    print(json.dumps({"gate_patterns_n30_c64": out}), flush=True)


def run_ncu_qft(args):
    """Profiling case: the QFT (29 qubits unless --n is given) with QS_FLAG_FUSE, twice; no timing."""
    import torch

    import paper_2411_18354_gb300 as qs
    import workloads as W

    qs.build()
    n = args.n if args.n != 30 else 29
    g = W.qft_circuit(n)
    flags = qs.QS_FLAG_FUSE | (qs.QS_FLAG_JIT if args.jit else 0)
    if args.jit:
        _compile(qs, n, g, None, "c64")
    with qs.State(n, "c64") as st:
        for _ in range(2):
            st.apply_circuit(g, flags=flags)
        torch.cuda.synchronize()
    print("ncu qft case done")


def main():
    args = parse_args()
    if args.ncu_case is not None:
        run_ncu_case(args)
        return
    if args.ncu_fused:
        run_ncu_fused(args)
        return
    if args.tile_costs:
        run_tile_costs(args)
        return
    if args.ncu_qft:
        run_ncu_qft(args)
        return
    if args.gate_patterns:
        run_gate_patterns(args)
        return
    if args.ncu_scale:
        run_ncu_scale(args)
        return
    if args.ncu_batch:
        run_ncu_batch(args)
        return
    if args.ncu_reduce:
        run_ncu_reduce(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
