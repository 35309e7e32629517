"""The autotuner on the GPU: its choices are legal, cached and restored, and runs with the
tuned settings still match the oracle."""
import json

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import ATOL_CIRCUIT, c128_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import paper_2411_18354_gb300 as q

    q.build()
    return q


@pytest.mark.parametrize("flags_name", ["interpreted", "compiled"])
def test_tune_fused_choices_cache_and_restore(qs, tmp_path, monkeypatch, flags_name):
    """tune_fused for the forward and the adjoint direction of an n = 12 ansatz: the chosen
    tile size is one of the candidates the library accepts, it is written to the cache and a
    second call is served from it; the context manager restores the tile size in force
    before; tuned fused runs match the oracle (state) and parameter shift (gradient)."""
    from paper_2411_18354_gb300 import autotune

    monkeypatch.setenv("QS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.delenv("QS_TILE_BITS", raising=False)
    extra = qs.QS_FLAG_JIT if flags_name == "compiled" else 0
    n, layers = 12, 3
    gates = W.hea_circuit(n, layers)
    th = W.hea_params(n, layers, seed=3)
    autotune.restore_defaults()
    default_fwd = qs.qs_get_tile_bits(qs.QS_C64, 0)
    default_adj = qs.qs_get_tile_bits(qs.QS_C64, 1)
    cands = (8, 10, 12, 14)  # 14 is too large for the adjoint's two tiles: skipped there
    for adjoint in (False, True):
        r = autotune.tune_fused(n, "c64", gates, th, adjoint=adjoint, candidates=cands, reps=1, flags=extra)
        assert r["tile_bits"] in cands and not r["cached"]
        assert qs.qs_get_tile_bits(qs.QS_C64, int(adjoint)) == r["tile_bits"]  # applied
        assert str(14) not in r["tried"] or not adjoint
        r2 = autotune.tune_fused(n, "c64", gates, th, adjoint=adjoint, candidates=cands, reps=1, flags=extra)
        assert r2["cached"] and r2["tile_bits"] == r["tile_bits"]
    cache = json.loads((tmp_path / "tune.json").read_text())
    assert len(cache) == 2
    # tuned settings in force: results still match the references
    ref = W.basis_state(n, 0)
    oracle.run_circuit(ref, n, gates, th)
    with qs.State(n, "c64") as st:
        st.apply_circuit(gates, th, qs.QS_FLAG_FUSE | extra)
        assert np.max(np.abs(c128_of(st.to_numpy()) - ref)) <= ATOL_CIRCUIT["c64"]
        st.set_basis(0)
        e, g = st.adjoint_grad(gates, th, qs.QS_FLAG_FUSE | extra)
    assert np.max(np.abs(g - oracle.param_shift_grad(n, gates, th))) <= 1e-4
    # apply=False and the context manager leave the previous setting in force
    autotune.restore_defaults()
    autotune.tune_fused(n, "c64", gates, th, candidates=cands, reps=1, flags=extra, use_cache=False, apply=False)
    assert qs.qs_get_tile_bits(qs.QS_C64, 0) == default_fwd
    with autotune.tuned_tile_bits(n, "c64", gates, th, adjoint=True, candidates=cands, reps=1, flags=extra) as ch:
        assert qs.qs_get_tile_bits(qs.QS_C64, 1) == ch["tile_bits"]
    assert qs.qs_get_tile_bits(qs.QS_C64, 1) == default_adj
    autotune.restore_defaults()


def test_tune_batch_choice_is_valid_and_cached(qs, tmp_path, monkeypatch):
    """tune_batch on a small uneven batch (n = 6..14, 2 ansatz layers): the chosen setting is
    one of the candidates, cached, and the batch built with it matches parameter shift for a
    few states (n <= 9) and the oracle energy for all of them."""
    import torch

    from paper_2411_18354_gb300 import autotune

    monkeypatch.setenv("QS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    rng = np.random.default_rng(44)
    ns = [int(v) for v in rng.integers(6, 15, size=24)]
    circuits = [W.hea_circuit(k, 2) for k in ns]
    nparams = [4 * k for k in ns]
    thetas = [rng.uniform(0, 2 * np.pi, size=p) for p in nparams]
    cands = ({"small_bits": 10, "tile_bits": 8, "max_pass_gates": 64},
             {"small_bits": 12, "tile_bits": 10, "max_pass_gates": 32},
             {"small_bits": 8, "tile_bits": 7, "max_pass_gates": 16})
    r = autotune.tune_batch(ns, circuits, nparams, thetas, "c64", candidates=cands, reps=1)
    cfg = {k: r[k] for k in ("small_bits", "tile_bits", "max_pass_gates")}
    assert cfg in [dict(c) for c in cands] and not r["cached"]
    assert autotune.tune_batch(ns, circuits, nparams, thetas, "c64", candidates=cands, reps=1)["cached"]
    b = qs.Batch(ns, circuits, nparams, "c64", **cfg)
    try:
        th = torch.tensor(np.concatenate(thetas), dtype=torch.float64, device="cuda")
        en = torch.empty(len(ns), dtype=torch.float64, device="cuda")
        gr = torch.empty(b.num_params, dtype=torch.float64, device="cuda")
        b.run(th, en, gr)
        torch.cuda.synchronize()
        en, gr = en.cpu().numpy(), gr.cpu().numpy()
    finally:
        b.close()
    off = np.concatenate([[0], np.cumsum(nparams)])
    checked = 0
    for s, k in enumerate(ns):
        assert abs(en[s] - oracle.energy(k, circuits[s], thetas[s])) <= 1e-5, s
        if k <= 9 and checked < 3:
            ps = oracle.param_shift_grad(k, circuits[s], thetas[s])
            assert np.max(np.abs(gr[off[s]:off[s + 1]] - ps)) <= 1e-4, s
            checked += 1
    assert checked > 0
