"""CPU checks of the C-ABI library: it builds, loads, exports every symbol that
include/*.h declares, and rejects bad arguments on the host before any CUDA call."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2411_18354_gb300 as qs
from paper_2411_18354_gb300 import _lib
from paper_2411_18354_gb300.build import LIB_PATH, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(qs_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_header_declares_the_interface():
    d = _declared()
    for name in ["qs_state_alloc", "qs_apply_gate", "qs_apply_circuit", "qs_expect_z", "qs_adjoint_grad"]:
        assert name in d


def test_library_exports_every_declared_symbol():
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = _declared() - exported
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert _declared() == set(_lib.exported_symbols())
    L = _lib.lib()
    for name in _declared():
        assert hasattr(L, name)


def test_package_reexports_every_declared_symbol():
    for name in _declared():
        assert callable(getattr(qs, name, None)), name


def test_gate_dtype_matches_struct_layout():
    g = qs.GATE_DTYPE
    assert g.itemsize == 96
    assert [g.fields[k][1] for k in ("target", "kind", "ctrl_mask", "ctrl_vals", "param", "reserved", "U")] == \
        [0, 4, 8, 16, 24, 28, 32]


# Host-side argument checks: these return before any CUDA call, so they run without a GPU.

def test_alloc_rejects_bad_sizes_on_host():
    for n in (0, -3, 41, 64):
        with pytest.raises(qs.QsError) as e:
            qs.qs_state_alloc(n, qs.QS_C64)
        assert e.value.status == _lib.QS_EINVAL
        assert "out of range" in qs.qs_last_error()
    with pytest.raises(qs.QsError) as e:
        qs.qs_state_alloc(4, 7)
    assert e.value.status == _lib.QS_EINVAL


def test_wrap_rejects_bad_buffers_on_host():
    with pytest.raises(qs.QsError):
        qs.qs_state_wrap(0, 1 << 20, 4, qs.QS_C64)  # NULL
    with pytest.raises(qs.QsError):
        qs.qs_state_wrap(0x1000 + 8, 1 << 20, 4, qs.QS_C64)  # misaligned
    with pytest.raises(qs.QsError) as e:
        qs.qs_state_wrap(0x100000, 100, 10, qs.QS_C128)  # too small
    assert "smaller" in str(e.value)


def test_calls_on_null_state_fail_cleanly():
    assert _lib.lib().qs_state_free(None) == 0
    U = np.eye(2)
    for fn in (lambda: qs.qs_apply_gate(0, 0, 0, 0, U), lambda: qs.qs_apply_x(0, 0),
               lambda: qs.qs_expect_z(0), lambda: qs.qs_state_set_basis(0, 0)):
        with pytest.raises(qs.QsError) as e:
            fn()
        assert e.value.status == _lib.QS_EINVAL


def test_wrapped_state_validates_gates_on_host():
    """A wrapped handle on a fake (never dereferenced) device address: gate validation
    fails on the host, so no kernel is launched and no CUDA call is made."""
    h = qs.qs_state_wrap(0x7f0000000000, 16 << 4, 4, qs.QS_C64)
    try:
        U = np.eye(2)
        bad = [
            (4, 0, 0, U),            # target out of range
            (-1, 0, 0, U),
            (1, 0b10, 0b10, U),      # control on the target
            (1, 0b10000, 0, U),      # control >= n
            (1, 0b100, 0b1000, U),   # vals outside mask
            (1, 0, 0, np.array([[np.nan, 0], [0, 1]])),
            (1, 0, 0, np.array([[1, np.inf], [0, 1]])),
        ]
        for t, m, v, u in bad:
            with pytest.raises(qs.QsError) as e:
                qs.qs_apply_gate(h, t, m, v, u)
            assert e.value.status == _lib.QS_EINVAL
        with pytest.raises(qs.QsError):
            qs.qs_apply_x(h, 0, 0b1, 0b1)
        # a circuit with one bad gate launches nothing
        import workloads as W
        gates = W.gate_list([W.make_gate(0, W.H_MATRIX), W.make_gate(9, W.H_MATRIX)])
        with pytest.raises(qs.QsError) as e:
            qs.qs_apply_circuit(h, gates)
        assert "gate 1" in str(e.value)
        # parameterised gate without theta
        gates = W.gate_list([W.make_gate(0, None, (), kind=W.KIND_RY, param=0)])
        with pytest.raises(qs.QsError):
            qs.qs_apply_circuit(h, gates)
        with pytest.raises(qs.QsError):
            qs.qs_adjoint_grad(h, gates, np.zeros(0))
        with pytest.raises(qs.QsError):
            qs.qs_apply_circuit(h, gates, np.zeros(1), flags=1 << 10)
        with pytest.raises(qs.QsError) as e:  # baseline schedule has no fused form
            qs.qs_apply_circuit(h, gates, np.zeros(1), flags=qs.QS_FLAG_FUSE | qs.QS_FLAG_MASKED)
        assert e.value.status == _lib.QS_EINVAL
    finally:
        qs.qs_state_free(h)  # wrapped memory is not freed by the library


def test_l2_fetch_setting_is_validated_on_host():
    before = qs.qs_get_l2_fetch_bytes()
    assert before in (0, 32, 64, 128)
    for bad in (1, 16, 48, 256, -32):
        with pytest.raises(qs.QsError) as e:
            qs.qs_set_l2_fetch_bytes(bad)
        assert e.value.status == _lib.QS_EINVAL
    try:
        for ok in (0, 64, 128, 32):
            qs.qs_set_l2_fetch_bytes(ok)
            assert qs.qs_get_l2_fetch_bytes() == ok
    finally:
        qs.qs_set_l2_fetch_bytes(before)


def test_tile_bits_setting_is_validated_on_host():
    for bad in (1, 4, 15, -2):
        with pytest.raises(qs.QsError):
            qs.qs_set_tile_bits(qs.QS_C64, 0, bad)
    qs.qs_set_tile_bits(qs.QS_C64, 1, 9)
    assert qs.qs_get_tile_bits(qs.QS_C64, 1) == 9
    qs.qs_set_tile_bits(qs.QS_C64, 1, 0)
    assert qs.qs_get_tile_bits(qs.QS_C64, 1) == 12
    # a block holds 2^bits amplitudes (twice for the adjoint's psi and lambda) and the pass's
    # gate tables in at most 227 KB of shared memory
    for dt, adj, largest in ((qs.QS_C64, 0, 14), (qs.QS_C64, 1, 13), (qs.QS_C128, 0, 13), (qs.QS_C128, 1, 12)):
        qs.qs_set_tile_bits(dt, adj, largest)
        assert qs.qs_get_tile_bits(dt, adj) == largest
        with pytest.raises(qs.QsError):
            qs.qs_set_tile_bits(dt, adj, largest + 1)
        qs.qs_set_tile_bits(dt, adj, 0)


def test_autotune_cache_roundtrip(tmp_path, monkeypatch):
    from paper_2411_18354_gb300 import autotune

    monkeypatch.setenv("QS_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    assert autotune._load() == {}
    autotune._save({"k": {"tile_bits": 11}})
    assert autotune._load() == {"k": {"tile_bits": 11}}
    assert autotune._sig(np.arange(3)) == autotune._sig(np.arange(3)) != autotune._sig(np.arange(4))
