"""The library's debug build on the GPU: bounds of every global access and the number of writes
per amplitude, for single gates at n = 1..16 (exactly the amplitudes of the reduced iteration
set written, each once), fused programs with interpreted and compiled passes, one-pass
programs (every amplitude written once) and gradients; the checks themselves are shown to
fire on a state declared smaller than its buffer. Runs tests/debug_checks_main.py in a child
process that loads libqs_debug.so."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_checks():
    env = dict(os.environ, QS_LIB_VARIANT="debug")
    env.pop("QS_TILE_BITS", None)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_checks_main.py")], env=env, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
    out = json.loads(line)
    assert out["debug_checks"] == "ok" and out["gates"] >= 300 and out["fused_runs"] >= 30
