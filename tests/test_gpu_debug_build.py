"""The DGT_DEBUG build (guard zones around every device allocation of the library and between
the regions of every workspace, checked after each kernel launch; include/dgt.h): built on
the GPU host and driven in a child process with DGT_DEBUG=1 through the coset, shear (both
branches), FIR, mixed-radix, real-signal, caller-workspace and dual-window paths against the
float64 oracle (tests/_debug_sweep.py); no guard word may be overwritten, the caller's
buffers must stay untouched outside their extent, and a guard word damaged inside the
library's own allocation must be reported by the next launch's check."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_sweep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    lib = build.build(debug=True)
    assert lib.endswith("libdgt_debug.so")
    env = dict(os.environ, DGT_DEBUG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_debug_sweep.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    assert rep["ok"] and rep["cases"] >= 20, rep
    det = [c for c in rep["report"] if c["path"] == "detector"][0]
    assert det["violations"] == 1 and det["kernel"] and det["after"] == 0, det
