"""The debug build of the library (device bounds checks that record the first
failing site and skip the access, never trapping) runs a set of parity cases
against the oracle in a process of its own: every processing tier, the orbit
tiles, top-K, generic circuits, two-word masks, both precisions.  A failed
check would make pp_propagate return PP_ERR_CUDA; a mismatch fails the case."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_parity_cases():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_20441_b300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, PP_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_parity_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("ok ")]
    assert len(lines) == 13, r.stdout
