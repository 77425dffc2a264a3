"""The bounds-checked debug build of libdp on the GPU (the stand-in for a device memory checker).

The build (-DDP_BOUNDS_CHECK, its own library under _build_bounds/) checks every neighbor, cell,
work-list and type index that its kernels read or derive before using it and records the first bad
one instead of accessing it.  Its cases run in a child process that loads that library
(DP_LIBRARY=bounds): every evaluation route, the wide nets, the force-loss gradient and an NVE run
with device list rebuilds must match the oracle as in the other GPU tests, and the record of bad
indexes must stay empty.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checked_build_runs_clean_and_matches_oracle():
    import paper_2005_00223_gb300 as pkg
    pkg.build(bounds_check=True)
    env = dict(os.environ, DP_LIBRARY="bounds")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["bounds"] == [0, 0, 0, 0]
    assert out["cases"] == ["water192", "cu500", "wide64", "grad", "md"]
