"""The N > 1 launch path of bench.py on CPU: two ranks under torch.distributed.run with gloo (the
reference arm), rank 0 alone runs and prints one JSON line, every rank exits 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.join(os.path.dirname(__file__), "..")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.timeout(600)
def test_reference_arm_two_ranks_gloo():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--workload", "water192"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["unit"] == "s/step/atom"
    assert out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
    # the base contract's keys, with the reference arm's e2e (no host-device copies)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in out, key
    assert out["higher_is_better"] is False and out["steps"] == 1 and out["warmup"] == 0
    assert out["config"]["workload"].startswith("64 H2O, 192 atoms")
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert out["cpu_baseline"]["value"] == out["value"] and out["cpu_baseline"]["cores"] >= 1
