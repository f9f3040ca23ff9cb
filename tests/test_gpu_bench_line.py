"""bench.py's JSON line on the GPU (a short lab run: 400 positions, 2 iterations per step):
every key of the result contract is present with a sensible value, the roofline is computed
from the run's own CUDA-event stage times, and the end-to-end arm moves the stack's bytes."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def line():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "2", "--warmup", "3", "--iters", "2",
           "--positions", "400", "--no-cpu-baseline", "--no-nrmse"]
    out = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_contract_keys(line):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks",
              "cpu_baseline"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["value"] > 0 and line["ms_per_step"] > 0
    # value = position-updates of the timed steps over their time
    J = line["config"]["positions"]
    assert line["value"] == pytest.approx(J * 2 / (line["ms_per_step"] / 1e3), rel=1e-3)
    assert line["gpu_launches"] > 0
    assert "workload" in line["config"]


def test_roofline_fields(line):
    r = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert 0 < r["frac"] < 1.5
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    # achieved = the kernel's algorithmic bytes per iteration over its measured time per iteration
    assert r["achieved"] == pytest.approx(
        r["bytes_per_position"] * r["positions_per_iteration"] / (r["ms_per_iteration"] / 1e3) / 1e9, rel=2e-3)
    assert 0 < r["iteration_view"]["frac"] < 1.5


def test_e2e_arm(line):
    e = line["e2e"]
    assert e["value"] > 0 and e["unit"] == line["unit"]
    J = line["config"]["positions"]
    # the raw stack (K exposures of N^2 uint16 per position) is copied every step
    assert e["h2d_bytes_per_step"] >= J * 5 * 256 * 256 * 2
    assert e["d2h_bytes_per_step"] >= 1024 * 1024 * 8      # the reconstructed object
