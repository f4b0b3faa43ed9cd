"""bench.py end to end on the GPU: one short run per streaming scheme prints a
single JSON line with the contract's keys, and the numbers are consistent
with each other (value from the events, roofline from the step kernel's own
events, launches counted)."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _run(*args):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), *args]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


@pytest.mark.parametrize("streaming", ["ab", "inplace"])
def test_bench_line_has_the_contract_keys(torch, streaming):
    d = _run("--steps", "3", "--warmup", "3", "--inner", "20", "--grid", "64", "--no-cpu-baseline",
             "--no-steady", "--warm-start-cases", "0", "--no-configs", "--streaming", streaming)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["unit"] == "MLUPS" and d["higher_is_better"] is True
    cells = 64 ** 3
    # value = cells x LBM steps / time
    assert abs(d["value"] - cells * 20 * 3 / (d["ms_per_step"] * 3 / 1e3) / 1e6) <= 1e-6 * d["value"]
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["bytes_per_cell"] == 208
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(r["frac_nominal"] - r["achieved"] / r["nominal_peak"]) < 1e-12
    assert abs(r["achieved"] - 208 * cells / (r["launch_us"] * 1e-6) / 1e9) <= 1e-6 * r["achieved"]
    # every timed benchmark step launches 20 step kernels, a residual (2) and a Nusselt (2)
    assert d["gpu_launches"] >= 3 * 20
    assert d["e2e"]["h2d_bytes_per_step"] == 20 * cells
    assert d["config"]["streaming"].startswith("two" if streaming == "ab" else "in place")
    # a walled box with even rows takes the paired kernels, named as such
    assert d["config"]["cells_per_thread"] == 2
    assert r["kernel"].startswith("step_pair_kernel<" if streaming == "ab" else "step_inplace_pair_kernel<")
