"""GPU: the benchmark's JSON line on a reduced stencil (64^3 grid over 4^3 ranks): every key
of the contract, the roofline of the standard exchange's kernel against the measured peak,
the end-to-end number through host buffers with its copy bytes, the CPU oracle baseline, the
kernel launch count and the clock record, and the same config dict as the reference arm."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import bench  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_contract():
    out = subprocess.run([sys.executable, "bench.py", "--edge", "16", "--ranks", "4", "--steps", "5", "--warmup", "3",
                          "--no-extras", "--e2e-steps", "2", "--cpu-sample-ranks", "8"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in d, k
    assert d["metric"] == bench.METRIC and d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True and d["data"] == "synthetic"
    p = bench.workload(16, 4)
    assert d["config"] == bench.workload_config(p, 16, 1, 4)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9 and 0 < r["frac"] < 1.5
    assert r["traffic"] is None   # counters are committed for the 512^3 launch only
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert d["gpu_launches"] == 5 * sum(f["launches"] for f in d["forms"].values())
    assert d["clocks"]["sm_max_mhz"] > 0
