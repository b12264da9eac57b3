"""bench.py's JSON line, as the full test run reads it: a short run of the default workload and of
the reference arm, every key of the contract present and consistent (the roofline fraction is
achieved / peak, the traffic is the committed profile's figure for these sources or null, the
end-to-end leg moves the state both ways, the clocks were sampled)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_default_line_keys():
    d = _run("--steps", "3", "--warmup", "3", "--no-cpu-baseline")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["data"] == "synthetic" and d["dtype"] == "f64"
    c = d["config"]
    assert c["workload"] == "grid_lognormal" and c["n_sd"] > 1.6e7 and "l2" in c
    assert d["value"] == pytest.approx(c["n_sd"] / (d["ms_per_step"] * 1e-3), rel=0.05)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-9)
    assert r["traffic"] == bench._profiled_traffic(r["kernel"], c["workload"], c["n_sd"])
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] >= 16 * c["n_sd"] and e["d2h_bytes_per_step"] >= 16 * c["n_sd"]
    assert d["gpu_launches"] >= 3 * d["steps"]
    k = d["clocks"]
    assert k["sm_mhz"] > 0 and k["sm_max_mhz"] > 0 and isinstance(k["reasons"], list)


def test_reference_arm_keys():
    d = _run("--impl", "reference", "--workload", "gravitational_box", "--steps", "2", "--warmup", "3")
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "gravitational_box"
