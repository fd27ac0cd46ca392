"""The benchmark's reference arm keeps the JSON-line contract on a machine without a GPU: one line with
impl = reference, the metric, unit and config of the GPU arm, a CPU baseline that states its cores and
sample, an end-to-end figure with no host-device copies, and an extrapolated per-step time that says so."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-seconds", "2"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    res = json.loads(lines[0])
    assert res["impl"] == "reference" and res["unit"] == "field·screen steps/s" and res["value"] > 0
    assert res["metric"].startswith("field·screen steps/s at N=1024")
    assert res["config"]["workload"].startswith("ar-evolution N=1024")
    cb = res["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["value"] == res["value"]
    assert res["e2e"] == {"value": res["value"], "unit": res["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "extrapolated" in res["ms_per_step_note"] and res["samples_timed"] == 1
