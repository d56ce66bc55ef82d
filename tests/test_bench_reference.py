"""The bench's reference arm (the FP64 oracle on the host cores) keeps the
line format the driver reads: one JSON line with the metric, unit, value,
impl = "reference", a cpu_baseline describing the run and an e2e object with
zero host-device bytes.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "plain_6x6", "--steps", "1", "--warmup", "3"], cwd=ROOT,
                         capture_output=True, text=True, timeout=600,
                         check=True).stdout.strip().splitlines()
    lines = [l for l in out if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "samples/s" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("plain_6x6")


def test_default_workload_is_the_metric_configuration(monkeypatch):
    """With no flags the bench times the learned-proposal workload (16x16,
    R = 2, chi = 128, 8192 chains) for a few seconds of steps."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.workload == "learned_16x16" and a.gpus == 1 and a.impl == "ours"
    assert a.warmup >= 3 and 1 <= a.steps <= 50
