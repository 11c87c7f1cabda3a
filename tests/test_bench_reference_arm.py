"""Host-side parts of bench.py, on the CPU. The reference arm (the CPU oracle timed on the
engine line's workload) prints one JSON line with the engine line's metric, unit and workload,
its own CPU baseline and end-to-end keys (no host-device copies); under a multi-rank launch
only rank 0 runs and prints (about a second). The roofline's DRAM traffic is read from the
committed ncu summary only while the kernel source matches the one profiled."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(rank):
    env = dict(os.environ, RANK=str(rank))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_the_engine_lines_metric_and_workload():
    lines = run_reference(0)
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "GOPS" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["config"]["grammars"] == ["Q1", "QSC"]
    # Algorithm 1's products over both closures (19 executions x 6 productions of Query 1,
    # 3 x 3 of the sc-only query): the count the engine's line reports too
    assert d["config"]["products_per_step"] == 123
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    assert run_reference(1) == []


def test_traffic_is_reported_only_for_the_profiled_kernel_source(tmp_path, monkeypatch):
    # the bench line's DRAM traffic per launch comes from the committed ncu summary, and only
    # while the tensor kernel's source is the one the counters were taken from
    import hashlib

    src = tmp_path / "kernel.cu"
    src.write_text("// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "profile.txt"
    prof.write_text(f"dram_bytes_per_launch_avg: 1234\ndram_bytes_per_launch_skip_avg: 56\nsource_sha256: {sha}\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(prof))
    monkeypatch.setattr(bench, "TC_SOURCE", str(src))
    assert bench.tc_traffic_per_launch(True) == 1234.0
    assert bench.tc_traffic_per_launch(False) == 56.0
    src.write_text("// kernel source, changed\n")
    assert bench.tc_traffic_per_launch(True) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.tc_traffic_per_launch(True) is None
