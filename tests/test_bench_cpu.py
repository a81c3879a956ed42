"""bench.py's reference arm (the oracle timed on the host cores) keeps the
JSON-line contract, without a GPU: one line with the metric, the whole-job
value, the timing fields (at least 3 warm-up steps), the workload config,
the cpu_baseline block and an e2e block with no host-device bytes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ, ET_REF_STEP_S="0.2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["metric"] == "views/s" and d["unit"] == "views/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] >= 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_tube_traffic_applies_only_to_its_launch_configuration():
    """The ncu traffic of the tube-count launch is reported only for the launch
    configuration it was captured on, and its HBM fraction is bytes over the
    kernel time against the measured copy bandwidth."""
    sys.path.insert(0, ROOT)
    import bench
    cap = bench.tube_run_key("batched", 256, [74, 621, 506], None, rows=2, ticket_origins=2)
    assert cap in bench.TUBE_DRAM_BYTES
    tuned = {"row_lists": 2, "ticket_origins": 2}
    assert bench.tube_run_key("batched", 256, (74, 621, 506), tuned) == cap
    assert bench.tube_run_key("batched", 32, (74, 621, 506), tuned) not in bench.TUBE_DRAM_BYTES
    assert bench.tube_run_key("batched", 256, (74, 506, 506), tuned) not in bench.TUBE_DRAM_BYTES
    assert bench.tube_run_key("batched", 256, (74, 621, 506), None, rows=1) not in bench.TUBE_DRAM_BYTES
    assert bench.tube_run_key("dense", 1, (68, 606, 606), {"row_lists": 2, "ticket_origins": 1})[1:] == \
        (1, (68, 606, 606), 2, 1)
    assert bench.hbm_roofline(None, 60.0, {}) is None
    h = bench.hbm_roofline(6.0e8, 60.0, {"hbm_gbs": 6000.0})
    assert abs(h["achieved_gbs"] - 10.0) < 1e-9 and abs(h["frac"] - 10.0 / 6000.0) < 1e-12
    assert h["peak_src"] == "of measured"
    assert bench.hbm_roofline(6.0e8, 60.0, {})["peak_src"] == "of fallback"
