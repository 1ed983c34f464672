"""bench.py's reference arm runs the CPU oracle and prints the contract's
JSON line (no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-sample", "1024"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "cpu_baseline", "e2e", "config"):
        assert key in line
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1


def _bench_module():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_issue_roofline_from_a_matching_capture(tmp_path, monkeypatch):
    b = _bench_module()
    prof = tmp_path / "prof.json"
    prof.write_text(json.dumps({"source_sha": b.kernel_source_hash(), "warp_instructions_per_launch": 4.0e7,
                                "dram_bytes_per_launch_full_size": 3.5e6}))
    monkeypatch.setattr(b, "TRAFFIC_FILE", str(prof))
    r = b.issue_roofline(0.1, {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0}, 152)
    # 4e7 instructions in 0.1 ms = 0.4 T/s; 4 x 152 x 2.0 GHz = 1.216 T/s
    assert abs(r["achieved"] - 0.4) < 1e-12 and abs(r["peak"] - 1.216) < 1e-12
    assert abs(r["frac"] - 0.4 / 1.216) < 1e-12 and r["bound"] == "issue"
    assert b.measured_traffic() == 3.5e6
    # a capture of another kernel source gives no number
    prof.write_text(json.dumps({"source_sha": "0" * 16, "warp_instructions_per_launch": 4.0e7}))
    assert b.issue_roofline(0.1, {"sm_mhz": 2000.0}, 152) is None and b.measured_traffic() is None
    # without a clock sample there is no peak
    prof.write_text(json.dumps({"source_sha": b.kernel_source_hash(), "warp_instructions_per_launch": 4.0e7}))
    assert b.issue_roofline(0.1, None, 152) is None
