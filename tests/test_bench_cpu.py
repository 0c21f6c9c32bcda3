"""The benchmark's host-side contract, without a GPU: the reference arm (the oracle timed on
the host cores) prints one JSON line with the keys the driver reads; the issue-rate roofline
is the committed record's instructions per cell over the kernel time against the derived
peak, and both it and the traffic are null without a record for the current source."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_json_line(oracle):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "blast",
                        "--n", "64", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "cell-updates/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["config"]["cells"] == 64 * 64
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_issue_roofline_arithmetic(monkeypatch):
    rec = {"source_hash": "x", "dram_bytes_per_cell": 75.0, "warp_inst_per_cell": 80.0}
    monkeypatch.setattr(bench, "traffic_record", lambda: rec)
    # the peak follows the device's SM count and the clock sampled during the timed region
    r = bench.issue_roofline(1_000_000, 1e-4, 148, {"sm_mhz": 1800.0, "sm_max_mhz": 2070.0, "reasons": []})
    peak = 148 * 4 * 1800e6
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(peak)
    assert r["sms"] == 148 and r["sm_mhz"] == 1800.0
    assert r["achieved"] == pytest.approx(80.0 * 1e6 / 1e-4)
    assert r["frac"] == pytest.approx(80.0 * 1e6 / 1e-4 / peak)
    # without a clock sample: the maximum SM clock, said so
    r = bench.issue_roofline(1_000_000, 1e-4, 152, None)
    assert r["peak"] == pytest.approx(152 * 4 * 2070e6) and "no clock sample" in r["clock_source"]
    assert bench.measured_traffic(1000) == pytest.approx(75_000.0)
    monkeypatch.setattr(bench, "traffic_record", lambda: None)
    assert bench.issue_roofline(1_000_000, 1e-4, 152, None) is None and bench.measured_traffic(1000) is None



def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    """The traffic record stays valid across comment edits of the kernel source and not
    across code edits (the hash covers the code with // comments and blank lines left out)."""
    csrc = tmp_path / "paper_1210_5246_gb300" / "csrc"
    csrc.mkdir(parents=True)
    dev = "inline int f(int x) { return x + 1; }  // one more\n"
    step = ("// header\ntemplate <int N> int g() { return N; }\n\n"
            "// ---------------------------------------------------------------- 2D kernel\n"
            "int after_the_cut = 0;\n")
    (csrc / "msh_device.cuh").write_text(dev)
    (csrc / "msh_step_kernels.cuh").write_text(step)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (csrc / "msh_device.cuh").write_text("// a new comment\n" + dev.replace("one more", "plus one") + "\n\n")
    (csrc / "msh_step_kernels.cuh").write_text(step.replace("after_the_cut = 0", "after_the_cut = 1"))
    assert bench.kernel_source_hash() == h0  # comments, blank lines, code past the 2D kernel
    (csrc / "msh_device.cuh").write_text(dev.replace("x + 1", "x + 2"))
    assert bench.kernel_source_hash() != h0
