"""Host logic of bench.py, on the CPU: the clock sampler's parsing and
rejection reasons (against a fake nvidia-smi), the committed ncu traffic
figure matching the committed kernel sources, and the reference arm's JSON
line (the FP64 oracle on two host threads, one short step).
"""
import json
import os
import stat
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def fake_smi(tmp_path, rows):
    script = tmp_path / "nvidia-smi"
    body = "".join(f"echo '{r}'\n" for r in rows)
    script.write_text("#!/bin/sh\n" + body + "sleep 5\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_clock_sampler_median_under_load_and_reasons(tmp_path, monkeypatch):
    rows = ["0, 2070, 2070, 450.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 460.0, 0x0, Not Active, Not Active, Not Active, Active",
            "0, 2055, 2070, 455.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 345, 2070, 90.0, 0x0, Not Active, Not Active, Not Active, Not Active"]   # idle sample
    monkeypatch.setenv("PATH", fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    c = s.stop()
    assert c["samples"] == 4
    assert c["sm_max_mhz"] == 2070.0
    assert c["sm_mhz"] == 2070.0            # median of the samples above half the maximum
    assert c["reasons"] == ["sw_power_cap"]
    assert c["power_w_max"] == 460.0


def test_clock_sampler_reports_thermal_slowdown(tmp_path, monkeypatch):
    rows = ["0, 1500, 2070, 700.0, 0x0, Active, Not Active, Active, Not Active"]
    monkeypatch.setenv("PATH", fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    c = s.stop()
    assert c["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_committed_traffic_figure():
    """profiles/k_sig_tc_traffic.json holds the ncu DRAM traffic of a
    k_sig_tc launch with the fingerprint of the sources it was taken on;
    bench.py scales it by ROIs while the fingerprint matches and reports null
    otherwise."""
    with open(bench.TRAFFIC_JSON) as fh:
        t = json.load(fh)
    assert t["kernel"] == "k_sig_tc" and t["captured_rois"] > 0 and t["dram_bytes_per_launch_captured"] > 0
    assert len(t["sources_sha256_16"]) == 16
    assert os.path.exists(os.path.join(ROOT, "profiles", t["summary"]))
    t8 = bench.tc_traffic_per_launch(8192)
    t1 = bench.tc_traffic_per_launch(1024)
    if bench.kernel_sources_sha16(t["sources"]) == t["sources_sha256_16"]:
        assert t8 is not None and np.isclose(t8, 8 * t1)
        assert np.isclose(t1 * t["scaled_rois"] / 1024, t["dram_bytes_per_launch_scaled"], rtol=1e-3)
    else:
        assert t8 is None and t1 is None


def test_traffic_figure_follows_the_fingerprint(tmp_path, monkeypatch):
    """A traffic record taken on other sources (one flipped fingerprint digit)
    gives null; the same record with the current fingerprint gives the
    captured bytes scaled by the ROI count."""
    with open(bench.TRAFFIC_JSON) as fh:
        t = json.load(fh)
    good = bench.kernel_sources_sha16(t["sources"])
    stale = dict(t, sources_sha256_16=("0" if good[0] != "0" else "1") + good[1:])
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(stale))
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(f))
    assert bench.tc_traffic_per_launch(8192) is None
    f.write_text(json.dumps(dict(t, sources_sha256_16=good)))
    got = bench.tc_traffic_per_launch(2 * t["captured_rois"])
    assert got is not None and np.isclose(got, 2 * t["dram_bytes_per_launch_captured"])


def test_reference_arm_json_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([x for x in out.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["unit"] == line["cpu_baseline"]["unit"] == line["e2e"]["unit"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 2
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["higher_is_better"] is True and line["dtype"] == "f64"
