"""The bench's accuracy metrics (Sec. IV-A, Eq. ea_ep): e_A is the mean angle and e_P(phi) the share of
angles at most phi, checked on vector pairs with known angles."""
import numpy as np

import bench


def test_ea_ep_on_known_angles():
    ang = np.array([0.0, 5.0, 9.0, 15.0, 25.0, 40.0])  # (none on a boundary)
    t = np.radians(ang)
    gt = np.stack([np.zeros_like(t), np.zeros_like(t), np.ones_like(t)])
    n = np.stack([np.sin(t), np.zeros_like(t), np.cos(t)]) * 3.0  # the metric ignores length
    r = bench.ea_ep(n, gt, np.ones(6, bool))
    assert r["m"] == 6
    assert abs(r["e_A_deg"] - ang.mean()) < 1e-3
    assert r["e_P_10"] == round(3 / 6, 4) and r["e_P_20"] == round(4 / 6, 4) and r["e_P_30"] == round(5 / 6, 4)


def test_ea_ep_selects_pixels():
    gt = np.zeros((3, 2, 2))
    gt[2] = 1
    n = gt.copy()
    n[:, 0, 0] = [1, 0, 0]  # 90 degrees off, but not selected
    sel = np.array([[False, True], [True, True]])
    r = bench.ea_ep(n, gt, sel)
    assert r["m"] == 3 and r["e_A_deg"] == 0.0 and r["e_P_10"] == 1.0


def test_clock_sampler_keeps_the_timed_window(tmp_path, monkeypatch):
    # a stand-in nvidia-smi that prints one reading per 20 ms: idle clocks first, load clocks later
    import os
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/usr/bin/env python3\n"
                    "import sys, time\n"
                    "k = 0\n"
                    "while True:\n"
                    "    sm = 345 if k < 10 else 2070\n"
                    "    cap = 'Active' if k >= 10 else 'Not Active'\n"
                    "    print(f'0, {sm}, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, {cap}', flush=True)\n"
                    "    k += 1\n"
                    "    time.sleep(0.02)\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    monkeypatch.setattr(bench.ClockSampler, "PERIOD_MS", 20)
    with bench.ClockSampler(0) as clk:
        assert clk.lines, "the sampler must be live before the caller's warm-up"
        time.sleep(0.5)  # past the idle readings
        clk.mark_start()
        time.sleep(0.1)
        clk.mark_end()
    s = clk.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"]
    assert 2 <= s["samples"] <= 12 and s["samples"] < len(clk.lines)
    assert 90 <= s["window_ms"] <= 400


def test_clock_sampler_short_window_gets_the_closing_reading(tmp_path, monkeypatch):
    import os
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/usr/bin/env python3\n"
                    "import time\n"
                    "while True:\n"
                    "    print('0, 1980, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active', flush=True)\n"
                    "    time.sleep(0.05)\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    monkeypatch.setattr(bench.ClockSampler, "PERIOD_MS", 50)
    with bench.ClockSampler(0) as clk:
        clk.mark_start()
        clk.mark_end()  # a region far shorter than the period
    s = clk.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 1980 and s["reasons"] == []


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    with bench.ClockSampler(0) as clk:
        clk.mark_start()
        clk.mark_end()
    assert clk.summary()["reasons"] == ["unsampled"]


def test_reference_arm_prints_the_contract_line():
    # the reference arm (the FP64 oracle on the host cores) runs without a GPU and prints one JSON
    # line with the keys the bench contract names
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "frames/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    for key in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "vs_baseline", "dtype", "data",
                "config"):
        assert key in d, key
