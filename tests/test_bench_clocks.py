"""bench.py's clock record: only nvidia-smi samples taken inside the timed
region count, and an active throttle reason outside it is not reported."""
import datetime

import bench


def _line(ts, mhz, hw):
    t = ts.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{t}, 0, {mhz}, 2070, 900.00, 0x0000000000000000, {hw}, Not Active, Not Active, Not Active"


def test_clock_record_keeps_only_samples_in_region():
    base = datetime.datetime(2026, 12, 3, 10, 0, 0)
    rows = [(1000, "Active"), (2070, "Not Active"), (2070, "Not Active"), (1965, "Not Active"), (900, "Active")]
    lines = [_line(base + datetime.timedelta(seconds=0.2 * i), mhz, hw) for i, (mhz, hw) in enumerate(rows)]
    lines.insert(2, "garbage line")
    t0 = (base + datetime.timedelta(seconds=0.2)).timestamp()
    t1 = (base + datetime.timedelta(seconds=0.6)).timestamp()
    rec = bench.parse_clock_csv(lines, t0, t1, slack=0.05)
    assert rec["samples"] == 3 and rec["samples_outside_region"] == 2
    assert rec["sm_mhz"] == 2070 and rec["sm_max_mhz"] == 2070
    assert rec["reasons"] == []
    every = bench.parse_clock_csv(lines)
    assert every["samples"] == 5 and every["reasons"] == ["hw_slowdown"]


def test_clock_record_without_readable_stamps_keeps_every_sample():
    lines = ["Thu Dec  3 10:00:00 2026, 0, 1980, 2070, 900.00, 0x0, Not Active, Not Active, Not Active, Active",
             "Thu Dec  3 10:00:01 2026, 0, 2070, 2070, 900.00, 0x0, Not Active, Not Active, Not Active, Not Active"]
    rec = bench.parse_clock_csv(lines, 0.0, 1.0)
    assert rec["samples"] == 2 and not rec["in_region_only"]
    assert rec["sm_mhz"] == 2025 and rec["reasons"] == ["sw_power_cap"]


def test_sampler_process_end_to_end(tmp_path, monkeypatch):
    """Clocks.start/begin/end/stop against a stand-in nvidia-smi that prints
    one stamped sample every 0.2 s (SM clock 2070 MHz, no reason active)."""
    import os
    import sys
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!" + sys.executable + "\n"
        "import datetime, sys, time\n"
        "while True:\n"
        "    t = datetime.datetime.now().strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]\n"
        "    print(f'{t}, 0, 2070, 2070, 950.00, 0x0, Not Active, Not Active, Not Active, Not Active', flush=True)\n"
        "    time.sleep(0.2)\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    c = bench.Clocks(0)
    c.start()
    time.sleep(0.3)
    c.begin()
    time.sleep(1.0)
    c.end()
    rec = c.stop()
    assert rec["in_region_only"] and 4 <= rec["samples"] <= 8
    assert rec["sm_mhz"] == 2070 and rec["reasons"] == [] and abs(rec["region_s"] - 1.0) < 0.2


def test_reference_arm_line_on_the_host():
    """`bench.py --impl reference` (the oracle on the host's cores, the
    driver's reference arm) prints one JSON line with the contract's keys:
    the metric of the default workload, impl, cpu_baseline, an e2e without
    host-device copies; small workload, one step."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                          "torus32x12", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=900, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "torus32x12" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["metric"] and d["unit"]
