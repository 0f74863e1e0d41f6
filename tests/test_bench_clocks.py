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
