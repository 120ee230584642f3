"""Host logic of bench.py that needs no GPU: the clock sampler's window, the
roofline traffic lookup and the reference arm's line."""

import datetime
import json
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler_with(lines, t0, t1):
    c = bench.ClockSampler(0)
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    with open(c.path, "w") as fh:
        fh.writelines(lines)
    c.proc = object()  # as if nvidia-smi had run
    c.t0, c.t1 = t0, t1
    return c


def _line(t, sm, cap=False, thermal=False):
    ts = t.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return (f"{ts}, 0, {sm}, 2070, 900.0, 0x0, Not Active, {'Active' if thermal else 'Not Active'}, Not Active, "
            f"{'Active' if cap else 'Not Active'}\n")


def test_clock_summary_keeps_only_the_timed_region():
    now = datetime.datetime(2026, 1, 1, 12, 0, 0)
    ms = datetime.timedelta(milliseconds=200)
    lines = [_line(now - 3 * ms, 1000, thermal=True)]  # before the region: ignored
    lines += [_line(now + k * ms, 2070 if k != 2 else 1980, cap=(k == 3)) for k in range(5)]
    lines += [_line(now + 9 * ms, 900)]  # after the region: ignored
    c = _sampler_with(lines, now, now + 4 * ms)
    s = c.summary()
    assert s["samples"] == 5 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]  # the thermal sample before the region does not count


def test_clock_summary_of_a_short_region_takes_the_next_sample():
    now = datetime.datetime(2026, 1, 1, 12, 0, 0)
    lines = [_line(now - datetime.timedelta(milliseconds=100), 1500), _line(now + datetime.timedelta(milliseconds=150), 2070)]
    c = _sampler_with(lines, now, now + datetime.timedelta(milliseconds=50))
    s = c.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 2070.0 and s["window"].startswith("first sample after")


def test_traffic_lookup_follows_kernel_workload_and_schedule():
    j = json.load(open(bench.TRAFFIC_FILE))
    sch = dict(zip(("sweep_kernel", "order", "ctas_per_sm"), j["schedule"]))
    nvox = int(j["voxels"])
    want = float(j["dram_read_bytes"]) + float(j["dram_write_bytes"])
    assert bench.measured_traffic("sweep_rows_kernel", 0, nvox, sch) == want
    assert bench.measured_traffic("sweep_rows_kernel", 0, nvox + 512, sch) is None  # another workload
    assert bench.measured_traffic("sweep_rows_kernel", 1, nvox, sch) is None  # another storage type
    other = dict(sch, ctas_per_sm=0)
    assert bench.measured_traffic("sweep_rows_kernel", 0, nvox, other) is None  # another schedule


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the C FP64 oracle on the host cores) prints one JSON
    line with the keys the driver reads: impl, value, the e2e block with no copies and a
    cpu_baseline describing the same run."""
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "voxel-updates/s" and d["dtype"] == "f64" and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["config"]["workload"] == bench.WORKLOAD
