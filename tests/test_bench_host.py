"""CPU tests of bench.py's host logic: the clock record taken during the
timed region (median SM clock, throttle reasons, the rejection rule) and the
traffic figure read from the committed ncu summary only while the kernel
source it was taken on is unchanged."""
import json
import os

import pytest

import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.out = "\n".join(lines)
    return s.summary()


def _line(sm, mx=2070, active="0x0", hw="Not Active", hwt="Not Active", swt="Not Active",
          cap="Not Active"):
    return "0, %s, %s, 900.5, %s, %s, %s, %s, %s" % (sm, mx, active, hw, hwt, swt, cap)


def test_clock_summary_and_rejection_rule():
    c = _sampler([_line(2070), _line(2055), _line(1980)])
    assert c["sm_mhz"] == 2055 and c["sm_max_mhz"] == 2070 and c["reasons"] == []
    assert c["samples"] == 3 and not bench.bad_clocks(c)
    # a power cap is kept and noted
    c = _sampler([_line(1800, cap="Active"), _line(1850, cap="Active")])
    assert c["reasons"] == ["sw_power_cap"] and not bench.bad_clocks(c)
    # thermal or hardware slowdown rejects the run
    for kw in ({"hw": "Active"}, {"hwt": "Active"}, {"swt": "Active"}):
        assert bench.bad_clocks(_sampler([_line(2000, **kw)]))
    # clocks stuck far below the maximum with no reason: a leftover clock lock
    assert bench.bad_clocks(_sampler([_line(900), _line(905)]))
    # no samples (no nvidia-smi): recorded as such, not a rejection
    c = _sampler(["garbage", ""])
    assert c["reasons"] == ["unsampled"] and not bench.bad_clocks(c)


def test_profiled_traffic_follows_the_source_hash(monkeypatch, tmp_path):
    # a record taken on the current kernel source is read back
    rec = tmp_path / "traffic.json"
    rec.write_text(json.dumps({"source_sha256_16": bench.kernel_source_sha(),
                               "dram_bytes_per_launch": 1.5e8, "command": "ncu ..."}))
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(rec))
    assert bench.profiled_traffic() == 1.5e8
    # once the kernel source differs from the one the counters were taken on,
    # the traffic is reported as unknown
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "ffffffffffffffff")
    assert bench.profiled_traffic() is None
    # a missing or malformed record is unknown too
    rec.write_text("{}")
    assert bench.profiled_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(tmp_path / "absent.json"))
    assert bench.profiled_traffic() is None


def test_committed_traffic_record_is_well_formed():
    if not os.path.exists(bench.TRAFFIC_JSON):
        pytest.skip("no traffic record committed")
    with open(bench.TRAFFIC_JSON) as f:
        rec = json.load(f)
    assert len(rec["source_sha256_16"]) == 16
    assert float(rec["dram_bytes_per_launch"]) > 0
    assert rec["command"].startswith("ncu ") and "--clock-control none" in rec["command"]


def test_source_hash_covers_the_layout_code():
    # the hash covers the kernel and the layout-deciding part of the setup only
    src = os.path.join(os.path.dirname(bench.__file__), "paper_1606_00545_gb300", "csrc",
                       "hec_setup.cpp")
    assert bench.LAYOUT_MARKER in open(src, "rb").read()
