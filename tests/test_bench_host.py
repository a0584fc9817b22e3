"""CPU tests of bench.py's host logic: the clock record taken during the
timed region (median SM clock, throttle reasons, the rejection rule), the
traffic figure read from the committed ncu record only while the kernel
source it was taken on is unchanged, and the algorithmic byte counts behind
the roofline figures."""
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


def test_trsv_method_bytes_counts_every_block_row():
    """The triangular-solve roofline's byte count: every stored factor entry
    (strict L, U with its diagonal) as value + int32 index, 4 values per block
    row (r read, y written and read back, z written) and 4 bytes per row and
    per level, recounted here from the factor and level queries of a small
    host-only preconditioner."""
    import numpy as np
    from paper_1606_00545_gb300 import hecgpu as H, synth
    A = synth.diffusion3d_7pt_lognormal(10, 2.0, 2)
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, 1, 4, 1)
    H.level_schedule(P)
    for vb in (8, 4):
        want = 0
        for b in range(4):
            rp, ci, _, _ = P.factor(b)
            rows = len(rp) - 1
            levels = sum(len(P.levels(b, w)[0]) - 1 for w in (H.FACTOR_L, H.FACTOR_U))
            want += len(ci) * (vb + 4) + rows * 4 * vb + 4 * (rows + levels)
        assert bench.trsv_method_bytes(H, P, vb) == want
    # it counts every row; the kernel's own count covers the needed rows only
    assert bench.trsv_method_bytes(H, P, 8) >= P.info()["apply_bytes"]


def test_c4_bytes_charges_the_third_gram_schmidt_pass():
    """Each Arnoldi step that took the third (re-orthogonalising) pass adds
    j + 3 vector passes at the cycle's mean j: with every step of a 30-step
    cycle re-orthogonalised, 30 * (14.5 + 3) vectors of n * nrhs FP32 values."""
    from paper_1606_00545_gb300 import synth
    Bs = synth.batch_diffusion2d(3, 16, 20, 2.0, 7)
    base = [{"iters": 30, "cycles": 1, "reorth": 0} for _ in range(3)]
    full = [{"iters": 30, "cycles": 1, "reorth": 30} for _ in range(3)]
    extra = bench.c4_bytes(Bs, full, 4, 30) - bench.c4_bytes(Bs, base, 4, 30)
    want = sum(30 * (29 / 2 + 3) * float(Bs.sys_ptr[s + 1] - Bs.sys_ptr[s]) * 4 * 4
               for s in range(3))
    assert abs(extra - want) <= 1e-9 * want
