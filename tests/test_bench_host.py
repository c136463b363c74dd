"""Host logic of bench.py that needs no GPU: the DRAM-traffic figure of the
roofline is reported only for the kernel source it was measured on, the
profile it cites carries the same figure, and the CPU baseline names the
full-size oracle timing only for the workload it was taken on."""
import argparse
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_reported_only_for_the_measured_kernel_source(monkeypatch):
    rec = bench.TRAFFIC["tc_gemm"]
    assert rec["src_hash"] == bench._src_hash("tc_gemm.cu")
    value, src = bench.traffic_for("tc_gemm")
    assert value == rec["bytes_per_launch"] and src == rec["profile"]
    # a capture taken on another kernel source is not reported
    monkeypatch.setitem(bench.TRAFFIC, "tc_gemm", dict(rec, src_hash="0" * 16))
    assert bench.traffic_for("tc_gemm") == (None, None)
    monkeypatch.setitem(bench.TRAFFIC, "tc_gemm", None)
    assert bench.traffic_for("tc_gemm") == (None, None)


def test_traffic_profile_matches_the_recorded_figure():
    rec = bench.TRAFFIC["tc_gemm"]
    with open(os.path.join(ROOT, rec["profile"])) as f:
        text = f.read()
    assert rec["src_hash"] in text
    mb = re.search(r"traffic per launch \(read \+ write\)\*\* \| \*\*([0-9.]+) MB\*\*", text)
    assert mb, "profile states the traffic per launch"
    assert abs(float(mb.group(1)) * 1e6 - rec["bytes_per_launch"]) < 0.1e6
    assert "--clock-control none" in text


def test_cpu_baseline_names_the_full_size_timing_only_for_its_workload():
    args = argparse.Namespace(sample_n=24, n=bench.ORACLE_FULL["n"])
    cb = bench.cpu_baseline(args)
    assert cb["kind"] == "oracle" and cb["extrapolated"] is True and cb["cores"] >= 1
    assert cb["full_size_measured"] == bench.ORACLE_FULL
    assert cb["value"] > 0.0
    args = argparse.Namespace(sample_n=24, n=1024)
    assert bench.cpu_baseline(args)["full_size_measured"] is None
