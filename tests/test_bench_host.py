"""Host logic of bench.py (no GPU): the DRAM traffic taken from the committed ncu summary is
reported only while the kernel's sources still hash to the value recorded with it."""
import json
import os
import shutil

import bench


def test_traffic_follows_the_sources(tmp_path, monkeypatch):
    root = tmp_path
    os.makedirs(root / "profiles")
    entry = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    key = "k_tc_gemm<KIND_CC,EPI_H> (stage 2)"
    for f in entry[key]["src_files"]:
        os.makedirs(root / os.path.dirname(f), exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, f), root / f)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), root / "profiles" / "traffic.json")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_traffic(key) == entry[key]["bytes"]
    # any change to a source the counters were taken from makes the figure stale
    with open(root / entry[key]["src_files"][0], "a") as fh:
        fh.write("\n")
    assert bench.kernel_traffic(key) is None
    assert bench.kernel_traffic("no such kernel") is None


def test_whole_job_value_is_all_ranks_over_the_slowest():
    # 2 ranks, 10 steps of 1e6 units each, slowest rank 5 ms in total: 4e9 units/s = 4 G
    assert abs(bench.whole_job_value(1e6, 10, 2, 5.0) - 4.0) < 1e-12
