"""Host logic of bench.py (no GPU): the DRAM traffic taken from the committed ncu summary is
reported only while the kernel's sources still hash to the value recorded with it; the
whole-job value; the clock record taken beside each number (from a fake nvidia-smi)."""
import json
import os

import bench


def test_traffic_follows_the_sources(tmp_path, monkeypatch):
    import hashlib
    root = tmp_path
    os.makedirs(root / "profiles")
    os.makedirs(root / "src")
    files = ["src/a.cu", "src/b.cuh"]
    for k, f in enumerate(files):
        (root / f).write_text(f"// kernel source {k}\n")
    h = hashlib.sha256()
    for f in files:
        h.update((root / f).read_bytes())
    key = "k_example"
    entry = {key: {"bytes": 12345.0, "source": "profiles/k_example.md", "src_files": files,
                   "src_hash": h.hexdigest()[:16]}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(entry))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_traffic(key) == 12345.0
    # any change to a source the counters were taken from makes the figure stale
    with open(root / files[1], "a") as fh:
        fh.write("\n")
    assert bench.kernel_traffic(key) is None
    assert bench.kernel_traffic("no such kernel") is None


def test_traffic_of_one_kernel_follows_its_definition_only(tmp_path, monkeypatch):
    """With a marker the hash covers the kernel's definition (its line to the next closing
    brace at column 0): edits elsewhere in the file keep the figure, edits inside drop it."""
    import hashlib
    root = tmp_path
    os.makedirs(root / "profiles")
    src = root / "k.cu"
    before = "__global__ void k_other() {\n  x = 1;\n}\n"
    body = "__global__ void k_mine(int* p) {\n  p[0] = 2;\n}\n"
    after = "int tail() {\n  return 3;\n}\n"
    src.write_text(before + body + after)
    entry = {"k_mine": {"bytes": 77.0, "source": "profiles/k.md", "src_files": ["k.cu"], "src_marker": "k_mine(",
                        "src_hash": hashlib.sha256(body.encode()).hexdigest()[:16]}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(entry))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_source_hash(["k.cu"], "k_mine(") == entry["k_mine"]["src_hash"]
    assert bench.kernel_traffic("k_mine") == 77.0
    src.write_text(before.replace("1", "5") + body + after + "// more\n")
    assert bench.kernel_traffic("k_mine") == 77.0
    src.write_text(before + body.replace("2", "4") + after)
    assert bench.kernel_traffic("k_mine") is None


def test_committed_traffic_entries_are_well_formed():
    entry = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for key, e in entry.items():
        assert e["bytes"] > 0 and len(e["src_hash"]) == 16, key
        bench.kernel_source_hash(e["src_files"], e.get("src_marker"))  # the marker is still in the sources
        assert os.path.exists(os.path.join(bench.ROOT, e["source"])), key
        for f in e["src_files"]:
            assert os.path.exists(os.path.join(bench.ROOT, f)), (key, f)


def test_whole_job_value_is_all_ranks_over_the_slowest():
    # 2 ranks, 10 steps of 1e6 units each, slowest rank 5 ms in total: 4e9 units/s = 4 G
    assert abs(bench.whole_job_value(1e6, 10, 2, 5.0) - 4.0) < 1e-12


def _fake_smi(tmp_path, lines):
    exe = tmp_path / "nvidia-smi"
    exe.write_text("#!/bin/sh\ncat <<'END'\n" + "\n".join(lines) + "\nEND\nexec sleep 30\n")
    exe.chmod(0o755)
    return str(tmp_path)


def test_clock_sampler_summarises_clocks_and_throttle_reasons(tmp_path, monkeypatch):
    """The clock record beside a bench number: median SM clock under load, the maximum, and
    every throttle reason seen in any sample (a fake nvidia-smi prints the samples)."""
    t = "2026/12/04 10:00:00.000"
    lines = [f"{t}, 0, 2070, 2070, 800.5, 0x0, Not Active, Not Active, Not Active, Not Active",
             f"{t}, 0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             f"{t}, 0, 1980, 2070, 1200.0, 0x8, Active, Not Active, Not Active, Not Active",
             "garbled line",
             f"{t}, 0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    import time
    time.sleep(0.5)
    s.stop()
    out = s.summary()
    assert out["samples"] == 3  # the garbled and the non-numeric samples are skipped
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070 and out["power_w_max"] == 1390.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi_says_so(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # no nvidia-smi here
    s = bench.ClockSampler(0)
    s.start()
    s.stop()
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
