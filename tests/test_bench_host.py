"""Host logic of bench.py (no GPU): the DRAM traffic taken from the committed ncu summary is
reported only while the kernel's sources still hash to the value recorded with it."""
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
