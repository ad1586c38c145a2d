"""Host logic of bench.py's roofline report, on CPU: which query kernel is reported, its
algorithmic work, the roofs it is measured against, and the committed ncu record that is
shown only for the source and workload it was measured on."""
import hashlib
import json
import os

import pytest

import bench


def _write_record(tmp_path, text, rec_for):
    src_dir = tmp_path / "paper_2508_19891_gb300" / "csrc"
    src_dir.mkdir(parents=True, exist_ok=True)
    (tmp_path / "profiles").mkdir(exist_ok=True)
    src = src_dir / "query.cu"
    src.write_text(text)
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    rec = {k: {"source": "query.cu", "source_sha": sha, "workloads": v} for k, v in rec_for.items()}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    return src


def test_longer_kernel_is_reported_with_its_roof():
    S, H = 1_000_000, 300_000
    agg = {"count": (2, 4.0), "write": (2, 6.0)}   # per launch: count 2 ms, write 3 ms
    dom, others = bench.query_rooflines(agg, S, H, 2, 1000.0, "measured", "no-such-workload", 100, 2000.0)
    assert dom["kernel"] == "write_kernel" and [o["kernel"] for o in others] == ["count_kernel"]
    # write: HBM-bound, 8 B per reported id, nothing for the hit mask
    assert dom["bound"] == "hbm" and dom["algorithmic_bytes"] == 8 * H
    assert dom["avg_launch_ms"] == pytest.approx(3.0)
    assert dom["achieved"] == pytest.approx(8 * H / 3e-3 / 1e9)
    assert dom["frac"] == pytest.approx(dom["achieved"] / 1000.0)
    assert dom["traffic"] is None and dom["dram_frac"] is None      # no record for this workload
    # count: issue-bound, 8 warp instructions per 32 scanned points against 4 per SM and cycle
    cnt = others[0]
    assert cnt["bound"] == "alu"
    assert cnt["algorithmic_inst"] == pytest.approx(8 * S / 32)
    assert cnt["peak"] == pytest.approx(100 * 4 * 2000e6 / 1e9)
    assert cnt["achieved"] == pytest.approx(8 * S / 32 / 2e-3 / 1e9)
    assert cnt["effective_gbs"] == pytest.approx(8 * S / 2e-3 / 1e9)
    agg = {"count": (1, 5.0), "write": (1, 1.0)}
    dom, _ = bench.query_rooflines(agg, S, H, 3, 1000.0, "measured")
    assert dom["kernel"] == "count_kernel" and dom["effective_gbs"] == pytest.approx(12 * S / 5e-3 / 1e9)


def test_dram_fraction_from_the_committed_record(tmp_path, monkeypatch):
    _write_record(tmp_path, "// kernel source\n",
                  {"write_kernel": {"w1": {"dram_bytes_per_launch": 6e9, "command": "ncu x"}},
                   "count_kernel": {"w1": {"dram_bytes_per_launch": 2e9, "inst_per_scanned_point": 0.5,
                                           "command": "ncu y"}}})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    agg = {"count": (1, 2.0), "write": (1, 3.0)}
    dom, others = bench.query_rooflines(agg, 10, 10, 2, 4000.0, "measured", "w1")
    assert dom["kernel"] == "write_kernel" and dom["traffic"] == 6e9
    assert dom["dram_gbs"] == pytest.approx(2000.0)
    assert dom["dram_frac"] == pytest.approx(0.5)
    assert dom["dram_frac_nominal"] == pytest.approx(0.25)
    assert others[0]["dram_frac"] == pytest.approx(0.25)
    assert others[0]["executed_inst_per_32_points"] == pytest.approx(16.0)


def test_record_only_for_the_measured_source_and_workload(tmp_path, monkeypatch):
    src = _write_record(tmp_path, "// kernel source\n",
                        {"write_kernel": {"w1": {"dram_bytes_per_launch": 123}}})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.committed_traffic("write_kernel", "w1")["dram_bytes_per_launch"] == 123
    assert bench.committed_traffic("write_kernel", "w2") is None     # another workload
    assert bench.committed_traffic("count_kernel", "w1") is None     # not recorded
    src.write_text("// kernel source, changed\n")
    assert bench.committed_traffic("write_kernel", "w1") is None     # source changed since


def test_record_hashes_every_listed_source(tmp_path, monkeypatch):
    """A record taken on two source files (the kernels and their header) holds only while
    neither changes."""
    src_dir = tmp_path / "paper_2508_19891_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src_dir / "query.cu").write_text("// kernels\n")
    (src_dir / "query.cuh").write_text("// constants\n")
    sha = hashlib.sha256(b"// kernels\n// constants\n").hexdigest()[:16]
    rec = {"write_kernel": {"source": ["query.cu", "query.cuh"], "source_sha": sha,
                            "workloads": {"w1": {"dram_bytes_per_launch": 5}}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.committed_traffic("write_kernel", "w1")["dram_bytes_per_launch"] == 5
    (src_dir / "query.cuh").write_text("// constants, changed\n")
    assert bench.committed_traffic("write_kernel", "w1") is None


def test_committed_record_has_both_query_kernels():
    """The committed record covers both query kernels, each with its source and the ncu
    command of every workload it holds."""
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for k in ("count_kernel", "write_kernel"):
        e = rec[k]
        assert e["source"] == ["query.cu", "query.cuh"] and len(e["source_sha"]) == 16
        assert e["workloads"]
        for w, r in e["workloads"].items():
            assert w in bench.WORKLOADS
            assert r["dram_bytes_per_launch"] > 0 and r["command"].startswith("ncu ")
            assert "--clock-control none" in r["command"]


def test_default_workload_is_the_learned_bounds_configuration():
    a = bench.parse([])
    assert a.workload == "mixed-1e8" and a.steps >= 10 and a.warmup >= 3
    assert bench.instance_seed(0) == 4 and bench.instance_seed(1) != 4


def test_tuning_flag():
    """--tuning CHUNK,BATCH,QBATCH pins the scan settings (with an explicit cover); malformed or
    misplaced uses are refused while parsing, before any work."""
    assert bench.pinned_tuning(bench.parse(["--tuning", "4096,16,2", "--cover", "1"])) == (4096, 16, 2)
    assert bench.pinned_tuning(bench.parse([])) is None
    for argv in (["--tuning", "4096,16,2"],                      # the autotuner would pick the cover
                 ["--tuning", "4096,16", "--cover", "1"],
                 ["--tuning", "4096,16,x", "--cover", "1"],
                 ["--tuning", "4096,16,2", "--cover", "1", "--workload", "dynamic-5e7"]):
        with pytest.raises(SystemExit):
            bench.parse(argv)
