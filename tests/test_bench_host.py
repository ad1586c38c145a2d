"""Host logic of bench.py's roofline report, on CPU: which query kernel is reported, its
algorithmic bytes, and the committed DRAM traffic that is shown only for the source it was
measured on."""
import hashlib
import json
import os

import pytest

import bench


def test_longer_kernel_is_reported():
    S, H = 1_000_000, 300_000
    agg = {"count": (2, 4.0), "write": (2, 6.0)}   # per launch: count 2 ms, write 3 ms
    dom, others = bench.query_rooflines(agg, S, H, 2, 1000.0, "measured")
    assert dom["kernel"] == "write_kernel" and [o["kernel"] for o in others] == ["count_kernel"]
    assert dom["algorithmic_bytes"] == 8 * H + S // 8
    assert dom["avg_launch_ms"] == pytest.approx(3.0)
    assert dom["achieved"] == pytest.approx((8 * H + S // 8) / 3e-3 / 1e9)
    assert dom["frac"] == pytest.approx(dom["achieved"] / 1000.0)
    cnt = others[0]
    assert cnt["algorithmic_bytes"] == 8 * S + S // 8
    agg = {"count": (1, 5.0), "write": (1, 1.0)}
    dom, _ = bench.query_rooflines(agg, S, H, 3, 1000.0, "measured")
    assert dom["kernel"] == "count_kernel" and dom["algorithmic_bytes"] == 12 * S + S // 8


def test_traffic_only_for_the_measured_source(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2508_19891_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "query.cu"
    src.write_text("// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    rec = {"write_kernel": {"source": "query.cu", "source_sha": sha, "dram_bytes_per_launch": 123}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.committed_traffic("write_kernel", 1) == 123.0
    assert bench.committed_traffic("count_kernel", 1) is None        # not recorded
    src.write_text("// kernel source, changed\n")
    assert bench.committed_traffic("write_kernel", 1) is None        # source changed since


def test_committed_record_has_both_query_kernels():
    """The committed record covers both query kernels, each with its source and command."""
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for k in ("count_kernel", "write_kernel"):
        e = rec[k]
        assert e["source"] == "query.cu" and len(e["source_sha"]) == 16
        assert e["dram_bytes_per_launch"] > 0 and e["command"].startswith("ncu ")
        assert "--clock-control none" in e["command"]
