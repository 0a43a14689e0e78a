"""Host logic of bench.py (no GPU): the reference arm's JSON line, the
digest that ties recorded DRAM traffic to the kernel code, and the reader of
the recorded traffic lines."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "Gedges/s"
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Gedges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.fixture
def source_copy(tmp_path, monkeypatch):
    dst = tmp_path / "paper_1708_07271_gb300" / "csrc"
    dst.mkdir(parents=True)
    for fn in bench.PRODUCT_SOURCES:
        shutil.copy(os.path.join(ROOT, "paper_1708_07271_gb300", "csrc", fn), dst / fn)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return dst


def test_digest_ignores_comments_not_code(source_copy):
    d0 = bench.kernel_source_digest()
    f = source_copy / "kernels.cuh"
    text = f.read_text()
    f.write_text(text + "\n// a remark\n/* a block\n   remark */\n\n")
    assert bench.kernel_source_digest() == d0
    f.write_text(text.replace("namespace bvg {", "namespace bvg {\nconstexpr int kUnused = 1;", 1))
    assert bench.kernel_source_digest() != d0


def test_code_only():
    src = "int a; // x\n/* y\n z */ int b;\n\n   \nint c; /* w */ int d;\n"
    assert bench.code_only(src) == "int a;\n int b;\nint c;  int d;"


def test_profile_traffic_reads_matching_lines(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "a.md").write_text("# x\n\ntraffic_bytes_per_launch: 123456 source: abcdef0123456789 kernel: push_fused k: 1\n")
    (prof / "b.txt").write_text("traffic_bytes_per_launch: 999 source: abcdef0123456789 kernel: pr_gather_pt k: 32\n")
    (prof / "c.csv").write_text("traffic_bytes_per_launch: 5 source: abcdef0123456789 kernel: push_fused k: 1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("push_fused", "abcdef0123456789", 1) == 123456.0
    assert bench.profile_traffic("pr_gather_pt", "abcdef0123456789", 32) == 999.0
    assert bench.profile_traffic("push_fused", "0000000000000000", 1) is None  # another code version
    assert bench.profile_traffic("push_fused", "abcdef0123456789", 32) is None
    assert bench.profile_traffic("pull_fused", "abcdef0123456789", 1) is None
