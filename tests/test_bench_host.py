"""Host-side logic of bench.py (no GPU): the reference arm's JSON line, the
rule that ties a measured DRAM traffic to the kernel's code lines, and the
graph storage flags."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "ba2000",
                        "--steps", "2", "--warmup", "0", "--ref-trees", "4"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "trees/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["config"]["workload"] == "ba2000"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["steps"] == 2 and d["ms_per_step"] > 0


def test_code_hash_ignores_comment_lines_only(tmp_path):
    b = _bench()
    p = tmp_path / "k.cu"
    p.write_text("// header\nint f() {\n    return 1;  // one\n}\n")
    h0 = b.code_hash(str(p))
    p.write_text("// a reworded header\n\n// and a new comment line\nint f() {\n    return 1;  // one\n}\n")
    assert b.code_hash(str(p)) == h0
    p.write_text("// header\nint f() {\n    return 2;  // one\n}\n")
    assert b.code_hash(str(p)) != h0


def test_traffic_is_reported_only_for_the_measured_code(tmp_path, monkeypatch):
    b = _bench()
    src = "walker.cu"
    cur = b.code_hash(os.path.join(ROOT, "paper_2510_20604_gb300", "csrc", src), *b.W_TREES_REGION[1:])
    monkeypatch.setitem(b.TRAFFIC_PER_DRAW, "grid", (250.0, "grid 256x256", src, cur))
    monkeypatch.setitem(b.TRAFFIC_PER_DRAW, "rmat", (99.0, "R-MAT 18", src, "0" * 64))
    assert b.traffic_per_draw("grid1024") == 250.0
    assert b.traffic_per_draw("rmat20") is None          # measured on other code
    assert b.traffic_per_draw("ba2000") is None          # never measured
    for fam, (nbytes, case, s, sha) in b.TRAFFIC_PER_DRAW.items():
        assert nbytes > 0 and case and s.endswith(".cu") and len(sha) == 64


def test_code_hash_of_a_region(tmp_path):
    b = _bench()
    p = tmp_path / "k.cu"
    p.write_text("int a() { return 0; }\n// BEGIN k\nint k() {\n  return 1;\n}\n// END\nint z() { return 2; }\n")
    h0 = b.code_hash(str(p), "BEGIN k", "END")
    p.write_text("int a() { return 5; }\n// BEGIN k\nint k() {\n  return 1;\n}\n// END\nint z() { return 7; }\n")
    assert b.code_hash(str(p), "BEGIN k", "END") == h0      # code outside the region changed
    p.write_text("int a() { return 5; }\n// BEGIN k\nint k() {\n  return 2;\n}\n// END\n")
    assert b.code_hash(str(p), "BEGIN k", "END") != h0


def test_algorithmic_bytes():
    b = _bench()
    assert b.bytes_per_draw(False, False) == 12
    assert b.bytes_per_draw(True, False) == 20
    assert b.bytes_per_draw(True, True) == 28
    # grid 1024^2 at 2000 trees with 42.56e9 draws: 527.5 GB
    got = b.algorithmic_bytes(42.56e9, 2000, 1 << 20, False, False)
    assert abs(got - (42.56e9 * 12 + 2000 * (1 << 20) * 8)) < 1


def test_graph_flags():
    b = _bench()
    import paper_2510_20604_gb300 as rwc
    assert b.graph_flags("rmat24", rwc) == rwc.GRAPH_INT64_OFFSETS
    assert b.graph_flags("grid1024", rwc) == 0
