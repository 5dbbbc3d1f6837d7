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
                        "--steps", "1", "--warmup", "0", "--ref-budget", "0.5"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "trees/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["config"]["workload"] == "ba2000"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_code_hash_ignores_comment_lines_only(tmp_path):
    b = _bench()
    p = tmp_path / "k.cu"
    p.write_text("// header\nint f() {\n    return 1;  // one\n}\n")
    h0 = b.code_hash(str(p))
    p.write_text("// a reworded header\n\n// and a new comment line\nint f() {\n    return 1;  // one\n}\n")
    assert b.code_hash(str(p)) == h0
    p.write_text("// header\nint f() {\n    return 2;  // one\n}\n")
    assert b.code_hash(str(p)) != h0


def test_traffic_is_reported_only_for_the_measured_code():
    b = _bench()
    key = ("grid1024+rmat20", "w_trees")
    assert key in b.TRAFFIC
    nbytes, src, sha = b.TRAFFIC[key]
    assert nbytes > 0
    cur = b.code_hash(os.path.join(ROOT, "paper_2510_20604_gb300", "csrc", src))
    assert b.traffic_for(*key) == (nbytes if cur == sha else None)
    assert b.traffic_for("no-such-workload", "w_trees") is None


def test_graph_flags():
    b = _bench()
    import paper_2510_20604_gb300 as rwc
    assert b.graph_flags("rmat24", rwc) == rwc.GRAPH_INT64_OFFSETS
    assert b.graph_flags("grid1024", rwc) == 0
