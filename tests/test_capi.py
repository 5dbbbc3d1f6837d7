"""C ABI: the library builds, loads and exports every symbol include/rwc.h
declares; host-side validation rejects malformed graphs before touching the
device (so these run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2510_20604_gb300 as rwc
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "rwc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:rwc_status|const char \*|int64_t)\s*(rwc_\w+)\s*\(", txt, re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2510_20604_gb300 import _build
    _build.build()
    L = ctypes.CDLL(rwc.lib_path)
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    assert "sm_103a" in rwc.rwc_version()


def test_binding_names_match_header():
    for s in declared_symbols():
        assert hasattr(rwc, s), s


def _create(rp, col, w=None, root=-1, flags=0):
    return rwc.rwc_graph_create(len(rp) - 1, rp[-1], np.array(rp, np.int64),
                                np.array(col, np.int32), w, root, flags)


@pytest.mark.parametrize("rp,col,w,why", [
    ([0, 1], [0], None, "n must be >= 2"),
    ([0, 2, 3], [0, 1, 0], None, "self-loop"),
    ([0, 1, 1], [1], None, "isolated|reverse"),
    ([0, 2, 3, 4], [2, 1, 0, 0], None, "sorted"),
    ([0, 2, 1, 2], [1, 2], None, "decreases"),
    ([0, 1, 2, 2], [1, 0], None, "isolated|reverse"),
    ([0, 1, 2], [1, 0], np.array([1.0, 2.0], np.float32), "different weights"),
    ([0, 1, 2], [1, 0], np.array([-1.0, -1.0], np.float32), "positive"),
    ([0, 1, 2], [1, 0], np.array([np.nan, np.nan], np.float32), "positive"),
    ([0, 2, 3, 4], [1, 2, 0, 1], None, "reverse"),
    ([0, 1, 2], [5, 0], None, "out of range"),
])
def test_validation_rejects(rp, col, w, why):
    with pytest.raises(rwc.RWCError) as e:
        _create(rp, col, w)
    assert e.value.status == 1
    assert re.search(why, str(e.value)), str(e.value)


def test_disconnected_graph_rejected():
    a = synth.from_edges(4, [0, 2], [1, 3])   # two components
    with pytest.raises(rwc.RWCError) as e:
        _create(a.row_ptr, a.col)
    assert e.value.status == 2


def test_bad_root_rejected():
    g = synth.path(5)
    with pytest.raises(rwc.RWCError) as e:
        _create(g.row_ptr, g.col, root=7)
    assert e.value.status == 1


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2510_20604_gb300 import _binding
    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding, "lib_path", "/nonexistent/librwc.so")
    with pytest.raises(rwc.RWCError):
        _binding.lib()


def test_evaluation_and_walk_entry_points_reject_bad_arguments():
    """Argument checks of rwc_mre, rwc_kendall, rwc_trap_walks and
    rwc_auto_params happen on the host, before any device work."""
    L = rwc.lib()
    d = ctypes.c_double(0.0)
    # rwc_mre: n >= 1 and non-NULL pointers
    assert L.rwc_mre(0, 8, 8, 8, None) == 1
    assert L.rwc_mre(5, None, 8, 8, None) == 1
    # rwc_kendall: 0 <= n <= 2^26, out pointer required
    assert L.rwc_kendall(-1, 8, 8, 8, None, None) == 1
    assert L.rwc_kendall((1 << 26) + 1, 8, 8, 8, None, None) == 1
    assert L.rwc_kendall(10, 8, 8, None, None, None) == 1
    assert "2^26" in rwc.rwc_last_error() or "NULL" in rwc.rwc_last_error()
    # rwc_trap_walks / rwc_auto_params: a graph is required
    assert L.rwc_trap_walks(None, 1, 4, 100, 8, None, None) == 1
    assert L.rwc_auto_params(None, 0.1, 0, 0.0, None, None) == 1


def test_status_pivot_and_sampling_entry_points_reject_bad_arguments():
    """rwc_sync_status, rwc_pivot_solve, rwc_sample_trees and the allocation-
    free sampler check their handles and ranges on the host, before any
    device work."""
    L = rwc.lib()
    assert L.rwc_sync_status(None, None) == 1
    assert "NULL" in rwc.rwc_last_error()
    assert L.rwc_pivot_solve(None, 1e-10, 8, None) == 1
    assert L.rwc_sample_trees(None, 1, 0, 4, 8, None, None, None, None, None) == 1
    assert L.rwc_sample_trees_noalloc(None, 1, 0, 4, 8, None, None, None) == 1
    assert L.rwc_estimate(None, 8, 4, 1e-10, 8, None, None) == 1
    assert L.rwc_recover(None, 8, 4, 8, 8, None) == 1


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of rwc_graph_info_t, rwc_options_t, rwc_stats_t and
    rwc_params_t have the C structs' sizes and field offsets (a C program
    compiled against include/rwc.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2510_20604_gb300 import _binding as B
    pairs = [("rwc_graph_info_t", B.GraphInfo), ("rwc_options_t", B.Options),
             ("rwc_stats_t", B.Stats), ("rwc_params_t", B.Params)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rwc.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
