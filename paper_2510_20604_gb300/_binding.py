"""ctypes marshalling for ``include/rwc.h``.  No computation happens here."""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(HERE, "librwc.so")

MODE_AUTO, MODE_GLOBAL, MODE_SHARED, MODE_WALKER = 0, 1, 2, 3
NPHASE = 6
PHASES = ("init", "walk", "classify", "pop", "finish", "accum")
GRAPH_INT64_OFFSETS, GRAPH_SKIP_CONNECTIVITY = 0x1, 0x2
_STATUS = {0: "OK", 1: "INVALID", 2: "NOT_CONNECTED", 3: "OOM", 4: "NOT_CONVERGED",
           5: "CUDA", 6: "UNSUPPORTED"}


class RWCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rwc status {status} ({_STATUS.get(status, '?')}): {msg}")
        self.status = status


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("root", ctypes.c_int32),
                ("weighted", ctypes.c_int32), ("offsets64", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("vol", ctypes.c_double), ("dmax", ctypes.c_double),
                ("device_bytes", ctypes.c_int64)]


class Options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("trees_per_chunk", ctypes.c_int64), ("use_jumps", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("memory_budget", ctypes.c_int64),
                ("profile", ctypes.c_int32), ("walker_policy", ctypes.c_int32),
                ("max_wait_ns", ctypes.c_int64), ("async_status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def __init__(self, mode=0, max_rounds=0, trees_per_chunk=0, use_jumps=-1, block_threads=0,
                 memory_budget=0, profile=0, walker_policy=0, max_wait_ns=0, async_status=0):
        super().__init__(mode, max_rounds, trees_per_chunk, use_jumps, block_threads,
                         memory_budget, profile, walker_policy, max_wait_ns, async_status, 0)


class Params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("mu", ctypes.c_double), ("t", ctypes.c_double),
                ("theta", ctypes.c_double), ("trees", ctypes.c_int64), ("diameter", ctypes.c_int64),
                ("sweep_end", ctypes.c_int32), ("iterations", ctypes.c_int32)]

    def as_dict(self):
        return {"lambda": self.lambda_, "mu": self.mu, "t": self.t, "theta": self.theta,
                "trees": self.trees, "diameter": self.diameter, "sweep_end": self.sweep_end,
                "iterations": self.iterations}


class Stats(ctypes.Structure):
    _fields_ = [("trees", ctypes.c_int64), ("draws", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("walk_steps", ctypes.c_int64), ("chunks", ctypes.c_int64), ("mode", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("marked", ctypes.c_int64),
                ("phase_ms", ctypes.c_double * NPHASE), ("phase_launches", ctypes.c_int64 * NPHASE),
                ("phase_units", ctypes.c_int64 * NPHASE), ("diag", ctypes.c_int64 * 8)]

    def as_dict(self):
        out = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            out[f] = list(v) if (f.startswith("phase_") or f == "diag") else v
        return out


_lib = None
_vp, _i64, _i32, _u32, _u64, _d = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                   ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double)


def lib():
    """Load librwc.so (raises RWCError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(lib_path):
        raise RWCError(5, f"CUDA library not built: {lib_path} is missing "
                          "(run __graft_entry__.build())")
    L = ctypes.CDLL(lib_path)
    sig = {
        "rwc_last_error": ([], ctypes.c_char_p),
        "rwc_version": ([], ctypes.c_char_p),
        "rwc_launch_count": ([], ctypes.c_int64),
        "rwc_graph_create": ([_i64, _i64, _vp, _vp, _vp, _i32, _u32, ctypes.POINTER(_vp)], _i32),
        "rwc_graph_info": ([_vp, ctypes.POINTER(GraphInfo)], _i32),
        "rwc_graph_destroy": ([_vp], _i32),
        "rwc_sync_status": ([_vp, _vp], _i32),
        "rwc_pivot_solve": ([_vp, ctypes.c_double, _vp, _vp], _i32),
        "rwc_sample_trees": ([_vp, _u64, _i64, _i64, _vp, _vp, _vp, ctypes.POINTER(Options),
                              ctypes.POINTER(Stats), _vp], _i32),
        "rwc_sample_trees_noalloc": ([_vp, _u64, _i64, _i64, _vp, _vp, _vp, _vp], _i32),
        "rwc_estimate": ([_vp, _vp, _i64, _d, _vp, _vp, _vp], _i32),
        "rwc_recover": ([_vp, _vp, _i64, _vp, _vp, _vp], _i32),
        "rwc_solve": ([_vp, _i32, _vp, _vp, _d, ctypes.POINTER(_i32), _vp], _i32),
        "rwc_grad": ([_vp, _vp, _i32, _u64, _d, _vp, _vp], _i32),
        "rwc_batch_create": ([_i32, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)], _i32),
        "rwc_batch_sample": ([_vp, _u64, _i64, _vp, _i32, _i32, ctypes.POINTER(Stats), _vp], _i32),
        "rwc_batch_roots": ([_vp, _vp], _i32),
        "rwc_autotune": ([_vp, ctypes.c_char_p, _vp], _i32),
        "rwc_batch_get_schedule": ([_vp, _vp], _i32),
        "rwc_batch_set_schedule": ([_vp, _i32, _i32, _i32, _i32, _i32], _i32),
        "rwc_batch_destroy": ([_vp], _i32),
        "rwc_mre": ([_i64, _vp, _vp, _vp, _vp], _i32),
        "rwc_auto_params": ([_vp, _d, _i32, _d, ctypes.POINTER(Params), _vp], _i32),
        "rwc_trap_walks": ([_vp, _u64, _i64, _i64, _vp, ctypes.POINTER(_i64), _vp], _i32),
        "rwc_predict_mre": ([_vp, _vp, _i64, _vp, _d, ctypes.POINTER(_d), ctypes.POINTER(_i64), _vp], _i32),
        "rwc_kendall": ([_i64, _vp, _vp, _vp, ctypes.POINTER(_d), _vp], _i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(st: int):
    if st != 0:
        raise RWCError(st, lib().rwc_last_error().decode())


def _dptr(x, dtype=None, name="buffer"):
    """Device pointer of a torch CUDA tensor (or an int), None for None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name}: expected a torch CUDA tensor")
    if not x.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if dtype is not None and x.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {x.dtype}")
    return x.data_ptr()


def _hptr(a, dtype):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def rwc_version() -> str:
    return lib().rwc_version().decode()


def rwc_launch_count() -> int:
    return int(lib().rwc_launch_count())


def rwc_last_error() -> str:
    return lib().rwc_last_error().decode()


def rwc_graph_create(n, nnz, row_ptr, col_idx, w=None, root=-1, flags=0):
    rp, prp = _hptr(row_ptr, np.int64)
    ci, pci = _hptr(col_idx, np.int32)
    ww, pw = _hptr(w, np.float32)
    out = _vp()
    _check(lib().rwc_graph_create(int(n), int(nnz), prp, pci, pw, int(root), int(flags),
                                  ctypes.byref(out)))
    return out.value


def rwc_graph_info(g) -> GraphInfo:
    info = GraphInfo()
    _check(lib().rwc_graph_info(g, ctypes.byref(info)))
    return info


def rwc_graph_destroy(g):
    _check(lib().rwc_graph_destroy(g))


def rwc_sample_trees(g, seed, tree0, num_trees, sums, parents=None, visits=None, opt=None,
                     stream=None):
    """Returns the call's Stats; None for an asynchronous call (opt.async_status
    = 1), whose device-side errors rwc_sync_status reports."""
    import torch
    asy = opt is not None and opt.async_status != 0
    st = None if asy else Stats()
    _check(lib().rwc_sample_trees(g, int(seed), int(tree0), int(num_trees),
                                  _dptr(sums, torch.float64, "sums"),
                                  _dptr(parents, torch.int32, "parents"),
                                  _dptr(visits, torch.int32, "visits"),
                                  ctypes.byref(opt) if opt is not None else None,
                                  ctypes.byref(st) if st is not None else None, _stream(stream)))
    return st


def rwc_sync_status(g, stream=None):
    """Synchronise the stream and raise the device-side error of the graph's
    asynchronous sampling calls, if any (the status word is cleared)."""
    _check(lib().rwc_sync_status(g, _stream(stream)))


def rwc_sample_trees_noalloc(g, seed, tree0, num_trees, sums, parents=None, visits=None,
                             stream=None):
    """Same trees as rwc_sample_trees, with all scratch in the library's static
    device array (no allocation during the call)."""
    import torch
    _check(lib().rwc_sample_trees_noalloc(g, int(seed), int(tree0), int(num_trees),
                                          _dptr(sums, torch.float64, "sums"),
                                          _dptr(parents, torch.int32, "parents"),
                                          _dptr(visits, torch.int32, "visits"), _stream(stream)))


def rwc_estimate(g, sums, num_trees, cg_tol, H_out, y_out=None, stream=None):
    import torch
    _check(lib().rwc_estimate(g, _dptr(sums, torch.float64, "sums"), int(num_trees),
                              float(cg_tol), _dptr(H_out, torch.float64, "H_out"),
                              _dptr(y_out, torch.float64, "y_out"), _stream(stream)))


def rwc_pivot_solve(g, cg_tol, y, stream=None):
    import torch
    _check(lib().rwc_pivot_solve(g, float(cg_tol), _dptr(y, torch.float64, "y"), _stream(stream)))


def rwc_recover(g, sums, num_trees, y, H_out, stream=None):
    import torch
    _check(lib().rwc_recover(g, _dptr(sums, torch.float64, "sums"), int(num_trees),
                             _dptr(y, torch.float64, "y"), _dptr(H_out, torch.float64, "H_out"),
                             _stream(stream)))


def rwc_solve(g, k, B, X, tol, stream=None) -> int:
    import torch
    it = _i32(0)
    _check(lib().rwc_solve(g, int(k), _dptr(B, torch.float64, "B"), _dptr(X, torch.float64, "X"),
                           float(tol), ctypes.byref(it), _stream(stream)))
    return it.value


def rwc_grad(g, c, k, sketch_seed, cg_tol, grad_w, stream=None):
    import torch
    _check(lib().rwc_grad(g, _dptr(c, torch.float64, "c"), int(k), int(sketch_seed),
                          float(cg_tol), _dptr(grad_w, torch.float32, "grad_w"), _stream(stream)))


def rwc_batch_create(G, graph_offsets, row_ptr, col_idx, w=None):
    go, pgo = _hptr(graph_offsets, np.int64)
    rp, prp = _hptr(row_ptr, np.int64)
    ci, pci = _hptr(col_idx, np.int32)
    ww, pw = _hptr(w, np.float32)
    out = _vp()
    _check(lib().rwc_batch_create(int(G), pgo, prp, pci, pw, ctypes.byref(out)))
    return out.value


def rwc_batch_sample(b, seed, trees_per_graph, sums, use_graph=1, per_graph_launch=0,
                     stream=None) -> Stats:
    import torch
    st = Stats()
    _check(lib().rwc_batch_sample(b, int(seed), int(trees_per_graph),
                                  _dptr(sums, torch.float64, "sums"), int(use_graph),
                                  int(per_graph_launch), ctypes.byref(st), _stream(stream)))
    return st


def rwc_batch_roots(b, G) -> np.ndarray:
    out = np.zeros(G, np.int32)
    _check(lib().rwc_batch_roots(b, out.ctypes.data))
    return out


def rwc_autotune(b, cache_path=None, stream=None):
    _check(lib().rwc_autotune(b, cache_path.encode() if cache_path else None, _stream(stream)))


def rwc_batch_get_schedule(b) -> tuple:
    """(large-class threads per block, split: largest n of the small class,
    trees per item, small class warp-per-tree, classes concurrent)."""
    out = np.zeros(5, np.int32)
    _check(lib().rwc_batch_get_schedule(b, out.ctypes.data))
    return tuple(int(x) for x in out)


def rwc_batch_set_schedule(b, threads, split, tile, warp=1, concurrent=1):
    _check(lib().rwc_batch_set_schedule(b, int(threads), int(split), int(tile), int(warp), int(concurrent)))


def rwc_batch_destroy(b):
    _check(lib().rwc_batch_destroy(b))


def rwc_trap_walks(g, seed, walks_per_node, sums, max_steps=1 << 32, stream=None) -> int:
    """Straightforward trap-walk estimator: sums[u] += visits to u of
    walks_per_node walks from u stopped at the pivot.  Returns total steps."""
    import torch
    steps = _i64(0)
    _check(lib().rwc_trap_walks(g, int(seed), int(walks_per_node), int(max_steps),
                                _dptr(sums, torch.float64, "sums"), ctypes.byref(steps), _stream(stream)))
    return steps.value


def rwc_predict_mre(g, sums, num_trees, H, target=0.01, stream=None):
    """(predicted MRE of the estimate H from num_trees trees, trees needed for
    the target MRE) by the variance law of the visit counts."""
    import torch
    m = _d(0.0)
    t = _i64(0)
    _check(lib().rwc_predict_mre(g, _dptr(sums, torch.float64, "sums"), int(num_trees),
                                 _dptr(H, torch.float64, "H"), float(target), ctypes.byref(m),
                                 ctypes.byref(t), _stream(stream)))
    return m.value, t.value


def rwc_auto_params(g, eps, max_iters=0, tol=0.0, stream=None) -> Params:
    """Sample size, solver accuracy, lambda and diameter for graph g."""
    p = Params()
    _check(lib().rwc_auto_params(g, float(eps), int(max_iters), float(tol), ctypes.byref(p),
                                 _stream(stream)))
    return p


def rwc_mre(H, H_est, out=None, stream=None):
    """Mean relative error of H_est against H (device FP64 [n]); returns the
    device scalar ``out`` (allocated when None)."""
    import torch
    n = H.numel()
    if H_est.numel() != n:
        raise ValueError("H and H_est differ in length")
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=H.device)
    _check(lib().rwc_mre(n, _dptr(H, torch.float64, "H"), _dptr(H_est, torch.float64, "H_est"),
                         _dptr(out, torch.float64, "out"), _stream(stream)))
    return out


def rwc_kendall(a, b, stream=None):
    """Kendall distance K of the rankings a, b (device FP64 [n]) and the exact
    alpha - beta; returns (K, alpha_minus_beta)."""
    import torch
    n = a.numel()
    if b.numel() != n:
        raise ValueError("a and b differ in length")
    diff = torch.empty((), dtype=torch.int64, device=a.device)
    tau = ctypes.c_double(0.0)
    _check(lib().rwc_kendall(n, _dptr(a, torch.float64, "a"), _dptr(b, torch.float64, "b"),
                             _dptr(diff, torch.int64, "out_diff"), ctypes.byref(tau), _stream(stream)))
    return tau.value, int(diff.item())
