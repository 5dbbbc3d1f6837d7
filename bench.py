#!/usr/bin/env python3
"""FastWalk hot-path benchmark on GB300.

One step = the whole hot path on every graph of the workload: sample T rooted
spanning trees (visit counts into FP64 sums) and run the pivot solve plus
recovery (Algorithm 1), with the graph already resident in HBM.  The default
workload is the 1024x1024 grid and the scale-20 R-MAT graph, 2000 trees each.

value    = trees per second over the timed steps (all ranks).
e2e      = the same metric through the public API from host buffers: graph
           upload from pinned host memory (rwc_graph_create), sampling,
           estimate, and the read-back of H, every step.
roofline = the sampler's algorithmic bytes (per successor draw: row bounds,
           arc head and, for weighted rows, the alias entry; per tree and
           vertex: parent and visit count) over the device time of its
           kernels, against the measured HBM copy bandwidth; the walker's own
           state-word traffic and the ncu-measured DRAM traffic are reported
           beside it.
extras   = the paper-size R-MAT 24 (500 trees), the 4096-graph batch
           (persistent launch against one launch per graph) and the gradient
           on the 1e5-vertex geometric graph, measured in the same run.

Under torchrun each rank samples its own tree range (weak scaling) and the
ranks add their visit sums before the estimate.  `--impl reference` times
the CPU oracle (sequential Wilson) on a bounded sample of the same workload
per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
T_START = time.perf_counter()
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: [(graph key, trees)]
    "grid1024+rmat20": [("grid1024", 2000), ("rmat20", 2000)],
    "grid1024": [("grid1024", 2000)],
    "rmat20": [("rmat20", 2000)],
    "ba2000": [("ba2000", 1000)],
    "grid512": [("grid512", 64)],
    # small cases of the default workload's graph families, for ncu captures
    "grid256": [("grid256", 2000)],
    "rmat18-2000": [("rmat18", 2000)],
    "rmat18": [("rmat18", 512)],
    "batch4096": [("batch4096", 256)],
    "rmat24": [("rmat24", 500)],
    # accuracy sweep (not a throughput workload): eps in EPS_SWEEP
    "eps-sweep": [("ba2000", 0)],
}
EPS_SWEEP = (0.3, 0.2, 0.1, 0.05, 0.02, 0.01)

PHASE_NAMES = ("init", "walk", "classify", "pop", "finish", "accum")
KERNEL_NAMES = {1: {"init": "g_init", "walk": "g_walk", "pop": "g_pop", "accum": "g_accum"},
                2: {"walk": "s_trees"},
                3: {"init": "w_init", "walk": "w_trees", "accum": "w_accum"}}


def bytes_per_draw(weighted, off64):
    """Algorithmic bytes of one successor draw (the method's own traffic): the
    row bounds of the vertex (2 x int32, or 2 x int64 offsets), the chosen
    arc's head (int32) and, for weighted rows, its alias threshold and alias
    (uint32 + int32)."""
    return (16 if off64 else 8) + 4 + (8 if weighted else 0)


# Per (tree, vertex): the tree's parent (int32) and visit count (int32).
BYTES_PER_TREE_VERTEX = 8
# Implementation traffic of the concurrent-walker sampler, not counted above:
# each draw reads and writes back the vertex's 8-byte state word.
IMPL_BYTES_PER_DRAW = 16


def algorithmic_bytes(draws, trees, n, weighted, off64):
    return draws * bytes_per_draw(weighted, off64) + trees * n * BYTES_PER_TREE_VERTEX


# DRAM traffic of the walker kernel per successor draw, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch divided by its
# draws) on a small case of each graph family; the benchmark scales it by the
# draws of its own launches.  Valid only for the kernel source it was measured
# on (code_hash of the .cu file), else reported as null.
TRAFFIC_PER_DRAW = {
    # family: (bytes per draw, case captured, source file, code hash of the kernel region)
    "grid": (266.2, "grid 256x256, 2000 trees, 64 walkers per tree: one w_trees launch "
                     "(565.0 GB over 2.123e9 draws)", "walker.cu",
             "ab1fdc759f922dfae00450c5610e7341609c15fbdcdfceea4077a8a0d4278a2e"),
    "rmat": (222.3, "R-MAT scale 18, 2000 trees, 64 walkers per tree: one w_trees launch "
                     "(171.0 GB over 7.693e8 draws)", "walker.cu",
             "ab1fdc759f922dfae00450c5610e7341609c15fbdcdfceea4077a8a0d4278a2e"),
}


def code_hash(path, begin=None, end=None):
    """SHA-256 of a source file's code: every line except blank lines and
    lines that hold only a // comment (so that rewording a comment keeps a
    measurement, while any change to the code voids it).  With begin/end,
    only the lines from the first line containing `begin` up to (not
    including) the first later line containing `end`: the measured kernel."""
    import hashlib
    lines = [ln.rstrip() for ln in open(path, encoding="utf-8")]
    if begin is not None:
        i = next(k for k, ln in enumerate(lines) if begin in ln)
        j = next((k for k in range(i + 1, len(lines)) if end in lines[k]), len(lines))
        lines = lines[i:j]
    code = [ln for ln in lines if ln.strip() and not ln.strip().startswith("//")]
    return hashlib.sha256("\n".join(code).encode()).hexdigest()


# the walker kernel's source region in walker.cu (what a traffic capture measured)
W_TREES_REGION = ("walker.cu", "struct DrawRow {",
                  "// visits_u = k_u + 1 over the chunk's trees")


def family(key):
    return "grid" if key.startswith("grid") else "rmat" if key.startswith("rmat") else key


def traffic_per_draw(key):
    """Measured DRAM bytes per draw of the walker kernel for this graph's
    family, or None (no capture, or the kernel changed since)."""
    ent = TRAFFIC_PER_DRAW.get(family(key))
    if not ent:
        return None
    nbytes, _case, src, sha = ent
    path = os.path.join(ROOT, "paper_2510_20604_gb300", "csrc", src)
    try:
        cur = code_hash(path, W_TREES_REGION[1], W_TREES_REGION[2])
    except (OSError, StopIteration):
        return None
    return nbytes if cur == sha else None


def make_graph(key):
    import synth
    if key == "grid1024":
        return synth.grid2d(1024, 1024)
    if key == "grid512":
        return synth.grid2d(512, 512)
    if key == "grid256":
        return synth.grid2d(256, 256)
    if key == "rmat20":
        return synth.rmat(20, 16, seed=0)
    if key == "rmat18":
        return synth.rmat(18, 16, seed=0)
    if key == "rmat24":
        return synth.rmat(24, 16, seed=0, sigma=1.0)
    if key == "ba2000":
        return synth.ba(2000, 3, seed=0)
    raise KeyError(key)


def graph_flags(key, rwc):
    """R-MAT 24 is stored with int64 arc offsets (its configuration asks for them)."""
    return rwc.GRAPH_INT64_OFFSETS if key == "rmat24" else 0


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.out = os.path.join("/tmp", f"rwc_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.out, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(workload, budget_s=20.0, graphs=None):
    """Oracle sequential Wilson on the host cores, bounded sample per graph
    (graphs: key -> graph already built, else made here).  Returns (trees/s
    for the workload's tree mix, details)."""
    from oracle import wilson as ow
    cores = ow.cores()
    per_tree = {}
    detail = []
    for key, T in WORKLOADS[workload]:
        g = graphs[key] if graphs else make_graph(key)
        s = ow.Sampler(g, seed=1)
        done, t_used, draws = 0, 0.0, 0
        tree0 = 1_000_000
        while t_used < budget_s / len(WORKLOADS[workload]) and done < T:
            k = min(cores, T - done)
            t0 = time.perf_counter()
            out = s.sample(tree0 + done, k, nthreads=cores)
            t_used += time.perf_counter() - t0
            done += k
            draws += out["draws"]
        per_tree[key] = t_used / done
        detail.append(f"{key}: {done} trees ({draws} draws) in {t_used:.2f} s")
    total_T = sum(T for _, T in WORKLOADS[workload])
    est = sum(per_tree[key] * T for key, T in WORKLOADS[workload])
    return total_T / est, cores, "; ".join(detail) + " (all cores, one tree per thread; scaled to the full tree counts)"


def cpu_single_thread(workload, budget_s=5.0, graphs=None):
    """The oracle on one host thread (the paper's setting), one tree at a
    time, bounded sample per graph (graphs as in cpu_baseline).  Returns
    (trees/s for the workload's tree mix, details)."""
    from oracle import wilson as ow
    per_tree = {}
    detail = []
    for key, T in WORKLOADS[workload]:
        g = graphs[key] if graphs else make_graph(key)
        s = ow.Sampler(g, seed=1)
        done, t_used, draws = 0, 0.0, 0
        while t_used < budget_s / len(WORKLOADS[workload]) and done < T:
            t0 = time.perf_counter()
            out = s.sample(2_000_000 + done, 1, nthreads=1)
            t_used += time.perf_counter() - t0
            done += 1
            draws += out["draws"]
        per_tree[key] = t_used / done
        detail.append(f"{key}: {done} trees ({draws} draws) in {t_used:.2f} s")
    total_T = sum(T for _, T in WORKLOADS[workload])
    est = sum(per_tree[key] * T for key, T in WORKLOADS[workload])
    return total_T / est, "; ".join(detail) + " (one thread; scaled to the full tree counts)"


def run_reference(args, rank):
    """The oracle (sequential Wilson, C, one tree per host thread) on a
    bounded sample of the workload per step: two trees per host core of every
    graph, so a step keeps the workload's mix of graphs.  value = trees of the
    step over its wall time, averaged over the timed steps."""
    if rank != 0:
        return
    from oracle import wilson as ow
    cores = ow.cores()
    built = {key: make_graph(key) for key, _ in WORKLOADS[args.workload]}
    samplers = {key: ow.Sampler(g, seed=1) for key, g in built.items()}
    per_graph = max(1, min(2 * cores, args.ref_trees)) if args.ref_trees else 2 * cores
    next_tree = {key: 1_000_000 for key in built}

    def ref_step():
        t0 = time.perf_counter()
        trees = 0
        for key, T in WORKLOADS[args.workload]:
            k = min(per_graph, T)
            samplers[key].sample(next_tree[key], k, nthreads=cores)
            next_tree[key] += k
            trees += k
        return trees, time.perf_counter() - t0

    for _ in range(args.warmup):
        ref_step()
    vals, secs = [], []
    trees = 0
    for _ in range(args.steps):
        trees, dt = ref_step()
        vals.append(trees / dt)
        secs.append(dt)
    value = float(np.mean(vals))
    sample = (f"{trees} trees per step ({', '.join(f'{min(per_graph, T)} of {key}' for key, T in WORKLOADS[args.workload])}), "
              f"{cores} threads, one tree per thread; {args.steps} steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "trees/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * float(np.mean(secs)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
        "config": {"workload": args.workload, "trees": dict(WORKLOADS[args.workload]),
                   "implementation": "oracle sequential Wilson (CPU), sampling only; each step a bounded "
                                     "sample with the workload's mix of graphs"},
        "cpu_baseline": {"value": value, "unit": "trees/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "trees/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


METRIC = "spanning trees/s and RWC nodes/s at <=1% mean rel err; % of HBM roofline"


def batch_measure(rwc, torch, dev, steps, warmup, world=1):
    """4096 small graphs (sizes log-uniform in [50, 20000], ER / BA / RGG),
    256 trees each, autotuned schedule: one CUDA-graph launch (two persistent
    kernels, one per size class, on forked streams) against one launch per
    graph, same trees, same sums."""
    import synth
    T = WORKLOADS["batch4096"][0][1]
    t0 = time.perf_counter()
    specs = synth.batch_specs(4096, seed=0)
    gs = [synth.batch_graph(i, n, kind, seed=0) for i, (n, kind) in enumerate(specs)]
    B = rwc.Batch(gs)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    B.autotune(None)
    tune_s = time.perf_counter() - t0
    sums = torch.zeros(B.N, dtype=torch.float64, device=dev)
    res = {}
    ref = None
    for name, kw in (("persistent_graph", dict(use_graph=1)), ("per_graph_launch", dict(per_graph_launch=1))):
        for _ in range(warmup):
            sums.zero_()
            B.sample(T, seed=1, sums=sums, **kw)
        torch.cuda.synchronize()
        t = []
        draws = 0
        for _ in range(steps):
            sums.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st = B.sample(T, seed=1, sums=sums, **kw)
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
            draws = st.draws
        if ref is None:
            ref = sums.clone()
        ms = float(np.mean(t))
        res[name] = {"ms_per_step": ms, "trees_per_s": world * 4096 * T / (ms / 1000.0),
                     "nodes_per_s": world * B.N / (ms / 1000.0), "draws_per_step": int(draws),
                     "same_sums": bool(torch.equal(ref, sums))}
    th, split, tile, warp, conc = B.schedule()
    return {"graphs": 4096, "total_vertices": int(B.N), "trees_per_graph": T,
            "schedule": {"large_class_threads": th, "small_class_up_to_n": split,
                         "small_class": "warp-per-tree" if warp else "block-per-tree", "trees_per_item": tile,
                         "classes": "concurrent" if conc else "sequential"},
            "persistent_graph": res["persistent_graph"], "per_graph_launch": res["per_graph_launch"],
            "speedup_vs_per_graph_launch": res["per_graph_launch"]["ms_per_step"] / res["persistent_graph"]["ms_per_step"],
            "steps": steps, "warmup": warmup, "generation_s": gen_s, "autotune_s": tune_s}


def run_batch(args, rwc, torch, dev, world, rank):
    res = batch_measure(rwc, torch, dev, args.steps, args.warmup, world)
    if rank == 0:
        line = {"metric": METRIC, "value": res["persistent_graph"]["trees_per_s"], "unit": "trees/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": res["persistent_graph"]["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
                "config": {"workload": "batch4096", "graphs": 4096, "total_vertices": res["total_vertices"],
                           "trees_per_graph": res["trees_per_graph"]},
                "batch": res}
        print(json.dumps(line), flush=True)


def rmat24_measure(rwc, torch, dev, hbm_peak, steps=2, warmup=1):
    """The paper-size stand-in: R-MAT scale 24, lognormal(0, 1) weights
    through the alias tables, int64 arc offsets, 500 trees per step, sampling
    plus the pivot solve and recovery."""
    key, T = "rmat24", WORKLOADS["rmat24"][0][1]
    t0 = time.perf_counter()
    g = make_graph(key)
    gen_s = time.perf_counter() - t0
    G = rwc.Graph.from_synth(g, flags=graph_flags(key, rwc))
    sums = torch.zeros(g.n, dtype=torch.float64, device=dev)
    opt = rwc.Options(profile=1)

    def one():
        sums.zero_()
        st = rwc.rwc_sample_trees(G.handle, 1, 0, T, sums, None, None, opt)
        return st, G.estimate(sums, T)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    ms, sample_ms, draws = [], [], 0
    H = None
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, H = one()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        sample_ms.append(sum(st.phase_ms))
        draws = st.draws
    mre, T1 = rwc.rwc_predict_mre(G.handle, sums, T, H, target=0.01)
    smp = float(np.mean(sample_ms))
    alg = algorithmic_bytes(draws, T, g.n, True, True)
    out = {"trees": T, "n": g.n, "arcs": g.nnz, "ms_per_step": float(np.mean(ms)),
           "trees_per_s": T / (float(np.mean(ms)) / 1000.0), "sample_ms": smp,
           "draws_per_tree": draws / T, "mre_pred": mre, "trees_for_1pct": int(T1),
           "roofline": {"kernel": "w_trees", "achieved": alg / (smp / 1000.0) / 1e9, "peak": hbm_peak,
                        "unit": "GB/s", "frac": alg / (smp / 1000.0) / 1e9 / hbm_peak,
                        "unit_bytes": {"per_draw": bytes_per_draw(True, True),
                                       "per_tree_vertex": BYTES_PER_TREE_VERTEX}},
           "steps": steps, "warmup": warmup, "generation_s": gen_s}
    del G, sums
    torch.cuda.empty_cache()
    return out


def grad_measure(rwc, torch, dev, steps=3):
    """rwc_grad on the 1e5-vertex random geometric graph (k = 64 sketch
    columns, CG to 1e-8): milliseconds per call; and the sketch's error
    against the exact gradient (k = 0, one solve per vertex) on the
    2000-vertex graph of the same generator, where the exact one is cheap."""
    import synth
    g = synth.rgg(100_000, 12.0, seed=0, sigma=0.5)
    G = rwc.Graph.from_synth(g)
    c = torch.tensor(synth.uniform_vector(g.n, 1), dtype=torch.float64, device=dev)
    G.grad(c, k=64, sketch_seed=77, tol=1e-8)
    torch.cuda.synchronize()
    t = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        G.grad(c, k=64, sketch_seed=77, tol=1e-8)
        e1.record()
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1))
    g2 = synth.rgg(2000, 12.0, seed=0, sigma=0.5)
    G2 = rwc.Graph.from_synth(g2)
    c2 = torch.tensor(synth.uniform_vector(g2.n, 1), dtype=torch.float64, device=dev)
    ex = G2.grad(c2, k=0, tol=1e-10).double()
    errs = []
    for sk_seed in range(8):
        sk = G2.grad(c2, k=64, sketch_seed=sk_seed, tol=1e-10).double()
        errs.append(((sk - ex).norm() / ex.norm()).item())
    med_edge = float(((sk - ex).abs() / ex.abs().clamp_min(1e-300)).median().item())
    return {"n": g.n, "edges": g.nnz // 2, "k": 64, "cg_tol": 1e-8, "ms_per_call": float(np.mean(t)),
            "calls": steps,
            "jl_error_k64": {"graph": "rgg n=2000 (same generator)", "rel_l2_mean_over_8_sketches": float(np.mean(errs)),
                             "rel_l2_min": float(np.min(errs)), "rel_l2_max": float(np.max(errs)),
                             "median_per_edge_rel": med_edge}}


def run_eps_sweep(args, rwc, torch, dev, rank):
    """Runtime, error and ranking quality against the accuracy target eps
    (the paper's Section 6 sweep over eps in [0.01, 0.3], on synthetic
    stand-ins).  The tree-count lemma's l is a worst-case bound (about 3e8
    trees at eps = 0.3 on BA-2000), so each eps gets the trees the variance
    law of the visit counts predicts for a mean relative error of eps
    (fastwalk_to_target).  BA n = 2000: measured MRE and Kendall distance
    against a ground truth of 4e6 trees (predicted MRE ~0.02%; the paper uses
    FastWalk at eps = 1e-4 the same way where no exact solve is possible).
    Grid 512^2 and R-MAT 18: trees and runtime per eps, measured while the
    tree count stays at most 4096, else from the per-tree time of that run."""
    import synth
    res = {}
    g = synth.ba(2000, 3, seed=0)
    G = rwc.Graph.from_synth(g)
    T_gt = 4_000_000
    t0 = time.perf_counter()
    Hgt, _ = rwc.fastwalk(G, T_gt, seed=777)
    torch.cuda.synchronize()
    gt_s = time.perf_counter() - t0
    rows = []
    for eps in EPS_SWEEP:
        rwc.fastwalk_to_target(G, eps, first_trees=8, seed=1)      # warm-up of the same call
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H, T, mre_pred = rwc.fastwalk_to_target(G, eps, first_trees=8, seed=1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        mre = float(rwc.rwc_mre(Hgt, H).item())
        tau, _ = rwc.rwc_kendall(H, Hgt)
        rows.append({"eps": eps, "trees": int(T), "seconds": dt, "mre_measured": mre,
                     "mre_predicted": float(mre_pred), "kendall": tau})
    res["ba2000"] = {"ground_truth_trees": T_gt, "ground_truth_s": gt_s, "rows": rows}
    for key in ("grid512", "rmat18"):
        gk = make_graph(key)
        Gk = rwc.Graph.from_synth(gk)
        T0 = 256
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sums, st, _, _ = Gk.sample(T0, seed=1, opt=rwc.Options(profile=1))
        Hk = Gk.estimate(sums, T0)
        torch.cuda.synchronize()
        base_s = time.perf_counter() - t0
        per_tree_s = sum(st.phase_ms) / 1000.0 / T0
        solve_s = max(0.0, base_s - per_tree_s * T0)
        mre0, _ = rwc.rwc_predict_mre(Gk.handle, sums, T0, Hk, target=0.01)
        krow = []
        for eps in EPS_SWEEP:
            need = max(1, int(np.ceil(T0 * (mre0 / eps) ** 2)))
            if need <= 4096:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                H, T, mp = rwc.fastwalk_to_target(Gk, eps, first_trees=need, seed=1)
                torch.cuda.synchronize()
                krow.append({"eps": eps, "trees": int(T), "seconds": time.perf_counter() - t0,
                             "mre_predicted": float(mp), "measured": True})
            else:
                krow.append({"eps": eps, "trees": need, "seconds": need * per_tree_s + solve_s,
                             "mre_predicted": eps, "measured": False})
        res[key] = {"pilot_trees": T0, "pilot_mre_predicted": float(mre0), "rows": krow}
        del Gk
    if rank == 0:
        line = {"metric": "RWC mean relative error, Kendall distance and runtime against eps",
                "value": rows[-1]["seconds"], "unit": "s at eps=0.01 (BA n=2000)", "n_gpus": 1,
                "steps": 1, "warmup": 1, "higher_is_better": False, "dtype": "int32/f64",
                "data": "synthetic", "config": {"workload": "eps-sweep", "eps": list(EPS_SWEEP)},
                "sweep": res}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid1024+rmat20", choices=list(WORKLOADS))
    ap.add_argument("--trees", type=int, default=0, help="override trees per graph")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=20.0, help="seconds of CPU baseline sampling")
    ap.add_argument("--ref-trees", type=int, default=0, help="reference arm: trees per graph per step (0 = 2 per core)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the R-MAT 24, batch and gradient measurements added to the line")
    ap.add_argument("--extras-budget", type=float, default=1200.0,
                    help="wall seconds after which the remaining extra measurements are skipped")
    ap.add_argument("--walkers", type=int, default=0, help="walkers per tree (0 = auto)")
    ap.add_argument("--policy", type=int, default=0, help="walker conflict policy (0 default: 3 up to 64 walkers per tree, else 1; 1 yield and wait, 2 wait, 3 yield and take a fresh start)")
    ap.add_argument("--diag", action="store_true", help="count walker loop iterations per state (slower)")
    args = ap.parse_args()
    if args.trees:
        WORKLOADS[args.workload] = [(k, args.trees) for k, _ in WORKLOADS[args.workload]]

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_2510_20604_gb300 as rwc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    hbm_peak, peak_src = load_peaks()

    if args.workload == "eps-sweep":
        run_eps_sweep(args, rwc, torch, dev, rank)
        return
    if args.workload == "batch4096":
        run_batch(args, rwc, torch, dev, world, rank)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    graphs = []
    for key, T in WORKLOADS[args.workload]:
        g = make_graph(key)
        G = rwc.Graph.from_synth(g, flags=graph_flags(key, rwc))
        sums = torch.zeros(g.n, dtype=torch.float64, device=dev)
        graphs.append((key, T, g, G, sums))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    opt = rwc.Options(profile=2 if args.diag else 1, block_threads=args.walkers, walker_policy=args.policy)
    from paper_2510_20604_gb300 import shard
    # weak scaling: every rank samples its own range of global tree ids
    tree_base = shard.tree_range(rank, world, max(T for _, T in WORKLOADS[args.workload]))[0]

    def step(stats_out=None):
        Hs = []
        for key, T, g, G, sums in graphs:
            sums.zero_()
            st = rwc.rwc_sample_trees(G.handle, 1, tree_base, T, sums, None, None, opt)
            if dist:
                # the one exchange of the path: add the ranks' visit sums
                # (exact integers), then estimate from all world * T trees
                shard.all_reduce_sums(sums)
            H = G.estimate(sums, world * T)
            Hs.append(H)
            if stats_out is not None:
                stats_out.append((key, st.as_dict()))
        return Hs

    for _ in range(args.warmup):
        step()
        flush.fill_(1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    launches0 = rwc.rwc_launch_count()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    all_stats = []
    t_wall0 = time.perf_counter()
    Hs = None
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        Hs = step(all_stats)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = rwc.rwc_launch_count() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(step_ms))
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    total_T = sum(T for _, T in WORKLOADS[args.workload])
    value = world * total_T / (ms / 1000.0)

    # accuracy: predicted MRE from the variance law of the visit counts (the
    # library's stopping rule) and the trees it needs for 1%
    acc = {}
    for (key, T, g, G, sums), H in zip(graphs, Hs):
        mre, T1 = rwc.rwc_predict_mre(G.handle, sums, world * T, H, target=0.01)
        acc[key] = {"mre_pred": mre, "trees_for_1pct": int(T1), "n": g.n,
                    "draws_per_tree": float(sums.sum().item() / (world * T))}

    # roofline of the sampler: the method's algorithmic bytes (per draw: row
    # bounds + arc head [+ alias entry]; per tree and vertex: parent + visit
    # count) over the device time of the sampler's kernels in the timed
    # region; the dominant kernel takes all but a fraction of a percent of it
    phase_ms = {p: 0.0 for p in PHASE_NAMES}
    per_graph = {}
    alg_total, impl_total, traffic_total, sampler_ms, launches_dom = 0.0, 0.0, 0.0, 0.0, 0
    traffic_known = True
    for key, st in all_stats:
        gi = [x for x in graphs if x[0] == key][0]
        n, info = gi[2].n, gi[3].info
        T_key = gi[1]
        ms_k = sum(st["phase_ms"])
        alg = algorithmic_bytes(st["draws"], T_key, n, bool(info.weighted), bool(info.offsets64))
        impl = st["draws"] * IMPL_BYTES_PER_DRAW if st["mode"] == 3 else 0
        tpd = traffic_per_draw(key) if st["mode"] == 3 else None
        traffic_known &= tpd is not None
        for i, p in enumerate(PHASE_NAMES):
            phase_ms[p] += st["phase_ms"][i]
        alg_total += alg
        impl_total += impl
        traffic_total += (tpd or 0.0) * st["draws"]
        sampler_ms += ms_k
        launches_dom += max(1, st["phase_launches"][1])
        pg = per_graph.setdefault(key, {"alg_bytes": 0.0, "ms": 0.0, "draws": 0})
        pg["alg_bytes"] += alg
        pg["ms"] += ms_k
        pg["draws"] += st["draws"]
    dom = max(PHASE_NAMES, key=lambda p: phase_ms[p])
    dom_mode = all_stats[-1][1]["mode"] if all_stats else 0
    kname = KERNEL_NAMES.get(dom_mode, {}).get(dom, dom)
    achieved = alg_total / (sampler_ms / 1000.0) / 1e9 if sampler_ms > 0 else 0.0
    traffic = traffic_total / launches_dom if traffic_known and launches_dom else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "kernel": kname,
                "algorithmic_bytes_per_launch": alg_total / max(1, launches_dom),
                "launch_ms": sampler_ms / max(1, launches_dom),
                "unit_bytes": {"per_draw": {k: bytes_per_draw(bool(G.info.weighted), bool(G.info.offsets64))
                                            for k, _T, _g, G, _s in graphs},
                               "per_tree_vertex": BYTES_PER_TREE_VERTEX},
                # the walker's own state-word traffic, not part of `achieved`
                "implementation_bytes_per_draw": IMPL_BYTES_PER_DRAW if dom_mode == 3 else 0,
                "implementation_gbs": impl_total / (sampler_ms / 1000.0) / 1e9 if sampler_ms > 0 else 0.0,
                # DRAM bytes actually moved (ncu per draw on a small case, scaled by the draws)
                "dram_gbs": traffic_total / (sampler_ms / 1000.0) / 1e9 if traffic_known and sampler_ms > 0 else None,
                "dram_frac": traffic_total / (sampler_ms / 1000.0) / 1e9 / hbm_peak if traffic_known and sampler_ms > 0 else None,
                "traffic_source": {f: TRAFFIC_PER_DRAW[f][1] for f in {family(k) for k, *_ in graphs} if f in TRAFFIC_PER_DRAW},
                "per_graph": {k: {"gbs": v["alg_bytes"] / (v["ms"] / 1000.0) / 1e9 if v["ms"] > 0 else 0.0,
                                  "frac": v["alg_bytes"] / (v["ms"] / 1000.0) / 1e9 / hbm_peak if v["ms"] > 0 else 0.0,
                                  "draws_per_s": v["draws"] / (v["ms"] / 1000.0) if v["ms"] > 0 else 0.0}
                              for k, v in per_graph.items()},
                "peak_source": f"{peak_src} hbm_gbs",
                "phase_share": {p: phase_ms[p] / max(sampler_ms, 1e-9) for p in PHASE_NAMES}}

    # RWC nodes/s at <= 1% MRE: trees needed for 1% from the variance law,
    # at the measured per-tree sampling time, plus the measured solve time
    nodes_at_1pct = None
    if all_stats:
        tot_time = 0.0
        for key, T, g, G, sums in graphs:
            per_tree = sum(sum(st["phase_ms"]) for k, st in all_stats if k == key) / args.steps / T / 1000.0
            step_share = per_tree * T
            tot_time += acc[key]["trees_for_1pct"] * per_tree
            acc[key]["sample_s_per_step"] = step_share
        solve_s = max(0.0, ms / 1000.0 - sum(a["sample_s_per_step"] for a in acc.values()))
        nodes = sum(a["n"] for a in acc.values())
        nodes_at_1pct = world * nodes / (tot_time + solve_s)

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        import ctypes
        pinned = []
        for key, T, g, G, sums in graphs:
            rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr, np.int64)).pin_memory()
            ci = torch.from_numpy(np.ascontiguousarray(g.col, np.int32)).pin_memory()
            ww = None if g.w is None else torch.from_numpy(np.ascontiguousarray(g.w, np.float32)).pin_memory()
            Hh = torch.empty(g.n, dtype=torch.float64).pin_memory()
            pinned.append((key, T, g, rp, ci, ww, Hh))
        h2d = sum(x[3].numel() * 8 + x[4].numel() * 4 + (0 if x[5] is None else x[5].numel() * 4) for x in pinned)
        d2h = sum(x[6].numel() * 8 for x in pinned)
        e_steps = max(1, min(args.steps, 2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            for key, T, g, rp, ci, ww, Hh in pinned:
                h = rwc.rwc_graph_create(g.n, g.nnz, rp.numpy(), ci.numpy(), None if ww is None else ww.numpy(),
                                         flags=graph_flags(key, rwc))
                try:
                    s = torch.zeros(g.n, dtype=torch.float64, device=dev)
                    rwc.rwc_sample_trees(h, 1, tree_base, T, s)
                    H = torch.empty(g.n, dtype=torch.float64, device=dev)
                    rwc.rwc_estimate(h, s, T, 1e-10, H)
                    Hh.copy_(H, non_blocking=True)
                    torch.cuda.synchronize()
                finally:
                    rwc.rwc_graph_destroy(h)
        e_s = (time.perf_counter() - t0) / e_steps
        if dist:
            t = torch.tensor([e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_s = float(t.item())
        e2e = {"value": world * total_T / e_s, "unit": "trees/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": e_steps,
               "includes": "host CSR validation, alias build, H2D upload, sampling, solve, D2H of H"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        built = {key: g for key, T, g, G, sums in graphs}
        v, cores, samp = cpu_baseline(args.workload, budget_s=args.ref_budget, graphs=built)
        cpu = {"value": v, "unit": "trees/s", "cores": cores, "kind": "oracle", "sample": samp}
        try:   # the paper's setting, reported beside the all-core baseline
            v1, samp1 = cpu_single_thread(args.workload, graphs=built)
            cpu["single_thread"] = {"value": v1, "unit": "trees/s", "cores": 1, "sample": samp1}
        except Exception as exc:  # a failed extra measurement must not cost the line
            cpu["single_thread"] = {"error": str(exc)[:200]}

    # further workloads measured in the same run (rank 0 at N = 1): the
    # paper-size R-MAT 24, the 4096-graph batch and the gradient; each is
    # skipped once the run has used its wall-time allowance
    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = {}
        for name, fn in (("rmat24", lambda: rmat24_measure(rwc, torch, dev, hbm_peak)),
                         ("batch4096", lambda: batch_measure(rwc, torch, dev, steps=3, warmup=1)),
                         ("grad_rgg100k", lambda: grad_measure(rwc, torch, dev))):
            if time.perf_counter() - T_START > args.extras_budget:
                extras[name] = {"skipped": f"run past {args.extras_budget:.0f} s of wall time"}
                continue
            try:
                extras[name] = fn()
            except Exception as exc:  # a failed extra must not cost the line
                extras[name] = {"error": str(exc)[:300]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32/f64", "data": "synthetic",
            "config": {"workload": args.workload, "trees": dict(WORKLOADS[args.workload]),
                       "l2": "256 MiB buffer written between steps; per-tree state exceeds L2",
                       "seed": 1, "pivot": "max degree, ties to smallest id"},
            "rwc_nodes_per_s_at_1pct": nodes_at_1pct,
            "accuracy": acc,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "extras": extras,
            "gpu_launches": int(launches),
            "clocks": clk,
            "wall_s_timed": t_wall,
            "step_ms": step_ms,
            "sampler_stats": [{"graph": k, "mode": st["mode"], "rounds_or_yields": st["rounds"],
                               "draws": st["draws"], "walk_steps": st["walk_steps"],
                               "chunks": st["chunks"], "walkers_per_tree": st["block_threads"],
                               "diag": st["diag"]}
                              for k, st in all_stats[-len(graphs):]],
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
