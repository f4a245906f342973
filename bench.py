#!/usr/bin/env python
"""Throughput of the linear-BVH segment/surface intersection on one GB300.

Workload (the paper's scale: ~2e4 triangles, 1e7 segments, Sec. 3.3): a
100 x 100-vertex heightfield with sinusoid + Gaussian-bump relief (19,602
triangles) and 1e7 segments, half crossing the surface and half wholly above
it, length U(0.05, 1), random directions -- seeded synthetic data standing in
for the paper's unavailable generator.

One step = the whole hot path on one batch: GPU build of the hierarchy
(extent, Morton codes, radix sort, radix tree, refit) + the boolean and the
intercept_count answer of every segment (FP32 traversal with the FP64
re-test of band segments).  The count pass yields the boolean answer too
(hit = count > 0; the boolean-mode ambiguity flag from the same pass), so
one traversal answers both modes (RSI_BOTH); the line also reports the step
with the two modes queried separately.  value = segments fully answered
(both modes) per second, summed over ranks.  The segments (240 MB) exceed the 129 MB L2, so no
flush is needed between steps.

--impl reference times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s (exact vs FP64 oracle) plain vs batched+learned on 1 GB300; % roofline"
WORKLOAD = ("c2: 100x100-vertex heightfield, 4 sinusoids + 8 Gaussian bumps (19,602 FP32 triangles); "
            "1e7 FP32 segments, 50% crossing / 50% above, length U(0.05,1), random directions; "
            "step = lbvh_build_ex (the paper's Karras build, then two treelet restructuring passes: "
            "same answers, fewer nodes met) + the boolean and intercept_count answers of every segment "
            "(one traversal answers both: rsi_query mode RSI_BOTH)")
W_DOC_PAPER = ("paper scale: 111x134-vertex heightfield, 4 sinusoids + 8 Gaussian bumps (14,874 vertices, "
               "29,260 triangles, the paper's counts); 1e7 segments, 50% crossing / 50% above")
BYTES_PER_RAY_COUNT = 28   # 24 B of segment in + 4 B of count out (algorithmic)
TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "k_query_fp32_count_c2.md")
TRAFFIC_SUMMARY_C3 = os.path.join(ROOT, "profiles", "k_query_fp32_count_c3.md")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash():
    """Hash of the traversal kernels' source: the region between their
    markers in query.cu (device code and the structures it reads) and the
    FP32 segment / box / triangle tests it includes (segtest.cuh)."""
    csrc = os.path.join(ROOT, "paper_2305_01867_gb300", "csrc")
    q = open(os.path.join(csrc, "query.cu")).read()
    b, e = q.index("// [traversal kernel: begin]"), q.index("// [traversal kernel: end]")
    t = open(os.path.join(csrc, "segtest.cuh")).read()
    return hashlib.sha256((q[b:e] + t).encode()).hexdigest()[:16]


def profile_values(path=None):
    """Figures of a committed ncu summary of the count traversal (the c2
    capture by default), if it was taken on the current source (else {})."""
    try:
        txt = open(path or TRAFFIC_SUMMARY).read()
    except OSError:
        return {}
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_hash") != source_hash():
        return {}
    out = {}
    for k, v in vals.items():
        try:
            out[k] = float(v)
        except ValueError:
            pass
    return out


def traffic_per_launch():
    """DRAM bytes per launch of the count traversal (ncu), or None."""
    return profile_values().get("dram_bytes_per_launch_full_size")


def issue_bound():
    """The measured L2 / issue bound of the count traversal (ncu, same
    source): fractions of peak issue slots, L1TEX and L2 throughput."""
    v = profile_values()
    if "issue_active_pct" not in v:
        return None
    return {"kernel": "k_query_fp32<count>", "issue_active_frac": v["issue_active_pct"] / 100,
            "l1tex_throughput_frac": v.get("l1tex_throughput_pct", float("nan")) / 100,
            "lts_throughput_frac": v.get("lts_throughput_pct", float("nan")) / 100,
            "source": "ncu --set full capture of the same kernel source (profiles/k_query_fp32_count_c2.md)"}


def second_bound():
    """The count traversal's binding limit, from the committed ncu capture of
    the same kernel source: the higher of L1TEX throughput and instruction
    issue (issue slots busy), each as a fraction of its peak.  A stale
    capture is reported as such (and on stderr), never silently dropped."""
    v = profile_values()
    if "issue_active_pct" not in v:
        msg = ("STALE: profiles/k_query_fp32_count_c2.md was captured on another traversal source "
               f"(current source_hash {source_hash()}); issue / L1 figures withheld")
        print("bench.py: " + msg, file=sys.stderr)
        return {"stale": msg}
    issue = v["issue_active_pct"] / 100
    l1 = v.get("l1tex_throughput_pct", 0.0) / 100
    if l1 >= issue:
        bound, unit = "l1tex", "fraction of peak L1TEX throughput"
    else:
        bound, unit = "issue", "issue slots busy"
    frac = max(l1, issue)
    return {"bound": bound, "achieved": frac, "peak": 1.0, "unit": unit, "frac": frac,
            "issue_frac": issue, "l1tex_frac": l1,
            "peak_source": "ncu l1tex__throughput / smsp__issue_active of the same kernel source "
                           "(profiles/k_query_fp32_count_c2.md)"}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(gpu_index)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def rank_seed(base_seed: int, rank: int) -> int:
    """Weak scaling: every rank answers its own batch of the same workload."""
    return base_seed + 1000 * rank


def max_over_ranks(pg, value: float, device) -> float:
    """The slowest rank's time (the job finishes when it does)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, values, device):
    """Element-wise sum of a few integer counters over all ranks: the one
    exchange of the sharded path (segments sent to the FP64 re-test and left
    ambiguous), taken after the timed region."""
    if pg is None:
        return [int(v) for v in values]
    import torch
    t = torch.tensor([int(v) for v in values], dtype=torch.int64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return [int(x) for x in t.tolist()]


def run_reference(args, ws, rank):
    """The FP64 oracle as it stands, on this machine's host cores."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    import workloads as W
    oracle.build()
    mesh = W.config_mesh("c2")
    spec = W.config_rays("c2")
    per_step = args.ref_rays
    times = []
    for k in range(args.warmup + args.steps):
        F, E = W.rays(spec, mesh, start=k * per_step, count=per_step)
        t0 = time.perf_counter()
        oracle.query(mesh.vertices, mesh.triangles, F, E)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = per_step / (ms / 1e3)
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_triangles": int(len(mesh.triangles)),
                       "rays_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} segments of the 1e7-segment batch per step, all "
                                       f"{len(mesh.triangles)} triangles each (brute force, both modes)"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_baseline(mesh, spec, n):
    import oracle
    import workloads as W
    F, E = W.rays(spec, mesh, start=0, count=n)
    t0 = time.perf_counter()
    oracle.query(mesh.vertices, mesh.triangles, F, E)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "rays/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {n} segments of the batch x all {len(mesh.triangles)} triangles, FP64 brute force "
                      f"(both modes in one pass), {dt:.1f} s"}


def measure_batched(rsi, torch, dev, c4, args):
    """64 independent heightfields with log-uniform triangle counts in
    [1e3, 1e5] and segment counts in [1e4, 1e7]: one graph-launched
    persistent traversal over all of them (rsi_query_batched), against the
    same work issued as 64 separate rsi_query calls."""
    jobs, rays = c4
    stream = torch.cuda.current_stream()
    meshes = [(torch.from_numpy(m.vertices).to(dev), torch.from_numpy(m.triangles).to(dev)) for m, _ in jobs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c4p = args.c4_treelet_passes
    for b in rsi.build_many(meshes, treelet_passes=c4p):   # warm-up
        b.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bvhs = rsi.build_many(meshes, treelet_passes=c4p)   # all 64 hierarchies in one build
    torch.cuda.synchronize()
    build_ms = 1e3 * (time.perf_counter() - t0)
    items = [(b, torch.from_numpy(F).to(dev), torch.from_numpy(E).to(dev)) for b, (F, E) in zip(bvhs, rays)]
    total = sum(int(f.shape[0]) for _, f, _ in items)
    steps = max(3, min(args.steps, 10))
    out = {"n_meshes": len(jobs), "triangles": int(sum(len(m.triangles) for m, _ in jobs)), "rays": total,
           "build_all_ms": build_ms, "steps": steps,
           "tree": (f"the paper's builds + {c4p} treelet restructuring pass(es) over all meshes at once "
                    "(lbvh_build_batched_ex)") if c4p else "as built"}

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    for mode in ("any_hit", "count"):
        t0 = time.perf_counter()
        tune = rsi.batch_autotune(items, mode)
        tune_s = time.perf_counter() - t0
        picked = {k: tune[k] for k in ("block", "blocks_per_sm", "node_width", "ray_sort_tile", "stack")}
        plan_default = rsi.BatchPlan(items, mode)
        ms_default = timed(plan_default.run)
        plan_default.close()
        plan = rsi.BatchPlan(items, mode, **picked)
        ms = timed(plan.run)
        outs = {}

        def sequential():
            for i, (b, f, t) in enumerate(items):
                key = "hit" if mode == "any_hit" else "count"
                buf = plan.hit[i] if mode == "any_hit" else plan.count[i]
                outs[i] = b.query(f, t, mode, **{key: buf}, ambiguous=plan.ambiguous[i])
        ms_seq = timed(sequential)
        st = plan.stats()
        out[mode] = {"rays_per_s": total / (ms / 1e3), "ms": ms, "autotuned": picked,
                     "autotune_s": tune_s, "autotune_candidates": tune["candidates"],
                     "default_plan_ms": ms_default, "gain_over_default": ms_default / ms,
                     "sequential_rays_per_s": total / (ms_seq / 1e3),
                     "sequential_ms": ms_seq, "band_rays": st["band_rays"], "ambiguous": st["ambiguous"]}
        plan.close()
    # build and query in one graph: a rebuilding plan (the batched build's
    # kernels in place, then the query) replayed every step
    tuned = out["any_hit"]["autotuned"]
    graph_ms = {}
    for passes in sorted({0, c4p}):   # a rebuild repeats the hierarchies' restructuring passes
        hs = bvhs if passes == c4p else rsi.build_many(meshes, treelet_passes=passes)
        its = [(b, f, t) for b, (_, f, t) in zip(hs, items)]
        plan = rsi.BatchPlan(its, "any_hit", rebuild=meshes, block=tuned["block"],
                             blocks_per_sm=tuned["blocks_per_sm"], ray_sort_tile=tuned["ray_sort_tile"])
        graph_ms[passes] = timed(plan.run)
        plan.close()
        if hs is not bvhs:
            for b in hs:
                b.close()
    out["build_and_query_one_graph_any_hit_ms"] = graph_ms[0]
    if c4p:
        out[f"build_and_query_one_graph_any_hit_ms_{c4p}_treelet_passes"] = graph_ms[c4p]
    out["build_and_query_one_graph_note"] = ("rsi_batch_create_rebuild: each launch rebuilds the 64 hierarchies "
                                             "in place from their mesh buffers (the paper's trees; with "
                                             "restructuring passes, which cost more than they save when every "
                                             "launch rebuilds, beside it), then runs the batched boolean query "
                                             "(the tuned launch shape; 128-entry stacks, child-pair nodes), one graph "
                                             "launch per step")

    for b in bvhs:
        b.close()

    # build and query in sequence, as a caller would: one batched build of
    # the 64 meshes, then one rsi_query_batched call on the new hierarchies
    # (a new plan each time: the hierarchies are new), wall clock
    def build_and_query(passes):
        hs = rsi.build_many(meshes, treelet_passes=passes)
        rsi.query_batched([(b, f, t) for b, (_, f, t) in zip(hs, items)], "any_hit")
        torch.cuda.synchronize()
        for b in hs:
            b.close()
    for passes in sorted({0, c4p}):
        build_and_query(passes)
        t0 = time.perf_counter()
        for _ in range(steps):
            build_and_query(passes)
        key = "build_then_query_any_hit_ms" + (f"_{passes}_treelet_passes" if passes else "")
        out[key] = 1e3 * (time.perf_counter() - t0) / steps
    out["build_then_query_note"] = ("wall clock of lbvh_build_batched_ex (the paper's trees; with restructuring "
                                    "passes beside it) + one rsi_query_batched call (plan, graph "
                                    "capture, launch) per step on new hierarchies; beside it, the rebuilding plan "
                                    "replays build and query of existing hierarchies in one graph")
    return out


def measure_nearest(rsi, torch, dev, pV, pT, pF, pE, dV, dT, dF, dE, args):
    """Barycentric mode on the same 1e7 segments: the device query
    (rsi_query_nearest: nearest triangle, t, point, distance) and, in the
    paper's end-to-end style (Sec. 3.3), host segments -> build -> nearest
    query -> compacted (rays, distances, triangles, points) -> host."""
    stream = torch.cuda.current_stream()
    n = dF.shape[0]
    steps = max(3, min(args.steps, 10))
    tp = args.treelet_passes
    bvh = rsi.LBVH(dV, dT, treelet_passes=tp)
    for _ in range(args.warmup):
        bvh.nearest(dF, dE)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    trav, fin = [], []
    e0.record(stream)
    for _ in range(steps):
        r = bvh.nearest(dF, dE, time_kernels=True)
        a, b = bvh.last_query_ms()
        trav.append(a)
        fin.append(b)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = bvh.nearest(dF, dE, stats=True)["stats"]
    hits = int((r["tri"] >= 0).sum())
    bvh.close()

    # page-locked host arrays for the compacted result (sized for every segment)
    h_out = (torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.float32).pin_memory(),
             torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, 3, dtype=torch.float32).pin_memory())

    def paper_style():
        b = rsi.LBVH(pV.to(dev, non_blocking=True), pT.to(dev, non_blocking=True), treelet_passes=tp)
        res = b.barycentric(pF.to(dev, non_blocking=True), pE.to(dev, non_blocking=True))
        k = res[0].shape[0]
        out = tuple(h[:k].copy_(r, non_blocking=True) for h, r in zip(h_out, res))
        torch.cuda.synchronize()
        b.close()
        return out

    for _ in range(args.warmup):
        paper_style()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        out = paper_style()
    e2e = 1e3 * (time.perf_counter() - t0) / steps
    assert out[0].shape[0] == hits
    return {"rays": n, "steps": steps, "ms": ms, "rays_per_s": n / (ms / 1e3), "treelet_passes": tp,
            "traverse_ms": statistics.median(trav), "fp64_and_finish_ms": statistics.median(fin),
            "hitting_rays": hits, "band_rays": st["band_rays"], "ambiguous": st["ambiguous"],
            "paper_style_e2e_ms": e2e,
            "paper_style_e2e": "pinned host segments and mesh -> build -> nearest -> compaction -> pinned host "
                               "(rays, distances, triangles, points)"}


def measure_builders(rsi, torch, dev, meshes, c4, reps=20):
    """Build time of the two tree constructions (Karras radix tree + refit,
    and the single bottom-up pass of Sec. 4.2 after Apetrei) on the c2 and
    c3 meshes and on all 64 c4 meshes: wall-clock per lbvh_build call
    (each call synchronizes its stream once), median over reps; and the 64
    c4 meshes in one lbvh_build_batched call."""
    def per_build(V, T, builder):
        for _ in range(3):
            rsi.LBVH(V, T, builder=builder).close()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b = rsi.LBVH(V, T, builder=builder)
            ts.append(1e3 * (time.perf_counter() - t0))
            b.close()
        return statistics.median(ts)

    out = {"reps": reps, "timing": "wall clock of one lbvh_build call (one stream synchronization inside)"}
    for name, m in meshes:
        V, T = torch.from_numpy(m.vertices).to(dev), torch.from_numpy(m.triangles).to(dev)
        out[name] = {"triangles": int(len(m.triangles)),
                     **{f"{b}_ms": per_build(V, T, b) for b in ("karras", "apetrei")}}
    if c4 is not None:
        jobs = [(torch.from_numpy(m.vertices).to(dev), torch.from_numpy(m.triangles).to(dev)) for m, _ in c4[0]]
        tot = {}
        for b in ("karras", "apetrei"):
            tot[f"{b}_ms"] = sum(per_build(V, T, b) for V, T in jobs)
        # all 64 in one build (lbvh_build_batched)
        for _ in range(3):
            for b in rsi.build_many(jobs):
                b.close()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hs = rsi.build_many(jobs)
            ts.append(1e3 * (time.perf_counter() - t0))
            for b in hs:
                b.close()
        tot["one_batched_build_ms"] = statistics.median(ts)
        out["c4_all_64"] = {"triangles": int(sum(len(m.triangles) for m, _ in c4[0])), **tot}
    return out


# The paper's own timings for 1e7 rays on its 29,260-triangle surface (Sec. 4,
# GPU not stated; the original CUDA program and the PyCUDA port), in ms.
PAPER_MS = {"boolean": {"cuda": 300.166, "pycuda": 355.094},
            "intercept_count": {"cuda": 334.192, "pycuda": 383.117},
            "barycentric": {"cuda": 308.625, "pycuda": 909.376}}


def measure_paper_scale(rsi, torch, dev, paper, args):
    """End to end in the paper's style (Sec. 3.3, Sec. 4) at the paper's
    scale: a surface with its vertex and triangle counts (111 x 134 grid,
    29,260 triangles) and 1e7 segments, all in pinned host memory; one run =
    build from host arrays + query + results back in host memory, per mode.
    Set beside the paper's own timings (other hardware, context only)."""
    mesh, (F, E) = paper
    pV, pT = torch.from_numpy(mesh.vertices).pin_memory(), torch.from_numpy(mesh.triangles).pin_memory()
    pF, pE = torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory()
    n = pF.shape[0]
    hh = torch.empty(n, dtype=torch.uint8).pin_memory()
    hc = torch.empty(n, dtype=torch.int32).pin_memory()
    ha = torch.empty(n, dtype=torch.uint8).pin_memory()
    steps = max(3, min(args.steps, 10))
    tp = args.treelet_passes

    def boolean():
        b = rsi.LBVH(pV, pT, treelet_passes=tp)
        b.query_host(pF, pE, "any_hit", hit=hh, ambiguous=ha)
        b.close()

    def intercept_count():
        b = rsi.LBVH(pV, pT, treelet_passes=tp)
        b.query_host(pF, pE, "count", count=hc, ambiguous=ha)
        b.close()

    h_out = (torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.float32).pin_memory(),
             torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, 3, dtype=torch.float32).pin_memory())

    def barycentric():
        b = rsi.LBVH(pV.to(dev, non_blocking=True), pT.to(dev, non_blocking=True), treelet_passes=tp)
        res = b.barycentric(pF.to(dev, non_blocking=True), pE.to(dev, non_blocking=True))
        k = res[0].shape[0]
        out = [h[:k].copy_(r, non_blocking=True) for h, r in zip(h_out, res)]
        torch.cuda.synchronize()
        b.close()
        return out

    out = {"workload": W_DOC_PAPER, "rays": n, "triangles": int(len(mesh.triangles)), "steps": steps,
           "timing": "wall clock, pinned host mesh and segments in, host results out, build included",
           "tree": f"the paper's Karras build + {tp} treelet restructuring pass(es)" if tp else "as built"}
    for name, fn in (("boolean", boolean), ("intercept_count", intercept_count), ("barycentric", barycentric)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / steps
        out[name] = {"ms": ms, "rays_per_s": n / (ms / 1e3), "paper_ms": PAPER_MS[name],
                     "paper_rays_per_s_cuda": n / (PAPER_MS[name]["cuda"] / 1e3)}
    out["hits"] = int(hh.sum())
    out["crossings"] = int(hc.sum())
    return out


def measure_precision_c3(rsi, torch, dev, c3, args):
    """The precision path on c3 (300 x 300 jittered heightfield, 178,802
    triangles; 1e8 segments, 1 % grazing): both modes with the FP64 re-test
    of band segments and without it (FP32 only), timed; then the FP64 oracle
    settles every segment where the two disagree (capped), every segment the
    GPU marked ambiguous (capped) and a random sample.  Flips are counted on
    segments the oracle does not mark ambiguous: with the re-test they must
    be 0, and since the re-tested answer equals the oracle on every checked
    segment, the FP32-only flips over the whole batch are the disagreements
    outside the ambiguous set."""
    import numpy as np
    import oracle
    mesh, (F, E) = c3
    n = F.shape[0]
    c3p = args.c3_treelet_passes
    bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).to(dev), torch.from_numpy(mesh.triangles).to(dev), morton_bits=63,
                   treelet_passes=c3p)
    dF, dE = torch.from_numpy(F).to(dev), torch.from_numpy(E).to(dev)
    stream = torch.cuda.current_stream()
    out = {"workload": "c3: 300x300-vertex jittered heightfield, 8 bumps (178,802 triangles); 1e8 segments, "
                       "50% crossing / 50% above, 1% grazing (end point within 1e-6 of an edge or vertex, or "
                       "nearly parallel to a face)", "rays": n, "triangles": int(len(mesh.triangles)), "morton_bits": 63,
           "tree": f"the paper's Karras build + {c3p} treelet restructuring pass(es)" if c3p else "as built",
           "tree_height": bvh.info()["height"]}
    res = {}
    for mode in ("any_hit", "count"):
        for fp32_only in (False, True):
            key = f"{mode}_{'fp32_only' if fp32_only else 'fp64_retest'}"
            r = bvh.query(dF, dE, mode, fp32_only=fp32_only)   # warm-up and the result
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                bvh.query(dF, dE, mode, fp32_only=fp32_only, hit=r["hit"], count=r["count"], ambiguous=r["ambiguous"])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
            st = bvh.query(dF, dE, mode, fp32_only=fp32_only, stats=True)["stats"]
            val = r["hit"] if mode == "any_hit" else r["count"]
            res[key] = (val.cpu().numpy(), r["ambiguous"].cpu().numpy())
            out[key] = {"ms": ms, "rays_per_s": n / (ms / 1e3), "band_rays": st["band_rays"],
                        "ambiguous": st["ambiguous"]}
    # the count traversal's roofline on this workload (CUDA events around the
    # kernel on the query's stream, median of 3)
    trav = []
    for _ in range(4):
        bvh.query(dF, dE, "count", time_kernels=True)
        trav.append(bvh.last_query_ms()[0])
    trav_ms = statistics.median(trav[1:])
    peak, peak_kind = peaks()
    achieved = BYTES_PER_RAY_COUNT * n / (trav_ms / 1e3) / 1e9
    out["roofline"] = {"kernel": "k_query_fp32<count> (FP32 traversal, intercept_count)", "bound": "hbm",
                       "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                       "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                       else "fallback 6.8 TB/s", "traffic": profile_values(TRAFFIC_SUMMARY_C3).get(
                           "dram_bytes_per_launch_full_size"), "algorithmic_bytes_per_ray": BYTES_PER_RAY_COUNT,
                       "kernel_ms": trav_ms}
    bvh.close()
    del dF, dE
    # end to end through the host-buffer calls: pinned mesh and segments in,
    # pinned results out; build + boolean + count per step, wall clock
    pV = torch.from_numpy(mesh.vertices).pin_memory()
    pT = torch.from_numpy(mesh.triangles).pin_memory()
    pF, pE = torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory()
    hh, ha = torch.empty(n, dtype=torch.uint8).pin_memory(), torch.empty(n, dtype=torch.uint8).pin_memory()
    hc = torch.empty(n, dtype=torch.int32).pin_memory()

    def step_e2e():
        b = rsi.LBVH(pV, pT, morton_bits=63, treelet_passes=c3p)
        b.query_host(pF, pE, "both", hit=hh, count=hc, ambiguous=ha)
        b.close()
    step_e2e()
    t0 = time.perf_counter()
    for _ in range(3):
        step_e2e()
    e2e_ms = 1e3 * (time.perf_counter() - t0) / 3
    same = bool(np.array_equal(hh.numpy(), res["any_hit_fp64_retest"][0])
                and np.array_equal(hc.numpy(), res["count_fp64_retest"][0])
                and np.array_equal(ha.numpy() & 1, res["any_hit_fp64_retest"][1])
                and np.array_equal(ha.numpy() >> 1, res["count_fp64_retest"][1]))
    out["e2e"] = {"value": n / (e2e_ms / 1e3), "unit": "rays/s",
                  "h2d_bytes_per_step": pV.numel() * 4 + pT.numel() * 4 + (pF.numel() + pE.numel()) * 4,
                  "d2h_bytes_per_step": n * (1 + 4 + 1), "ms_per_step": e2e_ms,
                  "step": "host mesh -> build -> boolean and intercept_count answers of the host segments in one "
                          "pass (RSI_BOTH) -> host results",
                  "matches_device_results": same}
    del pF, pE, hh, ha, hc
    rng = np.random.default_rng(31)
    checked = {}
    for mode in ("any_hit", "count"):
        a, amb = res[f"{mode}_fp64_retest"]
        b, _ = res[f"{mode}_fp32_only"]
        diff = np.flatnonzero(a != b)
        ambi = np.flatnonzero(amb)
        cap = args.c3_check
        pick = [diff if len(diff) <= cap else rng.choice(diff, cap, replace=False),
                ambi if len(ambi) <= cap // 4 else rng.choice(ambi, cap // 4, replace=False),
                rng.choice(n, cap // 2, replace=False)]
        checked[mode] = (diff, ambi, np.unique(np.concatenate(pick)))
    idx = np.unique(np.concatenate([c[2] for c in checked.values()]))
    t0 = time.perf_counter()
    ref = oracle.query(mesh.vertices, mesh.triangles, F[idx], E[idx])
    oracle_s = time.perf_counter() - t0
    pos = {int(i): k for k, i in enumerate(idx)}
    for mode in ("any_hit", "count"):
        diff, ambi, sel = checked[mode]
        k = np.array([pos[int(i)] for i in sel])
        rv, ra = (ref["hit"], ref["amb_hit"]) if mode == "any_hit" else (ref["count"], ref["amb_count"])
        a, amb = res[f"{mode}_fp64_retest"]
        b, _ = res[f"{mode}_fp32_only"]
        ok = ra[k] == 0
        kd = np.array([pos[int(i)] for i in diff if int(i) in pos], dtype=np.int64)
        out[mode] = {"checked_by_oracle": int(len(sel)), "disagreements_fp32_only_vs_retest": int(len(diff)),
                     "disagreements_checked": int(len(kd)),
                     "flips_with_fp64_retest": int(np.sum(a[sel][ok] != rv[k][ok])),
                     "ambiguous_marks_differ": int(np.sum(amb[sel] != ra[k])),
                     "flips_fp32_only_checked": int(np.sum(b[sel][ok] != rv[k][ok])),
                     "flips_fp32_only_whole_batch": int(np.sum(ref["amb_hit" if mode == "any_hit" else "amb_count"][kd] == 0))
                     if len(kd) == len(diff) else None,
                     "gpu_ambiguous": int(len(ambi))}
    out["oracle"] = {"segments": int(len(idx)), "seconds": oracle_s, "cores": oracle.num_threads()}
    return out


MLP_FLOP_PER_SEGMENT = 2 * (6 * 128 + 128 * 128 + 128 * 256)   # algorithmic (unpadded) multiply-adds x 2


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1900.0, 1700.0, "fallback"


def measure_learned(rsi, torch, dev, c5, args):
    """The c1 mesh: train the proposal network on labelled segments, then
    time the boolean query over fresh segments with and without it (answers
    identical by construction) and the tensor-core forward alone."""
    mesh, ((Ft, Et), (Fe, Ee)) = c5
    stream = torch.cuda.current_stream()
    bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).to(dev), torch.from_numpy(mesh.triangles).to(dev))
    dFt, dEt = torch.from_numpy(Ft).to(dev), torch.from_numpy(Et).to(dev)
    labels = rsi.cluster_labels(bvh, dFt, dEt)
    net = rsi.MLP(5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.fit(bvh, dFt, dEt, labels, epochs=2, batch=8192, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del dFt, dEt, labels
    dF, dE = torch.from_numpy(Fe).to(dev), torch.from_numpy(Ee).to(dev)
    n = dF.shape[0]
    hit = torch.empty(n, dtype=torch.uint8, device=dev)
    amb = torch.empty(n, dtype=torch.uint8, device=dev)
    steps = max(3, min(args.steps, 10))

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_plain = timed(lambda: bvh.query(dF, dE, "any_hit", hit=hit, ambiguous=amb))
    plain_hit = hit.clone()
    ms_learned = timed(lambda: rsi.query_learned(bvh, net, dF, dE, hit=hit, ambiguous=amb))
    same = bool(torch.equal(hit, plain_hit))
    st = rsi.query_learned(bvh, net, dF, dE, hit=hit, ambiguous=amb, stats=True)["stats"]
    st_plain = bvh.query(dF, dE, "any_hit", hit=hit, ambiguous=amb, stats=True)["stats"]
    top4 = torch.empty(n, 4, dtype=torch.uint8, device=dev)
    ms_fwd = timed(lambda: net.forward(bvh, dF, dE, logits=False, top4=True))
    tflops = MLP_FLOP_PER_SEGMENT * n / (ms_fwd / 1e3) / 1e12
    burst, sustained, kind = bf16_peak()
    hits = int(plain_hit.sum())
    bvh.close()
    work = {"plain": {"node_visits_per_segment": st_plain["node_visits"] / n,
                      "tri_tests_per_segment": st_plain["tri_tests"] / n},
            "learned": {"node_visits_per_segment": st["node_visits"] / n,
                        "tri_tests_per_segment": st["tri_tests"] / n,
                        "note": "tri_tests include the proposal's verification tests"}}
    return {"train_segments": int(Ft.shape[0]), "epochs": 2, "batch": 8192, "train_s": train_s,
            "train_note": "train_s: 2 epochs over 1e7 labelled segments on the GPU's SIMT training kernels "
                          "(one-off set-up, not part of the query)",
            "loss_per_epoch": losses, "eval_segments": n, "steps": steps, "work": work,
            "plain_any_hit": {"ms": ms_plain, "rays_per_s": n / (ms_plain / 1e3)},
            "learned_any_hit": {"ms": ms_learned, "rays_per_s": n / (ms_learned / 1e3), "matches_plain": same},
            "proposal_confirmed": st["proposal_confirmed"], "hits": hits,
            "confirmed_share_of_hits": st["proposal_confirmed"] / max(hits, 1), "fallback_rays": st["fallback_rays"],
            "mlp_forward_tc": {"ms": ms_fwd, "tflops": tflops, "flop_per_segment": MLP_FLOP_PER_SEGMENT,
                               "peak_tflops": sustained, "frac": tflops / sustained,
                               "peak_source": f"{kind} bf16 sustained"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rays", type=int, default=10_000_000)
    ap.add_argument("--ref-rays", type=int, default=20_000)
    ap.add_argument("--cpu-sample", type=int, default=600_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-nearest", action="store_true")
    ap.add_argument("--no-builders", action="store_true")
    ap.add_argument("--no-paper-scale", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--c3-rays", type=int, default=100_000_000)
    ap.add_argument("--c3-check", type=int, default=20_000)
    ap.add_argument("--learned-rays", type=int, default=100_000_000)
    ap.add_argument("--train-rays", type=int, default=10_000_000)
    ap.add_argument("--c3-only", action="store_true",
                    help="run the c3 precision leg alone and print its object (for profiler captures)")
    ap.add_argument("--treelet-passes", type=int, default=2,
                    help="restructuring passes after the c2 build (0: the paper's tree as built)")
    ap.add_argument("--c3-treelet-passes", type=int, default=2,
                    help="restructuring passes after the c3 build (1e8 segments per build)")
    ap.add_argument("--c4-treelet-passes", type=int, default=2,
                    help="restructuring passes after the batched c4 build (7.7e7 segments per build)")
    ap.add_argument("--order", action="store_true",
                    help="walk the segments in midpoint-cell order in the timed step (rsi_segment_order inside it)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        if pg:
            pg.barrier()
            pg.destroy_process_group()
        return

    import numpy as np
    import torch

    import paper_2305_01867_gb300 as rsi
    import workloads as W

    if args.c3_only:   # the c3 leg by itself: its own JSON object, no contract line
        m3 = W.config_mesh("c3")
        c3 = (m3, W.rays_many([(m3, W.config_rays("c3", args.c3_rays))])[0])
        torch.cuda.set_device(local)
        print(json.dumps({"precision_c3": measure_precision_c3(rsi, torch, torch.device("cuda", local), c3, args)}))
        return

    mesh = W.config_mesh("c2")
    spec = W.config_rays("c2", args.rays)
    spec.seed = rank_seed(spec.seed, rank)       # each rank its own batch (weak scaling)
    F, E = W.rays(spec, mesh)
    c4 = None
    if not args.no_batched and rank == 0:
        jobs = W.batched_meshes(n_meshes=64, seed=4)
        c4 = (jobs, W.rays_many(jobs))           # process pool before any GPU call
    c3 = None
    if not args.no_precision and rank == 0:
        m3 = W.config_mesh("c3")
        c3 = (m3, W.rays_many([(m3, W.config_rays("c3", args.c3_rays))])[0])
    paper = None
    if not args.no_paper_scale and rank == 0:
        pm = W.config_mesh("paper")
        paper = (pm, W.rays_many([(pm, W.config_rays("paper"))])[0])
    c5 = None
    if not args.no_learned and rank == 0:
        m1 = W.config_mesh("c1")
        jobs = [(m1, W.RaySpec("uniform_box", args.train_rays, seed=11)),
                (m1, W.RaySpec("uniform_box", args.learned_rays, seed=12))]
        c5 = (m1, W.rays_many(jobs))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = len(F)
    pF, pE = torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory()
    pV, pT = torch.from_numpy(mesh.vertices).pin_memory(), torch.from_numpy(mesh.triangles).pin_memory()
    dV, dT = pV.to(dev), pT.to(dev)
    dF, dE = pF.to(dev), pE.to(dev)
    hit = torch.empty(n, dtype=torch.uint8, device=dev)
    amb_h = torch.empty(n, dtype=torch.uint8, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    amb_c = torch.empty(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    amb2 = torch.empty(n, dtype=torch.uint8, device=dev)
    step_order = torch.empty(n, dtype=torch.int32, device=dev) if args.order else None

    tp = args.treelet_passes

    def step(evs=None, trav=None, passes=None):
        if evs:
            evs[0].record(stream)
        bvh = rsi.LBVH(dV, dT, morton_bits=30, treelet_passes=tp if passes is None else passes)
        if evs:
            evs[1].record(stream)
        if step_order is not None:
            bvh.segment_order(dF, dE, out=step_order)
        bvh.query(dF, dE, "both", hit=hit, count=cnt, ambiguous=amb2, time_kernels=trav is not None,
                  order=step_order)
        if evs:
            evs[2].record(stream)
        if trav is not None:
            trav.append(bvh.last_query_ms()[0])
        bvh.close()

    def step_separate(evs=None):
        if evs:
            evs[0].record(stream)
        bvh = rsi.LBVH(dV, dT, morton_bits=30, treelet_passes=tp)
        if evs:
            evs[1].record(stream)
        bvh.query(dF, dE, "any_hit", hit=hit, ambiguous=amb_h)
        if evs:
            evs[2].record(stream)
        bvh.query(dF, dE, "count", count=cnt, ambiguous=amb_c)
        if evs:
            evs[3].record(stream)
        bvh.close()

    def barrier():
        torch.cuda.synchronize()
        if pg:
            pg.barrier()

    # the clock sampler starts (and its NVML set-up finishes) before the warm-up,
    # so only its steady 50 ms sampling overlaps the timed region
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    time.sleep(0.5)
    for _ in range(args.warmup):
        step()
    barrier()
    n_ev = args.steps
    phase = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_ev)]
    trav = []
    l0 = rsi.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for k in range(args.steps):
        step(phase[k], trav)
    e1.record(stream)
    barrier()
    launches = rsi.kernel_launches() - l0
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(pg, e0.elapsed_time(e1) / args.steps, dev)
    value = ws * n / (ms / 1e3)
    build_ms = statistics.median(p[0].elapsed_time(p[1]) for p in phase)
    both_ms = statistics.median(p[1].elapsed_time(p[2]) for p in phase)
    trav_ms = statistics.mean(trav)
    # the same step with the two modes queried separately (context): the
    # answers must be those of the combined pass
    for _ in range(3):
        step_separate()
    sep = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    for k in range(args.steps):
        step_separate(sep[k])
    torch.cuda.synchronize()
    separate = {"step_ms": statistics.median(p[0].elapsed_time(p[3]) for p in sep),
                "any_hit_query_ms": statistics.median(p[1].elapsed_time(p[2]) for p in sep),
                "count_query_ms": statistics.median(p[2].elapsed_time(p[3]) for p in sep)}
    bvh = rsi.LBVH(dV, dT, morton_bits=30, treelet_passes=tp)
    bvh.query(dF, dE, "both", hit=hit, count=cnt, ambiguous=amb2)
    both_hit, both_cnt, both_amb = hit.clone(), cnt.clone(), amb2.clone()
    bvh.query(dF, dE, "any_hit", hit=hit, ambiguous=amb_h)
    bvh.query(dF, dE, "count", count=cnt, ambiguous=amb_c)
    separate["answers_equal_combined_pass"] = bool(
        torch.equal(both_hit, hit) and torch.equal(both_cnt, cnt) and torch.equal(both_amb & 1, amb_h)
        and torch.equal(both_amb >> 1, amb_c))
    bvh.close()

    # end to end through the host-buffer C-ABI calls: mesh and segments in
    # pinned host memory, results back in pinned host memory, every step
    hh = torch.empty(n, dtype=torch.uint8).pin_memory()
    ha = torch.empty(n, dtype=torch.uint8).pin_memory()
    hc = torch.empty(n, dtype=torch.int32).pin_memory()

    def step_e2e():
        bvh = rsi.LBVH(pV, pT, morton_bits=30, treelet_passes=tp)
        bvh.query_host(pF, pE, "both", hit=hh, count=hc, ambiguous=ha)
        bvh.close()

    for _ in range(args.warmup):
        step_e2e()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    barrier()
    e2e_ms = max_over_ranks(pg, 1e3 * (time.perf_counter() - t0) / args.steps, dev)
    same = bool(torch.equal(hh, both_hit.cpu()) and torch.equal(hc, both_cnt.cpu())
                and torch.equal(ha, both_amb.cpu()))
    h2d = (pV.numel() * 4 + pT.numel() * 4) + (pF.numel() + pE.numel()) * 4
    d2h = n * (1 + 4 + 1)

    # the same step on the paper's tree as built (no restructuring): context
    plain_tree = None
    if tp:
        for _ in range(3):
            step(passes=0)
        pl = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(10)]
        for k in range(10):
            step(pl[k], passes=0)
        torch.cuda.synchronize()
        b0 = rsi.LBVH(dV, dT, morton_bits=30)
        plain_tree = {"step_ms": statistics.median(p[0].elapsed_time(p[2]) for p in pl),
                      "build_ms": statistics.median(p[0].elapsed_time(p[1]) for p in pl),
                      "both_modes_query_ms": statistics.median(p[1].elapsed_time(p[2]) for p in pl),
                      "node_visits_per_ray_count": b0.query(dF, dE, "count", stats=True)["stats"]["node_visits"] / n,
                      "tree_height": b0.info()["height"]}
        b0.close()

    # counters of one extra (untimed) pass
    bvh = rsi.LBVH(dV, dT, morton_bits=30, treelet_passes=tp)
    st_c = bvh.query(dF, dE, "count", stats=True)["stats"]
    st_a = bvh.query(dF, dE, "any_hit", stats=True)["stats"]
    job_counts = sum_over_ranks(pg, [st_c["band_rays"], st_c["ambiguous"], st_a["band_rays"], st_a["ambiguous"]],
                                dev)
    height = bvh.info()["height"]
    # traversal kernel time by node width (child-pair, compressed child-pair,
    # four-wide), same answers; on the paper's tree (compressed nodes need its
    # numbering) and, child-pair only, on the restructured one
    widths = {}
    bp = rsi.LBVH(dV, dT, morton_bits=30)
    for w in (2, 3, 4):
        st_w = bp.query(dF, dE, "count", stats=True, node_width=w)["stats"]
        per = {}
        for mode in ("any_hit", "count"):
            ts = []
            for _ in range(5):
                bp.query(dF, dE, mode, hit=hit, count=cnt, ambiguous=amb_c, time_kernels=True, node_width=w)
                ts.append(bp.last_query_ms()[0])
            per[f"{mode}_traverse_ms"] = statistics.median(ts[1:])
        per["node_fetches_per_ray_count"] = st_w["node_visits"] / n
        widths[str(w)] = per
    bp.close()
    if tp:
        per = {}
        for mode in ("any_hit", "count"):
            ts = []
            for _ in range(5):
                bvh.query(dF, dE, mode, hit=hit, count=cnt, ambiguous=amb_c, time_kernels=True)
                ts.append(bvh.last_query_ms()[0])
            per[f"{mode}_traverse_ms"] = statistics.median(ts[1:])
        per["node_fetches_per_ray_count"] = st_c["node_visits"] / n
        widths[f"2_restructured_{tp}_pass"] = per
    # the same queries walking the segments in midpoint-cell order
    # (rsi_segment_order), and a whole step with the order computed in it
    order = bvh.segment_order(dF, dE)
    ordered = {}
    for mode in ("any_hit", "count"):
        ts = []
        for _ in range(5):
            bvh.query(dF, dE, mode, hit=hit, count=cnt, ambiguous=amb_c, time_kernels=True, order=order)
            ts.append(bvh.last_query_ms()[0])
        ordered[f"{mode}_traverse_ms"] = statistics.median(ts[1:])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        bvh.segment_order(dF, dE, out=order)
    e0.record(stream)
    for _ in range(5):
        bvh.segment_order(dF, dE, out=order)
    e1.record(stream)
    torch.cuda.synchronize()
    ordered["order_ms"] = e0.elapsed_time(e1) / 5

    def step_ordered():
        b = rsi.LBVH(dV, dT, morton_bits=30, treelet_passes=tp)
        b.segment_order(dF, dE, out=order)
        b.query(dF, dE, "both", hit=hit, count=cnt, ambiguous=amb2, order=order)
        b.close()
    for _ in range(3):
        step_ordered()
    e0.record(stream)
    for _ in range(10):
        step_ordered()
    e1.record(stream)
    torch.cuda.synchronize()
    ordered["step_ms"] = e0.elapsed_time(e1) / 10
    bvh.close()

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    peak, peak_kind = peaks()
    achieved = BYTES_PER_RAY_COUNT * n / (trav_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_triangles": int(len(mesh.triangles)), "rays_per_gpu": n,
                   "morton_bits": 30, "l2": "inputs larger than L2 (240 MB of segments per batch), no flush",
                   "segment_order": bool(args.order),
                   "tree": (f"the paper's Karras build + {tp} treelet restructuring pass(es) (depth-tiled treelets of "
                            "up to 7 subtrees; answers identical to the plain tree's)") if tp
                   else "the paper's Karras build as built",
                   "fp64_retest": "on (band segments re-tested in FP64)"},
        "roofline": {"kernel": "k_query_fp32<count> (FP32 traversal, intercept_count)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s",
                     "traffic": traffic_per_launch(), "algorithmic_bytes_per_ray": BYTES_PER_RAY_COUNT,
                     "kernel_ms": trav_ms, "second_bound": second_bound()},
        "l2_issue_bound": issue_bound(),
        "e2e": {"value": ws * n / (e2e_ms / 1e3), "unit": "rays/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "matches_device_results": same},
        "gpu_launches": launches,
        "clocks": clocks,
        "phases_ms": {"build": build_ms, "both_modes_query": both_ms},
        "query_rays_per_s": {"both_modes": n / (both_ms / 1e3),
                             "any_hit_alone": n / (separate["any_hit_query_ms"] / 1e3),
                             "count_alone": n / (separate["count_query_ms"] / 1e3)},
        "separate_queries": separate,
        "plain_tree": plain_tree,
        "counters": {"tree_height": height, "node_visits_per_ray_count": st_c["node_visits"] / n,
                     "tri_tests_per_ray_count": st_c["tri_tests"] / n, "band_rays_count": st_c["band_rays"],
                     "ambiguous_count": st_c["ambiguous"], "node_visits_per_ray_any": st_a["node_visits"] / n,
                     "band_rays_any": st_a["band_rays"], "ambiguous_any": st_a["ambiguous"]},
        "counters_all_ranks": dict(zip(("band_rays_count", "ambiguous_count", "band_rays_any", "ambiguous_any"),
                                       job_counts)),
        "node_width": widths,
        "segment_order": ordered,
    }
    if not args.no_builders:
        line["builders"] = measure_builders(rsi, torch, dev, [("c2", mesh), ("c3", W.config_mesh("c3"))],
                                            c4, reps=max(5, min(args.steps, 20)))
    if paper is not None:
        line["paper_scale_e2e"] = measure_paper_scale(rsi, torch, dev, paper, args)
    if c3 is not None:
        line["precision_c3"] = measure_precision_c3(rsi, torch, dev, c3, args)
        c3 = None
    if not args.no_nearest:
        line["barycentric_c2"] = measure_nearest(rsi, torch, dev, pV, pT, pF, pE, dV, dT, dF, dE, args)
    if c4 is not None:
        line["batched_c4"] = measure_batched(rsi, torch, dev, c4, args)
    if c5 is not None:
        line["learned_c5"] = measure_learned(rsi, torch, dev, c5, args)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mesh, W.config_rays("c2"), args.cpu_sample)
    print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
