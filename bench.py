"""Benchmark of the metadata triangle survey on one B300 (or N, one process each).

A step is one pass of the whole hot path over the R-MAT scale-24 workload:
build G+ on the device from the resident edge arrays (dedup, degree order,
orientation, CSR, in-edge lists, survey plan), run the survey (closure-time
histogram + edge-type triples inside the window covering the middle half of
time), release the graph.  One JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tripoll|reference]

--impl reference times the CPU oracle (the plain C node-iterator) on the
host cores over a bounded sample of the same workload family.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "triangles surveyed/s"
UNIT = "triangles/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic of the survey per algorithmic byte, from the last ncu capture of
# survey_block_kernel on R-MAT scale 22 (6.39 GB read, 3.4 MB written, for 9.92 GB
# of algorithmic bytes), valid only for the survey source it was taken on (first 16
# hex digits of the SHA-256 of the kernels and their dispatch); any other source
# reports null.
PROFILED_SURVEY = {"sha256_16": "e993e1b8d415a105", "dram_per_alg_byte": (6.386344e9 + 3.368448e6) / 9.917552541e9,
                   "capture": "ncu, survey_block_kernel, R-MAT scale 22, scaled by algorithmic bytes"}


# The batched family's survey is one survey_warp_kernel launch; DRAM bytes of the
# timed launch over 2000 graphs of the same family (ncu), per algorithmic byte.
PROFILED_BATCHED_SURVEY = {"sha256_16": "e993e1b8d415a105", "dram_per_alg_byte": (1108644352 + 404736) / 3459588372,
                           "capture": "ncu, survey_warp_kernel, the same family at 2000 graphs, scaled by "
                                      "algorithmic bytes"}


def survey_source_sha16() -> str:
    """First 16 hex digits of the SHA-256 of the survey kernels' source (kernels, then dispatch)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("survey_kernels.cuh", "survey.cu"):
        with open(os.path.join(ROOT, "paper_2107_12330_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def survey_traffic(alg_bytes: int, profiled=None):
    profiled = profiled or PROFILED_SURVEY
    sha = survey_source_sha16()
    if sha != profiled["sha256_16"]:
        return None, "survey source changed since the last ncu capture"
    return alg_bytes * profiled["dram_per_alg_byte"], profiled["capture"]


def algorithmic_bytes(st: dict, wedge_checks: int, triangles_in_window: int) -> int:
    """Bytes one survey launch must move: the compulsory G+ once (offsets and
    label 9 B per vertex; out-list id, timestamp, edge label and target label
    10 B and the in-edge record 16 B per edge), one 4-byte candidate id per
    wedge check of the window, and the (p,r) edge's timestamp and label (5 B)
    per triangle in the window."""
    n, m = st["num_vertices"], st["num_edges"]
    return 9 * n + (10 + 16) * m + 4 * wedge_checks + 5 * triangles_in_window


def merge_path_bytes(st: dict, triangles_in_window: int) -> int:
    """The bytes a merge-path survey would move: offsets, pivot label and the
    augmented out-list of every pivot once (9 B per vertex, 9 B per edge), the whole out-list of q once per
    directed edge (p,q) (4 B per entry: sum over (p,q) of d+(q)) plus q's label, and 6 B per triangle.  This
    library never re-reads Adj+(q) per in-edge -- it stages it once on chip and probes it with the pivots'
    suffixes -- so this figure counts reads it does not make; it is reported beside the method's own bytes."""
    n, m = st["num_vertices"], st["num_edges"]
    return 9 * n + 9 * m + 4 * st["q_list_words"] + m + 6 * triangles_in_window


def compulsory_bytes(st: dict) -> int:
    """The part of the algorithmic bytes that does not depend on the window:
    G+ with its metadata and in-edge records read once."""
    return 9 * st["num_vertices"] + (10 + 16) * st["num_edges"]


def use_tuned_plan(tp, workload):
    """Start new graphs with the plan the autotuner stored for this workload (tuned_plans.json), if any."""
    from paper_2107_12330_b300 import tuning
    plan = tuning.plan_for(workload)
    tp.tripoll_set_default_plan(plan)
    return {"plan": plan or dict(tp.DEFAULT_PLAN),
            "plan_source": f"autotuned ({workload}, tuned_plans.json v{tuning.FORMAT_VERSION})" if plan else "defaults"}


def run_tripoll(args):
    import torch
    import torch.distributed as dist
    import paper_2107_12330_b300 as tp
    from paper_2107_12330_b300.shard import sharded_survey

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = tp.load_library()

    g = synth.rmat(args.scale, 1)
    kinds = g.kinds
    t_lo, t_hi = g.window
    m_in = g.m_in
    src = torch.from_numpy(g.src).to(dev)
    dst = torch.from_numpy(g.dst).to(dev)
    ts = torch.from_numpy(g.ts).to(dev)
    el = torch.from_numpy(g.elabel).to(dev)
    vl = torch.from_numpy(g.vlabel).to(dev)
    words = tp.tripoll_result_words(kinds, g.num_vlabels, g.num_elabels, g.n)
    result = torch.zeros(words, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = use_tuned_plan(tp, f"rmat{args.scale}")

    def build():
        return tp.tripoll_graph_create(src, dst, ts, el, vl, g.n, g.num_vlabels, g.num_elabels, stream=stream)

    # shard the pivots across ranks (one graph replica each); one sum at the end
    h0 = build()
    info = tp.tripoll_graph_stats(h0)
    wedge_checks = tp.tripoll_wedge_checks(h0, t_lo, t_hi, stream=stream)
    bounds = tp.tripoll_partition_pivots(h0, world)
    tp.tripoll_destroy(h0)

    phases = []

    def step(ev=None):
        h = build()

        def survey_range(lo, hi, out):
            if ev is not None:
                ev[0].record(stream)
                phases.append(tp.tripoll_survey_timed(h, kinds, t_lo, t_hi, lo, hi, out, stream=stream))
                ev[1].record(stream)
            else:
                tp.tripoll_survey_range(h, kinds, t_lo, t_hi, lo, hi, out, stream=stream)

        sharded_survey(survey_range, bounds, rank, result, dist.all_reduce if world > 1 else (lambda x: None))
        tp.tripoll_destroy(h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    res0 = result.cpu().numpy().view(np.uint64).copy()
    triangles = int(res0[0])

    clocks = ClockSampler(local)
    launches0 = tp.tripoll_launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = tp.tripoll_launch_count() - launches0
    ms = start.elapsed_time(end) / args.steps
    survey_ms = [a.elapsed_time(b) for a, b in evs]
    survey_avg = sum(survey_ms) / len(survey_ms)
    survey_med = float(np.percentile(survey_ms, 50))
    survey_p99 = float(np.percentile(survey_ms, 99))
    ph = np.mean(np.array(phases), axis=0) if phases else np.zeros(4)
    t = torch.tensor([ms, survey_avg, survey_med, survey_p99] + list(ph), dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms, survey_avg, survey_med, survey_p99 = float(t[0]), float(t[1]), float(t[2]), float(t[3])
    ph = [float(x) for x in t[4:8]]
    res1 = result.cpu().numpy().view(np.uint64)
    assert np.array_equal(res0, res1), "survey result changed between steps"

    # end-to-end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if rank == 0 and world == 1 and args.e2e_steps > 0:
        # the step's inputs and result in page-locked host memory
        pinned = [None if x is None else torch.from_numpy(x).pin_memory() for x in (g.src, g.dst, g.ts, g.elabel,
                                                                                    g.vlabel)]
        hsrc, hdst, hts, hel, hvl = [None if x is None else x.numpy() for x in pinned]
        res_pinned = torch.zeros(words, dtype=torch.int64).pin_memory()
        host_res = res_pinned.numpy().view(np.uint64)
        for _ in range(1):
            h = tp.tripoll_graph_create(hsrc, hdst, hts, hel, hvl, g.n, g.num_vlabels, g.num_elabels)
            tp.tripoll_survey(h, kinds, t_lo, t_hi, host_res)
            tp.tripoll_destroy(h)
        times = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            h = tp.tripoll_graph_create(hsrc, hdst, hts, hel, hvl, g.n, g.num_vlabels, g.num_elabels)
            tp.tripoll_survey(h, kinds, t_lo, t_hi, host_res)
            tp.tripoll_destroy(h)
            times.append(time.perf_counter() - t0)
        assert int(host_res[0]) == triangles
        e2e_s = sum(times) / len(times)
        e2e = {"value": triangles / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(g.src.nbytes + g.dst.nbytes + g.ts.nbytes + g.elabel.nbytes + g.vlabel.nbytes),
               "d2h_bytes_per_step": int(words * 8), "ms_per_step": e2e_s * 1e3}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    meta_cost = metadata_cost(tp, build, stream) if world == 1 and args.metadata_cost else None
    peak, peak_kind = _peaks()
    alg = algorithmic_bytes(info, wedge_checks, triangles)
    achieved = alg / (survey_avg * 1e-3) / 1e9
    merge_bytes = merge_path_bytes(info, triangles)
    traffic, traffic_src = survey_traffic(alg)
    value = triangles / (ms * 1e-3)
    l2_note = ("inputs larger than L2 (126 MB): %.2f GB of edge records, %.2f GB of graph"
               % (m_in * 13 / 1e9, info["device_bytes"] / 1e9)) if info["device_bytes"] > 126e6 else \
        "graph smaller than L2 (126 MB); the edge records are rebuilt into it every step"
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u32/u64 integer", "data": "synthetic",
        "config": {"workload": rmat_workload(args.scale),
                   "step": "build G+ from device-resident edge arrays + survey + release",
                   "input_edges": m_in, "edges": info["num_edges"], "wedges": info["wedges"], "wedge_checks_in_window": wedge_checks,
                   "triangles_in_window": triangles, "l2": l2_note,
                   "parallelism": f"pivot shards x{world}", **plan},
        "survey_ms": survey_avg, "survey_ms_p50": survey_med, "survey_ms_p99": survey_p99,
        "survey_latency": {"p50_ms": survey_med, "p99_ms": survey_p99, "over": f"{args.steps} timed surveys"},
        "survey_phases_ms": {"window_view": ph[0], "survey_warp_kernel": ph[1], "survey_block_kernel": ph[2],
                             "survey_block_kernel_long_lists": ph[3]},
        "build_ms": ms - survey_avg,
        "survey_triangles_per_s": triangles / (survey_avg * 1e-3),
        "wedge_checks_per_s": wedge_checks / (survey_avg * 1e-3),
        "roofline": {"bound": "hbm",
                     "kernel": "survey launch group on one stream (window view, warp-item kernel, block-item "
                               "kernel, long-list kernel); survey_block_kernel dominates (survey_phases_ms)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind, "algorithmic_bytes": alg,
                     "algorithmic_bytes_formula": "9n + 26m + 4 wedge checks of the window subgraph "
                                                  "+ 5 per triangle in the window",
                     "merge_path_bytes": merge_bytes,
                     "merge_path_frac": merge_bytes / (survey_avg * 1e-3) / 1e9 / peak,
                     "compulsory_bytes": compulsory_bytes(info), "traffic": traffic,
                     "traffic_source": traffic_src},
        "metadata_cost": meta_cost,
        "clocks": clk, "gpu_launches": int(launches), "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    if world > 1:
        dist.destroy_process_group()
    return out


def metadata_cost(tp, build, stream):
    """The cost of metadata in the survey (the paper's Sec. 5.10 measures a degree-triple callback against
    the plain count and finds just under 2x): device time of the full-window survey with the count alone,
    with the count and the degree-log triples, and with the count, closing-time histogram and vertex- and
    edge-label triples, on the same graph (median of 3 after one warm-up each)."""
    import torch
    h = build()
    try:
        st = tp.tripoll_graph_stats(h)
        out = {}
        for name, kinds in (("count", tp.TRIPOLL_COUNT),
                            ("count_degree_triples", tp.TRIPOLL_COUNT | tp.TRIPOLL_DEGREE_TRIPLES),
                            ("count_hist_label_triples", tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST |
                             tp.TRIPOLL_VLABEL_TRIPLES | tp.TRIPOLL_ELABEL_TRIPLES)):
            w = tp.tripoll_result_words(kinds, st["num_vlabels"], max(1, st["num_elabels"]), st["num_vertices"])
            res = torch.zeros(w, dtype=torch.int64, device="cuda")
            times = []
            for k in range(4):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                tp.tripoll_survey(h, kinds, 0, 0xFFFFFFFF, res, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if k:
                    times.append(a.elapsed_time(b))
            out[name + "_ms"] = float(np.median(times))
        out["degree_triples_over_count"] = out["count_degree_triples_ms"] / out["count_ms"]
        out["label_tables_over_count"] = out["count_hist_label_triples_ms"] / out["count_ms"]
        out["window"] = "full (every triangle)"
        return out
    finally:
        tp.tripoll_destroy(h)


def cpu_model() -> str:
    """The host CPU's model name, as the kernel reports it (empty when unknown)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return ""


def cpu_baseline(args, scale=None):
    """The oracle as it stands on the host cores, over a bounded sample: the same
    R-MAT recipe at a smaller scale (the full scale-24 survey takes the oracle
    tens of minutes)."""
    import oracle
    scale = scale or args.cpu_scale
    g = synth.rmat(scale, 1)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.survey_graph(g, threads=cores, extras=())
    dt = time.perf_counter() - t0
    tri = int(r["count"][0])
    # the same oracle on one thread, over a smaller sample so that it stays within seconds
    s1 = max(10, scale - 2)
    g1 = synth.rmat(s1, 1)
    t0 = time.perf_counter()
    r1 = oracle.survey_graph(g1, threads=1, extras=())
    dt1 = time.perf_counter() - t0
    tri1 = int(r1["count"][0])
    return {"value": tri / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"R-MAT scale {scale} with the same recipe (seed 1), full survey incl. build, "
                      f"{tri} triangles in {dt:.2f} s",
            "single_thread": {"value": tri1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"R-MAT scale {s1}, same recipe, {tri1} triangles in {dt1:.2f} s"}}


def rmat_workload(scale):
    return (f"R-MAT scale {scale}, edge factor 16, a/b/c/d .57/.19/.19/.05, seed 1; ts uniform [0,2^30), "
            "vlabel 16, etype Zipf(1.2) over 8; survey = count + closure histogram + edge-type triples in window "
            "[2^28, 3*2^28-1]")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    g = synth.rmat(args.cpu_scale, 1)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.survey_graph(g, threads=cores, extras=())
    times = []
    tri = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.survey_graph(g, threads=cores, extras=())
        times.append(time.perf_counter() - t0)
        tri = int(r["count"][0])
    s = sum(times) / len(times)
    v = tri / s
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": s * 1e3, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "u32/u64 integer", "data": "synthetic",
            "config": {"workload": rmat_workload(args.scale),
                       "step": "the oracle on the host cores over a bounded sample of the workload",
                       "parallelism": f"{cores} host threads"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": f"each step: R-MAT scale {args.cpu_scale} with the same recipe (seed 1), "
                                       f"full survey including the build, {tri} triangles"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def batched_inputs(num_graphs):
    graphs = [synth.batched_graph(i) for i in range(num_graphs)]
    eoff = np.zeros(num_graphs + 1, np.uint64)
    eoff[1:] = np.cumsum([g.m_in for g in graphs])
    nv = np.array([g.n for g in graphs], np.uint32)
    cat = {k: np.concatenate([getattr(g, k) for g in graphs]) for k in ("src", "dst", "ts", "vlabel")}
    return graphs, eoff, nv, cat


def run_batched(args):
    """The batched workload: many small graphs built together and surveyed in one
    launch pair with per-graph records, against one survey launch per graph."""
    import torch
    import paper_2107_12330_b300 as tp
    lib = tp.load_library()
    dev = torch.device("cuda", 0)
    kinds = tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST
    G = args.graphs
    graphs, eoff, nv, cat = batched_inputs(G)
    d = {k: torch.from_numpy(v).to(dev) for k, v in cat.items()}
    w = tp.tripoll_result_words(kinds, 4, 1, 0)
    result = torch.zeros(w * G, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = use_tuned_plan(tp, f"batched{G}")

    def build():
        return tp.tripoll_batch_create(d["src"], d["dst"], d["ts"], None, eoff, d["vlabel"], nv, 4, 0, stream=stream)

    h0 = build()
    info = tp.tripoll_graph_stats(h0)
    wedge_checks = tp.tripoll_wedge_checks(h0, stream=stream)
    tp.tripoll_destroy(h0)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step(ev=None):
        h = build()
        if ev:
            ev[0].record(stream)
        tp.tripoll_survey(h, kinds, 0, 0xFFFFFFFF, result, stream=stream)
        if ev:
            ev[1].record(stream)
        tp.tripoll_destroy(h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = tp.tripoll_launch_count()
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = tp.tripoll_launch_count() - l0
    ms = start.elapsed_time(end) / args.steps
    survey_ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    res = result.cpu().numpy().view(np.uint64).reshape(G, w)
    triangles = int(res[:, 0].sum())

    # one survey launch per graph over the same graphs, each built alone beforehand
    P = min(G, args.plain_graphs)
    handles = [tp.tripoll_graph_create(g.src, g.dst, g.ts, None, g.vlabel, g.n, 4, 0) for g in graphs[:P]]
    outs = torch.zeros(w * P, dtype=torch.int64, device=dev)
    for i, h in enumerate(handles[:8]):
        tp.tripoll_survey(h, kinds, 0, 0xFFFFFFFF, outs[i * w:(i + 1) * w], stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i, h in enumerate(handles):
        tp.tripoll_survey(h, kinds, 0, 0xFFFFFFFF, outs[i * w:(i + 1) * w], stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    plain_survey_ms = a.elapsed_time(b)
    plain = outs.cpu().numpy().view(np.uint64).reshape(P, w)
    assert np.array_equal(plain, res[:P]), "batched and per-graph surveys differ"
    sample = graphs[:max(1, min(G, args.plain_build_graphs))]
    t0 = time.perf_counter()
    for g in sample:
        h = tp.tripoll_graph_create(g.src, g.dst, g.ts, None, g.vlabel, g.n, 4, 0)
        tp.tripoll_survey(h, kinds, 0, 0xFFFFFFFF, outs[:w], stream=stream)
        tp.tripoll_destroy(h)
    torch.cuda.synchronize()
    plain_full_s = (time.perf_counter() - t0) / len(sample)
    for h in handles:
        tp.tripoll_destroy(h)
    batched_graphs_per_s = G / (survey_ms * 1e-3)
    plain_graphs_per_s = P / (plain_survey_ms * 1e-3)
    peak, peak_kind = _peaks()
    alg = algorithmic_bytes(info, wedge_checks, triangles)
    achieved = alg / (survey_ms * 1e-3) / 1e9
    traffic, traffic_src = survey_traffic(alg, PROFILED_BATCHED_SURVEY)
    return {
        "metric": "graphs surveyed/s (batched)", "value": G / (ms * 1e-3), "unit": "graphs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 integer", "data": "synthetic",
        "config": {"workload": f"{G} Chung-Lu graphs, exponent 2.5, n log-uniform [32,8192], mean degree "
                               "uniform [4,64], seeds 0..; ts uniform [0,2^20), vlabel 4; per-graph count + "
                               "closure histogram", "input_edges": int(eoff[-1]), "edges": info["num_edges"],
                   "wedges": info["wedges"], "triangles": triangles,
                   "step": "batched build + one survey launch pair + release", **plan},
        "triangles_per_s": triangles / (ms * 1e-3), "survey_ms": survey_ms, "build_ms": ms - survey_ms,
        "survey_graphs_per_s": batched_graphs_per_s,
        "plain_path": {"graphs": P, "survey_graphs_per_s": plain_graphs_per_s,
                       "batched_over_plain_survey": batched_graphs_per_s / plain_graphs_per_s,
                       "build_and_survey_ms_per_graph": plain_full_s * 1e3,
                       "batched_over_plain_build_and_survey": (G / (ms * 1e-3)) * plain_full_s},
        "roofline": {"bound": "hbm", "kernel": "survey (one launch pair, all graphs)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                     "algorithmic_bytes": alg, "compulsory_bytes": compulsory_bytes(info), "traffic": traffic,
                     "traffic_source": traffic_src},
        "clocks": clk, "gpu_launches": int(launches),
    }


def run_chunglu(args):
    """The 50M-vertex Chung-Lu graph (exponent 2.1, ~1B unique edges): build and
    full survey (count, closure histogram, vertex- and edge-label triples)."""
    import torch
    import paper_2107_12330_b300 as tp
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    g = synth.chung_lu_50m(m_samples=args.samples)
    gen_s = time.perf_counter() - t0
    dev = [torch.from_numpy(x).cuda() for x in (g.src, g.dst, g.ts, g.elabel, g.vlabel)]
    stream = torch.cuda.current_stream()
    w = tp.tripoll_result_words(g.kinds, g.num_vlabels, g.num_elabels, g.n)
    out = torch.zeros(w, dtype=torch.int64, device="cuda")
    times = []
    for k in range(args.warmup + args.steps):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        h = tp.tripoll_graph_create(*dev, g.n, g.num_vlabels, g.num_elabels, stream=stream)
        b.record(stream)
        tp.tripoll_survey(h, g.kinds, 0, 0xFFFFFFFF, out, stream=stream)
        c.record(stream)
        torch.cuda.synchronize()
        if k == 0:
            info = tp.tripoll_graph_stats(h)
        tp.tripoll_destroy(h)
        if k >= args.warmup:
            times.append((a.elapsed_time(b), b.elapsed_time(c)))
    res = out.cpu().numpy().view(np.uint64)
    parts = tp.split_result(res, g.kinds, g.num_vlabels, g.num_elabels)
    tri = int(parts["count"][0])
    for k in ("hist", "vtri", "etri"):
        assert int(parts[k].sum()) == tri, k
    build_ms = sum(t[0] for t in times) / len(times)
    survey_ms = sum(t[1] for t in times) / len(times)
    return {"metric": METRIC, "value": tri / ((build_ms + survey_ms) * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": build_ms + survey_ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32/u64 integer",
            "data": "synthetic",
            "config": {"workload": f"Chung-Lu exponent 2.1, 50M vertices, {args.samples} sampled pairs; ts Poisson "
                                   "over 3.15e8 s; vlabel Zipf(1.1) over 64; elabel uniform over 8; full survey",
                       "input_edges": g.m_in, "edges": info["num_edges"], "wedges": info["wedges"],
                       "dplus_max": info["dplus_max"], "degree_max": info["degree_max"], "triangles": tri,
                       "generate_s": gen_s},
            "build_ms": build_ms, "survey_ms": survey_ms, "survey_triangles_per_s": tri / (survey_ms * 1e-3),
            "device_bytes": info["device_bytes"]}


def run_serve(args):
    """The serving workload: resident R-MAT graphs and a Poisson stream of survey
    requests (4 kinds, random windows), served by the library's continuous-
    batching server, against one request per launch in arrival order."""
    import torch
    import paper_2107_12330_b300 as tp
    torch.cuda.set_device(0)
    scales = [int(x) for x in args.serve_scales.split(",")]
    handles, infos = [], []
    for i, sc in enumerate(scales):
        g = synth.rmat_graph(sc, 16, i + 1, ts_bits=24, num_vlabels=16, num_elabels=8)
        dev = [torch.from_numpy(x).cuda() for x in (g.src, g.dst, g.ts, g.elabel, g.vlabel)]
        handles.append(tp.tripoll_graph_create(*dev, g.n, 16, 8))
        infos.append((g.n, sc))
        del dev
        torch.cuda.synchronize()
    kinds_set = [tp.TRIPOLL_COUNT, tp.TRIPOLL_CLOSURE_HIST, tp.TRIPOLL_VLABEL_TRIPLES, tp.TRIPOLL_ELABEL_TRIPLES]
    R = args.requests
    draws = [synth.draw(99, 1, i) for i in range(4 * R)]
    reqs = []
    for i in range(R):
        gi = (draws[4 * i] >> 32) * len(scales) >> 32
        kind = kinds_set[(draws[4 * i + 1] >> 32) * 4 >> 32]
        lo = (draws[4 * i + 2] >> 40) % ((1 << 24) + 1)
        hi = (draws[4 * i + 3] >> 40) % ((1 << 24) + 1)
        reqs.append((int(gi), kind, int(min(lo, hi)), int(max(lo, hi))))
    words = [tp.tripoll_result_words(k, 16, 8, infos[gi][0]) for gi, k, _, _ in reqs]

    # one request per launch, in order, each to completion
    outs_plain = []
    t0 = time.perf_counter()
    lat_plain = []
    for (gi, k, lo, hi), w in zip(reqs, words):
        o = np.zeros(w, np.uint64)
        s = time.perf_counter()
        tp.tripoll_survey(handles[gi], k, lo, hi, o)
        lat_plain.append(time.perf_counter() - s)
        outs_plain.append(o)
    plain_s = time.perf_counter() - t0

    srv = tp.tripoll_server_create(args.scratch_gb << 30, args.max_inflight)
    slots = [tp.tripoll_server_add_graph(srv, h) for h in handles]
    # burst: every request queued at once -> throughput
    t0 = time.perf_counter()
    ids = [tp.tripoll_server_submit(srv, slots[gi], k, lo, hi) for gi, k, lo, hi in reqs]
    lat_burst = []
    for rid, w, want in zip(ids, words, outs_plain):
        o = np.zeros(w, np.uint64)
        lat_burst.append(tp.tripoll_server_wait(srv, rid, o, 600000) * 1e-9)
        assert np.array_equal(o, want), "served result differs from the request alone"
    served_s = time.perf_counter() - t0
    burst_stats = tp.tripoll_server_stats(srv)
    # Poisson arrivals at fractions of the served capacity -> latency under load
    def poisson(load, stream):
        rate = load * R / served_s
        gaps = [-np.log(1.0 - ((synth.draw(7, stream, i) >> 11) * 2.0 ** -53)) / rate for i in range(R)]
        before = tp.tripoll_server_stats(srv)
        ids = []
        t_next = time.perf_counter()
        for (gi, k, lo, hi), gap in zip(reqs, gaps):
            t_next += gap
            while time.perf_counter() < t_next:
                pass
            ids.append(tp.tripoll_server_submit(srv, slots[gi], k, lo, hi))
        lat = []
        for rid, w in zip(ids, words):
            o = np.zeros(w, np.uint64)
            lat.append(tp.tripoll_server_wait(srv, rid, o, 600000) * 1e-9)
        after = tp.tripoll_server_stats(srv)
        return rate, lat, {k: after[k] - before[k] for k in after}

    loads = [float(x) for x in args.loads.split(",")] if args.loads else []
    if args.load not in loads:
        loads.append(args.load)
    sweep = []
    for j, load in enumerate(sorted(loads)):
        rate, lat, st = poisson(load, 2 + j)
        sweep.append({"load": load, "rate_per_s": rate, "lat": lat, "server": st})
    tp.tripoll_server_destroy(srv)
    for h in handles:
        tp.tripoll_destroy(h)

    def pct(x, q):
        return float(np.percentile(np.array(x) * 1e3, q))

    return {
        "metric": "survey requests/s (served)", "value": R / served_s, "unit": "requests/s", "n_gpus": 1,
        "steps": 1, "warmup": 0, "ms_per_step": served_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32/u64 integer", "data": "synthetic",
        "config": {"workload": f"resident R-MAT graphs scales {scales} (edge factor 16, seeds 1..), ts uniform "
                               "[0,2^24), vlabel 16, etype Zipf(1.2) over 8; requests: kind uniform over count / "
                               "closure histogram / vertex-label triples / edge-label triples, windows uniform "
                               "in [0,2^24]", "requests": R, "scratch_cap_gb": args.scratch_gb,
                   "max_inflight": args.max_inflight},
        "plain_path": {"requests_per_s": R / plain_s, "p50_ms": pct(lat_plain, 50), "p99_ms": pct(lat_plain, 99)},
        "served_burst": {"requests_per_s": R / served_s, "p50_ms": pct(lat_burst, 50), "p99_ms": pct(lat_burst, 99),
                         "server": burst_stats},
        "served_poisson": next({"load": r["load"], "rate_per_s": r["rate_per_s"], "p50_ms": pct(r["lat"], 50),
                                "p99_ms": pct(r["lat"], 99), "server": r["server"]}
                               for r in sweep if r["load"] == args.load),
        "served_poisson_sweep": [{"load": r["load"], "rate_per_s": r["rate_per_s"], "p50_ms": pct(r["lat"], 50),
                                  "p99_ms": pct(r["lat"], 99)} for r in sweep],
        "served_over_plain": plain_s / served_s,
    }


def _ensure_built():
    """Compile libtripoll.so (nvcc, sm_103a, in tree) if this checkout has none."""
    from paper_2107_12330_b300 import build as libbuild
    if not os.path.exists(libbuild.LIB):
        libbuild.build()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tripoll", choices=["tripoll", "reference"])
    ap.add_argument("--workload", default="rmat", choices=["rmat", "batched", "serve", "chunglu"])
    ap.add_argument("--samples", type=int, default=1_200_000_000)
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--cpu-scale", type=int, default=19)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-metadata-cost", dest="metadata_cost", action="store_false")
    ap.add_argument("--graphs", type=int, default=20000)
    ap.add_argument("--plain-graphs", type=int, default=20000)
    ap.add_argument("--plain-build-graphs", type=int, default=200)
    ap.add_argument("--serve-scales", default="16,18,20,22,24,26,16,18")
    ap.add_argument("--requests", type=int, default=400)
    ap.add_argument("--scratch-gb", type=int, default=40)
    ap.add_argument("--max-inflight", type=int, default=32)
    ap.add_argument("--load", type=float, default=0.7)
    ap.add_argument("--loads", default="0.3,0.5,0.9",
                    help="serve: further Poisson loads (fractions of the served capacity) for the latency sweep")
    args = ap.parse_args()
    if args.impl != "reference":
        _ensure_built()
    if args.impl == "reference":
        out = run_reference(args)
    elif args.workload == "batched":
        out = run_batched(args)
    elif args.workload == "serve":
        out = run_serve(args)
    elif args.workload == "chunglu":
        out = run_chunglu(args)
    else:
        out = run_tripoll(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
