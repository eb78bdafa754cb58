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


def algorithmic_bytes(st: dict, triangles_in_window: int) -> int:
    """Bytes the survey must move per launch (measurement):
    the compulsory G+ once (offsets 8 B/vertex, label 1 B/vertex, out-list ids,
    timestamps and edge labels 9 B/edge, in-edge records 16 B/edge), one 4-byte
    candidate id per wedge check (|W+|), and 5 bytes per triangle for the (p,r)
    edge's timestamp and label gathered at the hit."""
    n, m, w = st["num_vertices"], st["num_edges"], st["wedges"]
    return 9 * n + (9 + 16) * m + 4 * w + 5 * triangles_in_window


def run_tripoll(args):
    import torch
    import torch.distributed as dist
    import paper_2107_12330_b300 as tp

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

    def build():
        return tp.tripoll_graph_create(src, dst, ts, el, vl, g.n, g.num_vlabels, g.num_elabels, stream=stream)

    # shard the pivots across ranks (one graph replica each); one sum at the end
    h0 = build()
    info = tp.tripoll_graph_stats(h0)
    bounds = tp.tripoll_partition_pivots(h0, world)
    p_lo, p_hi = int(bounds[rank]), int(bounds[rank + 1])
    tp.tripoll_destroy(h0)

    def step(ev=None):
        h = build()
        if ev is not None:
            ev[0].record(stream)
        tp.tripoll_survey_range(h, kinds, t_lo, t_hi, p_lo, p_hi, result, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        if world > 1:
            dist.all_reduce(result)
        tp.tripoll_destroy(h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    res0 = result.cpu().numpy().view(np.uint64).copy()
    triangles = int(res0[0])

    clocks = ClockSampler(local)
    launches0 = lib.tripoll_launch_count()
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
    launches = lib.tripoll_launch_count() - launches0
    ms = start.elapsed_time(end) / args.steps
    survey_ms = [a.elapsed_time(b) for a, b in evs]
    survey_avg = sum(survey_ms) / len(survey_ms)
    t = torch.tensor([ms, survey_avg], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms, survey_avg = float(t[0]), float(t[1])
    res1 = result.cpu().numpy().view(np.uint64)
    assert np.array_equal(res0, res1), "survey result changed between steps"

    # end-to-end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if rank == 0 and world == 1 and args.e2e_steps > 0:
        host_res = np.zeros(words, np.uint64)
        for _ in range(1):
            h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels)
            tp.tripoll_survey(h, kinds, t_lo, t_hi, host_res)
            tp.tripoll_destroy(h)
        times = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels)
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
    peak, peak_kind = _peaks()
    alg = algorithmic_bytes(info, triangles)
    achieved = alg / (survey_avg * 1e-3) / 1e9
    value = triangles / (ms * 1e-3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u32/u64 integer", "data": "synthetic",
        "config": {"workload": f"R-MAT scale {args.scale}, edge factor 16, a/b/c/d .57/.19/.19/.05, seed 1; "
                               "ts uniform [0,2^30), vlabel 16, etype Zipf(1.2) over 8; survey = count + "
                               "closure histogram + edge-type triples in window [2^28, 3*2^28-1]",
                   "step": "build G+ from device-resident edge arrays + survey + release",
                   "input_edges": m_in, "edges": info["num_edges"], "wedges": info["wedges"],
                   "triangles_in_window": triangles, "l2": "inputs larger than L2 (126 MB)",
                   "parallelism": f"pivot shards x{world}"},
        "survey_ms": survey_avg, "build_ms": ms - survey_avg,
        "survey_triangles_per_s": triangles / (survey_avg * 1e-3),
        "wedge_checks_per_s": info["wedges"] / (survey_avg * 1e-3),
        "roofline": {"bound": "hbm", "kernel": "survey (wedge-check + fold kernels, one launch pair)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind, "algorithmic_bytes": alg, "traffic": None},
        "clocks": clk, "gpu_launches": int(launches), "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    if world > 1:
        dist.destroy_process_group()
    return out


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
    return {"value": tri / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"R-MAT scale {scale} with the same recipe (seed 1), full survey incl. build, "
                      f"{tri} triangles in {dt:.2f} s"}


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
            "config": {"workload": f"R-MAT scale {args.cpu_scale} sample of the scale-24 recipe"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"R-MAT scale {args.cpu_scale}, same recipe, per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tripoll", choices=["tripoll", "reference"])
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--cpu-scale", type=int, default=19)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    out = run_reference(args) if args.impl == "reference" else run_tripoll(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
