"""Tuned survey plans, kept in a versioned JSON file beside the library.

``tuned_plans.json`` maps a workload name to the plan tripoll_tune chose for
it on a B300 (the four tripoll_plan fields), with the measured survey times
of the tuned and the default plan and the GPU it ran on.  The file carries a
format version; a file of another version is ignored.

  python -m paper_2107_12330_b300.tuning rmat24 [--out PATH]

tunes the named workload on cuda:0 and writes (or updates) its entry.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
PLANS_PATH = os.path.join(HERE, "tuned_plans.json")
FORMAT_VERSION = 1
PLAN_FIELDS = ("warp_max_dplus", "block_item_in_edges", "long_list_min_dplus", "window_view")


def load_plans(path: str = PLANS_PATH) -> dict:
    """Workload name -> entry; empty when the file is absent or of another format version."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    if data.get("version") != FORMAT_VERSION:
        return {}
    return data.get("plans", {})


def plan_for(workload: str, path: str = PLANS_PATH):
    """The tuned plan of a workload (a dict of the tripoll_plan fields), or None."""
    e = load_plans(path).get(workload)
    if not e or not all(k in e.get("plan", {}) for k in PLAN_FIELDS):
        return None
    return {k: int(e["plan"][k]) for k in PLAN_FIELDS}


def store_plan(workload: str, entry: dict, path: str = PLANS_PATH) -> None:
    plans = load_plans(path)
    plans[workload] = entry
    with open(path, "w") as f:
        json.dump({"version": FORMAT_VERSION, "plans": plans}, f, indent=1, sort_keys=True)
        f.write("\n")


def _workload(name: str):
    """(graph inputs, kinds, window, batched offsets or None) of a named workload."""
    root = os.path.dirname(HERE)
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    import synth
    if name.startswith("rmat"):
        return synth.rmat(int(name[4:]), 1), None
    if name.startswith("batched"):
        G = int(name[7:])
        graphs = [synth.batched_graph(i) for i in range(G)]
        eoff = np.zeros(G + 1, np.uint64)
        eoff[1:] = np.cumsum([g.m_in for g in graphs])
        nv = np.array([g.n for g in graphs], np.uint32)
        cat = {k: np.concatenate([getattr(g, k) for g in graphs]) for k in ("src", "dst", "ts", "vlabel")}
        return cat, (eoff, nv)
    raise ValueError(f"unknown workload {name}")


def tune(name: str, reps: int = 3, out: str = PLANS_PATH) -> dict:
    import torch
    import paper_2107_12330_b300 as tp
    torch.cuda.set_device(0)
    g, batch = _workload(name)
    if batch is None:
        dev = [torch.from_numpy(x).cuda() for x in (g.src, g.dst, g.ts, g.elabel, g.vlabel)]
        h = tp.tripoll_graph_create(*dev, g.n, g.num_vlabels, g.num_elabels)
        kinds, (lo, hi) = g.kinds, g.window
    else:
        eoff, nv = batch
        d = {k: torch.from_numpy(v).cuda() for k, v in g.items()}
        h = tp.tripoll_batch_create(d["src"], d["dst"], d["ts"], None, eoff, d["vlabel"], nv, 4, 0)
        kinds, (lo, hi) = tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST, (0, 0xFFFFFFFF)
    try:
        tp.tripoll_set_plan(h, tp.DEFAULT_PLAN)
        plan, best_ms, start_ms = tp.tripoll_tune(h, kinds, lo, hi, reps)
    finally:
        tp.tripoll_destroy(h)
    entry = {"plan": plan, "survey_ms": best_ms, "default_plan_ms": start_ms, "kinds": kinds, "window": [lo, hi],
             "gpu": torch.cuda.get_device_name(0), "reps": reps,
             "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    store_plan(name, entry, out)
    return entry


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", nargs="+", help="rmat<scale> or batched<graphs>")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=PLANS_PATH)
    args = ap.parse_args()
    for w in args.workload:
        print(w, json.dumps(tune(w, args.reps, args.out)), flush=True)


if __name__ == "__main__":
    main()
