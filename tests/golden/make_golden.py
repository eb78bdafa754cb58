"""Write the stored expected surveys of the full-size workloads.

Every value in tests/golden/*.json comes from this script, which calls only
the CPU oracle (oracle/) on inputs from the seeded generators (synth/):

  python tests/golden/make_golden.py rmat24 [--threads N]

Each file holds the oracle's survey tables for the workload's kinds and
window, the G+ statistics, and the recipe name, so a GPU test can compare the
library's full-size result word by word.
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

RECIPES = {
    "rmat24": synth.rmat24,
    "rmat20": lambda: synth.rmat(20, 1),
    "rmat22": lambda: synth.rmat(22, 1),
    # the 50M-vertex Chung-Lu recipe at 2M vertices (28 sampled pairs per vertex, as at full size)
    "chunglu2m": lambda: synth.chung_lu_50m(m_samples=56_000_000, n=2_000_000),
    # the full 50M-vertex Chung-Lu workload (1.2G sampled pairs, about 995M unique edges)
    "chunglu50m": lambda: synth.chung_lu_50m(),
}
# workloads whose result vector is stored by digest (large label-triple tables)
DIGEST_ONLY = {"chunglu2m", "chunglu50m"}


BATCH_KINDS = synth.COUNT | synth.CLOSURE_HIST


def _batched_one(i):
    g = synth.batched_graph(i)
    r = oracle.survey_graph(g, extras=())
    return oracle.result_vector(r, BATCH_KINDS, g.num_vlabels, g.num_elabels)


def batched(num_graphs, procs):
    """Per-graph oracle surveys of the batched family, graphs 0..num_graphs-1."""
    import hashlib
    import multiprocessing as mp
    import numpy as np
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        vecs = pool.map(_batched_one, range(num_graphs), chunksize=64)
    dt = time.time() - t0
    allv = np.concatenate(vecs).astype("<u8")
    out = {"workload": f"batched{num_graphs}", "kinds": BATCH_KINDS, "num_graphs": num_graphs,
           "words_per_graph": int(vecs[0].shape[0]),
           "sha256": hashlib.sha256(allv.tobytes()).hexdigest(),
           "counts": [int(v[0]) for v in vecs],
           "hist_total": [int(x) for x in allv.reshape(num_graphs, -1)[:, 1:].sum(axis=0)],
           "oracle_seconds": round(dt, 1), "oracle_procs": procs}
    path = os.path.join(HERE, f"batched{num_graphs}_survey.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, sum(out["counts"]), f"{dt:.1f}s")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(RECIPES) + ["batched"])
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("--graphs", type=int, default=20000)
    args = ap.parse_args()
    if args.name == "batched":
        batched(args.graphs, args.threads)
        return
    g = RECIPES[args.name]()
    t0 = time.time()
    r = oracle.survey_graph(g, threads=args.threads, extras=())
    dt = time.time() - t0
    vec = oracle.result_vector(r, g.kinds, g.num_vlabels, g.num_elabels)
    out = {"workload": args.name, "kinds": g.kinds, "window": list(g.window), "n": g.n, "m_in": g.m_in,
           "num_vlabels": g.num_vlabels, "num_elabels": g.num_elabels, "stats": r["stats"],
           "oracle_seconds": round(dt, 1), "oracle_threads": args.threads}
    if args.name in DIGEST_ONLY:
        import hashlib
        import numpy as np
        out["sha256"] = hashlib.sha256(np.asarray(vec, dtype="<u8").tobytes()).hexdigest()
        out["words"] = int(len(vec))
        out["count"] = int(r["count"][0])
        out["hist"] = [int(x) for x in r["hist"]]
        out["etri"] = [int(x) for x in r["etri"]]
    else:
        out["result"] = [int(x) for x in vec]
    path = os.path.join(HERE, f"{args.name}_survey.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, int(vec[0]) if len(vec) else 0, f"{dt:.1f}s")


if __name__ == "__main__":
    main()
