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
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(RECIPES))
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    args = ap.parse_args()
    g = RECIPES[args.name]()
    t0 = time.time()
    r = oracle.survey_graph(g, threads=args.threads, extras=())
    dt = time.time() - t0
    vec = oracle.result_vector(r, g.kinds, g.num_vlabels, g.num_elabels)
    out = {"workload": args.name, "kinds": g.kinds, "window": list(g.window), "n": g.n, "m_in": g.m_in,
           "num_vlabels": g.num_vlabels, "num_elabels": g.num_elabels, "stats": r["stats"],
           "result": [int(x) for x in vec], "oracle_seconds": round(dt, 1), "oracle_threads": args.threads}
    path = os.path.join(HERE, f"{args.name}_survey.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, int(vec[0]) if len(vec) else 0, f"{dt:.1f}s")


if __name__ == "__main__":
    main()
