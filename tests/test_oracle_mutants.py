"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle.c`` (a dropped term, a
wrong sign or index, a transposed operand, an off-by-one), builds it with gcc
into a temporary directory and runs the pin suite of ``test_oracle.py``
against that build in a child process.  The pins pass on the real oracle (its
own test file), so every mutant here must make at least one of them fail.
Nothing in this file touches a GPU or the survey library.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, exact text in oracle.c, replacement)
MUTANTS = [
    # closing-time bin: floor(log2) instead of ceil(log2) (Alg. 4)
    ("bin_floor", "while (k < 64 && ((uint64_t)1 << k) < x) ++k;",
     "while (k < 63 && ((uint64_t)2 << k) <= x) ++k;"),
    # closing-time bin: one too many
    ("bin_plus_one", "while (k < 64 && ((uint64_t)1 << k) < x) ++k;",
     "while (k < 64 && ((uint64_t)1 << k) <= x) ++k;"),
    # dedup keeps the latest record instead of the first
    ("dedup_latest", "if (x->ts != y->ts) return x->ts < y->ts ? -1 : 1;",
     "if (x->ts != y->ts) return x->ts > y->ts ? -1 : 1;"),
    # dedup ties on the timestamp keep the largest edge label
    ("dedup_label_max", "if (x->el != y->el) return x->el < y->el ? -1 : 1;",
     "if (x->el != y->el) return x->el > y->el ? -1 : 1;"),
    # dedup on the first endpoint only
    ("dedup_u_only", "rec[i].u != rec[i - 1].u || rec[i].v != rec[i - 1].v",
     "rec[i].u != rec[i - 1].u"),
    # self loops kept
    ("loops_kept", "if (src[i] == dst[i]) continue;", ";"),
    # window with an exclusive upper end
    ("window_exclusive", "t3 > w->t_hi)", "t3 >= w->t_hi)"),
    # window ignores the first edge
    ("window_drops_edge", "if (t1 < w->t_lo || t1 > w->t_hi || t2", "if (t2"),
    # closing time measured from the middle timestamp
    ("close_from_t2", "o->hist[ceil_log2((uint64_t)(t3 - t1))]", "o->hist[ceil_log2((uint64_t)(t3 - t2))]"),
    # joint table transposed (open, close) -> (close, open)
    ("joint_transposed",
     "joint[ceil_log2((uint64_t)(t2 - t1)) * HIST_BINS + ceil_log2((uint64_t)(t3 - t1))]",
     "joint[ceil_log2((uint64_t)(t3 - t1)) * HIST_BINS + ceil_log2((uint64_t)(t2 - t1))]"),
    # distinct vertex labels checked on two pairs only
    ("maxel_two_pairs", "lp != lq && lq != lr && lp != lr", "lp != lq && lq != lr"),
    # minimum edge label instead of the maximum
    ("maxel_min", "uint32_t mx = ea > eb ? ea : eb;", "uint32_t mx = ea < eb ? ea : eb;"),
    # vertex-label triple not sorted
    ("vtri_unsorted", "sort3_u32(&a, &b, &c);\n        o->vtri[", "o->vtri["),
    # wrong edge for the third edge label
    ("etri_wrong_edge", "ec = w->eel ? w->eel[e_qr] : 0;", "ec = w->eel ? w->eel[e_pr] : 0;"),
    # degree triple takes q twice
    ("degtri_wrong_vertex", "c = (uint32_t)ceil_log2(w->deg[r]);", "c = (uint32_t)ceil_log2(w->deg[q]);"),
    # degree counted at one endpoint only
    ("degree_one_end", "deg[ev[i]] += 1;", ";"),
    # per-vertex participation credits q for r
    ("vlocal_wrong_vertex", "o->vlocal[r] += 1;", "o->vlocal[q] += 1;"),
    # merge skips the element right after q
    ("merge_skips_one", "uint64_t a = i + 1, b = 0;", "uint64_t a = i + 2, b = 0;"),
    # |W+| without the -1 of C(d, 2)
    ("wedges_formula", "wedges += d * (d ? d - 1 : 0) / 2;", "wedges += d * d / 2;"),
    # thread blocks overlap
    ("threads_overlap", "% w->stride != w->t) continue;", "% w->stride > w->t) continue;"),
    # per-edge participation credits (p,r) to (p,q)
    ("elocal_wrong_edge", "o->elocal[e_pr] += 1;", "o->elocal[e_pq] += 1;"),
    # per-thread vertex tables merged short by one
    ("vtri_index_transposed", "o->vtri[((uint64_t)a * w->Lv + b) * w->Lv + c] += 1;",
     "o->vtri[((uint64_t)a * w->Lv + c) * w->Lv + b] += 1;"),
    ("etri_index_transposed", "o->etri[((uint64_t)a * w->Le + b) * w->Le + c] += 1;",
     "o->etri[((uint64_t)c * w->Le + b) * w->Le + a] += 1;"),
    ("degtri_index_transposed", "o->degtri[((uint64_t)a * HIST_BINS + b) * HIST_BINS + c] += 1;",
     "o->degtri[((uint64_t)b * HIST_BINS + a) * HIST_BINS + c] += 1;"),
    ("merge_vlocal_short", "add_into(out->vlocal, o->vlocal, n);", "add_into(out->vlocal, o->vlocal, n ? n - 1 : 0);"),
]


def _mutant_source(old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique or missing: {old!r}"
    return text.replace(old, new)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, tmp_path):
    src = tmp_path / f"oracle_{name}.c"
    src.write_text(_mutant_source(old, new))
    lib = tmp_path / f"liboracle_{name}.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-pthread", str(src), "-o", str(lib)])
    env = dict(os.environ, ORACLE_LIBRARY=str(lib), PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    proc = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle.py"), "-x", "-q",
                           "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=300)
    assert proc.returncode == 1, f"mutant {name} survived the pins:\n{proc.stdout[-2000:]}"
