"""Helpers shared by the GPU tests: run the library on a synth.Graph and the
oracle on the same arrays.  Per-edge counts (TRIPOLL_EDGE_LOCAL) come from the
library by CSR position of G+ and from the oracle by unique edge in (min id,
max id) order; `survey` reorders the library's to the oracle's order, using the
exported G+ to name each position's endpoints."""
import numpy as np

import oracle
import paper_2107_12330_b300 as tp


def words(kinds, g, num_edges=0):
    return tp.tripoll_result_words(kinds, g.num_vlabels, g.num_elabels, g.n, num_edges)


def edges_in_pair_order(h):
    """Permutation taking CSR positions of G+ to unique edges in (min id, max id) order."""
    off, col, _, _, order = tp.tripoll_graph_export(h)
    n = len(order)
    src = np.repeat(np.arange(n), np.diff(off.astype(np.int64)))
    u = order[src].astype(np.int64)
    v = order[col].astype(np.int64)
    return np.argsort(np.minimum(u, v) * max(n, 1) + np.maximum(u, v), kind="stable")


def build(g, device_inputs=False):
    import torch
    arrs = [g.src, g.dst, g.ts, g.elabel, g.vlabel]
    if device_inputs:
        arrs = [None if a is None else torch.from_numpy(a).cuda() for a in arrs]
    h = tp.tripoll_graph_create(arrs[0], arrs[1], arrs[2], arrs[3], arrs[4], g.n, g.num_vlabels,
                                g.num_elabels if g.elabel is not None else 0)
    if device_inputs:
        torch.cuda.synchronize()
    return h


def survey(h, g, kinds, window=None, host_result=False, pivot_range=None):
    import torch
    lo, hi = window if window is not None else g.window
    m = tp.tripoll_graph_stats(h)["num_edges"] if kinds & tp.TRIPOLL_EDGE_LOCAL else 0
    w = words(kinds, g, m)
    if host_result:
        out = np.zeros(w, np.uint64)
    else:
        out = torch.zeros(max(w, 1), dtype=torch.int64, device="cuda")
    if pivot_range is None:
        tp.tripoll_survey(h, kinds, lo, hi, out)
    else:
        tp.tripoll_survey_range(h, kinds, lo, hi, pivot_range[0], pivot_range[1], out)
    if not host_result:
        torch.cuda.synchronize()
        out = out.cpu().numpy().view(np.uint64)[:w].copy()
    if m:  # the per-edge table is last in the record
        out[w - m:] = out[w - m:][edges_in_pair_order(h)]
    return out


def oracle_vector(g, kinds, window=None, threads=1):
    lo, hi = window if window is not None else g.window
    extras = ("joint", "maxel", "degtri", "vlocal") + (("elocal",) if kinds & tp.TRIPOLL_EDGE_LOCAL else ())
    r = oracle.survey(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels,
                      t_lo=lo, t_hi=hi, threads=threads, extras=extras)
    parts = []
    for bit, key in ((1, "count"), (2, "hist"), (4, "vtri"), (8, "etri"), (16, "joint"), (32, "maxel"),
                     (64, "degtri"), (128, "vlocal"), (256, "elocal")):
        if kinds & bit:
            parts.append(r[key])
    return np.concatenate(parts) if parts else np.zeros(0, np.uint64), r


def assert_equal_tables(got, want, kinds, g):
    """Bit-exact comparison; on mismatch name the first differing table."""
    if np.array_equal(got, want):
        return
    m = len(got) - words(kinds & ~tp.TRIPOLL_EDGE_LOCAL, g) if kinds & tp.TRIPOLL_EDGE_LOCAL else 0
    a = tp.split_result(got, kinds, g.num_vlabels, g.num_elabels, g.n, m)
    b = tp.split_result(want, kinds, g.num_vlabels, g.num_elabels, g.n, m)
    for k in a:
        if not np.array_equal(a[k], b[k]):
            idx = np.nonzero(a[k] != b[k])[0][:8]
            raise AssertionError(f"{g.name}: table {k} differs at {idx.tolist()}: "
                                 f"gpu {a[k][idx].tolist()} oracle {b[k][idx].tolist()}")
    raise AssertionError("length mismatch")
