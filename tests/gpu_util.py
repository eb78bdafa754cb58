"""Helpers shared by the GPU tests: run the library on a synth.Graph and the
oracle on the same arrays."""
import numpy as np

import oracle
import paper_2107_12330_b300 as tp


def words(kinds, g):
    return tp.tripoll_result_words(kinds, g.num_vlabels, g.num_elabels, g.n)


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
    w = words(kinds, g)
    if host_result:
        out = np.zeros(w, np.uint64)
    else:
        out = torch.zeros(max(w, 1), dtype=torch.int64, device="cuda")
    if pivot_range is None:
        tp.tripoll_survey(h, kinds, lo, hi, out)
    else:
        tp.tripoll_survey_range(h, kinds, lo, hi, pivot_range[0], pivot_range[1], out)
    if host_result:
        return out
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)[:w]


def oracle_vector(g, kinds, window=None, threads=1):
    lo, hi = window if window is not None else g.window
    r = oracle.survey(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels,
                      t_lo=lo, t_hi=hi, threads=threads)
    parts = []
    for bit, key in ((1, "count"), (2, "hist"), (4, "vtri"), (8, "etri"), (16, "joint"), (32, "maxel"),
                     (64, "degtri"), (128, "vlocal")):
        if kinds & bit:
            parts.append(r[key])
    return np.concatenate(parts) if parts else np.zeros(0, np.uint64), r


def assert_equal_tables(got, want, kinds, g):
    """Bit-exact comparison; on mismatch name the first differing table."""
    if np.array_equal(got, want):
        return
    a = tp.split_result(got, kinds, g.num_vlabels, g.num_elabels, g.n)
    b = tp.split_result(want, kinds, g.num_vlabels, g.num_elabels, g.n)
    for k in a:
        if not np.array_equal(a[k], b[k]):
            idx = np.nonzero(a[k] != b[k])[0][:8]
            raise AssertionError(f"{g.name}: table {k} differs at {idx.tolist()}: "
                                 f"gpu {a[k][idx].tolist()} oracle {b[k][idx].tolist()}")
    raise AssertionError("length mismatch")
