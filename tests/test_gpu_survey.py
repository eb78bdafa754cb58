"""GPU parity: the CUDA survey path against the CPU oracle, bit-exact.

All survey arithmetic is integer, so every table must match exactly
(no tolerance).  Inputs are seeded synthetic graphs from ``synth``.
"""
import dataclasses
import itertools

import numpy as np
import pytest

import synth
import paper_2107_12330_b300 as tp
from gpu_util import assert_equal_tables, build, oracle_vector, survey, words

pytestmark = pytest.mark.gpu

ALL = tp.TRIPOLL_ALL_KINDS
BASIC = tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_VLABEL_TRIPLES | tp.TRIPOLL_ELABEL_TRIPLES


def check(g, kinds, window=None, **kw):
    h = build(g, device_inputs=kw.pop("device_inputs", False))
    try:
        got = survey(h, g, kinds, window=window, **kw)
    finally:
        tp.tripoll_destroy(h)
    want, _ = oracle_vector(g, kinds, window=window)
    assert_equal_tables(got, want, kinds, g)
    return got


def test_rmat12_survey():
    """R-MAT scale 12: count + closure histogram + vertex-label triples."""
    g = synth.rmat12()
    got = check(g, g.kinds)
    assert got[0] > 0


def test_rmat12_all_kinds_with_edge_labels():
    g = synth.rmat_graph(12, 16, 7, ts_bits=24, num_vlabels=4, num_elabels=5)
    check(g, ALL)


@pytest.mark.parametrize("seed,n,m", [(1, 2, 3), (2, 3, 10), (3, 5, 40), (4, 17, 200), (5, 64, 1500),
                                      (6, 200, 6000), (7, 1000, 30000), (8, 40, 2000)])
def test_tiny_graphs_all_kinds(seed, n, m):
    g = synth.tiny_random_graph(seed, n, m, ts_bits=6, num_vlabels=3, num_elabels=4)
    check(g, ALL)


@pytest.mark.parametrize("window", [(0, 0xFFFFFFFF), (10, 40), (0, 0), (63, 63), (20, 21)])
def test_windows(window):
    g = synth.tiny_random_graph(11, 300, 20000, ts_bits=6, num_vlabels=2, num_elabels=3)
    check(g, BASIC, window=window)


@pytest.mark.parametrize("window", [(0, 0xFFFFFFFF), (0xFFFFFFFF, 0xFFFFFFFF), (1, 0xFFFFFFFE), (0, 0),
                                    (0x80000000, 0xFFFFFFFF)])
def test_full_range_timestamps(window):
    """Timestamps over the whole uint32 range with 0 and 2^32-1 planted: closing times up to 2^32-1 fill the
    last histogram bin (32), and windows start or end at the extreme timestamps."""
    g = synth.tiny_random_graph(21, 120, 6000, ts_bits=32, num_vlabels=3, num_elabels=4)
    ts = g.ts.copy()
    ts[::7] = 0
    ts[3::11] = 0xFFFFFFFF
    g = dataclasses.replace(g, ts=ts)
    got = check(g, ALL, window=window)
    if window == (0, 0xFFFFFFFF):
        assert got[1 + 32] > 0  # the count word, then bins 0..32


@pytest.mark.parametrize("log2", ["0", "4"])
def test_shared_mirror_moves_leave_results_unchanged(log2, monkeypatch):
    """A block sums into a 32-bit shared-memory mirror of the result record; to keep it below 2^32, a warp
    moves it into the 64-bit record (exchanging each word with 0) every 2^k work items its block (or, in the
    warp kernel, the warp) takes.  With k forced to 0 or 4 the moves happen thousands of times while other
    warps keep adding; the result must still equal the oracle's."""
    monkeypatch.setenv("TRIPOLL_MIRROR_MOVE_LOG2", log2)
    g = synth.rmat_graph(14, 16, 5, ts_bits=24, num_vlabels=4, num_elabels=5)
    check(g, ALL)
    check(g, BASIC, window=(1 << 22, 3 << 22))


def test_host_and_device_results_and_inputs_agree():
    g = synth.rmat_graph(11, 16, 3, ts_bits=20, num_vlabels=4, num_elabels=8)
    a = check(g, BASIC, host_result=True)
    b = check(g, BASIC, device_inputs=True)
    assert np.array_equal(a, b)


def test_empty_and_degenerate_graphs():
    # no edges at all, only loops, a single repeated edge, isolated vertices
    for src, dst, n in [([], [], 0), ([], [], 5), ([0, 1, 2], [0, 1, 2], 3), ([0, 0, 1, 1], [1, 1, 0, 0], 4),
                        ([0, 1, 2], [1, 2, 0], 1000)]:
        src = np.array(src, np.uint32)
        dst = np.array(dst, np.uint32)
        ts = np.arange(len(src), dtype=np.uint32)
        g = synth.Graph("degenerate", n, src, dst, ts, None, None, 1, 1, 3)
        check(g, tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_VLABEL_TRIPLES)


def test_complete_graph_long_out_lists():
    """K_1100: out-lists longer than one on-chip chunk (chunked middle vertices)."""
    n = 1100
    iu = np.triu_indices(n, 1)
    src = iu[0].astype(np.uint32)
    dst = iu[1].astype(np.uint32)
    m = len(src)
    ts = synth.uniform_bits(5, synth.STREAM_TS, m, 16)
    el = synth.uniform_labels(5, synth.STREAM_ELABEL, m, 3)
    vl = synth.uniform_labels(5, synth.STREAM_VLABEL, n, 3)
    g = synth.Graph("K1100", n, src, dst, ts, vl, el, 3, 3, BASIC)
    got = check(g, BASIC)
    assert int(got[0]) == n * (n - 1) * (n - 2) // 6
    # a window: the chunks' value ranges come from their in-window entries only
    check(g, ALL & ~tp.TRIPOLL_VERTEX_LOCAL, window=(1 << 14, 3 << 14))
    check(g, tp.TRIPOLL_COUNT | tp.TRIPOLL_VERTEX_LOCAL | tp.TRIPOLL_EDGE_LOCAL, window=(0, 1 << 12))


def test_out_lists_past_the_long_list_threshold():
    """K_4200: every degree is 4199, so <+ is the id order and vertex i has 4199 - i out-edges; the first 103
    vertices pass 4096 and are surveyed by the 2048-entry-table kernel, in parts.  Too many triangles for the
    oracle (12.3 G), so the counts are checked against closed forms: C(n,3) triangles, all in bin 0 of the
    closing-time histogram (equal timestamps), and vertex-label triples as products of binomials of the label
    classes; a window that holds every edge gives the same tables."""
    import math
    n, sizes = 4200, [1400, 1500, 1300]
    iu = np.triu_indices(n, 1)
    src, dst = iu[0].astype(np.uint32), iu[1].astype(np.uint32)
    ts = np.full(len(src), 77, np.uint32)
    vl = np.repeat(np.arange(3), sizes).astype(np.uint8)
    g = synth.Graph("K4200", n, src, dst, ts, vl, None, 3, 1, BASIC)
    kinds = tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_VLABEL_TRIPLES
    h = build(g)
    try:
        assert tp.tripoll_graph_stats(h)["dplus_max"] == n - 1
        want = np.zeros(1 + 33 + 27, np.uint64)
        want[0] = math.comb(n, 3)
        want[1] = math.comb(n, 3)
        for a, b, c in itertools.combinations_with_replacement(range(3), 3):
            x = 1
            for lab in set((a, b, c)):
                x *= math.comb(sizes[lab], (a, b, c).count(lab))
            want[34 + (a * 3 + b) * 3 + c] = x
        for window in [(0, 0xFFFFFFFF), (77, 77)]:
            got = survey(h, g, kinds, window=window)
            assert np.array_equal(got, want), window
    finally:
        tp.tripoll_destroy(h)


def test_edge_local_counts_view_in_place_and_shards():
    """Per-edge participation through the window view, in place (full window), and as pivot-range shards."""
    g = synth.rmat(13, 3)
    kinds = tp.TRIPOLL_COUNT | tp.TRIPOLL_VERTEX_LOCAL | tp.TRIPOLL_EDGE_LOCAL
    check(g, kinds)
    full = check(g, kinds | tp.TRIPOLL_CLOSURE_HIST, window=(0, 0xFFFFFFFF))
    m = len(full) - words((kinds | tp.TRIPOLL_CLOSURE_HIST) & ~tp.TRIPOLL_EDGE_LOCAL, g)
    assert int(full[-m:].sum()) == 3 * int(full[0])
    h = build(g)
    try:
        bounds = tp.tripoll_partition_pivots(h, 3)
        acc = np.zeros_like(full)
        for lo, hi in zip(bounds[:-1], bounds[1:]):
            acc += survey(h, g, kinds | tp.TRIPOLL_CLOSURE_HIST, window=(0, 0xFFFFFFFF), pivot_range=(int(lo), int(hi)))
        assert np.array_equal(acc, full)
    finally:
        tp.tripoll_destroy(h)


def _numpy_window_wedges(g, lo, hi):
    """Sum over pivots p of C(k_p, 2), k_p the in-window edges of Adj+(p): dedup keeping the
    first record, (degree, id) order, orientation low -> high, all in numpy."""
    u = np.minimum(g.src, g.dst).astype(np.int64)
    v = np.maximum(g.src, g.dst).astype(np.int64)
    el = g.elabel if g.elabel is not None else np.zeros(len(u), np.uint8)
    keep = u != v
    u, v, t, e = u[keep], v[keep], g.ts[keep].astype(np.int64), el[keep]
    o = np.lexsort((e, t, v, u))
    u, v, t = u[o], v[o], t[o]
    first = np.ones(len(u), bool)
    first[1:] = (u[1:] != u[:-1]) | (v[1:] != v[:-1])
    u, v, t = u[first], v[first], t[first]
    deg = np.bincount(u, minlength=g.n) + np.bincount(v, minlength=g.n)
    rank = np.empty(g.n, np.int64)
    rank[np.lexsort((np.arange(g.n), deg))] = np.arange(g.n)
    piv = np.where(rank[u] < rank[v], u, v)
    inw = (t >= lo) & (t <= hi)
    k = np.bincount(piv[inw], minlength=g.n).astype(np.int64)
    return int((k * (k - 1) // 2).sum()), int(len(u))


def test_wedge_checks_of_a_window():
    g = synth.rmat(13, 3)
    h = build(g)
    try:
        st = tp.tripoll_graph_stats(h)
        assert tp.tripoll_wedge_checks(h) == st["wedges"]
        for lo, hi in [g.window, (0, 0), (1 << 29, 0xFFFFFFFF)]:
            want, m = _numpy_window_wedges(g, lo, hi)
            assert m == st["num_edges"]
            assert tp.tripoll_wedge_checks(h, lo, hi) == want
    finally:
        tp.tripoll_destroy(h)


def test_rmat16_window_edge_label_triples():
    g = synth.rmat(16, 2)
    check(g, g.kinds)


def test_shards_sum_to_full_survey():
    g = synth.rmat(14, 4)
    h = build(g)
    try:
        full = survey(h, g, g.kinds)
        bounds = tp.tripoll_partition_pivots(h, 5)
        assert bounds[0] == 0 and bounds[-1] == g.n and np.all(np.diff(bounds.astype(np.int64)) >= 0)
        acc = np.zeros_like(full)
        for lo, hi in zip(bounds[:-1], bounds[1:]):
            acc += survey(h, g, g.kinds, pivot_range=(int(lo), int(hi)))
    finally:
        tp.tripoll_destroy(h)
    assert np.array_equal(acc, full)
    want, _ = oracle_vector(g, g.kinds)
    assert np.array_equal(full, want)


def test_pivot_range_matches_oracle():
    g = synth.rmat_graph(12, 16, 9, ts_bits=24, num_vlabels=4, num_elabels=4)
    h = build(g)
    try:
        got = survey(h, g, BASIC, pivot_range=(1000, 3000))
    finally:
        tp.tripoll_destroy(h)
    r = __import__("oracle").survey(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 4, 4, pivot_range=(1000, 3000))
    want = np.concatenate([r["count"], r["hist"], r["vtri"], r["etri"]])
    assert np.array_equal(got, want)


def test_batched_graphs_match_each_alone():
    graphs = [synth.batched_graph(i) for i in range(40)]
    src = np.concatenate([g.src for g in graphs])
    dst = np.concatenate([g.dst for g in graphs])
    ts = np.concatenate([g.ts for g in graphs])
    vl = np.concatenate([g.vlabel for g in graphs])
    eoff = np.zeros(len(graphs) + 1, np.uint64)
    eoff[1:] = np.cumsum([g.m_in for g in graphs])
    nv = np.array([g.n for g in graphs], np.uint32)
    kinds = tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_VLABEL_TRIPLES
    h = tp.tripoll_batch_create(src, dst, ts, None, eoff, vl, nv, 4, 0)
    window = (1 << 18, 3 << 18)  # the window view of a batched graph
    try:
        w = tp.tripoll_result_words(kinds, 4, 1, 0)
        out = np.zeros(w * len(graphs), np.uint64)
        tp.tripoll_survey(h, kinds, 0, 0xFFFFFFFF, out)
        outw = np.zeros(w * len(graphs), np.uint64)
        tp.tripoll_survey(h, kinds, window[0], window[1], outw)
    finally:
        tp.tripoll_destroy(h)
    for i, g in enumerate(graphs):
        want, _ = oracle_vector(g, kinds, window=(0, 0xFFFFFFFF))
        assert_equal_tables(out[i * w:(i + 1) * w], want, kinds, g)
        want, _ = oracle_vector(g, kinds, window=window)
        assert_equal_tables(outw[i * w:(i + 1) * w], want, kinds, g)


def test_largest_label_counts():
    """256 vertex and 256 edge labels: triple tables of 256^3 words, far past the on-chip record mirror."""
    g = synth.tiny_random_graph(21, 400, 30000, ts_bits=10, num_vlabels=256, num_elabels=256)
    check(g, ALL & ~(tp.TRIPOLL_VERTEX_LOCAL | tp.TRIPOLL_EDGE_LOCAL))
    check(g, BASIC, window=(100, 700))


def test_errors_are_reported_not_faulted():
    src = np.array([0, 1], np.uint32)
    dst = np.array([1, 5], np.uint32)
    ts = np.zeros(2, np.uint32)
    with pytest.raises(tp.TripollError) as e:
        tp.tripoll_graph_create(src, dst, ts, None, None, 3, 1, 0)
    assert e.value.status == tp.TRIPOLL_ERR_VERTEX_RANGE
    with pytest.raises(tp.TripollError) as e:
        tp.tripoll_graph_create(src, np.array([1, 2], np.uint32), ts, np.array([0, 9], np.uint8), None, 3, 1, 4)
    assert e.value.status == tp.TRIPOLL_ERR_LABEL_RANGE
    h = tp.tripoll_graph_create(src, np.array([1, 2], np.uint32), ts, None, None, 3, 1, 0)
    try:
        out = np.zeros(64, np.uint64)
        with pytest.raises(tp.TripollError) as e:
            tp.tripoll_survey(h, tp.TRIPOLL_COUNT, 5, 4, out)
        assert e.value.status == tp.TRIPOLL_ERR_INVALID_ARG
        with pytest.raises(tp.TripollError) as e:
            tp.tripoll_survey(h, tp.TRIPOLL_ELABEL_TRIPLES, 0, 9, out)
        assert e.value.status == tp.TRIPOLL_ERR_NO_EDGE_LABELS
    finally:
        tp.tripoll_destroy(h)


def test_builder_matches_independent_construction():
    """The exported G+ equals a plain numpy construction of dedup, (degree, id) order and CSR."""
    g = synth.rmat_graph(11, 16, 5, ts_bits=10, num_vlabels=1, num_elabels=6)
    h = build(g)
    try:
        off, col, ts, el, order = tp.tripoll_graph_export(h)
    finally:
        tp.tripoll_destroy(h)
    u = np.minimum(g.src, g.dst).astype(np.int64)
    v = np.maximum(g.src, g.dst).astype(np.int64)
    keep = u != v
    u, v, t, e = u[keep], v[keep], g.ts[keep].astype(np.int64), g.elabel[keep].astype(np.int64)
    o = np.lexsort((e, t, v, u))
    u, v, t, e = u[o], v[o], t[o], e[o]
    first = np.ones(len(u), bool)
    first[1:] = (u[1:] != u[:-1]) | (v[1:] != v[:-1])
    u, v, t, e = u[first], v[first], t[first], e[first]
    deg = np.bincount(u, minlength=g.n) + np.bincount(v, minlength=g.n)
    ordr = np.lexsort((np.arange(g.n), deg))
    rank = np.empty(g.n, np.int64)
    rank[ordr] = np.arange(g.n)
    s, d = np.minimum(rank[u], rank[v]), np.maximum(rank[u], rank[v])
    o = np.lexsort((d, s))
    assert np.array_equal(order, ordr.astype(np.uint32))
    assert np.array_equal(col, d[o].astype(np.uint32))
    assert np.array_equal(ts, t[o].astype(np.uint32))
    assert np.array_equal(el, e[o].astype(np.uint8))
    want_off = np.zeros(g.n + 1, np.uint64)
    want_off[1:] = np.cumsum(np.bincount(s, minlength=g.n))
    assert np.array_equal(off, want_off)


def test_graph_stats():
    g = synth.rmat12()
    h = build(g)
    try:
        st = tp.tripoll_graph_stats(h)
    finally:
        tp.tripoll_destroy(h)
    _, r = oracle_vector(g, 1)
    assert st["num_edges"] == r["stats"]["m"]
    assert st["wedges"] == r["stats"]["wedges"]
    assert st["dplus_max"] == r["stats"]["dplus_max"]
    assert st["degree_max"] == r["stats"]["dmax"]


def test_vertex_ids_past_2_to_the_28_take_the_wide_record_path():
    """With n = 2^29 the builder's pair keys take 58 bits, too wide to carry the payload's top byte beside
    them, so its sorts move the payload as a full 64-bit value instead of the packed 12-byte record.  A
    sparse graph on 3,000 ids spread over [0, 2^29) must survey exactly like the same graph relabelled onto
    0..2999 (every table here is invariant under relabelling, Sec. 3), which the oracle surveys."""
    small = synth.tiny_random_graph(71, 3000, 60000, ts_bits=16, num_vlabels=1, num_elabels=6)
    n_big = 1 << 29
    ids = np.unique(synth.uniform_bits(72, synth.STREAM_TS, 4000, 29).astype(np.uint64))[:3000]
    assert len(ids) == 3000
    ids = ids[np.argsort(synth.uniform_bits(73, synth.STREAM_TS, 3000, 31), kind="stable")].astype(np.uint32)
    big = dataclasses.replace(small, name="sparse-2^29", n=n_big, src=ids[small.src], dst=ids[small.dst],
                              vlabel=None)
    small = dataclasses.replace(small, vlabel=None)
    kinds = (tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_ELABEL_TRIPLES | tp.TRIPOLL_OPEN_CLOSE_HIST |
             tp.TRIPOLL_DEGREE_TRIPLES)
    h = tp.tripoll_graph_create(big.src, big.dst, big.ts, big.elabel, None, n_big, 1, 6)
    try:
        st = tp.tripoll_graph_stats(h)
        for window in [(0, 0xFFFFFFFF), (1 << 13, 3 << 13)]:
            got = np.zeros(tp.tripoll_result_words(kinds, 1, 6, n_big), np.uint64)
            tp.tripoll_survey(h, kinds, window[0], window[1], got)
            want, r = oracle_vector(small, kinds, window=window)
            assert_equal_tables(got, want, kinds, small)
        # (|W+| is not compared: equal degrees are ordered by id, and relabelling changes that orientation)
        assert st["num_edges"] == r["stats"]["m"]
    finally:
        tp.tripoll_destroy(h)
