"""Pins of the CPU oracle against what the paper and the mathematics fix.

The oracle is the reference the CUDA path is compared with, so it is checked
here against things other than itself: a brute-force O(n^3) enumeration
written straight from the definitions (Sec. 3), closed forms (K_n, bipartite
and star graphs), trace(A^3)/6, hand-computed closing-time bins (Alg. 4),
invariances the survey must have (relabelling, edge order, duplicates, the
tie-break of the order <+), and the window = filtered-subgraph identity.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

ALL_EXTRAS = ("joint", "maxel", "degtri", "vlocal", "elocal")


def run(src, dst, ts, el, vl, n, Lv, Le, **kw):
    return oracle.survey(np.asarray(src, np.uint32), np.asarray(dst, np.uint32), np.asarray(ts, np.uint32),
                         None if el is None else np.asarray(el, np.uint8),
                         None if vl is None else np.asarray(vl, np.uint8), n, Lv, Le, **kw)


def ceil_log2_by_hand(d):
    """Closing-time bin: the smallest k with 2^k >= d, and 0 for d in {0, 1}."""
    k = 0
    while (1 << k) < d:
        k += 1
    return k


def brute_force(src, dst, ts, el, vl, n, Lv, Le, t_lo=0, t_hi=0xFFFFFFFF):
    """The survey from its definition: simple graph by dict, every vertex triple."""
    edges = {}
    for u, v, t, e in zip(src, dst, ts, el if el is not None else [0] * len(src)):
        u, v, t, e = int(u), int(v), int(t), int(e)
        if u == v:
            continue
        key = (min(u, v), max(u, v))
        if key not in edges or (t, e) < edges[key]:
            edges[key] = (t, e)
    deg = [0] * n
    for (u, v) in edges:
        deg[u] += 1
        deg[v] += 1
    lab = [int(x) for x in vl] if vl is not None else [0] * n
    index = {key: i for i, key in enumerate(sorted(edges))}  # unique edges in (min id, max id) order
    res = {"count": 0, "hist": [0] * 33, "vtri": [0] * Lv ** 3, "etri": [0] * Le ** 3, "joint": [0] * 33 * 33,
           "maxel": [0] * Le, "degtri": [0] * 33 ** 3, "vlocal": [0] * n, "elocal": [0] * len(edges)}
    for x, y, z in itertools.combinations(range(n), 3):
        if (x, y) in edges and (x, z) in edges and (y, z) in edges:
            (t1, e1), (t2, e2), (t3, e3) = edges[(x, y)], edges[(x, z)], edges[(y, z)]
            if not all(t_lo <= t <= t_hi for t in (t1, t2, t3)):
                continue
            a, b, c = sorted((t1, t2, t3))
            res["count"] += 1
            res["hist"][ceil_log2_by_hand(c - a)] += 1
            res["joint"][ceil_log2_by_hand(b - a) * 33 + ceil_log2_by_hand(c - a)] += 1
            la, lb, lc = sorted((lab[x], lab[y], lab[z]))
            res["vtri"][(la * Lv + lb) * Lv + lc] += 1
            ea, eb, ec = sorted((e1, e2, e3))
            res["etri"][(ea * Le + eb) * Le + ec] += 1
            if lab[x] != lab[y] and lab[y] != lab[z] and lab[x] != lab[z]:
                res["maxel"][max(e1, e2, e3)] += 1
            da, db, dc = sorted(ceil_log2_by_hand(deg[w]) for w in (x, y, z))
            res["degtri"][(da * 33 + db) * 33 + dc] += 1
            for w in (x, y, z):
                res["vlocal"][w] += 1
            for key in ((x, y), (x, z), (y, z)):
                res["elocal"][index[key]] += 1
    return res


def same(r, b, keys=("count", "hist", "vtri", "etri") + ALL_EXTRAS):
    for k in keys:
        got = [int(x) for x in np.atleast_1d(r[k])]
        want = [b[k]] if k == "count" else b[k]
        assert got == want, f"table {k}"


def test_closing_time_bins_by_hand():
    # one triangle with timestamps (0, 0, d): the closing time is d (Alg. 4)
    table = {0: 0, 1: 0, 2: 1, 3: 2, 4: 2, 5: 3, 8: 3, 9: 4, 1023: 10, 1024: 10, 1025: 11,
             2 ** 31: 31, 2 ** 31 + 1: 32, 2 ** 32 - 1: 32}
    for d, k in table.items():
        r = run([0, 0, 1], [1, 2, 2], [0, 0, d], None, None, 3, 1, 1)
        assert int(r["count"][0]) == 1
        assert np.nonzero(r["hist"])[0].tolist() == [k], d


def test_single_triangle_worked_example():
    # ts {0, 5, 9}: t1=0, t2=5, t3=9 -> open = ceil(log2 5) = 3, close = ceil(log2 9) = 4
    r = run([0, 1, 2], [1, 2, 0], [0, 5, 9], [2, 0, 1], [1, 0, 2], 3, 3, 3)
    assert int(r["count"][0]) == 1
    assert np.nonzero(r["hist"])[0].tolist() == [4]
    assert np.nonzero(r["joint"])[0].tolist() == [3 * 33 + 4]
    assert np.nonzero(r["vtri"])[0].tolist() == [(0 * 3 + 1) * 3 + 2]
    assert np.nonzero(r["etri"])[0].tolist() == [(0 * 3 + 1) * 3 + 2]
    assert r["maxel"].tolist() == [0, 0, 1]  # labels pairwise distinct; max edge label 2
    assert r["vlocal"].tolist() == [1, 1, 1]
    assert np.nonzero(r["degtri"])[0].tolist() == [(1 * 33 + 1) * 33 + 1]  # degree 2 -> bin 1


@pytest.mark.parametrize("seed,n,m", [(1, 6, 20), (2, 9, 40), (3, 12, 90), (4, 16, 150), (5, 24, 300),
                                      (6, 30, 200), (7, 40, 700)])
def test_brute_force_all_tables(seed, n, m):
    g = synth.tiny_random_graph(seed, n, m, ts_bits=5, num_vlabels=3, num_elabels=4)
    r = oracle.survey_graph(g, extras=ALL_EXTRAS)
    b = brute_force(g.src, g.dst, g.ts, g.elabel, g.vlabel, n, 3, 4)
    same(r, b)


@pytest.mark.parametrize("window", [(3, 20), (0, 0), (31, 31), (10, 11)])
def test_brute_force_windows(window):
    g = synth.tiny_random_graph(17, 20, 250, ts_bits=5, num_vlabels=2, num_elabels=2)
    r = oracle.survey(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 2, 2, t_lo=window[0], t_hi=window[1],
                      extras=ALL_EXTRAS)
    same(r, brute_force(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 2, 2, *window))


def test_complete_graph_closed_forms():
    n = 30
    iu = np.triu_indices(n, 1)
    m = len(iu[0])
    sizes = [5, 10, 15]  # vertex label classes
    vl = np.repeat(np.arange(3), sizes).astype(np.uint8)
    r = run(iu[0], iu[1], np.full(m, 7), None, vl, n, 3, 1)
    assert int(r["count"][0]) == math.comb(n, 3)
    assert r["hist"][0] == math.comb(n, 3) and r["hist"][1:].sum() == 0  # all timestamps equal
    for a, b, c in itertools.combinations_with_replacement(range(3), 3):
        want = 1
        for lab in set((a, b, c)):
            want *= math.comb(sizes[lab], (a, b, c).count(lab))
        assert r["vtri"][(a * 3 + b) * 3 + c] == want
    assert r["vlocal"].tolist() == [math.comb(n - 1, 2)] * n
    assert r["degtri"][(5 * 33 + 5) * 33 + 5] == math.comb(n, 3)  # degree 29 -> ceil(log2 29) = 5


def test_complete_graph_over_several_thread_blocks():
    """K_600 with 4 threads: pivots fall in three blocks of 256, so every per-thread table is merged."""
    n = 600
    iu = np.triu_indices(n, 1)
    r = run(iu[0], iu[1], np.arange(len(iu[0])), None, None, n, 1, 1, threads=4, extras=ALL_EXTRAS)
    assert int(r["count"][0]) == math.comb(n, 3)
    assert r["vlocal"].tolist() == [math.comb(n - 1, 2)] * n
    assert r["elocal"].tolist() == [n - 2] * math.comb(n, 2)  # every edge closes with each of the other n - 2
    assert int(r["degtri"][(10 * 33 + 10) * 33 + 10]) == math.comb(n, 3)  # degree 599 -> bin 10


def test_bipartite_and_star_have_no_triangles():
    a, b = np.meshgrid(np.arange(10), np.arange(10, 25))
    r = run(a.ravel(), b.ravel(), np.zeros(a.size), None, None, 25, 1, 1)
    assert int(r["count"][0]) == 0
    r = run(np.zeros(50), np.arange(1, 51), np.zeros(50), None, None, 51, 1, 1)
    assert int(r["count"][0]) == 0


def test_count_equals_trace_of_a_cubed_over_six():
    """R-MAT scale 12: triangles = trace(A^3)/6 (exact in float64: all partial sums < 2^53)."""
    g = synth.rmat12()
    r = oracle.survey_graph(g, extras=())
    A = np.zeros((g.n, g.n))
    keep = g.src != g.dst
    A[g.src[keep], g.dst[keep]] = 1
    A[g.dst[keep], g.src[keep]] = 1
    tr = float(np.sum((A @ A) * A))
    assert tr % 6 == 0
    assert int(r["count"][0]) == int(tr) // 6


def test_table_sums_and_marginals():
    g = synth.rmat_graph(10, 16, 2, ts_bits=16, num_vlabels=4, num_elabels=3)
    r = oracle.survey_graph(g, extras=ALL_EXTRAS)
    c = int(r["count"][0])
    assert c > 0
    for k in ("hist", "vtri", "etri", "joint", "degtri"):
        assert int(r[k].sum()) == c, k
    assert int(r["vlocal"].sum()) == 3 * c
    assert int(r["elocal"].sum()) == 3 * c
    assert np.array_equal(r["joint"].reshape(33, 33).sum(axis=0), r["hist"])  # marginal over open time
    assert int(r["maxel"].sum()) <= c


def _relabelled(g, seed):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n).astype(np.uint32)
    vl = np.empty_like(g.vlabel)
    vl[perm] = g.vlabel
    return perm[g.src], perm[g.dst], vl


def test_invariances():
    g = synth.rmat_graph(10, 8, 5, ts_bits=12, num_vlabels=3, num_elabels=3)
    base = oracle.survey_graph(g, extras=("joint", "maxel", "degtri"))
    keys = ("count", "hist", "vtri", "etri", "joint", "maxel", "degtri")

    def eq(r):
        for k in keys:
            assert np.array_equal(r[k], base[k]), k

    # vertex relabelling (labels carried)
    s, d, vl = _relabelled(g, 1)
    eq(oracle.survey(s, d, g.ts, g.elabel, vl, g.n, 3, 3, extras=("joint", "maxel", "degtri")))
    # edge order permutation and reversed endpoints
    p = np.random.default_rng(2).permutation(g.m_in)
    eq(oracle.survey(g.dst[p], g.src[p], g.ts[p], g.elabel[p], g.vlabel, g.n, 3, 3,
                     extras=("joint", "maxel", "degtri")))
    # duplicates that are later in time change nothing (the first record is kept)
    eq(oracle.survey(np.concatenate([g.src, g.dst]), np.concatenate([g.dst, g.src]),
                     np.concatenate([g.ts, g.ts + 1]), np.concatenate([g.elabel, (g.elabel + 1) % 3]),
                     g.vlabel, g.n, 3, 3, extras=("joint", "maxel", "degtri")))
    # the tie-break of <+ and even the degree itself only change the orientation (Sec. 3)
    for mode in (1, 2):
        eq(oracle.survey_graph(g, order_mode=mode, extras=("joint", "maxel", "degtri")))


def test_degree_triples_under_a_window_use_the_whole_graphs_degrees():
    """The window selects triangles, not degrees: d(v) is the degree in the whole simple graph (Sec. 3, Sec.
    5.9), so a window that leaves out edges at a vertex does not change its degree bin."""
    # triangle {0,1,2} at ts 5; edges (0,3), (0,4) at ts 50 lie outside the window [0, 10]
    r = run([0, 1, 0, 0, 0], [1, 2, 2, 3, 4], [5, 5, 5, 50, 50], None, None, 5, 1, 1, t_lo=0, t_hi=10)
    assert int(r["count"][0]) == 1
    # d(0) = 4 -> bin 2; d(1) = d(2) = 2 -> bin 1: the sorted triple (1, 1, 2), not (1, 1, 1)
    assert np.nonzero(r["degtri"])[0].tolist() == [(1 * 33 + 1) * 33 + 2]


def test_window_equals_filtered_subgraph():
    g = synth.rmat_graph(10, 16, 8, ts_bits=10, num_vlabels=2, num_elabels=4)
    lo, hi = 200, 700
    a = oracle.survey(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 2, 4, t_lo=lo, t_hi=hi, extras=())
    # the window applies after dedup: keep the first record of each pair, then filter
    u = np.minimum(g.src, g.dst).astype(np.int64)
    v = np.maximum(g.src, g.dst).astype(np.int64)
    o = np.lexsort((g.elabel, g.ts, v, u))
    u, v, t, e = u[o], v[o], g.ts[o], g.elabel[o]
    first = np.ones(len(u), bool)
    first[1:] = (u[1:] != u[:-1]) | (v[1:] != v[:-1])
    keep = first & (t >= lo) & (t <= hi)
    b = oracle.survey(u[keep], v[keep], t[keep], e[keep], g.vlabel, g.n, 2, 4, extras=())
    for k in ("count", "hist", "vtri", "etri"):
        assert np.array_equal(a[k], b[k]), k
    full = oracle.survey(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 2, 4, t_lo=0, t_hi=0xFFFFFFFF, extras=())
    assert int(full["count"][0]) >= int(a["count"][0])


def test_pivot_ranges_and_threads_partition_the_survey():
    g = synth.rmat_graph(11, 16, 3, ts_bits=20, num_vlabels=4, num_elabels=2)
    full = oracle.survey_graph(g, extras=ALL_EXTRAS)
    cuts = [0, 100, 900, 1500, g.n]
    acc = {k: np.zeros_like(full[k]) for k in ("count", "hist", "vtri", "etri") + ALL_EXTRAS}
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        part = oracle.survey_graph(g, pivot_range=(lo, hi), extras=ALL_EXTRAS)
        for k in acc:
            acc[k] += part[k]
    for k in acc:
        assert np.array_equal(acc[k], full[k]), k
    thr = oracle.survey_graph(g, threads=4, extras=ALL_EXTRAS)
    for k in acc:
        assert np.array_equal(thr[k], full[k]), k


def test_graph_statistics():
    g = synth.rmat12()
    r = oracle.survey_graph(g, extras=())
    st = r["stats"]
    # |W+| from its definition on an independent numpy orientation
    u = np.minimum(g.src, g.dst).astype(np.int64)
    v = np.maximum(g.src, g.dst).astype(np.int64)
    keep = u != v
    key = np.unique(u[keep] * g.n + v[keep])
    U, V = key // g.n, key % g.n
    deg = np.bincount(U, minlength=g.n) + np.bincount(V, minlength=g.n)
    rank = np.empty(g.n, np.int64)
    rank[np.lexsort((np.arange(g.n), deg))] = np.arange(g.n)
    piv = np.where(rank[U] < rank[V], U, V)
    dplus = np.bincount(piv, minlength=g.n)
    assert st["m"] == len(key)
    assert st["wedges"] == int((dplus * (dplus - 1) // 2).sum())
    assert st["dplus_max"] == int(dplus.max())
    assert st["dmax"] == int(deg.max())


def test_invalid_inputs_rejected():
    with pytest.raises(ValueError):
        run([0], [5], [0], None, None, 3, 1, 1)
    with pytest.raises(ValueError):
        run([0], [1], [0], [7], None, 3, 1, 4)
    with pytest.raises(ValueError):
        run([0], [1], [0], None, [9, 0, 0], 3, 2, 1)


def test_per_vertex_counts_match_networkx_triangles():
    """A library routine as an independent pin: networkx.triangles gives the number of triangles at every
    vertex of the simple graph; the oracle's per-vertex participation (Sec. 5.3) and total count must agree on
    an R-MAT graph with loops and duplicate records (scale 11, about 30 k records)."""
    nx = pytest.importorskip("networkx")
    g = synth.rmat_graph(11, 16, 9, ts_bits=20, num_vlabels=3, num_elabels=1)
    r = run(g.src, g.dst, g.ts, None, g.vlabel, g.n, 3, 1, extras=("vlocal",))
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from((int(u), int(v)) for u, v in zip(g.src, g.dst) if u != v)
    want = nx.triangles(G)
    got = r["vlocal"]
    assert [int(got[v]) for v in range(g.n)] == [want[v] for v in range(g.n)]
    assert int(r["count"][0]) == sum(want.values()) // 3 > 0
