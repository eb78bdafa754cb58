"""Full-size parity: the benchmark workload (R-MAT scale 24, 268M input edges),
built and surveyed in the launch configuration bench.py times, against the
oracle's stored survey (tests/golden/*_survey.json, written by
tests/golden/make_golden.py from the oracle alone).  Bit-exact.  The Chung-Lu
workload at its full size (about 1G edges; the oracle took 39 minutes on 7
host threads) is compared through the SHA-256 of the whole result and its
small tables, plus properties that hold at any size."""
import json
import os

import numpy as np
import pytest

import synth
import paper_2107_12330_b300 as tp

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    path = os.path.join(HERE, "golden", f"{name}_survey.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored survey {path}")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("name,make", [("rmat24", synth.rmat24)])
def test_full_size_survey_matches_stored_oracle(name, make):
    import torch
    gold = _golden(name)
    g = make()
    assert g.kinds == gold["kinds"] and list(g.window) == gold["window"] and g.m_in == gold["m_in"]
    dev = [torch.from_numpy(x).cuda() for x in (g.src, g.dst, g.ts, g.elabel, g.vlabel)]
    h = tp.tripoll_graph_create(*dev, g.n, g.num_vlabels, g.num_elabels)
    try:
        st = tp.tripoll_graph_stats(h)
        w = tp.tripoll_result_words(g.kinds, g.num_vlabels, g.num_elabels, g.n)
        out = torch.zeros(w, dtype=torch.int64, device="cuda")
        tp.tripoll_survey(h, g.kinds, g.window[0], g.window[1], out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
    finally:
        tp.tripoll_destroy(h)
    assert st["num_edges"] == gold["stats"]["m"]
    assert st["wedges"] == gold["stats"]["wedges"]
    assert st["dplus_max"] == gold["stats"]["dplus_max"]
    want = np.array(gold["result"], dtype=np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"words {bad[:10].tolist()} differ: gpu {got[bad[:10]].tolist()} oracle {want[bad[:10]].tolist()}"


def test_chung_lu_recipe_matches_stored_oracle():
    """The 50M-vertex Chung-Lu recipe (exponent 2.1, heavy hubs, 64 vertex labels) at
    2M vertices: all four tables, against the oracle's digest and small tables."""
    import hashlib
    import torch
    gold = _golden("chunglu2m")
    g = synth.chung_lu_50m(m_samples=gold["m_in"], n=gold["n"])
    dev = [torch.from_numpy(x).cuda() for x in (g.src, g.dst, g.ts, g.elabel, g.vlabel)]
    h = tp.tripoll_graph_create(*dev, g.n, g.num_vlabels, g.num_elabels)
    try:
        st = tp.tripoll_graph_stats(h)
        w = tp.tripoll_result_words(g.kinds, g.num_vlabels, g.num_elabels, g.n)
        assert w == gold["words"]
        out = torch.zeros(w, dtype=torch.int64, device="cuda")
        tp.tripoll_survey(h, g.kinds, 0, 0xFFFFFFFF, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
    finally:
        tp.tripoll_destroy(h)
    assert st["num_edges"] == gold["stats"]["m"] and st["wedges"] == gold["stats"]["wedges"]
    parts = tp.split_result(got, g.kinds, g.num_vlabels, g.num_elabels)
    assert int(parts["count"][0]) == gold["count"]
    assert parts["hist"].tolist() == gold["hist"]
    assert parts["etri"].tolist() == gold["etri"]
    assert hashlib.sha256(got.astype("<u8").tobytes()).hexdigest() == gold["sha256"]


def test_full_batched_family_matches_stored_oracle():
    """All 20,000 graphs of the batched family in one build and one survey launch
    pair: per-graph records against the oracle's, by SHA-256 of the whole result
    and by per-graph triangle counts."""
    import hashlib
    import torch
    gold = _golden("batched20000")
    G = gold["num_graphs"]
    graphs = [synth.batched_graph(i) for i in range(G)]
    eoff = np.zeros(G + 1, np.uint64)
    eoff[1:] = np.cumsum([g.m_in for g in graphs])
    nv = np.array([g.n for g in graphs], np.uint32)
    cat = [torch.from_numpy(np.concatenate([getattr(g, k) for g in graphs])).cuda()
           for k in ("src", "dst", "ts", "vlabel")]
    del graphs
    kinds = gold["kinds"]
    h = tp.tripoll_batch_create(cat[0], cat[1], cat[2], None, eoff, cat[3], nv, 4, 0)
    try:
        w = tp.tripoll_result_words(kinds, 4, 1, 0)
        assert w == gold["words_per_graph"]
        out = torch.zeros(w * G, dtype=torch.int64, device="cuda")
        tp.tripoll_survey(h, kinds, 0, 0xFFFFFFFF, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64).reshape(G, w)
    finally:
        tp.tripoll_destroy(h)
    counts = got[:, 0].astype(np.int64)
    want = np.array(gold["counts"], dtype=np.int64)
    bad = np.nonzero(counts != want)[0]
    assert bad.size == 0, f"graphs {bad[:10].tolist()} differ in count"
    assert got[:, 1:].sum(axis=0).tolist() == gold["hist_total"]
    assert hashlib.sha256(got.astype("<u8").tobytes()).hexdigest() == gold["sha256"]


def test_chunglu_50m_matches_stored_oracle_at_full_size():
    """The Chung-Lu workload at its benchmark size (50M vertices, 1.2G sampled pairs, 995M edges, 53.9G
    triangles): the whole survey (count, closing-time histogram, 64^3 vertex-label and 8^3 edge-label
    triples) against the oracle's digest and small tables.  Then properties that hold at any size: every
    table sums to the count, the per-vertex participation sums to three times the count, and pivot-range
    shards add up to the full survey."""
    import hashlib
    import torch
    gold = _golden("chunglu50m")
    g = synth.chung_lu_50m()
    assert g.m_in == gold["m_in"] and g.n == gold["n"] and g.kinds == gold["kinds"]
    dev = [torch.from_numpy(x).cuda() for x in (g.src, g.dst, g.ts, g.elabel, g.vlabel)]
    h = tp.tripoll_graph_create(*dev, g.n, g.num_vlabels, g.num_elabels)
    del dev
    try:
        kinds = g.kinds | tp.TRIPOLL_VERTEX_LOCAL
        w = tp.tripoll_result_words(kinds, g.num_vlabels, g.num_elabels, g.n)
        out = torch.zeros(w, dtype=torch.int64, device="cuda")
        tp.tripoll_survey(h, kinds, 0, 0xFFFFFFFF, out)
        torch.cuda.synchronize()
        st = tp.tripoll_graph_stats(h)
        assert st["num_edges"] == gold["stats"]["m"] and st["wedges"] == gold["stats"]["wedges"]
        assert st["dplus_max"] == gold["stats"]["dplus_max"] and st["degree_max"] == gold["stats"]["dmax"]
        parts = tp.split_result(out.cpu().numpy().view(np.uint64), kinds, g.num_vlabels, g.num_elabels, g.n)
        count = int(parts["count"][0])
        assert count == gold["count"]
        assert parts["hist"].tolist() == gold["hist"]
        assert parts["etri"].tolist() == gold["etri"]
        tables = np.concatenate([parts[k] for k in ("count", "hist", "vtri", "etri")])
        assert len(tables) == gold["words"]
        assert hashlib.sha256(tables.astype("<u8").tobytes()).hexdigest() == gold["sha256"]
        for k in ("hist", "vtri", "etri"):
            assert int(parts[k].sum(dtype=np.uint64)) == count, k
        assert int(parts["vlocal"].sum(dtype=np.uint64)) == 3 * count
        full = np.concatenate([parts[k] for k in ("count", "hist", "vtri", "etri")])
        bounds = tp.tripoll_partition_pivots(h, 3)
        acc = np.zeros_like(full)
        w2 = tp.tripoll_result_words(g.kinds, g.num_vlabels, g.num_elabels, g.n)
        for lo, hi in zip(bounds[:-1], bounds[1:]):
            part = torch.zeros(w2, dtype=torch.int64, device="cuda")
            tp.tripoll_survey_range(h, g.kinds, 0, 0xFFFFFFFF, int(lo), int(hi), part)
            torch.cuda.synchronize()
            acc += part.cpu().numpy().view(np.uint64)
        assert np.array_equal(acc, full)
    finally:
        tp.tripoll_destroy(h)
