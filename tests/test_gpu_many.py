"""Several requests on one graph in one pass (tripoll_survey_many, the unit the
server batches): every request's tables must equal the oracle's survey of that
request alone, bit for bit, for random kinds and windows, duplicate and
degenerate windows, the full window, 64 requests at once, records past the
on-chip mirror (word cache), and forced moves of the on-chip partial sums."""
import numpy as np
import pytest

import synth
import paper_2107_12330_b300 as tp
from gpu_util import assert_equal_tables, oracle_vector

pytestmark = pytest.mark.gpu

FUSABLE = [tp.TRIPOLL_COUNT, tp.TRIPOLL_CLOSURE_HIST, tp.TRIPOLL_VLABEL_TRIPLES, tp.TRIPOLL_ELABEL_TRIPLES,
           tp.TRIPOLL_OPEN_CLOSE_HIST, tp.TRIPOLL_MAX_ELABEL, tp.TRIPOLL_DEGREE_TRIPLES,
           tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_ELABEL_TRIPLES]


def _requests(seed, count, ts_max, kinds=FUSABLE):
    reqs = []
    for i in range(count):
        d = [synth.draw(seed, 4, 4 * i + j) for j in range(4)]
        k = kinds[d[0] % len(kinds)]
        lo, hi = sorted((d[1] % (ts_max + 1), d[2] % (ts_max + 1)))
        if d[3] % 9 == 0:
            lo, hi = 0, 0xFFFFFFFF
        reqs.append((k, lo, hi))
    return reqs


def _check_many(g, reqs, device=False):
    import torch
    h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels)
    try:
        words = [tp.tripoll_result_words(k, g.num_vlabels, g.num_elabels, g.n) for k, _, _ in reqs]
        if device:
            outs = [torch.full((w,), -1, dtype=torch.int64, device="cuda") for w in words]
        else:
            outs = [np.full(w, 5, np.uint64) for w in words]
        tp.tripoll_survey_many(h, [r[0] for r in reqs], [r[1] for r in reqs], [r[2] for r in reqs], outs)
        if device:
            torch.cuda.synchronize()
            outs = [o.cpu().numpy().view(np.uint64) for o in outs]
        for (k, lo, hi), got in zip(reqs, outs):
            want, _ = oracle_vector(g, k, window=(lo, hi))
            assert_equal_tables(got, want, k, g)
            alone = np.zeros_like(got)
            tp.tripoll_survey(h, k, lo, hi, alone)
            assert np.array_equal(alone, got)
    finally:
        tp.tripoll_destroy(h)


@pytest.mark.parametrize("count", [1, 2, 7, 64])
def test_many_requests_on_rmat_match_the_oracle(count):
    g = synth.rmat_graph(11, 16, 5, ts_bits=16, num_vlabels=4, num_elabels=5)
    _check_many(g, _requests(40 + count, count, 1 << 16), device=count % 2 == 0)


def test_many_requests_on_tiny_graphs_with_shared_and_degenerate_windows():
    g = synth.tiny_random_graph(61, 300, 20000, ts_bits=6, num_vlabels=3, num_elabels=4)
    reqs = [(tp.TRIPOLL_COUNT, 10, 40), (tp.TRIPOLL_CLOSURE_HIST, 10, 40), (tp.TRIPOLL_COUNT, 10, 40),
            (tp.TRIPOLL_COUNT, 0, 0), (tp.TRIPOLL_VLABEL_TRIPLES, 63, 63), (tp.TRIPOLL_ELABEL_TRIPLES, 20, 21),
            (tp.TRIPOLL_COUNT | tp.TRIPOLL_ELABEL_TRIPLES, 0, 0xFFFFFFFF), (tp.TRIPOLL_MAX_ELABEL, 5, 60),
            (tp.TRIPOLL_DEGREE_TRIPLES, 30, 31), (tp.TRIPOLL_OPEN_CLOSE_HIST, 0, 63)]
    _check_many(g, reqs)


def test_many_requests_with_large_tables_and_forced_mirror_moves(monkeypatch):
    """64 vertex labels (a 262,144-word triple table) make every cell record pass through the word cache;
    moving the on-chip sums after every work item exercises the moves of cache and mirror together."""
    monkeypatch.setenv("TRIPOLL_MIRROR_MOVE_LOG2", "0")
    g = synth.rmat_graph(10, 16, 9, ts_bits=12, num_vlabels=64, num_elabels=8)
    reqs = [(tp.TRIPOLL_VLABEL_TRIPLES | tp.TRIPOLL_COUNT, 0, 4095), (tp.TRIPOLL_VLABEL_TRIPLES, 100, 3000),
            (tp.TRIPOLL_ELABEL_TRIPLES, 500, 4000), (tp.TRIPOLL_DEGREE_TRIPLES, 0, 2000)]
    _check_many(g, reqs)


def test_many_rejects_what_it_cannot_fuse():
    g = synth.rmat_graph(8, 8, 2, ts_bits=12, num_vlabels=2, num_elabels=2)
    h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 2, 2)
    try:
        out = [np.zeros(tp.tripoll_result_words(tp.TRIPOLL_VERTEX_LOCAL, 2, 2, g.n), np.uint64)]
        with pytest.raises(tp.TripollError) as e:
            tp.tripoll_survey_many(h, [tp.TRIPOLL_VERTEX_LOCAL], [0], [10], out)
        assert e.value.status == tp.TRIPOLL_ERR_INVALID_ARG
        outs = [np.zeros(1, np.uint64) for _ in range(65)]
        with pytest.raises(tp.TripollError) as e:
            tp.tripoll_survey_many(h, [tp.TRIPOLL_COUNT] * 65, [0] * 65, [10] * 65, outs)
        assert e.value.status == tp.TRIPOLL_ERR_INVALID_ARG
        with pytest.raises(tp.TripollError) as e:
            tp.tripoll_survey_many(h, [tp.TRIPOLL_COUNT], [5], [4], [np.zeros(1, np.uint64)])
        assert e.value.status == tp.TRIPOLL_ERR_INVALID_ARG
    finally:
        tp.tripoll_destroy(h)
