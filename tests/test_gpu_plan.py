"""Survey plans and the autotuner.  The plan (warp-item limit, in-edges per
block item, long-list limit, window strategy) moves work between kernels but
never changes a result: under every extreme plan the survey must equal the
oracle's, bit for bit; tripoll_tune must end with a valid plan whose survey
still equals the oracle's; a default plan reaches the graphs built after it."""
import numpy as np
import pytest

import synth
import paper_2107_12330_b300 as tp
from gpu_util import assert_equal_tables, oracle_vector

pytestmark = pytest.mark.gpu

ALL = tp.TRIPOLL_ALL_KINDS & ~tp.TRIPOLL_EDGE_LOCAL
PLANS = [
    {"warp_max_dplus": 32, "block_item_in_edges": 256, "long_list_min_dplus": 1024, "window_view": 0},
    {"warp_max_dplus": 256, "block_item_in_edges": 2048, "long_list_min_dplus": 65536, "window_view": 1},
    {"warp_max_dplus": 64, "block_item_in_edges": 512, "long_list_min_dplus": 2048, "window_view": 1},
]


def _survey(h, g, kinds, window):
    out = np.zeros(tp.tripoll_result_words(kinds, g.num_vlabels, g.num_elabels, g.n), np.uint64)
    tp.tripoll_survey(h, kinds, window[0], window[1], out)
    return out


def test_every_plan_gives_the_oracles_survey():
    graphs = [synth.rmat_graph(12, 16, 7, ts_bits=20, num_vlabels=4, num_elabels=5)]
    # a dense graph whose out-lists pass every threshold (K_1200: d+ up to 1199)
    n = 1200
    iu = np.triu_indices(n, 1)
    m = len(iu[0])
    graphs.append(synth.Graph("K1200", n, iu[0].astype(np.uint32), iu[1].astype(np.uint32),
                              synth.uniform_bits(3, synth.STREAM_TS, m, 16),
                              synth.uniform_labels(3, synth.STREAM_VLABEL, n, 3),
                              synth.uniform_labels(3, synth.STREAM_ELABEL, m, 3), 3, 3, 15))
    for g in graphs:
        kinds = ALL if g.name != "K1200" else tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_ELABEL_TRIPLES
        windows = [(0, 0xFFFFFFFF), (1 << 12, 3 << 12)]
        wants = {w: oracle_vector(g, kinds, window=w)[0] for w in windows}
        h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels)
        try:
            for plan in PLANS:
                tp.tripoll_set_plan(h, plan)
                assert tp.tripoll_get_plan(h) == plan
                for w in windows:
                    assert_equal_tables(_survey(h, g, kinds, w), wants[w], kinds, g)
        finally:
            tp.tripoll_destroy(h)


def test_autotuner_ends_with_a_valid_plan_and_the_same_survey():
    g = synth.rmat_graph(13, 16, 8, ts_bits=20, num_vlabels=4, num_elabels=5)
    kinds = tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_ELABEL_TRIPLES
    window = (1 << 18, 3 << 18)
    h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels)
    try:
        plan, best_ms, start_ms = tp.tripoll_tune(h, kinds, window[0], window[1], reps=2)
        assert tp.tripoll_get_plan(h) == plan
        assert 0 < best_ms <= start_ms
        assert plan["warp_max_dplus"] in (32, 64, 128, 256)
        assert plan["block_item_in_edges"] in (512, 1024, 2048)
        assert plan["long_list_min_dplus"] in (2048, 4096, 8192)
        got = _survey(h, g, kinds, window)
        want, _ = oracle_vector(g, kinds, window=window)
        assert_equal_tables(got, want, kinds, g)
    finally:
        tp.tripoll_destroy(h)


def test_default_plan_reaches_new_graphs():
    g = synth.rmat_graph(9, 8, 2, ts_bits=12, num_vlabels=2, num_elabels=2)
    try:
        tp.tripoll_set_default_plan(PLANS[0])
        h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 2, 2)
        try:
            assert tp.tripoll_get_plan(h) == PLANS[0]
        finally:
            tp.tripoll_destroy(h)
    finally:
        tp.tripoll_set_default_plan(None)
    h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 2, 2)
    try:
        assert tp.tripoll_get_plan(h) == tp.DEFAULT_PLAN
    finally:
        tp.tripoll_destroy(h)
