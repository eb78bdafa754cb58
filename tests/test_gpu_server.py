"""Serving: resident graphs and continuously batched requests.  Every result a
request gets in a mix of concurrent requests (different graphs, kinds and
windows, submitted from several threads while others run) must equal the
survey of that request alone, bit for bit, and both must equal the CPU
oracle's survey of the request (on the graphs the oracle finishes quickly)."""
import threading

import numpy as np
import pytest

import synth
import paper_2107_12330_b300 as tp
from gpu_util import oracle_vector

pytestmark = pytest.mark.gpu
KINDS = [tp.TRIPOLL_COUNT, tp.TRIPOLL_CLOSURE_HIST, tp.TRIPOLL_VLABEL_TRIPLES, tp.TRIPOLL_ELABEL_TRIPLES,
         tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_ELABEL_TRIPLES]


def _graphs():
    """Small graphs, and one (scale 22, about 64M edges) past the size from which the server runs requests one
    at a time while small ones overlap them."""
    out = []
    for i, sc in enumerate([10, 12, 14, 22]):
        g = synth.rmat_graph(sc, 16, i + 1, ts_bits=24, num_vlabels=16, num_elabels=8)
        h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 16, 8)
        out.append((g, h))
    return out


def test_requests_in_a_mix_equal_requests_alone():
    graphs = _graphs()
    try:
        reqs = []
        for i in range(60):
            d = [synth.draw(5, 9, 4 * i + j) for j in range(4)]
            gi = d[0] % len(graphs)
            k = KINDS[d[1] % len(KINDS)]
            lo, hi = sorted(((d[2] >> 40) % (1 << 24), (d[3] >> 40) % (1 << 24)))
            if i % 7 == 0:
                lo, hi = 0, 0xFFFFFFFF
            reqs.append((gi, k, lo, hi))
        alone = []
        checked = 0
        for gi, k, lo, hi in reqs:
            g, h = graphs[gi]
            o = np.zeros(tp.tripoll_result_words(k, 16, 8, g.n), np.uint64)
            tp.tripoll_survey(h, k, lo, hi, o)
            alone.append(o)
            if g.n <= 1 << 14:  # the request against the oracle (Sec. 3 triangle set, Alg. 4 closing time)
                want, _ = oracle_vector(g, k, window=(lo, hi))
                assert np.array_equal(o, want), f"request {(gi, k, lo, hi)} differs from the oracle"
                checked += 1
        assert checked >= 30
        srv = tp.tripoll_server_create(1 << 30, 8)
        try:
            slots = [tp.tripoll_server_add_graph(srv, h) for _, h in graphs]
            ids = [None] * len(reqs)

            def submit(part):
                for i in part:
                    gi, k, lo, hi = reqs[i]
                    ids[i] = tp.tripoll_server_submit(srv, slots[gi], k, lo, hi)

            threads = [threading.Thread(target=submit, args=(range(t, len(reqs), 3),)) for t in range(3)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            for i, (gi, k, lo, hi) in enumerate(reqs):
                g, _ = graphs[gi]
                o = np.zeros(tp.tripoll_result_words(k, 16, 8, g.n), np.uint64)
                lat = tp.tripoll_server_wait(srv, ids[i], o, 120000)
                assert lat > 0
                assert np.array_equal(o, alone[i]), f"request {i} differs in the mix"
            with pytest.raises(tp.TripollError) as e:
                tp.tripoll_server_wait(srv, 10 ** 9, None, 10)
            assert e.value.status == tp.TRIPOLL_ERR_NOT_FOUND
        finally:
            tp.tripoll_server_destroy(srv)
    finally:
        for _, h in graphs:
            tp.tripoll_destroy(h)


def test_requests_beyond_the_scratch_budget_are_refused():
    graphs = _graphs()
    try:
        srv = tp.tripoll_server_create(1024, 4)  # 1 KB of scratch: a 33-word histogram fits, 4096 triples do not
        try:
            slot = tp.tripoll_server_add_graph(srv, graphs[0][1])
            rid = tp.tripoll_server_submit(srv, slot, tp.TRIPOLL_CLOSURE_HIST)
            o = np.zeros(33, np.uint64)
            tp.tripoll_server_wait(srv, rid, o, 60000)
            assert o.sum() > 0
            with pytest.raises(tp.TripollError) as e:
                tp.tripoll_server_submit(srv, slot, tp.TRIPOLL_VLABEL_TRIPLES)
            assert e.value.status == tp.TRIPOLL_ERR_NO_MEMORY
        finally:
            tp.tripoll_server_destroy(srv)
    finally:
        for _, h in graphs:
            tp.tripoll_destroy(h)


def test_requests_without_room_for_a_window_view_match_the_oracle():
    """A budget that holds a request's result but not the window view makes the server survey in place
    (out-of-window edges skipped where they are met); those results must equal the oracle's too."""
    graphs = [(g, h) for g, h in _graphs() if g.n <= 1 << 14]
    srv = tp.tripoll_server_create(64 << 10, 4)
    try:
        slots = [tp.tripoll_server_add_graph(srv, h) for _, h in graphs]
        reqs = []
        for i in range(16):
            d = [synth.draw(6, 3, 4 * i + j) for j in range(4)]
            gi = d[0] % len(graphs)
            k = KINDS[d[1] % len(KINDS)]
            lo, hi = sorted(((d[2] >> 40) % (1 << 24), (d[3] >> 40) % (1 << 24)))
            reqs.append((gi, k, lo, hi, tp.tripoll_server_submit(srv, slots[gi], k, lo, hi)))
        for gi, k, lo, hi, rid in reqs:
            g, _ = graphs[gi]
            o = np.zeros(tp.tripoll_result_words(k, 16, 8, g.n), np.uint64)
            tp.tripoll_server_wait(srv, rid, o, 120000)
            want, _ = oracle_vector(g, k, window=(lo, hi))
            assert np.array_equal(o, want), f"request {(gi, k, lo, hi)} differs from the oracle"
    finally:
        tp.tripoll_server_destroy(srv)
        for _, h in graphs:
            tp.tripoll_destroy(h)


def test_wait_times_out_and_the_request_stays_queued():
    """A wait shorter than the request's run returns TRIPOLL_ERR_TIMEOUT (a bounded wait on the host, no
    GPU involvement); the request stays queued and a later wait returns its result."""
    g = synth.rmat_graph(22, 16, 4, ts_bits=24, num_vlabels=16, num_elabels=8)
    h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 16, 8)
    srv = tp.tripoll_server_create(1 << 30, 4)
    try:
        slot = tp.tripoll_server_add_graph(srv, h)
        k = tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST
        ids = [tp.tripoll_server_submit(srv, slot, k) for _ in range(3)]
        o = np.zeros(tp.tripoll_result_words(k, 16, 8, g.n), np.uint64)
        with pytest.raises(tp.TripollError) as e:
            tp.tripoll_server_wait(srv, ids[-1], o, 0)
        assert e.value.status == tp.TRIPOLL_ERR_TIMEOUT
        alone = np.zeros_like(o)
        tp.tripoll_survey(h, k, 0, 0xFFFFFFFF, alone)
        for rid in ids:
            o[:] = 0
            tp.tripoll_server_wait(srv, rid, o, 120000)
            assert np.array_equal(o, alone)
    finally:
        tp.tripoll_server_destroy(srv)
        tp.tripoll_destroy(h)


def test_batches_without_room_for_the_union_window_view_match_the_oracle():
    """A budget that holds several requests' cell records but not the union window's view: the server still
    runs each graph's requests as one batch, skipping out-of-window edges in place; results equal the oracle."""
    g = synth.rmat_graph(13, 16, 12, ts_bits=24, num_vlabels=16, num_elabels=8)
    h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, 16, 8)
    srv = tp.tripoll_server_create(2 << 20, 64)  # 2 MB: records and results fit, a view of 130K edges does not
    try:
        slot = tp.tripoll_server_add_graph(srv, h)
        reqs = []
        for i in range(12):
            d = [synth.draw(8, 1, 3 * i + j) for j in range(3)]
            k = [tp.TRIPOLL_COUNT, tp.TRIPOLL_CLOSURE_HIST, tp.TRIPOLL_ELABEL_TRIPLES][d[0] % 3]
            lo, hi = sorted(((d[1] >> 40) % (1 << 24), (d[2] >> 40) % (1 << 24)))
            reqs.append((k, lo, hi, tp.tripoll_server_submit(srv, slot, k, lo, hi)))
        for k, lo, hi, rid in reqs:
            o = np.zeros(tp.tripoll_result_words(k, 16, 8, g.n), np.uint64)
            tp.tripoll_server_wait(srv, rid, o, 120000)
            want, _ = oracle_vector(g, k, window=(lo, hi))
            assert np.array_equal(o, want), f"request {(k, lo, hi)} differs from the oracle"
    finally:
        tp.tripoll_server_destroy(srv)
        tp.tripoll_destroy(h)
