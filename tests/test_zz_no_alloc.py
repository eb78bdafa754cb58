"""tripoll_survey_static: the survey for callers that cannot allocate device
memory where they survey -- request loops that must never enter an allocator,
and hosts whose device memory belongs to another framework.  Its scratch is a
static device array instead of allocated memory, so its results must equal
tripoll_survey's, call after call, although every call reuses the array the
previous one left behind.  It skips out-of-window edges in place (no window
view), so it is also compared with the oracle directly.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import synth
import paper_2107_12330_b300 as tp
from gpu_util import assert_equal_tables, oracle_vector

pytestmark = pytest.mark.gpu


def test_static_scratch_survey_equals_allocating_survey_twice():
    import torch
    g = synth.rmat_graph(13, 16, 11, ts_bits=20, num_vlabels=4, num_elabels=5)
    kinds = tp.TRIPOLL_ALL_KINDS & ~(tp.TRIPOLL_VERTEX_LOCAL | tp.TRIPOLL_EDGE_LOCAL)
    dev = [torch.from_numpy(a).cuda() for a in (g.src, g.dst, g.ts, g.elabel, g.vlabel)]
    h = tp.tripoll_graph_create(*dev, g.n, g.num_vlabels, g.num_elabels)
    try:
        w = tp.tripoll_result_words(kinds, g.num_vlabels, g.num_elabels, g.n)
        for window in [(0, 0xFFFFFFFF), (1 << 18, 3 << 18)]:
            ref = torch.zeros(w, dtype=torch.int64, device="cuda")
            tp.tripoll_survey(h, kinds, window[0], window[1], ref)
            torch.cuda.synchronize()
            want = ref.cpu().numpy().view(np.uint64)
            assert want[0] > 0
            for _ in range(2):  # the second call starts from the first call's leftovers
                out_dev = torch.full((w,), -1, dtype=torch.int64, device="cuda")
                tp.tripoll_survey_static(h, kinds, window[0], window[1], out_dev)
                torch.cuda.synchronize()
                assert np.array_equal(out_dev.cpu().numpy().view(np.uint64), want)
                out_host = np.full(w, 7, np.uint64)
                tp.tripoll_survey_static(h, kinds, window[0], window[1], out_host)
                assert np.array_equal(out_host, want)
    finally:
        tp.tripoll_destroy(h)


@pytest.mark.parametrize("make,window", [
    (lambda: synth.rmat_graph(12, 16, 9, ts_bits=20, num_vlabels=4, num_elabels=5), (1 << 18, 3 << 18)),
    (lambda: synth.rmat_graph(12, 16, 9, ts_bits=20, num_vlabels=4, num_elabels=5), (0, 1 << 17)),
    (lambda: synth.tiny_random_graph(31, 300, 20000, ts_bits=6, num_vlabels=3, num_elabels=4), (10, 40)),
    (lambda: synth.tiny_random_graph(32, 1000, 30000, ts_bits=8, num_vlabels=3, num_elabels=4), (0, 0)),
])
def test_static_scratch_survey_matches_the_oracle(make, window):
    """The in-place window path (in-edges and (q,r) entries outside the window skipped where they are met,
    no compacted view) against the oracle's survey over the same window."""
    g = make()
    kinds = tp.TRIPOLL_ALL_KINDS & ~(tp.TRIPOLL_VERTEX_LOCAL | tp.TRIPOLL_EDGE_LOCAL)
    h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels)
    try:
        out = np.zeros(tp.tripoll_result_words(kinds, g.num_vlabels, g.num_elabels, g.n), np.uint64)
        for _ in range(2):
            out[:] = 3
            tp.tripoll_survey_static(h, kinds, window[0], window[1], out)
            want, _ = oracle_vector(g, kinds, window=window)
            assert_equal_tables(out, want, kinds, g)
    finally:
        tp.tripoll_destroy(h)


def test_static_scratch_survey_calls_no_allocator():
    """With a caller's allocator installed, tripoll_survey_static never calls it (tripoll_survey does, for its
    result record and window view)."""
    g = synth.rmat_graph(11, 16, 5, ts_bits=20, num_vlabels=4, num_elabels=5)
    kinds = tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_ELABEL_TRIPLES
    h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels)
    calls = []
    alloc, free = tp.torch_caching_allocator()
    try:
        out = np.zeros(tp.tripoll_result_words(kinds, g.num_vlabels, g.num_elabels, g.n), np.uint64)
        tp.tripoll_survey_static(h, kinds, 1 << 18, 3 << 18, out)  # first call on the device: set-up
        tp.tripoll_set_allocator(lambda n, s: calls.append(n) or alloc(n, s), free)
        try:
            static = np.zeros_like(out)
            tp.tripoll_survey_static(h, kinds, 1 << 18, 3 << 18, static)
            assert calls == []
            tp.tripoll_survey(h, kinds, 1 << 18, 3 << 18, out)
            assert len(calls) > 0
        finally:
            tp.tripoll_set_allocator(None, None)
        assert np.array_equal(static, out)
    finally:
        tp.tripoll_destroy(h)


def test_static_scratch_rejects_results_beyond_its_size():
    import torch
    # per-vertex local counts of 2^21 vertices need 16 MiB: more than the 8 MiB array
    g = synth.rmat_graph(21, 2, 3, ts_bits=20, num_vlabels=1, num_elabels=0)
    dev = [torch.from_numpy(a).cuda() for a in (g.src, g.dst, g.ts)]
    h = tp.tripoll_graph_create(*dev, None, None, g.n, 1, 0)
    try:
        w = tp.tripoll_result_words(tp.TRIPOLL_VERTEX_LOCAL, 1, 1, g.n)
        out = torch.zeros(w, dtype=torch.int64, device="cuda")
        with pytest.raises(tp.TripollError) as e:
            tp.tripoll_survey_static(h, tp.TRIPOLL_VERTEX_LOCAL, 0, 0xFFFFFFFF, out)
        assert e.value.status == tp.TRIPOLL_ERR_NO_MEMORY
        assert "static scratch" in str(e.value)
    finally:
        tp.tripoll_destroy(h)
