"""tripoll_survey_static: the survey for callers that cannot allocate device
memory (stream capture in progress, allocator-free request loops, memory owned
by another framework).  Its scratch is a static device array instead of the
stream-ordered pool, so its results must equal tripoll_survey's, call after
call, although every call reuses the array the previous one left behind.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import synth
import paper_2107_12330_b300 as tp

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
