"""Device memory from the caller's allocator (tripoll_set_allocator), and
allocation failures injected on the host.

A counting allocator on top of torch's caching allocator records every block
the library takes and gives back.  A build and a windowed survey through it
must equal the oracle, and every block must be back once the graph is
destroyed.  Then each allocation of a build + survey is made to fail in turn
(the allocator returns NULL): every call must fail with
TRIPOLL_ERR_NO_MEMORY and leave no block behind, and the library must work
normally afterwards.  No GPU fault is involved: the failure is a NULL
returned on the host."""
import numpy as np
import pytest

import synth
import paper_2107_12330_b300 as tp
from gpu_util import assert_equal_tables, oracle_vector

pytestmark = pytest.mark.gpu

KINDS = tp.TRIPOLL_COUNT | tp.TRIPOLL_CLOSURE_HIST | tp.TRIPOLL_VLABEL_TRIPLES | tp.TRIPOLL_ELABEL_TRIPLES


class CountingAllocator:
    """Blocks from torch's caching allocator, counted; optionally the fail_at-th request returns NULL."""

    def __init__(self, fail_at=None):
        self._alloc, self._free = tp.torch_caching_allocator()
        self.live = {}
        self.calls = 0
        self.errors = []
        self.fail_at = fail_at

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return 0
        p = self._alloc(nbytes, stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, nbytes, stream):
        if self.live.pop(ptr, None) != nbytes:
            self.errors.append((ptr, nbytes))
        self._free(ptr, nbytes, stream)


def _graph():
    return synth.rmat_graph(11, 16, 4, ts_bits=20, num_vlabels=4, num_elabels=4)


def _build_and_survey(g, window):
    h = tp.tripoll_graph_create(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels)
    try:
        out = np.zeros(tp.tripoll_result_words(KINDS, g.num_vlabels, g.num_elabels, g.n), np.uint64)
        tp.tripoll_survey(h, KINDS, window[0], window[1], out)
    finally:
        tp.tripoll_destroy(h)
    return out


def test_build_and_survey_through_the_callers_allocator():
    import torch
    g = _graph()
    window = (1 << 18, 3 << 18)
    c = CountingAllocator()
    tp.tripoll_set_allocator(c.alloc, c.free)
    try:
        out = _build_and_survey(g, window)
        torch.cuda.synchronize()
    finally:
        tp.tripoll_set_allocator(None, None)
    assert c.calls > 10, "the build and the window view should take their memory from the allocator"
    assert not c.live, f"{len(c.live)} blocks not returned"
    assert not c.errors
    want, _ = oracle_vector(g, KINDS, window=window)
    assert_equal_tables(out, want, KINDS, g)


def test_each_failed_allocation_leaves_nothing_allocated():
    import torch
    g = _graph()
    window = (1 << 18, 3 << 18)
    probe = CountingAllocator()
    tp.tripoll_set_allocator(probe.alloc, probe.free)
    try:
        want = _build_and_survey(g, window)
    finally:
        tp.tripoll_set_allocator(None, None)
    total = probe.calls
    assert total > 10
    for k in range(1, total + 1):
        c = CountingAllocator(fail_at=k)
        tp.tripoll_set_allocator(c.alloc, c.free)
        try:
            with pytest.raises(tp.TripollError) as e:
                _build_and_survey(g, window)
            torch.cuda.synchronize()
        finally:
            tp.tripoll_set_allocator(None, None)
        assert e.value.status == tp.TRIPOLL_ERR_NO_MEMORY, (k, e.value)
        assert not c.live, f"allocation {k} of {total} failed and {len(c.live)} blocks were left"
        assert not c.errors
    # the library is unaffected: the same survey from its own pool
    assert np.array_equal(_build_and_survey(g, window), want)
