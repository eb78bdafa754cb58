"""The C ABI library loads and exports every entry point include/tripoll.h
declares; host-only helpers behave as documented (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import paper_2107_12330_b300 as tp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "tripoll.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tripoll_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = tp.load_library()
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(tp.EXPORTS)
    # the Python binding carries the same names as the C entry points
    unbound = [n for n in names if not callable(getattr(tp, n, None))]
    assert not unbound, unbound


def test_result_words_layout():
    assert tp.tripoll_result_words(tp.TRIPOLL_COUNT, 4, 8) == 1
    assert tp.tripoll_result_words(tp.TRIPOLL_CLOSURE_HIST, 4, 8) == 33
    assert tp.tripoll_result_words(1 | 2 | 4, 4, 1) == 1 + 33 + 64
    assert tp.tripoll_result_words(2 | 8, 16, 8) == 33 + 512
    assert tp.tripoll_result_words(tp.TRIPOLL_ALL_KINDS, 2, 3, 10, 7) == 1 + 33 + 8 + 27 + 33 * 33 + 3 + 33 ** 3 + 10 + 7
    assert tp.tripoll_result_words(tp.TRIPOLL_EDGE_LOCAL, 1, 1, 10, 7) == 7


def test_status_strings():
    assert tp.tripoll_status_string(0) == "ok"
    assert "vertex" in tp.tripoll_status_string(tp.TRIPOLL_ERR_VERTEX_RANGE)
    assert tp.tripoll_status_string(-99) == "unknown status"


def test_split_result_views():
    import numpy as np
    v = np.arange(1 + 33 + 8, dtype=np.uint64)
    parts = tp.split_result(v, 1 | 2 | 4, 2, 1)
    assert parts["count"].tolist() == [0]
    assert parts["hist"][0] == 1 and len(parts["hist"]) == 33
    assert len(parts["vtri"]) == 8


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    # no fallback path: without the shared library every call raises
    monkeypatch.setattr(tp, "_lib", None)
    with pytest.raises(OSError):
        tp.load_library(str(tmp_path / "libtripoll.so"))


def test_split_result_matches_the_library_layout_for_every_kind_mask():
    """The binding's table layout and the library's record size agree for all 2^9 kind masks: the parts
    split_result cuts out are contiguous, in the header's order, and end exactly at tripoll_result_words."""
    for Lv, Le, n, m in [(1, 1, 0, 0), (2, 3, 5, 7), (16, 8, 1000, 4000), (64, 16, 3, 2)]:
        for mask in range(1, tp.TRIPOLL_ALL_KINDS + 1):
            words = tp.tripoll_result_words(mask, Lv, Le, n, m)
            vec = np.arange(words, dtype=np.uint64)
            parts = tp.split_result(vec, mask, Lv, Le, n, m)
            assert sum(len(p) for p in parts.values()) == words, (mask, Lv, Le)
            o = 0
            for p in parts.values():
                assert len(p) == 0 or int(p[0]) == o
                o += len(p)


def test_invalid_arguments_are_rejected_before_any_gpu_work():
    """Argument checks of the C ABI run on the host before the library touches the device, so on any machine
    each bad call returns TRIPOLL_ERR_INVALID_ARG with a message, and nothing is built or launched."""
    src = np.array([0, 1], np.uint32)
    dst = np.array([1, 2], np.uint32)
    ts = np.array([1, 2], np.uint32)
    el = np.array([0, 1], np.uint8)
    z = np.zeros(1, np.uint64)
    cases = {
        "no vertex label classes": lambda: tp.tripoll_graph_create(src, dst, ts, None, None, 3, 0, 1),
        "257 vertex label classes": lambda: tp.tripoll_graph_create(src, dst, ts, None, None, 3, 257, 1),
        "edge labels without classes": lambda: tp.tripoll_graph_create(src, dst, ts, el, None, 3, 1, 0),
        "257 edge label classes": lambda: tp.tripoll_graph_create(src, dst, ts, el, None, 3, 1, 257),
        "batch offsets not from 0": lambda: tp.tripoll_batch_create(
            src, dst, ts, None, np.array([1, 2], np.uint64), None, np.array([3], np.uint32), 1, 1),
        "batch offsets decreasing": lambda: tp.tripoll_batch_create(
            np.r_[src, src], np.r_[dst, dst], np.r_[ts, ts], None, np.array([0, 3, 2], np.uint64), None,
            np.array([3, 3], np.uint32), 1, 1),
        "survey of no graph": lambda: tp.tripoll_survey(None, tp.TRIPOLL_COUNT, 0, 1, z),
        "pivot range of no graph": lambda: tp.tripoll_survey_range(None, tp.TRIPOLL_COUNT, 0, 1, 0, 1, z),
        "static survey of no graph": lambda: tp.tripoll_survey_static(None, tp.TRIPOLL_COUNT, 0, 1, z),
        "several requests on no graph": lambda: tp.tripoll_survey_many(None, [tp.TRIPOLL_COUNT], [0], [1], [z]),
        "wedge checks of no graph": lambda: tp.tripoll_wedge_checks(None),
        "statistics of no graph": lambda: tp.tripoll_graph_stats(None),
        "partition of no graph": lambda: tp.tripoll_partition_pivots(None, 2),
        "server without budget": lambda: tp.tripoll_server_create(0, 4),
        "server without requests in flight": lambda: tp.tripoll_server_create(1 << 20, 0),
        "allocator without its free": lambda: tp.tripoll_set_allocator(lambda n, s: 0, None),
        "free without its allocator": lambda: tp.tripoll_set_allocator(None, lambda p, n, s: None),
    }
    for what, call in cases.items():
        with pytest.raises(tp.TripollError) as e:
            call()
        assert e.value.status == tp.TRIPOLL_ERR_INVALID_ARG, what


def test_allocator_hook_installs_and_restores_on_the_host():
    """Installing an allocator and restoring the library's pool are host-side settings: both succeed
    without a device, and no allocation is made by installing one."""
    calls = []
    tp.tripoll_set_allocator(lambda n, s: calls.append(n) or 0, lambda p, n, s: calls.append(-1))
    try:
        assert calls == []
    finally:
        tp.tripoll_set_allocator(None, None)


def test_plans_outside_their_bounds_are_rejected_on_the_host():
    """The plan bounds keep every on-chip 32-bit partial sum below 2^32: plans outside them are refused."""
    good = dict(tp.DEFAULT_PLAN)
    bad = [("warp_max_dplus", 16), ("warp_max_dplus", 512), ("block_item_in_edges", 300),
           ("block_item_in_edges", 4096), ("long_list_min_dplus", 512), ("long_list_min_dplus", 1 << 17),
           ("window_view", 2)]
    for field, value in bad:
        p = dict(good, **{field: value})
        with pytest.raises(tp.TripollError) as e:
            tp.tripoll_set_default_plan(p)
        assert e.value.status == tp.TRIPOLL_ERR_INVALID_ARG, (field, value)
    tp.tripoll_set_default_plan(dict(good, warp_max_dplus=256, block_item_in_edges=256))
    tp.tripoll_set_default_plan(None)


def test_tuned_plan_file_round_trip(tmp_path):
    from paper_2107_12330_b300 import tuning
    path = str(tmp_path / "plans.json")
    assert tuning.plan_for("rmat24", path) is None
    tuning.store_plan("rmat24", {"plan": dict(tp.DEFAULT_PLAN, warp_max_dplus=64), "survey_ms": 1.0}, path)
    assert tuning.plan_for("rmat24", path)["warp_max_dplus"] == 64
    import json
    with open(path) as f:
        data = json.load(f)
    data["version"] = tuning.FORMAT_VERSION + 1
    with open(path, "w") as f:
        json.dump(data, f)
    assert tuning.plan_for("rmat24", path) is None  # another format version is ignored
