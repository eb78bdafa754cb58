"""Python binding of libtripoll.so, the B300 metadata triangle survey library.

Argument marshalling only: every function forwards to the C entry point of
the same name declared in ``include/tripoll.h``.  Arrays may be torch tensors
(device or host) or numpy arrays (host); the library copies host data itself.
Streams default to torch's current CUDA stream.  There is no fallback: if the
shared library is missing or fails to load, importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtripoll.so")

TRIPOLL_OK = 0
TRIPOLL_ERR_INVALID_ARG = -1
TRIPOLL_ERR_VERTEX_RANGE = -2
TRIPOLL_ERR_LABEL_RANGE = -3
TRIPOLL_ERR_NO_MEMORY = -4
TRIPOLL_ERR_CUDA = -5
TRIPOLL_ERR_TIMEOUT = -6
TRIPOLL_ERR_NO_EDGE_LABELS = -7
TRIPOLL_ERR_NOT_FOUND = -8

TRIPOLL_COUNT = 1
TRIPOLL_CLOSURE_HIST = 2
TRIPOLL_VLABEL_TRIPLES = 4
TRIPOLL_ELABEL_TRIPLES = 8
TRIPOLL_OPEN_CLOSE_HIST = 16
TRIPOLL_MAX_ELABEL = 32
TRIPOLL_DEGREE_TRIPLES = 64
TRIPOLL_VERTEX_LOCAL = 128
TRIPOLL_EDGE_LOCAL = 256
TRIPOLL_ALL_KINDS = 511
TRIPOLL_HIST_BINS = 33
FULL_WINDOW = (0, 0xFFFFFFFF)

# every symbol include/tripoll.h declares
EXPORTS = (
    "tripoll_graph_create", "tripoll_batch_create", "tripoll_result_words", "tripoll_survey",
    "tripoll_survey_range", "tripoll_partition_pivots", "tripoll_graph_stats", "tripoll_graph_export",
    "tripoll_destroy", "tripoll_server_create", "tripoll_server_add_graph", "tripoll_server_submit",
    "tripoll_server_wait", "tripoll_server_destroy", "tripoll_status_string", "tripoll_last_error",
    "tripoll_launch_count", "tripoll_wedge_checks", "tripoll_survey_static", "tripoll_set_allocator",
    "tripoll_survey_timed", "tripoll_survey_many", "tripoll_server_stats", "tripoll_get_plan",
    "tripoll_set_plan", "tripoll_set_default_plan", "tripoll_tune",
)

# C signatures of the allocator hook (tripoll_alloc_fn, tripoll_free_fn)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class TripollError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class GraphInfo(ctypes.Structure):
    _fields_ = [
        ("num_vertices", ctypes.c_uint64), ("num_input_edges", ctypes.c_uint64),
        ("num_edges", ctypes.c_uint64), ("wedges", ctypes.c_uint64), ("dplus_max", ctypes.c_uint64),
        ("degree_max", ctypes.c_uint64), ("q_list_words", ctypes.c_uint64),
        ("num_graphs", ctypes.c_uint64), ("num_vlabels", ctypes.c_uint32),
        ("num_elabels", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Plan(ctypes.Structure):
    """tripoll_plan: the survey plan of a graph (see tripoll.h)."""
    _fields_ = [("warp_max_dplus", ctypes.c_uint32), ("block_item_in_edges", ctypes.c_uint32),
                ("long_list_min_dplus", ctypes.c_uint32), ("window_view", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}

    @classmethod
    def of(cls, d):
        return d if isinstance(d, cls) else cls(**{k: int(d[k]) for k, _ in cls._fields_})


DEFAULT_PLAN = {"warp_max_dplus": 128, "block_item_in_edges": 2048, "long_list_min_dplus": 4096, "window_view": 1}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtripoll.so (raises OSError if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not built; run `python -m paper_2107_12330_b300.build`")
    lib = ctypes.CDLL(path)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    pvp = ctypes.POINTER(ctypes.c_void_p)
    lib.tripoll_graph_create.argtypes = [vp, vp, vp, vp, u64, vp, u32, u32, u32, vp, pvp]
    lib.tripoll_batch_create.argtypes = [vp, vp, vp, vp, vp, vp, vp, u32, u32, u32, vp, pvp]
    lib.tripoll_result_words.argtypes = [u32, u32, u32, u64, u64]
    lib.tripoll_result_words.restype = u64
    lib.tripoll_survey.argtypes = [vp, u32, u32, u32, vp, vp]
    lib.tripoll_survey_range.argtypes = [vp, u32, u32, u32, u64, u64, vp, vp]
    lib.tripoll_partition_pivots.argtypes = [vp, u32, vp, vp]
    lib.tripoll_graph_stats.argtypes = [vp, ctypes.POINTER(GraphInfo)]
    lib.tripoll_graph_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.tripoll_destroy.argtypes = [vp]
    lib.tripoll_destroy.restype = None
    lib.tripoll_server_create.argtypes = [u64, u32, pvp]
    lib.tripoll_server_add_graph.argtypes = [vp, vp, ctypes.POINTER(u32)]
    lib.tripoll_server_submit.argtypes = [vp, u32, u32, u32, u32, ctypes.POINTER(u64)]
    lib.tripoll_server_wait.argtypes = [vp, u64, vp, ctypes.POINTER(u64), u32]
    lib.tripoll_server_destroy.argtypes = [vp]
    lib.tripoll_server_destroy.restype = None
    lib.tripoll_status_string.argtypes = [i32]
    lib.tripoll_status_string.restype = ctypes.c_char_p
    lib.tripoll_last_error.argtypes = []
    lib.tripoll_last_error.restype = ctypes.c_char_p
    lib.tripoll_wedge_checks.argtypes = [vp, u32, u32, ctypes.POINTER(u64), vp]
    lib.tripoll_survey_static.argtypes = [vp, u32, u32, u32, vp, vp]
    lib.tripoll_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    lib.tripoll_survey_timed.argtypes = [vp, u32, u32, u32, u64, u64, vp, vp, vp]
    lib.tripoll_survey_many.argtypes = [vp, u32, vp, vp, vp, vp, vp]
    lib.tripoll_server_stats.argtypes = [vp, vp]
    pplan = ctypes.POINTER(Plan)
    lib.tripoll_get_plan.argtypes = [vp, pplan]
    lib.tripoll_set_plan.argtypes = [vp, pplan, vp]
    lib.tripoll_set_default_plan.argtypes = [pplan]
    lib.tripoll_tune.argtypes = [vp, u32, u32, u32, u32, pplan, ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_float), vp]
    lib.tripoll_launch_count.argtypes = []
    lib.tripoll_launch_count.restype = u64
    for name in ("tripoll_graph_create", "tripoll_batch_create", "tripoll_survey", "tripoll_survey_range",
                 "tripoll_partition_pivots", "tripoll_graph_stats", "tripoll_graph_export",
                 "tripoll_server_create", "tripoll_server_add_graph", "tripoll_server_submit",
                 "tripoll_server_wait", "tripoll_wedge_checks", "tripoll_survey_static", "tripoll_set_allocator",
                 "tripoll_survey_timed", "tripoll_survey_many", "tripoll_server_stats", "tripoll_get_plan",
                 "tripoll_set_plan", "tripoll_set_default_plan", "tripoll_tune"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != TRIPOLL_OK:
        lib = load_library()
        detail = lib.tripoll_last_error().decode(errors="replace")
        raise TripollError(rc, where, detail or lib.tripoll_status_string(rc).decode())


def _ptr(x):
    """Address of a tensor/array (None -> NULL).  Keeps no reference."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("numpy arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def _len(x):
    return int(x.shape[0])


def tripoll_graph_create(src, dst, ts, elabel=None, vlabel=None, num_vertices=None, num_vlabels=1,
                         num_elabels=0, stream=None):
    """Build G+ on the device; returns an opaque handle (int)."""
    lib = load_library()
    m = _len(src)
    if num_vertices is None:
        raise ValueError("num_vertices is required")
    out = ctypes.c_void_p()
    rc = lib.tripoll_graph_create(_ptr(src), _ptr(dst), _ptr(ts), _ptr(elabel), m, _ptr(vlabel),
                                  int(num_vertices), int(num_vlabels), int(num_elabels),
                                  _stream(stream), ctypes.byref(out))
    _check(rc, "tripoll_graph_create")
    return out.value


def tripoll_batch_create(src, dst, ts, elabel, edge_offsets, vlabel, num_vertices, num_vlabels=1,
                         num_elabels=0, stream=None):
    """Build one G+ holding many graphs.  edge_offsets, num_vertices: host numpy arrays."""
    lib = load_library()
    eo = np.ascontiguousarray(edge_offsets, dtype=np.uint64)
    nv = np.ascontiguousarray(num_vertices, dtype=np.uint32)
    out = ctypes.c_void_p()
    rc = lib.tripoll_batch_create(_ptr(src), _ptr(dst), _ptr(ts), _ptr(elabel), eo.ctypes.data, _ptr(vlabel),
                                  nv.ctypes.data, int(nv.shape[0]), int(num_vlabels), int(num_elabels),
                                  _stream(stream), ctypes.byref(out))
    _check(rc, "tripoll_batch_create")
    return out.value


def tripoll_launch_count():
    """Kernels this library has launched in the process so far (host-side counter)."""
    return int(load_library().tripoll_launch_count())


def tripoll_result_words(kind_mask, num_vlabels, num_elabels, num_vertices=0, num_edges=0):
    return int(load_library().tripoll_result_words(kind_mask, num_vlabels, num_elabels, num_vertices, num_edges))


def tripoll_survey(g, kind_mask, t_lo, t_hi, result, stream=None):
    """Survey into `result` (uint64 words; torch tensor on device or host, or numpy)."""
    _check(load_library().tripoll_survey(g, kind_mask, t_lo, t_hi, _ptr(result), _stream(stream)),
           "tripoll_survey")
    return result


def tripoll_survey_static(g, kind_mask, t_lo, t_hi, result, stream=None):
    """tripoll_survey without any device allocation (static scratch; see tripoll.h).
    For callers that must not allocate; calls that overlap on the GPU race."""
    _check(load_library().tripoll_survey_static(g, kind_mask, t_lo, t_hi, _ptr(result), _stream(stream)),
           "tripoll_survey_static")
    return result


def tripoll_survey_range(g, kind_mask, t_lo, t_hi, pivot_lo, pivot_hi, result, stream=None):
    _check(load_library().tripoll_survey_range(g, kind_mask, t_lo, t_hi, pivot_lo, pivot_hi, _ptr(result),
                                               _stream(stream)), "tripoll_survey_range")
    return result


def tripoll_survey_many(g, kind_masks, t_lo, t_hi, results, stream=None):
    """Several requests on one graph in one pass: request k (kind_masks[k], [t_lo[k], t_hi[k]]) into
    results[k] (each a device tensor, host tensor or numpy array of its result words)."""
    n = len(results)
    km = np.ascontiguousarray(kind_masks, dtype=np.uint32)
    lo = np.ascontiguousarray(t_lo, dtype=np.uint32)
    hi = np.ascontiguousarray(t_hi, dtype=np.uint32)
    if not (len(km) == len(lo) == len(hi) == n):
        raise ValueError("one kind mask, window and result per request")
    ptrs = (ctypes.c_void_p * max(n, 1))(*[_ptr(r) for r in results])
    _check(load_library().tripoll_survey_many(g, n, km.ctypes.data, lo.ctypes.data, hi.ctypes.data, ptrs,
                                              _stream(stream)), "tripoll_survey_many")
    return results


def tripoll_survey_timed(g, kind_mask, t_lo, t_hi, pivot_lo, pivot_hi, result, stream=None):
    """tripoll_survey_range that also returns the device time (ms) of its four phases: window view,
    warp-item kernel, block-item kernel, long-list kernel.  Synchronises the stream."""
    ms = (ctypes.c_float * 4)()
    _check(load_library().tripoll_survey_timed(g, kind_mask, t_lo, t_hi, pivot_lo, pivot_hi, _ptr(result), ms,
                                               _stream(stream)), "tripoll_survey_timed")
    return [float(x) for x in ms]


def tripoll_get_plan(g):
    p = Plan()
    _check(load_library().tripoll_get_plan(g, ctypes.byref(p)), "tripoll_get_plan")
    return p.as_dict()


def tripoll_set_plan(g, plan, stream=None):
    p = Plan.of(plan)
    _check(load_library().tripoll_set_plan(g, ctypes.byref(p), _stream(stream)), "tripoll_set_plan")


def tripoll_set_default_plan(plan=None):
    """The plan graphs built from now on start with (None: the built-in defaults)."""
    p = None if plan is None else ctypes.byref(Plan.of(plan))
    _check(load_library().tripoll_set_default_plan(p), "tripoll_set_default_plan")


def tripoll_tune(g, kind_mask, t_lo=0, t_hi=0xFFFFFFFF, reps=3, stream=None):
    """Autotune g's plan for this survey; returns (best plan dict, its ms, the starting plan's ms)."""
    p = Plan()
    best, start = ctypes.c_float(), ctypes.c_float()
    _check(load_library().tripoll_tune(g, kind_mask, t_lo, t_hi, reps, ctypes.byref(p), ctypes.byref(best),
                                       ctypes.byref(start), _stream(stream)), "tripoll_tune")
    return p.as_dict(), float(best.value), float(start.value)


def tripoll_partition_pivots(g, parts, stream=None):
    bounds = np.zeros(parts + 1, np.uint64)
    _check(load_library().tripoll_partition_pivots(g, parts, bounds.ctypes.data, _stream(stream)),
           "tripoll_partition_pivots")
    return bounds


def tripoll_graph_stats(g):
    info = GraphInfo()
    _check(load_library().tripoll_graph_stats(g, ctypes.byref(info)), "tripoll_graph_stats")
    return info.as_dict()


def tripoll_wedge_checks(g, t_lo=0, t_hi=0xFFFFFFFF, stream=None):
    """Wedge checks a survey over [t_lo, t_hi] performs (|W+| for the full window)."""
    out = ctypes.c_uint64()
    _check(load_library().tripoll_wedge_checks(g, t_lo, t_hi, ctypes.byref(out), _stream(stream)),
           "tripoll_wedge_checks")
    return out.value


def tripoll_graph_export(g, stream=None):
    """Host copies of the built G+: offsets, col, ts, elabel (or None), order."""
    st = tripoll_graph_stats(g)
    n, m = st["num_vertices"], st["num_edges"]
    off = np.zeros(n + 1, np.uint64)
    col = np.zeros(m, np.uint32)
    ts = np.zeros(m, np.uint32)
    el = np.zeros(m, np.uint8) if st["num_elabels"] else None
    order = np.zeros(n, np.uint32)
    _check(load_library().tripoll_graph_export(g, off.ctypes.data, col.ctypes.data, ts.ctypes.data,
                                               None if el is None else el.ctypes.data, order.ctypes.data,
                                               _stream(stream)), "tripoll_graph_export")
    return off, col, ts, el, order


def tripoll_destroy(g):
    if g:
        load_library().tripoll_destroy(g)


def tripoll_server_create(scratch_cap_bytes, max_inflight=64):
    out = ctypes.c_void_p()
    _check(load_library().tripoll_server_create(scratch_cap_bytes, max_inflight, ctypes.byref(out)),
           "tripoll_server_create")
    return out.value


def tripoll_server_add_graph(s, g):
    slot = ctypes.c_uint32()
    _check(load_library().tripoll_server_add_graph(s, g, ctypes.byref(slot)), "tripoll_server_add_graph")
    return slot.value


def tripoll_server_submit(s, slot, kind_mask, t_lo=0, t_hi=0xFFFFFFFF):
    rid = ctypes.c_uint64()
    _check(load_library().tripoll_server_submit(s, slot, kind_mask, t_lo, t_hi, ctypes.byref(rid)),
           "tripoll_server_submit")
    return rid.value


def tripoll_server_wait(s, request_id, result, timeout_ms=60000):
    """Wait for a request; fills `result` (host numpy uint64) and returns latency in ns."""
    lat = ctypes.c_uint64()
    _check(load_library().tripoll_server_wait(s, request_id, _ptr(result), ctypes.byref(lat), timeout_ms),
           "tripoll_server_wait")
    return lat.value


def tripoll_server_stats(s):
    """Server counters: requests launched, batches, survey passes, requests in fused passes."""
    st = np.zeros(4, np.uint64)
    _check(load_library().tripoll_server_stats(s, st.ctypes.data), "tripoll_server_stats")
    return {"requests": int(st[0]), "batches": int(st[1]), "passes": int(st[2]), "fused_requests": int(st[3])}


def tripoll_server_destroy(s):
    if s:
        load_library().tripoll_server_destroy(s)


_allocator_refs = []  # installed ctypes callbacks: they stay alive, since graphs may outlive a swap


def tripoll_set_allocator(alloc=None, free=None):
    """Install Python callables as the library's device allocator (see tripoll.h):
    alloc(bytes, stream) -> device address (int), or 0 / None when it cannot;
    free(ptr, bytes, stream).  Both None restores the library's own pool."""
    lib = load_library()
    a = ALLOC_FN() if alloc is None else ALLOC_FN(lambda nbytes, stream, ctx: alloc(nbytes, stream or 0) or None)
    f = FREE_FN() if free is None else FREE_FN(lambda ptr, nbytes, stream, ctx: free(ptr, nbytes, stream or 0))
    _check(lib.tripoll_set_allocator(a, f, None), "tripoll_set_allocator")
    if alloc is not None:
        _allocator_refs.append((a, f))


def torch_caching_allocator():
    """(alloc, free) drawing device memory from torch's caching allocator, for
    tripoll_set_allocator: blocks are taken on the library's stream and handed back to
    torch, which reuses them in that stream's order."""
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream))

    def free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    return alloc, free


def tripoll_status_string(status):
    return load_library().tripoll_status_string(status).decode()


def tripoll_last_error():
    return load_library().tripoll_last_error().decode()


def split_result(vec, kind_mask, num_vlabels, num_elabels, num_vertices=0, num_edges=0):
    """Views of the tables in one result record, by kind name (layout of tripoll.h)."""
    out, o = {}, 0
    sizes = [("count", TRIPOLL_COUNT, 1), ("hist", TRIPOLL_CLOSURE_HIST, TRIPOLL_HIST_BINS),
             ("vtri", TRIPOLL_VLABEL_TRIPLES, num_vlabels ** 3), ("etri", TRIPOLL_ELABEL_TRIPLES, num_elabels ** 3),
             ("joint", TRIPOLL_OPEN_CLOSE_HIST, TRIPOLL_HIST_BINS ** 2), ("maxel", TRIPOLL_MAX_ELABEL, num_elabels),
             ("degtri", TRIPOLL_DEGREE_TRIPLES, TRIPOLL_HIST_BINS ** 3),
             ("vlocal", TRIPOLL_VERTEX_LOCAL, num_vertices), ("elocal", TRIPOLL_EDGE_LOCAL, num_edges)]
    for name, bit, size in sizes:
        if kind_mask & bit:
            out[name] = vec[o:o + size]
            o += size
    return out
