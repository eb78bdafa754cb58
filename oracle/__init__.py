"""TEST INFRASTRUCTURE: Python handle on the plain CPU oracle (``oracle.c``).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  The survey library never does, and the oracle never
imports the library: they share no code.

``survey`` returns a dict of numpy uint64 arrays (``count``, ``hist`` [33],
``vtri`` [Lv^3], ``etri`` [Le^3], and on request ``joint`` [33*33], ``maxel``
[Le], ``degtri`` [33^3], ``vlocal`` [n], ``elocal`` [m], the unique edges in
ascending (min id, max id) order) plus the graph statistics of G+.  What
each one means is stated in ``oracle.c`` with the paper passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

HIST_BINS = 33
_lib = None


class _Out(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("count", "hist", "vtri", "etri", "joint", "maxel", "degtri", "vlocal", "elocal")]


class _Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("m", "wedges", "dplus_max", "dmax")]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11 + pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-pthread", _SRC,
                               "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    """The compiled oracle.  ``ORACLE_LIBRARY`` names another build of ``oracle.c`` to load
    instead: the mutation tests point it at copies with a planted mistake."""
    global _lib
    if _lib is None:
        path = os.environ.get("ORACLE_LIBRARY") or build()
        lib = ctypes.CDLL(path)
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        lib.oracle_survey.argtypes = [vp, vp, vp, vp, u64, vp, u32, u32, u32, u32, u32, i32, u32,
                                      u32, i32, ctypes.POINTER(_Out), ctypes.POINTER(_Stats)]
        lib.oracle_survey.restype = i32
        _lib = lib
    return _lib


def _arr(a, dtype):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=dtype)


def survey(src, dst, ts, elabel, vlabel, n, num_vlabels=1, num_elabels=1, t_lo=0,
           t_hi=0xFFFFFFFF, order_mode=0, pivot_range=None, threads=1,
           extras=("joint", "maxel", "degtri", "vlocal")):
    """Run the oracle survey; returns dict of uint64 arrays and G+ statistics."""
    lib = _load()
    src = _arr(src, np.uint32)
    dst = _arr(dst, np.uint32)
    ts = _arr(ts, np.uint32)
    el = _arr(elabel, np.uint8)
    vl = _arr(vlabel, np.uint8)
    m_in = int(src.shape[0])
    Lv, Le = int(num_vlabels), int(num_elabels)
    res = {
        "count": np.zeros(1, np.uint64),
        "hist": np.zeros(HIST_BINS, np.uint64),
        "vtri": np.zeros(Lv ** 3, np.uint64),
        "etri": np.zeros(Le ** 3, np.uint64),
    }
    if "joint" in extras:
        res["joint"] = np.zeros(HIST_BINS * HIST_BINS, np.uint64)
    if "maxel" in extras:
        res["maxel"] = np.zeros(Le, np.uint64)
    if "degtri" in extras:
        res["degtri"] = np.zeros(HIST_BINS ** 3, np.uint64)
    if "vlocal" in extras:
        res["vlocal"] = np.zeros(max(n, 1), np.uint64)
    if "elocal" in extras:  # the unique edge count is at most m_in; trimmed below
        res["elocal"] = np.zeros(max(m_in, 1), np.uint64)
    out = _Out(*[res[k].ctypes.data if k in res else None for k in
                 ("count", "hist", "vtri", "etri", "joint", "maxel", "degtri", "vlocal", "elocal")])
    st = _Stats()
    lo, hi = (0, n) if pivot_range is None else pivot_range
    rc = lib.oracle_survey(
        src.ctypes.data, dst.ctypes.data, ts.ctypes.data, None if el is None else el.ctypes.data,
        m_in, None if vl is None else vl.ctypes.data, n, Lv, Le, t_lo, t_hi, order_mode, lo, hi,
        threads, ctypes.byref(out), ctypes.byref(st))
    if rc == -1:
        raise ValueError("oracle_survey: invalid arguments")
    if rc != 0:
        raise MemoryError("oracle_survey: out of host memory")
    if "vlocal" in res:
        res["vlocal"] = res["vlocal"][:n]
    if "elocal" in res:
        res["elocal"] = res["elocal"][:int(st.m)]
    res["stats"] = dict(m=int(st.m), wedges=int(st.wedges), dplus_max=int(st.dplus_max),
                        dmax=int(st.dmax))
    return res


def survey_graph(g, threads=1, **kw):
    """Oracle survey of a ``synth.Graph`` over its window."""
    lo, hi = g.window
    return survey(g.src, g.dst, g.ts, g.elabel, g.vlabel, g.n, g.num_vlabels, g.num_elabels,
                  t_lo=lo, t_hi=hi, threads=threads, **kw)


def result_vector(res, kinds, num_vlabels, num_elabels):
    """The oracle's survey laid out like the library's result buffer:
    [count][hist 33][vtri Lv^3][etri Le^3], requested kinds only, in that order."""
    parts = []
    if kinds & 1:
        parts.append(res["count"])
    if kinds & 2:
        parts.append(res["hist"])
    if kinds & 4:
        parts.append(res["vtri"])
    if kinds & 8:
        parts.append(res["etri"])
    return np.concatenate(parts) if parts else np.zeros(0, np.uint64)
