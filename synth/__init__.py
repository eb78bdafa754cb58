"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only shapes inputs: decorated temporal graphs in the form of edge
arrays (src, dst, ts, elabel) and a vertex-label array.  It holds none of the
survey's arithmetic (no dedup, orientation, intersection or fold), so the CPU
oracle and the CUDA path can both read its arrays without sharing any code.

The generators live in ``synth.c`` (counter-based SplitMix64 draws, R-MAT and
Chung-Lu edge samplers) and are compiled on first use with gcc.

Workload recipes (sizes, distributions) follow the paper's inputs: R-MAT graphs
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05) for the weak-scaling family (Sec. 5.2,
Sec. 5.5) and Chung-Lu power-law graphs standing in for the scale-free real
graphs of Table 2, with uint32 timestamps and uint8 labels as edge/vertex
metadata (Sec. 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")

# substream ids
STREAM_EDGES = 1
STREAM_TS = 2
STREAM_VLABEL = 3
STREAM_ELABEL = 4
STREAM_PARAMS = 6

# survey kind bits (the same values the C-ABI uses; plain enumeration, no arithmetic)
COUNT = 1
CLOSURE_HIST = 2
VLABEL_TRIPLES = 4
ELABEL_TRIPLES = 8

FULL_WINDOW = (0, 0xFFFFFFFF)

_lib = None


def build(force: bool = False) -> str:
    """Compile libsynth.so with gcc (OpenMP); returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i32, u32, dbl, vp = (ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32,
                                  ctypes.c_double, ctypes.c_void_p)
        lib.synth_stream_key.argtypes = [u64, u64]
        lib.synth_stream_key.restype = u64
        lib.synth_splitmix64_at.argtypes = [u64, u64]
        lib.synth_splitmix64_at.restype = u64
        lib.synth_draw.argtypes = [u64, u64, u64]
        lib.synth_draw.restype = u64
        lib.synth_rmat.argtypes = [u64, u64, i32, u64, dbl, dbl, dbl, vp, vp]
        lib.synth_bits_u32.argtypes = [u64, u64, u64, i32, vp]
        lib.synth_scaled_u32.argtypes = [u64, u64, u64, dbl, vp]
        lib.synth_uniform_u8.argtypes = [u64, u64, u64, u32, vp]
        lib.synth_zipf_u8.argtypes = [u64, u64, u64, u32, dbl, vp]
        lib.synth_chung_lu.argtypes = [u64, u64, u32, dbl, u64, vp, vp]
        lib.synth_chung_lu.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def splitmix64_at(state: int, i: int) -> int:
    return int(_load().synth_splitmix64_at(state, i))


def draw(seed: int, stream: int, i: int) -> int:
    return int(_load().synth_draw(seed, stream, i))


def rmat_edges(seed: int, scale: int, m: int, a=0.57, b=0.19, c=0.19):
    src = np.empty(m, np.uint32)
    dst = np.empty(m, np.uint32)
    _load().synth_rmat(seed, STREAM_EDGES, scale, m, a, b, c, _ptr(src), _ptr(dst))
    return src, dst


def chung_lu_edges(seed: int, n: int, gamma: float, m: int):
    src = np.empty(m, np.uint32)
    dst = np.empty(m, np.uint32)
    if _load().synth_chung_lu(seed, STREAM_EDGES, n, gamma, m, _ptr(src), _ptr(dst)) != 0:
        raise MemoryError("synth_chung_lu: out of host memory")
    return src, dst


def uniform_bits(seed: int, stream: int, count: int, bits: int) -> np.ndarray:
    out = np.empty(count, np.uint32)
    _load().synth_bits_u32(seed, stream, count, bits, _ptr(out))
    return out


def scaled_times(seed: int, stream: int, count: int, horizon: float) -> np.ndarray:
    out = np.empty(count, np.uint32)
    _load().synth_scaled_u32(seed, stream, count, horizon, _ptr(out))
    return out


def uniform_labels(seed: int, stream: int, count: int, L: int) -> np.ndarray:
    out = np.empty(count, np.uint8)
    _load().synth_uniform_u8(seed, stream, count, L, _ptr(out))
    return out


def zipf_labels(seed: int, stream: int, count: int, K: int, s: float) -> np.ndarray:
    out = np.empty(count, np.uint8)
    _load().synth_zipf_u8(seed, stream, count, K, s, _ptr(out))
    return out


@dataclass
class Graph:
    """A decorated temporal graph as raw input arrays (before any dedup)."""
    name: str
    n: int
    src: np.ndarray
    dst: np.ndarray
    ts: np.ndarray
    vlabel: np.ndarray | None
    elabel: np.ndarray | None
    num_vlabels: int
    num_elabels: int
    kinds: int
    window: tuple = FULL_WINDOW
    meta: dict = field(default_factory=dict)

    @property
    def m_in(self) -> int:
        return int(self.src.shape[0])


def rmat_graph(scale: int, edge_factor: int = 16, seed: int = 1, ts_bits: int = 24,
               num_vlabels: int = 4, num_elabels: int = 0, elabel_zipf: float = 1.2,
               kinds: int = COUNT | CLOSURE_HIST | VLABEL_TRIPLES, window=FULL_WINDOW,
               name: str | None = None) -> Graph:
    n = 1 << scale
    m = edge_factor * n
    src, dst = rmat_edges(seed, scale, m)
    ts = uniform_bits(seed, STREAM_TS, m, ts_bits)
    vl = uniform_labels(seed, STREAM_VLABEL, n, num_vlabels) if num_vlabels > 1 else None
    el = zipf_labels(seed, STREAM_ELABEL, m, num_elabels, elabel_zipf) if num_elabels > 1 else None
    return Graph(name or f"rmat{scale}", n, src, dst, ts, vl, el,
                 num_vlabels if vl is not None else 1, num_elabels if el is not None else 1,
                 kinds, tuple(window), dict(scale=scale, edge_factor=edge_factor, seed=seed))


def small_chung_lu_params(g: int):
    """Per-graph size of the batched family: n log-uniform in [32, 8192],
    mean degree uniform in [4, 64], number of sampled pairs round(n * dbar / 2)."""
    key_u = draw(g, STREAM_PARAMS, 0)
    key_d = draw(g, STREAM_PARAMS, 1)
    u = (key_u >> 11) * 2.0 ** -53
    ud = (key_d >> 11) * 2.0 ** -53
    n = int(round(32.0 * 256.0 ** u))
    dbar = 4.0 + 60.0 * ud
    m = int(round(n * dbar / 2.0))
    return n, dbar, m


def chung_lu_graph(seed: int, n: int, gamma: float, m_samples: int, ts=None, vlabel=None,
                   elabel=None, num_vlabels=1, num_elabels=1, kinds=COUNT | CLOSURE_HIST,
                   window=FULL_WINDOW, name: str | None = None) -> Graph:
    src, dst = chung_lu_edges(seed, n, gamma, m_samples)
    return Graph(name or f"chunglu{n}", n, src, dst, ts, vlabel, elabel, num_vlabels, num_elabels,
                 kinds, tuple(window), dict(seed=seed, gamma=gamma, m_samples=m_samples))


def batched_graph(g: int, ts_bits: int = 20, num_vlabels: int = 4) -> Graph:
    """Graph g of the batched family: Chung-Lu, exponent 2.5, timestamps uniform in
    [0, 2^20), vertex labels uniform in {0..3}; survey = count + closure histogram."""
    n, dbar, m = small_chung_lu_params(g)
    ts = uniform_bits(g, STREAM_TS, m, ts_bits)
    vl = uniform_labels(g, STREAM_VLABEL, n, num_vlabels)
    return chung_lu_graph(g, n, 2.5, m, ts=ts, vlabel=vl, num_vlabels=num_vlabels,
                          kinds=COUNT | CLOSURE_HIST, name=f"cl_batch{g}")


# -- the five workloads ----------------------------------------------------------------------

def rmat12() -> Graph:
    """R-MAT scale 12, edge factor 16, seed 1; ts uniform [0, 2^24); vertex labels
    uniform {0..3}; survey = count + closure histogram + vertex-label triples."""
    return rmat_graph(12, 16, 1, ts_bits=24, num_vlabels=4, num_elabels=0,
                      kinds=COUNT | CLOSURE_HIST | VLABEL_TRIPLES, name="rmat12")


RMAT24_WINDOW = (1 << 28, 3 * (1 << 28) - 1)


def rmat(scale: int, seed: int = 1) -> Graph:
    """R-MAT at `scale` with the scale-24 recipe: ts uniform [0, 2^30), vertex labels
    uniform {0..15}, edge types Zipf(1.2) over {0..7}; survey = count + closure histogram
    + edge-type triples inside the window covering the middle half of time."""
    return rmat_graph(scale, 16, seed, ts_bits=30, num_vlabels=16, num_elabels=8,
                      kinds=COUNT | CLOSURE_HIST | ELABEL_TRIPLES, window=RMAT24_WINDOW,
                      name=f"rmat{scale}")


def rmat24() -> Graph:
    return rmat(24, 1)


def serving_graph(i: int) -> Graph:
    """Resident graph i of the serving mix: R-MAT scales 16,18,20,22,24,26,16,18,
    seeds 1..8, ts uniform [0, 2^24), vertex labels uniform {0..15}, edge types
    Zipf(1.2) over {0..7}."""
    scales = [16, 18, 20, 22, 24, 26, 16, 18]
    return rmat_graph(scales[i], 16, i + 1, ts_bits=24, num_vlabels=16, num_elabels=8,
                      kinds=COUNT | CLOSURE_HIST | VLABEL_TRIPLES | ELABEL_TRIPLES,
                      name=f"serve{i}_rmat{scales[i]}")


def chung_lu_50m(m_samples: int = 1_200_000_000, n: int = 50_000_000) -> Graph:
    """Chung-Lu exponent 2.1 at 50M vertices; ts = Poisson arrivals over 3.15e8 s;
    vertex labels Zipf(1.1) over {0..63}; edge labels uniform {0..7}; full survey."""
    seed = 3
    src, dst = chung_lu_edges(seed, n, 2.1, m_samples)
    ts = scaled_times(seed, STREAM_TS, m_samples, 3.15e8)
    vl = zipf_labels(seed, STREAM_VLABEL, n, 64, 1.1)
    el = uniform_labels(seed, STREAM_ELABEL, m_samples, 8)
    return Graph("chunglu50m", n, src, dst, ts, vl, el, 64, 8,
                 COUNT | CLOSURE_HIST | VLABEL_TRIPLES | ELABEL_TRIPLES, FULL_WINDOW,
                 dict(seed=seed, gamma=2.1, m_samples=m_samples))


def tiny_random_graph(seed: int, n: int, m: int, ts_bits: int = 8, num_vlabels: int = 3,
                      num_elabels: int = 3, kinds: int = 15, window=FULL_WINDOW) -> Graph:
    """Uniform random multigraph on n vertices (loops and repeats included): test input."""
    src = uniform_bits(seed, 11, m, 32) % np.uint32(n) if n > 0 else np.zeros(m, np.uint32)
    dst = uniform_bits(seed, 12, m, 32) % np.uint32(n) if n > 0 else np.zeros(m, np.uint32)
    ts = uniform_bits(seed, STREAM_TS, m, ts_bits)
    vl = uniform_labels(seed, STREAM_VLABEL, n, num_vlabels) if num_vlabels > 1 else None
    el = uniform_labels(seed, STREAM_ELABEL, m, num_elabels) if num_elabels > 1 else None
    return Graph(f"tiny{seed}", n, src.astype(np.uint32), dst.astype(np.uint32), ts, vl, el,
                 num_vlabels if vl is not None else 1, num_elabels if el is not None else 1,
                 kinds, tuple(window))
