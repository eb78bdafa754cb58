"""The seeded input generators: published SplitMix64 outputs, determinism, and
the shape of the workloads (sizes and value ranges)."""
import numpy as np

import synth


def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 from state 1234567 (Steele, Lea & Flood 2014,
    # as printed by the reference implementations of the generator)
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert [synth.splitmix64_at(1234567, i) for i in range(5)] == want


def test_generators_are_deterministic():
    a = synth.rmat_graph(10, 16, 3, ts_bits=20, num_vlabels=4, num_elabels=5)
    b = synth.rmat_graph(10, 16, 3, ts_bits=20, num_vlabels=4, num_elabels=5)
    for k in ("src", "dst", "ts", "vlabel", "elabel"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    c = synth.rmat_graph(10, 16, 4, ts_bits=20, num_vlabels=4, num_elabels=5)
    assert not np.array_equal(a.src, c.src)


def test_rmat_shape():
    g = synth.rmat12()
    assert g.n == 4096 and g.m_in == 65536
    assert g.src.max() < g.n and g.dst.max() < g.n
    assert g.ts.max() < 2 ** 24 and set(np.unique(g.vlabel)) <= {0, 1, 2, 3}
    # quadrant a = 0.57 at the top level: about 57% of edges have both top bits 0
    top = ((g.src >> 11) == 0) & ((g.dst >> 11) == 0)
    assert 0.55 < top.mean() < 0.59


def test_zipf_and_uniform_labels():
    z = synth.zipf_labels(1, 4, 200000, 8, 1.2)
    p = np.bincount(z, minlength=8) / len(z)
    w = np.arange(1, 9) ** -1.2
    assert np.allclose(p, w / w.sum(), atol=0.005)
    u = synth.uniform_labels(1, 3, 200000, 16)
    assert np.allclose(np.bincount(u, minlength=16) / len(u), 1 / 16, atol=0.004)


def test_batched_family_sizes():
    sizes = [synth.small_chung_lu_params(g) for g in range(500)]
    ns = np.array([s[0] for s in sizes])
    dbar = np.array([s[1] for s in sizes])
    assert ns.min() >= 32 and ns.max() <= 8192
    assert dbar.min() >= 4 and dbar.max() <= 64
    # log-uniform: about half the graphs below the geometric midpoint 512
    assert 0.4 < (ns < 512).mean() < 0.6


def test_chung_lu_power_law_head():
    src, dst = synth.chung_lu_edges(7, 10000, 2.1, 200000)
    deg = np.bincount(np.concatenate([src, dst]), minlength=10000)
    # expected endpoint share of vertex 0 is w_0 / sum(w), w_i = (i+1)^(-1/1.1)
    w = np.arange(1, 10001, dtype=np.float64) ** (-1 / 1.1)
    share = deg[0] / deg.sum()
    assert abs(share - w[0] / w.sum()) < 0.01
