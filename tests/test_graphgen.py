"""The shared input generator: deterministic, shaped as the workloads state, no method arithmetic."""
import numpy as np

import graphgen


def test_bernoulli_deterministic_and_shaped():
    a = graphgen.bernoulli(600, 0.1, 1, 100, 11)
    b = graphgen.bernoulli(600, 0.1, 1, 100, 11)
    c = graphgen.bernoulli(600, 0.1, 1, 100, 12)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.w, b.w)
    assert not (a.m == c.m and np.array_equal(a.src, c.src))
    assert (a.src < a.dst).all()
    assert a.w.min() >= 1 and a.w.max() <= 100
    pairs = 600 * 599 // 2
    assert abs(a.m - 0.1 * pairs) < 5 * np.sqrt(pairs * 0.1 * 0.9)
    # pairs listed once, in row-major order
    key = a.src.astype(np.int64) * 600 + a.dst
    assert (np.diff(key) > 0).all()


def test_bernoulli_extremes():
    assert graphgen.bernoulli(50, 0.0, 1, 5, 1).m == 0
    full = graphgen.bernoulli(50, 1.0, 1, 5, 1)
    assert full.m == 50 * 49 // 2


def test_outdeg_shape():
    e = graphgen.outdeg(2000, 8, 1, 10000, 3)
    assert e.directed
    assert (e.src != e.dst).all()
    assert e.m <= 16000 and e.m > 15900
    assert e.w.min() >= 1 and e.w.max() <= 10000
    counts = np.bincount(e.src, minlength=2000)
    assert counts.max() <= 8


def test_sources_distinct():
    s = graphgen.sources(8192, 256, 4)
    assert len(set(s.tolist())) == 256 and s.min() >= 0 and s.max() < 8192
    assert np.array_equal(s, graphgen.sources(8192, 256, 4))
    assert sorted(graphgen.sources(5, 5, 9).tolist()) == [0, 1, 2, 3, 4]


def test_bounded_is_uniform():
    x = graphgen.bounded(1, 0, 200000, 10)
    h = np.bincount(x, minlength=10)
    assert h.min() > 19000 and h.max() < 21000


def test_serving_trace_shape():
    tr = graphgen.serving_trace(64, 10000, 500.0, 5)
    assert tr.graph_n.min() >= 512 and tr.graph_n.max() <= 16384
    assert (tr.graph_p >= 0.01).all() and (tr.graph_p <= 0.5).all()
    assert (tr.req_source < tr.graph_n[tr.req_graph]).all()
    assert (np.diff(tr.req_arrival_s) > 0).all()
    mean_gap = tr.req_arrival_s[-1] / 10000
    assert abs(mean_gap - 1 / 500.0) < 0.1 / 500.0
