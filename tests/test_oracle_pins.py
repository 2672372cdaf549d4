"""Pins for the CPU oracle: each check below compares it with something other than itself.

The paper's worked matrices (Section III-A) and padded example (Section III-B)
come from tests/golden; the remaining references are brute force (Floyd-Warshall,
Bellman-Ford), scipy's shortest-path routine, BFS for unit weights, the
predecessor closed form and the optimality invariants (see tests/_pins.py).
"""
import numpy as np
import pytest

import _pins as P


def test_worked_matrices_fill_from_edges(orc):
    g = P.parse_golden("worked_4node.txt")
    e = g["edges"]
    assert np.array_equal(orc.build_matrix(4, e[:, 0], e[:, 1], e[:, 2], False), g["matrices"]["undirected"])
    assert np.array_equal(orc.build_matrix(4, e[:, 0], e[:, 1], e[:, 2], True), g["matrices"]["directed"])


@pytest.mark.parametrize("fixture", ["worked_4node.txt", "padded_6node.txt"])
def test_golden_solves(orc, fixture):
    g = P.parse_golden(fixture)
    assert g["expect"]
    for kind, s, dist, pred in g["expect"]:
        G = g["matrices"][kind]
        d, p = orc.dijkstra(G, s)
        assert np.array_equal(d, dist), (kind, s, d)
        assert np.array_equal(p, pred), (kind, s, p)
        # the hand-derived rows themselves agree with brute force
        assert np.array_equal(P.floyd_warshall(G)[s], dist.astype(np.int64))


def test_worked_example_distances_from_node_0(orc):
    g = P.parse_golden("worked_4node.txt")
    d, _ = orc.dijkstra(g["matrices"]["undirected"], 0)
    assert d.tolist() == [0, 2, 3, 5]


def test_full_pin_suite(orc):
    fails = P.run_pin_suite(orc.build_matrix, orc.dijkstra)
    assert fails == []


def test_many_matches_single(orc):
    rng = np.random.default_rng(7)
    G = P.random_matrix(rng, 50, 0.2, tuple(range(1, 30)), True)
    srcs = np.array([0, 7, 49, 7], dtype=np.int32)
    D, Pr = orc.dijkstra_many(G, srcs)
    for i, s in enumerate(srcs):
        d, p = orc.dijkstra(G, int(s))
        assert np.array_equal(D[i], d) and np.array_equal(Pr[i], p)


def test_threaded_many_matches_single(orc):
    """The threaded driver only schedules independent serial solves: every row equals dijkstra()."""
    rng = np.random.default_rng(8)
    G = P.random_matrix(rng, 70, 0.15, tuple(range(1, 9)), False)
    srcs = np.array([3, 0, 69, 3, 41, 12, 5], dtype=np.int32)
    for threads in (1, 3, 16):
        D, Pr, used = orc.dijkstra_many_threads(G, srcs, threads)
        assert 1 <= used <= min(threads, len(srcs))
        for i, s in enumerate(srcs):
            d, p = orc.dijkstra(G, int(s))
            assert np.array_equal(D[i], d) and np.array_equal(Pr[i], p)


def test_fill_rejects_bad_edges(orc):
    one = np.array([0], dtype=np.int32)
    with pytest.raises(ValueError):
        orc.build_matrix(2, one, np.array([2], dtype=np.int32), one, False)
    with pytest.raises(ValueError):
        orc.build_matrix(2, one, one + 1, np.array([-1], dtype=np.int32), False)
    with pytest.raises(ValueError):
        orc.build_matrix(2, one, one + 1, np.array([P.INF], dtype=np.int32), False)


def test_generated_workload_invariants(orc):
    """A synthetic dense workload at the smallest bench shape: invariants and the pred closed form."""
    import graphgen
    spec = graphgen.WORKLOADS["dense_n1024_p0.1"]
    e = graphgen.make_graph(spec)
    G = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    s = graphgen.workload_source(spec)
    d, p = orc.dijkstra(G, s)
    assert P.check_invariants(G, s, d, p) == []
    assert np.array_equal(p, P.pred_closed_form(G, s, d))
    assert np.array_equal(d.astype(np.int64), P.scipy_distances(G, s))
