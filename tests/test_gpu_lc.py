"""Label-correcting solve (the paper's CUDA variant, Algorithms 3 and 4): dist bit-exact
against the CPU oracle, pred a shortest-path tree.

The paper's variant is a Bellman-Ford fixed point; its dist are the exact shortest
distances, its pred is any tree of shortest paths.  So dist is compared element by
element with Algorithm 1's, and pred is checked against the invariants of a
shortest-path tree (dist[pred[v]] + G[pred[v]][v] == dist[v], no improvable edge,
-1 at the source and the unreachable nodes) computed from the oracle's matrix.
"""
import numpy as np
import pytest

import _pins as P
import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dj():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_03667_gb300 import dj as _dj
    torch.cuda.set_device(0)
    return _dj


def solve_lc(dj, g, s):
    import torch
    n = dj.dj_graph_get_info(g)["n"]
    dist = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    pred = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    dj.dj_sssp_lc(g, s, dist, pred)
    dj.dj_sync()
    return dist.cpu().numpy(), pred.cpu().numpy()


def check(W, s, got, ref, what):
    d, p = got
    assert np.array_equal(d, ref[0]), f"{what}: dist differs at {np.count_nonzero(d != ref[0])} nodes"
    errs = P.check_invariants(W, s, d, p)
    assert errs == [], f"{what}: {errs}"
    assert (p[d == P.INF] == -1).all(), f"{what}: unreachable node with a pred"


def test_worked_matrices(dj):
    gold = P.parse_golden("worked_4node.txt")
    e = gold["edges"]
    for kind, directed in (("undirected", False), ("directed", True)):
        G = dj.dj_load_edges(4, e[:, 0], e[:, 1], e[:, 2], directed)
        W = gold["matrices"][kind]
        for k, s, dist, pred in gold["expect"]:
            if k == kind:
                check(W, s, solve_lc(dj, G, s), (dist, pred), f"{kind} s={s}")
        G.free()


@pytest.mark.parametrize("n", [1, 2, 5, 97, 1000, 4099, 5003])
def test_ragged_tie_heavy_and_zero_weights(dj, orc, n):
    for directed in (False, True):
        for wlo in (0, 1):
            m = int(min(n * (n - 1) // 2, 6 * n))
            e = graphgen.random_edges(n, m, wlo, 3, seed=2000 + n + int(directed) + 7 * wlo, directed=directed)
            G = dj.dj_load_edges(n, e.src, e.dst, e.w, directed)
            W = orc.build_matrix(n, e.src, e.dst, e.w, directed)
            for s in sorted({0, n - 1, n // 2}):
                check(W, s, solve_lc(dj, G, s), orc.dijkstra(W, s), f"n={n} directed={directed} wlo={wlo} s={s}")
            G.free()


def test_dense_n16384_and_sweeps(dj, orc):
    spec = graphgen.WORKLOADS["dense_n16384_p0.5"]
    e = graphgen.make_graph(spec)
    s = graphgen.workload_source(spec)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    check(W, s, solve_lc(dj, G, s), orc.dijkstra(W, s), "n=16384 p=0.5")
    assert 1 < dj.dj_last_phases() < e.n


def test_sparse_directed_n32768(dj, orc):
    spec = graphgen.WORKLOADS["sparse_directed_n32768_deg8"]
    e = graphgen.make_graph(spec)
    s = graphgen.workload_source(spec)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    check(W, s, solve_lc(dj, G, s), orc.dijkstra(W, s), "n=32768 directed")
