"""Compressed-row graphs: dj_sssp on a graph kept without its n x n matrix gives the
oracle's dist and pred bit for bit, with the same fill rules (repeats keep their
smallest weight, self-loops dropped, undirected fills both directions)."""
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


def solve(dj, g, s, mode=0):
    import torch
    n = dj.dj_graph_get_info(g)["n"]
    dist = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    pred = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    dj.dj_sssp_ex(g, s, dist, pred, dj.make_solve_opts(mode=mode))
    dj.dj_sync()
    return dist.cpu().numpy(), pred.cpu().numpy()


def same(got, ref, what):
    assert np.array_equal(got[0], ref[0]), f"{what}: dist differs at {np.count_nonzero(got[0] != ref[0])} nodes"
    assert np.array_equal(got[1], ref[1]), f"{what}: pred differs at {np.count_nonzero(got[1] != ref[1])} nodes"


@pytest.mark.parametrize("mode", [1, 2], ids=["phase", "plain"])
def test_worked_matrices(dj, mode):
    gold = P.parse_golden("worked_4node.txt")
    e = gold["edges"]
    for kind, directed in (("undirected", False), ("directed", True)):
        G = dj.dj_load_edges_csr(4, e[:, 0], e[:, 1], e[:, 2], directed)
        assert dj.dj_graph_get_info(G)["format"] == dj.DJ_FORMAT_CSR
        for k, s, dist, pred in gold["expect"]:
            if k == kind:
                same(solve(dj, G, s, mode), (dist, pred), f"{kind} s={s}")
        G.free()


@pytest.mark.parametrize("n", [1, 2, 5, 97, 1000, 4099, 5003])
def test_ragged_ties_repeats_zero_weights(dj, orc, n):
    rng = np.random.default_rng(n)
    for directed in (False, True):
        for wlo in (0, 1):
            m = int(min(n * (n - 1) // 2, 6 * n)) + 5
            e = graphgen.random_edges(n, m, wlo, 3, seed=3000 + n + int(directed) + 7 * wlo, directed=directed)
            # plant repeats with larger weights and self-loops: both must be ignored
            src = np.concatenate([e.src, e.src[:5], np.arange(min(n, 3), dtype=np.int32)])
            dst = np.concatenate([e.dst, e.dst[:5], np.arange(min(n, 3), dtype=np.int32)])
            w = np.concatenate([e.w, e.w[:5] + 7, np.zeros(min(n, 3), dtype=np.int32)])
            G = dj.dj_load_edges_csr(n, src, dst, w, directed)
            W = orc.build_matrix(n, src, dst, w, directed)
            for s in sorted({0, n - 1, int(rng.integers(0, n))}):
                ref = orc.dijkstra(W, s)
                for mode in (1, 2) if n <= 1000 else (1,):
                    same(solve(dj, G, s, mode), ref, f"n={n} directed={directed} wlo={wlo} s={s} mode={mode}")
            G.free()


def test_sparse_directed_n32768_full(dj, orc):
    spec = graphgen.WORKLOADS["sparse_directed_n32768_deg8"]
    e = graphgen.make_graph(spec)
    s = graphgen.workload_source(spec)
    Gc = dj.dj_load_edges_csr(e.n, e.src, e.dst, e.w, e.directed)
    info = dj.dj_graph_get_info(Gc)
    assert info["bytes"] < 8 * e.m + 16 * e.n + 64  # 8 bytes per edge, no matrix
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    ref = orc.dijkstra(W, s)
    same(solve(dj, Gc, s), ref, "n=32768 directed, compressed rows")
    Gd = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
    same(solve(dj, Gd, 12345), solve(dj, Gc, 12345), "dense and compressed rows agree")


def test_dense_only_calls_reject_compressed_rows(dj):
    import torch
    e = graphgen.random_edges(300, 1500, 1, 9, seed=5, directed=False)
    G = dj.dj_load_edges_csr(300, e.src, e.dst, e.w, False)
    d = torch.empty(300, dtype=torch.int32, device="cuda")
    p = torch.empty_like(d)
    for call in (lambda: dj.dj_graph_download(G), lambda: dj.dj_sssp_lc(G, 0, d, p),
                 lambda: dj.dj_sssp_noalloc(G, 0, d, p), lambda: dj.dj_sssp_batch([G], [0], [d], [p])):
        with pytest.raises(dj.DjError) as ei:
            call()
        assert ei.value.status == dj.DJ_EUNSUPPORTED
    G.free()
