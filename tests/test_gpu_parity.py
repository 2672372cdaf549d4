"""GPU parity: dist and pred from the CUDA path equal the CPU oracle bit for bit.

All arithmetic is int32, so the tolerance is zero: every element must match.
Inputs are the paper's worked matrices and padded example, seeded synthetic
graphs at ragged sizes (spanning several CTA slices and a partial last tile),
tie-heavy and zero-weight graphs, weights at the int32 overflow limit, and the
full-size dense and sparse workloads.  Every call goes through the C ABI.
"""
import numpy as np
import pytest

import _pins as P
import graphgen

pytestmark = pytest.mark.gpu

ENGINES = [("grid", 1), ("cluster", 2)]
MODES = [("phase", 1), ("plain", 2)]


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


def solve(dj, g, s, engine=0, mode=0, cluster_size=0, live=0, rowsplit=0, rowpush=0, settle=0):
    import torch
    n = dj.dj_graph_get_info(g)["n"]
    dist = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    pred = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    dj.dj_sssp_ex(g, s, dist, pred, dj.make_solve_opts(mode=mode, engine=engine, cluster_size=cluster_size,
                                                       live=live, rowsplit=rowsplit, rowpush=rowpush,
                                                       settle=settle))
    dj.dj_sync()
    return dist.cpu().numpy(), pred.cpu().numpy()


def assert_same(got, ref, what=""):
    d, p = got
    dr, pr = ref
    if not np.array_equal(d, dr):
        bad = np.nonzero(d != dr)[0]
        raise AssertionError(f"{what}: dist differs at {bad.size} nodes, first {bad[:5]}: {d[bad[:5]]} vs {dr[bad[:5]]}")
    if not np.array_equal(p, pr):
        bad = np.nonzero(p != pr)[0]
        raise AssertionError(f"{what}: pred differs at {bad.size} nodes, first {bad[:5]}: {p[bad[:5]]} vs {pr[bad[:5]]}")


@pytest.mark.parametrize("engine", [e for _, e in ENGINES], ids=[n for n, _ in ENGINES])
@pytest.mark.parametrize("mode", [m for _, m in MODES], ids=[n for n, _ in MODES])
def test_worked_matrices(dj, engine, mode):
    g = P.parse_golden("worked_4node.txt")
    e = g["edges"]
    for kind, directed in (("undirected", False), ("directed", True)):
        G = dj.dj_load_edges(4, e[:, 0], e[:, 1], e[:, 2], directed)
        assert np.array_equal(dj.dj_graph_download(G), g["matrices"][kind])
        for k, s, dist, pred in g["expect"]:
            if k == kind:
                assert_same(solve(dj, G, s, engine, mode), (dist, pred), f"{kind} s={s}")
        G.free()


@pytest.mark.parametrize("engine", [e for _, e in ENGINES], ids=[n for n, _ in ENGINES])
def test_padded_example_dense_load(dj, engine):
    g = P.parse_golden("padded_6node.txt")
    G = dj.dj_load_dense(g["matrices"]["padded"])
    for _, s, dist, pred in g["expect"]:
        assert_same(solve(dj, G, s, engine), (dist, pred), f"padded s={s}")


@pytest.mark.parametrize("engine", [e for _, e in ENGINES], ids=[n for n, _ in ENGINES])
@pytest.mark.parametrize("mode", [m for _, m in MODES], ids=[n for n, _ in MODES])
def test_dense_n1024(dj, orc, engine, mode):
    spec = graphgen.WORKLOADS["dense_n1024_p0.1"]
    e = graphgen.make_graph(spec)
    s = graphgen.workload_source(spec)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    assert np.array_equal(dj.dj_graph_download(G), W)
    ref = orc.dijkstra(W, s)
    assert_same(solve(dj, G, s, engine, mode), ref, "n=1024")
    for s2 in (1, 511, 1023):
        assert_same(solve(dj, G, s2, engine, mode), orc.dijkstra(W, s2), f"n=1024 s={s2}")


RAGGED = [1, 2, 3, 5, 31, 33, 64, 97, 255, 1000, 1025, 2047, 4099, 5003]


@pytest.mark.parametrize("n", RAGGED)
def test_ragged_sizes_ties_and_unreachable(dj, orc, n):
    rng = np.random.default_rng(n)
    for directed in (False, True):
        m = int(min(n * (n - 1) // 2, 6 * n))
        e = graphgen.random_edges(n, m, 1, 3, seed=1000 + n + int(directed), directed=directed)  # heavy ties
        G = dj.dj_load_edges(n, e.src, e.dst, e.w, directed)
        W = orc.build_matrix(n, e.src, e.dst, e.w, directed)
        srcs = sorted({0, n - 1, int(rng.integers(0, n))})
        for s in srcs:
            ref = orc.dijkstra(W, s)
            for ename, engine in ENGINES:
                for mname, mode in MODES:
                    if mode == 2 and n > 1100:
                        continue
                    assert_same(solve(dj, G, s, engine, mode), ref, f"n={n} {ename}/{mname} directed={directed} s={s}")
        G.free()


@pytest.mark.parametrize("cluster_size", [1, 2, 4, 8, 16])
def test_cluster_sizes(dj, orc, cluster_size):
    e = graphgen.bernoulli(3001, 0.02, 1, 50, seed=77)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
    assert_same(solve(dj, G, 123, 2, 1, cluster_size), orc.dijkstra(W, 123), f"C={cluster_size}")


def test_zero_weights(dj, orc):
    for n, seed in ((40, 1), (700, 2), (5000, 3)):
        e = graphgen.random_edges(n, 5 * n, 0, 2, seed=seed, directed=bool(seed % 2))
        G = dj.dj_load_edges(n, e.src, e.dst, e.w, e.directed)
        W = orc.build_matrix(n, e.src, e.dst, e.w, e.directed)
        assert dj.dj_graph_get_info(G)["min_weight"] == 0
        for s in (0, n // 2):
            ref = orc.dijkstra(W, s)
            for _, engine in ENGINES:
                assert_same(solve(dj, G, s, engine), ref, f"zero weights n={n} s={s}")


def test_weights_at_overflow_limit(dj, orc):
    """Large weights shrink the packing span: the capped settle bound must stay exact."""
    n = 3000
    wmax = (2**31 - 2) // (n - 1)
    e = graphgen.random_edges(n, 8 * n, wmax // 2, wmax, seed=5, directed=True)
    G = dj.dj_load_edges(n, e.src, e.dst, e.w, True)
    W = orc.build_matrix(n, e.src, e.dst, e.w, True)
    for s in (0, 1234):
        ref = orc.dijkstra(W, s)
        for _, engine in ENGINES:
            assert_same(solve(dj, G, s, engine), ref, f"near-overflow s={s}")


def test_complete_equal_weights_and_path(dj, orc):
    n = 2000
    W = np.full((n, n), 9, dtype=np.int32)
    np.fill_diagonal(W, 0)
    G = dj.dj_load_dense(W)
    d, p = solve(dj, G, 7)
    assert (np.delete(d, 7) == 9).all() and (np.delete(p, 7) == 7).all() and d[7] == 0 and p[7] == -1
    src = np.arange(n - 1, dtype=np.int32)
    G2 = dj.dj_load_edges(n, src, src + 1, np.full(n - 1, 3, dtype=np.int32), True)
    d, p = solve(dj, G2, 0)
    assert np.array_equal(d, 3 * np.arange(n)) and np.array_equal(p, np.arange(n) - 1)


PATHS = [("ring", -1, -1, -1), ("auto", 0, 0, 0), ("gather", 1 << 20, -1, -1), ("rowsplit", -1, 1, -1),
         ("rowpush", -1, -1, 1)]


@pytest.mark.parametrize("live,rowsplit,rowpush", [(lv, rs, rp) for _, lv, rs, rp in PATHS],
                         ids=[n for n, _, _, _ in PATHS])
def test_relaxation_paths(dj, orc, live, rowsplit, rowpush):
    """Grid engine relaxation paths: streaming every settled row's slice (ring), the default (skip a
    slice with no live column, load only the live groups when few, row split for big phases of
    dense graphs, row push for those of sparser ones), loading only the live groups in every phase
    (gather), row split in every phase and row push in every phase all give Algorithm 1's dist
    and pred.  Dense graphs with weights 1..3 make ties on both dist and pred
    pervasive; zero weights turn the IN bound off; narrow weight ranges give columns a few
    dozen rows of their minimum in-weight, the tie sources the gather path settles tie-only
    columns from."""
    cases = [
        ("dense ties", graphgen.bernoulli(4096, 0.5, 1, 3, seed=91), (0, 1, 2)),
        ("directed ties", graphgen.random_edges(5003, 6 * 5003, 1, 3, seed=92, directed=True), (0, 1)),
        ("zero weights", graphgen.random_edges(4099, 5 * 4099, 0, 2, seed=93, directed=False), (0, 1)),
        ("sparse wide weights", graphgen.bernoulli(6000, 0.01, 1, 1000, seed=94), (0, 1)),
        # ~22 rows of weight 1 into each column: most columns list their tie sources, some overflow
        ("tie sources", graphgen.bernoulli(3000, 0.3, 1, 40, seed=96), (0, 1)),
        ("directed tie sources", graphgen.random_edges(4000, 40 * 4000, 1, 20, seed=97, directed=True), (0, 1)),
    ]
    for what, e, modes in cases:
        G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
        W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
        for s in (0, e.n // 3, e.n - 1):
            ref = orc.dijkstra(W, s)
            for mode in modes:
                if mode == 2 and s != 0:
                    continue
                assert_same(solve(dj, G, s, engine=1, mode=mode, live=live, rowsplit=rowsplit, rowpush=rowpush),
                            ref, f"{what} s={s} mode={mode}")
        G.free()


def test_dense_n16384_full(dj, orc):
    spec = graphgen.WORKLOADS["dense_n16384_p0.5"]
    e = graphgen.make_graph(spec)
    s = graphgen.workload_source(spec)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    ref = orc.dijkstra(W, s)
    got = solve(dj, G, s)  # the engine and launch the benchmark times
    assert_same(got, ref, "n=16384 p=0.5")
    assert_same(solve(dj, G, s, engine=1, live=-1, rowsplit=-1), ref, "n=16384 p=0.5, filter and row split off")
    assert_same(solve(dj, G, s, engine=1, rowsplit=1), ref, "n=16384 p=0.5, row split in every phase")
    assert P.check_invariants(W, s, *got) == []
    assert dj.dj_last_phases() > 0


def test_sparse_directed_n32768_full(dj, orc):
    spec = graphgen.WORKLOADS["sparse_directed_n32768_deg8"]
    e = graphgen.make_graph(spec)
    s = graphgen.workload_source(spec)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    ref = orc.dijkstra(W, s)
    assert_same(solve(dj, G, s), ref, "n=32768 directed")  # the launch the benchmark times
    dyn_phases = dj.dj_last_phases()
    assert_same(solve(dj, G, s, engine=1, settle=2), ref, "n=32768 directed, static IN bound")
    static_phases = dj.dj_last_phases()
    assert dyn_phases < static_phases  # the dynamic IN bound settles more per phase
    assert_same(solve(dj, G, s, engine=1, rowpush=-1), ref, "n=32768 directed, row push off")
    assert_same(solve(dj, G, s, engine=1, rowpush=1), ref, "n=32768 directed, row push in every phase")
    assert_same(solve(dj, G, s, engine=2, cluster_size=16), ref, "n=32768 directed, cluster engine")


def test_batch_matches_single_and_oracle(dj, orc):
    import torch
    spec = graphgen.WORKLOADS["multisource_n8192_p0.05_k256"]
    e = graphgen.make_graph(spec)
    srcs = graphgen.sources(e.n, spec["k"], spec["seed"])
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    k = len(srcs)
    D = torch.full((k, e.n), -5, dtype=torch.int32, device="cuda")
    Pr = torch.full((k, e.n), -5, dtype=torch.int32, device="cuda")
    dj.dj_sssp_batch([G] * k, srcs, list(D), list(Pr))
    dj.dj_sync()
    D, Pr = D.cpu().numpy(), Pr.cpu().numpy()
    # every one of the 256 sources against the CPU oracle (independent serial solves on all host cores)
    Dr, Prr, _ = orc.dijkstra_many_threads(W, srcs)
    for i in range(k):
        assert_same((D[i], Pr[i]), (Dr[i], Prr[i]), f"batch source #{i}")
    for i in range(1, k, 8):  # alone vs in the mix
        assert_same((D[i], Pr[i]), solve(dj, G, int(srcs[i])), f"batch vs single #{i}")


def test_batch_uneven_graphs(dj, orc):
    import torch
    sizes = [5000, 33, 1, 1024, 2999, 64, 7000, 300]
    graphs, Ws, srcs, dists, preds = [], [], [], [], []
    for i, n in enumerate(sizes):
        e = graphgen.bernoulli(n, min(1.0, 20.0 / max(n, 1)), 1, 100, seed=900 + i)
        graphs.append(dj.dj_load_edges(n, e.src, e.dst, e.w, False))
        Ws.append(orc.build_matrix(n, e.src, e.dst, e.w, False))
        srcs.append((7 * i) % n)
        dists.append(torch.full((n,), -5, dtype=torch.int32, device="cuda"))
        preds.append(torch.full((n,), -5, dtype=torch.int32, device="cuda"))
    for mode in (1, 2):
        b = dj.dj_batch_create(graphs, srcs, dists, preds, mode=mode)
        dj.dj_batch_launch(b)
        dj.dj_sync()
        for i in range(len(sizes)):
            assert_same((dists[i].cpu().numpy(), preds[i].cpu().numpy()), orc.dijkstra(Ws[i], srcs[i]),
                        f"uneven batch #{i} n={sizes[i]} mode={mode}")
        b.free()


def test_batch_in_cuda_graph(dj, orc):
    import torch
    e = graphgen.bernoulli(4000, 0.05, 1, 1000, seed=31)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
    srcs = graphgen.sources(e.n, 12, 31)
    D = torch.full((12, e.n), -5, dtype=torch.int32, device="cuda")
    Pr = torch.full((12, e.n), -5, dtype=torch.int32, device="cuda")
    b = dj.dj_batch_create([G] * 12, srcs, list(D), list(Pr))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dj.dj_batch_launch(b, s)  # warm-up outside capture
    s.synchronize()
    D.fill_(-5)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        dj.dj_batch_launch(b, s)
    cg.replay()
    cg.replay()
    torch.cuda.synchronize()
    for i in range(12):
        assert_same((D[i].cpu().numpy(), Pr[i].cpu().numpy()), orc.dijkstra(W, int(srcs[i])), f"graph replay #{i}")


def test_argument_errors(dj):
    import torch
    one = np.array([0], dtype=np.int32)
    with pytest.raises(dj.DjError) as ei:
        dj.dj_load_edges(2, one, np.array([2], dtype=np.int32), one, False)
    assert ei.value.status == dj.DJ_EINVAL
    with pytest.raises(dj.DjError) as ei:
        dj.dj_load_edges(2, one, one + 1, np.array([-3], dtype=np.int32), False)
    assert ei.value.status == dj.DJ_EINVAL
    with pytest.raises(dj.DjError) as ei:
        dj.dj_load_edges(3, one, one + 1, np.array([2**30], dtype=np.int32), False)
    assert ei.value.status == dj.DJ_EOVERFLOW
    G = dj.dj_load_edges(3, one, one + 1, np.array([5], dtype=np.int32), False)
    d = torch.empty(3, dtype=torch.int32, device="cuda")
    with pytest.raises(dj.DjError) as ei:
        dj.dj_sssp(G, 3, d, d.clone())
    assert ei.value.status == dj.DJ_EINVAL
    with pytest.raises(dj.DjError):
        dj.dj_load_dense(np.array([[0, -1], [1, 0]], dtype=np.int32))


def test_bounded_barrier_timeout_reports_and_recovers(dj, orc):
    """One CTA never arrives at the first grid barrier: the others give up after 50 ms,
    the host reads DJ_ETIMEOUT, and the next solve on the same context is exact."""
    import torch
    e = graphgen.bernoulli(5000, 0.01, 1, 100, seed=3)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
    d = torch.empty(e.n, dtype=torch.int32, device="cuda")
    p = torch.empty(e.n, dtype=torch.int32, device="cuda")
    dj.dj_sssp_ex(G, 0, d, p, dj.make_solve_opts(engine=1, timeout_ns=50_000_000, debug_skip_cta=1))
    with pytest.raises(dj.DjError) as ei:
        dj.dj_sync()
    assert ei.value.status == dj.DJ_ETIMEOUT
    dj.dj_sync()  # the error word was cleared
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
    assert_same(solve(dj, G, 0, engine=1), orc.dijkstra(W, 0), "after timeout")


def test_host_result_entry_point(dj, orc):
    e = graphgen.bernoulli(2500, 0.05, 1, 100, seed=8)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
    d, p = dj.dj_sssp_host(G, 42)
    assert_same((d, p), orc.dijkstra(W, 42), "host buffers")
    # upload a modified matrix into the same graph and solve again
    W2 = W.copy()
    W2[42, :] = np.where(W2[42, :] == P.INF, P.INF, 1)  # the graph is undirected: keep it symmetric
    W2[:, 42] = W2[42, :]
    W2[42, 42] = 0
    dj.dj_graph_upload(G, W2)
    d, p = dj.dj_sssp_host(G, 42)
    assert_same((d, p), orc.dijkstra(W2, 42), "after upload")


@pytest.mark.parametrize("directed", [True, False], ids=["directed", "undirected"])
def test_pinned_upload_strides(dj, orc, directed):
    """dj_graph_upload from pinned host memory copies the rows with a kernel that takes their row
    minima on the way (and, on an undirected graph, the tie sources from them): with a row stride
    that is a multiple of 4 (16-byte pieces and an n mod 4 tail), an odd one (entry by entry) and
    none, on a sparse graph and a dense tie-heavy one, the matrix downloads unchanged and both
    engines, and the gather in every phase, solve it as the oracle does."""
    import torch
    sparse = graphgen.random_edges(1003, 8 * 1003, 1, 9, seed=131 + int(directed), directed=directed)
    # columns with a few dozen rows of their minimum in-weight: the gather's column pass (phases
    # of at least 1024 candidates) decides tie-only columns from them
    dense = (graphgen.random_edges(3001, 40 * 3001, 1, 20, seed=133, directed=True) if directed
             else graphgen.bernoulli(3001, 0.3, 1, 40, seed=134))
    rng = np.random.default_rng(7)
    for kind, e, hi in (("sparse", sparse, 20), ("dense, tie-heavy", dense, 40)):
        n = e.n
        G = dj.dj_load_edges(n, e.src, e.dst, e.w, directed)
        W = orc.build_matrix(n, e.src, e.dst, e.w, directed)
        for ld in ((n + 8) // 4 * 4, n + 2 if n % 2 else n + 1, n):
            W2 = W.copy()
            fin = W2 < P.INF
            W2[fin] = rng.integers(1, hi, size=int(fin.sum()), dtype=np.int32)  # new weights, same edges
            np.fill_diagonal(W2, 0)
            if not directed:
                W2 = np.minimum(W2, W2.T)
            buf = torch.full((n, ld), -7, dtype=torch.int32).pin_memory()
            buf[:, :n] = torch.from_numpy(W2)
            dj.dj_graph_upload(G, buf[:, :n])
            dj.dj_sync()
            assert np.array_equal(dj.dj_graph_download(G), W2), f"{kind} ld={ld}: download"
            for s in (0, n // 2, n - 1):
                ref = orc.dijkstra(W2, s)
                for _, engine in ENGINES:
                    assert_same(solve(dj, G, s, engine), ref, f"{kind} ld={ld} engine={engine} s={s}")
                # the gather in every phase: its column pass decides tie-only columns from the tie
                # sources listed by the upload
                assert_same(solve(dj, G, s, 1, live=1 << 20), ref, f"{kind} ld={ld} gather s={s}")
        G.free()


def test_back_to_back_small_solves_keep_stream_order(dj, orc):
    """Small-graph solves start while the previous kernel on the stream is still running (they
    are programmatic dependents) and wait for it only before writing their results.  Back to back
    on one stream: solves into separate buffers each equal the oracle; solves into one shared
    buffer pair leave the last solve's result; a copy taken by an ordinary kernel between two
    solves sees the earlier solve's result complete, never a mix."""
    import torch
    e = graphgen.bernoulli(1024, 0.1, 1, 100, seed=61)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
    srcs = [int(x) for x in graphgen.sources(e.n, 24, 62)]
    Dr, Prr, _ = orc.dijkstra_many_threads(W, np.array(srcs, dtype=np.int32))
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        D = torch.full((len(srcs), e.n), -5, dtype=torch.int32, device="cuda")
        Pr = torch.full((len(srcs), e.n), -5, dtype=torch.int32, device="cuda")
        for i, s in enumerate(srcs):
            dj.dj_sssp(G, s, D[i], Pr[i], st)
        d1 = torch.full((e.n,), -5, dtype=torch.int32, device="cuda")
        p1 = torch.full((e.n,), -5, dtype=torch.int32, device="cuda")
        snaps = []
        for s in srcs:
            dj.dj_sssp(G, s, d1, p1, st)
            snaps.append((d1.clone(), p1.clone()))  # ordinary kernels between the solves
    dj.dj_sync(st)
    for i in range(len(srcs)):
        assert_same((D[i].cpu().numpy(), Pr[i].cpu().numpy()), (Dr[i], Prr[i]), f"separate buffers #{i}")
        assert_same((snaps[i][0].cpu().numpy(), snaps[i][1].cpu().numpy()), (Dr[i], Prr[i]), f"snapshot #{i}")
    assert_same((d1.cpu().numpy(), p1.cpu().numpy()), (Dr[-1], Prr[-1]), "shared buffers")
    G.free()


def test_cuda_graph_capture_and_replay(dj, orc):
    """Single solves captured into a CUDA graph and replayed (the host's per-call work leaves the
    loop): on the cluster engine (n=1024, no device memory per solve) and the grid engine (n=4096,
    a stream-ordered workspace inside the graph), every replay writes the oracle's dist and pred."""
    import torch
    for n, pr, seed in ((1024, 0.1, 71), (4096, 0.2, 72)):
        e = graphgen.bernoulli(n, pr, 1, 100, seed=seed)
        G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
        W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
        srcs = [int(x) for x in graphgen.sources(n, 6, seed + 1)]
        Dr, Prr, _ = orc.dijkstra_many_threads(W, np.array(srcs, dtype=np.int32))
        st = torch.cuda.Stream()
        D = torch.full((len(srcs), n), -5, dtype=torch.int32, device="cuda")
        P = torch.full((len(srcs), n), -5, dtype=torch.int32, device="cuda")
        dj.dj_sssp(G, srcs[0], D[0], P[0], st)  # first launch: the kernel's one-time set-up
        dj.dj_sync(st)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=st):
            for i, s in enumerate(srcs):
                dj.dj_sssp(G, s, D[i], P[i], st)
        for rep in range(2):
            with torch.cuda.stream(st):
                D.fill_(-5)
                P.fill_(-5)
                cg.replay()
            dj.dj_sync(st)
            for i in range(len(srcs)):
                assert_same((D[i].cpu().numpy(), P[i].cpu().numpy()), (Dr[i], Prr[i]), f"n={n} replay {rep} #{i}")
        del cg
        G.free()


def test_back_to_back_grid_solves_and_upload(dj, orc):
    """Grid-engine solves launched back to back (each a programmatic dependent of the previous
    kernel, sharing the stream's workspace), then a matrix upload followed at once by solves on
    both engines: every result equals the oracle on the matrix in force when it was enqueued."""
    import torch
    e = graphgen.bernoulli(4096, 0.3, 1, 50, seed=63)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
    srcs = [int(x) for x in graphgen.sources(e.n, 6, 64)]
    st = torch.cuda.Stream()
    D = torch.full((len(srcs), e.n), -5, dtype=torch.int32, device="cuda")
    Pr = torch.full((len(srcs), e.n), -5, dtype=torch.int32, device="cuda")
    for i, s in enumerate(srcs):
        dj.dj_sssp(G, s, D[i], Pr[i], st)
    dj.dj_sync(st)
    Dr, Prr, _ = orc.dijkstra_many_threads(W, np.array(srcs, dtype=np.int32))
    for i in range(len(srcs)):
        assert_same((D[i].cpu().numpy(), Pr[i].cpu().numpy()), (Dr[i], Prr[i]), f"grid b2b #{i}")
    # a small graph: upload a changed matrix, then solve right away on the same stream
    e2 = graphgen.bernoulli(1500, 0.1, 1, 100, seed=65)
    G2 = dj.dj_load_edges(e2.n, e2.src, e2.dst, e2.w, False)
    W2 = orc.build_matrix(e2.n, e2.src, e2.dst, e2.w, False)
    W3 = W2.copy()
    W3[:7, :] = np.where(W3[:7, :] == P.INF, P.INF, 1)  # edges at nodes 0..6 get weight 1 (kept symmetric)
    W3[:, :7] = W3[:7, :].T
    np.fill_diagonal(W3, 0)
    Wh = torch.from_numpy(W3).pin_memory()
    d = torch.full((e2.n,), -5, dtype=torch.int32, device="cuda")
    p = torch.full((e2.n,), -5, dtype=torch.int32, device="cuda")
    dj.dj_sssp(G2, 3, d, p, st)  # on the old matrix
    dj.dj_graph_upload(G2, Wh, st)
    d2 = torch.full((e2.n,), -5, dtype=torch.int32, device="cuda")
    p2 = torch.full((e2.n,), -5, dtype=torch.int32, device="cuda")
    dj.dj_sssp(G2, 3, d2, p2, st)  # on the new one
    dj.dj_sync(st)
    assert_same((d.cpu().numpy(), p.cpu().numpy()), orc.dijkstra(W2, 3), "before upload")
    assert_same((d2.cpu().numpy(), p2.cpu().numpy()), orc.dijkstra(W3, 3), "after upload")
    G.free()
    G2.free()


def test_dynamic_in_bound(dj, orc):
    """On graphs that are not dense the grid engine takes the IN bound from the smallest in-weight
    of the rows still unsettled (each column's four smallest in-weights listed at load).  Static,
    dynamic and OUT-only settle bounds, on ragged tie-heavy directed and undirected graphs, columns
    with more in-edges than listed and fewer, all give Algorithm 1's dist and pred; the dynamic
    bound never takes more phases than the static one."""
    cases = [
        ("directed ties", graphgen.random_edges(5003, 6 * 5003, 1, 3, seed=101, directed=True)),
        ("undirected ties", graphgen.random_edges(4099, 5 * 4099, 1, 4, seed=102, directed=False)),
        ("directed wide weights", graphgen.outdeg(6000, 8, 1, 10000, seed=103)),
        ("in-degree about 40", graphgen.random_edges(4000, 40 * 4000, 1, 20, seed=104, directed=True)),
        ("few in-edges", graphgen.random_edges(3001, 2 * 3001, 1, 9, seed=105, directed=True)),
    ]
    for what, e in cases:
        G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
        W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
        for s in (0, e.n // 2, e.n - 1):
            ref = orc.dijkstra(W, s)
            assert_same(solve(dj, G, s, engine=1, settle=3), ref, f"{what} s={s} dynamic IN")
            ph_dyn = dj.dj_last_phases()
            assert_same(solve(dj, G, s, engine=1, settle=4), ref, f"{what} s={s} dynamic IN and OUT")
            assert_same(solve(dj, G, s, engine=1, settle=4, rowpush=1), ref, f"{what} s={s} dynamic both, row push")
            assert_same(solve(dj, G, s, engine=1, settle=4, live=1 << 20, rowpush=-1), ref,
                        f"{what} s={s} dynamic both, gather")
            assert_same(solve(dj, G, s, engine=1, settle=2), ref, f"{what} s={s} static IN")
            ph_static = dj.dj_last_phases()
            assert_same(solve(dj, G, s, engine=1, settle=1), ref, f"{what} s={s} OUT only")
            assert_same(solve(dj, G, s, engine=1, settle=3, rowpush=1), ref, f"{what} s={s} dynamic IN, row push")
            assert_same(solve(dj, G, s, engine=1, settle=3, live=1 << 20, rowpush=-1), ref,
                        f"{what} s={s} dynamic IN, gather")
            assert ph_dyn <= ph_static, (what, s, ph_dyn, ph_static)
        G.free()
