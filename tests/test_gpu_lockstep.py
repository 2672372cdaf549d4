"""Lockstep multi-source engine: every source's dist and pred equal the CPU oracle bit for bit.

Many sources of one graph advance phase by phase together, each matrix row a phase needs read
once for every source that settles it.  Cases: the benchmark's 256-source batch (every source
checked), ragged n and several source groups, tie-heavy and zero-weight graphs, weights too large
for the 16-bit tie record (IN bound off), the OUT bound only, directed graphs, repeated sources,
one source, the one-shot dj_sssp_batch path and the autotuner's choice.
"""
import numpy as np
import pytest

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


def run_batch(dj, G, n, srcs, **kw):
    import torch
    k = len(srcs)
    D = torch.full((k, n), -5, dtype=torch.int32, device="cuda")
    P = torch.full((k, n), -5, dtype=torch.int32, device="cuda")
    b = dj.dj_batch_create([G] * k, srcs, list(D), list(P), **kw)
    eng = dj.dj_batch_get_engine(b)
    dj.dj_batch_launch(b)
    dj.dj_sync()
    out = (D.cpu().numpy(), P.cpu().numpy())
    b.free()
    return out, eng


def check(orc, W, srcs, got, what):
    D, P = got
    Dr, Pr, _ = orc.dijkstra_many_threads(W, np.asarray(srcs, dtype=np.int32))
    for i in range(len(srcs)):
        if not np.array_equal(D[i], Dr[i]):
            bad = np.nonzero(D[i] != Dr[i])[0]
            raise AssertionError(f"{what}: source #{i} ({srcs[i]}) dist differs at {bad.size} nodes, first {bad[:5]}")
        if not np.array_equal(P[i], Pr[i]):
            bad = np.nonzero(P[i] != Pr[i])[0]
            raise AssertionError(f"{what}: source #{i} ({srcs[i]}) pred differs at {bad.size} nodes, first {bad[:5]}: "
                                 f"{P[i][bad[:5]]} vs {Pr[i][bad[:5]]}")


def test_bench_batch_all_sources(dj, orc):
    spec = graphgen.WORKLOADS["multisource_n8192_p0.05_k256"]
    e = graphgen.make_graph(spec)
    srcs = [int(x) for x in graphgen.sources(e.n, spec["k"], spec["seed"])]
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
    got, eng = run_batch(dj, G, e.n, srcs, engine=dj.DJ_BATCH_ENGINE_LOCKSTEP)
    assert eng == "lockstep"
    check(orc, W, srcs, got, "n=8192 p=0.05, 256 sources")
    assert dj.dj_last_phases() > 0
    G.free()


@pytest.mark.parametrize("n", [1, 5, 33, 257, 1000, 3001, 5003])
def test_ragged_ties_directed(dj, orc, n):
    for directed in (False, True):
        m = int(min(n * (n - 1) // 2, 6 * n))
        e = graphgen.random_edges(n, m, 1, 3, seed=3000 + n + int(directed), directed=directed)
        G = dj.dj_load_edges(n, e.src, e.dst, e.w, directed)
        W = orc.build_matrix(n, e.src, e.dst, e.w, directed)
        k = min(n, 37)
        srcs = [int(x) for x in graphgen.sources(n, k, 71 + n)]
        got, eng = run_batch(dj, G, n, srcs, engine=dj.DJ_BATCH_ENGINE_LOCKSTEP)
        assert eng == "lockstep"
        check(orc, W, srcs, got, f"n={n} directed={directed}")
        G.free()


def test_several_groups_and_repeated_sources(dj, orc):
    """More sources than one group holds (n > 8192 keeps fewer per group), repeats included."""
    e = graphgen.bernoulli(9000, 0.02, 1, 200, seed=81)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
    srcs = [int(x) for x in graphgen.sources(e.n, 300, 82)] + [5, 5, 8999]
    got, _ = run_batch(dj, G, e.n, srcs, engine=dj.DJ_BATCH_ENGINE_LOCKSTEP)
    check(orc, W, srcs, got, "n=9000, 303 sources")
    G.free()


def test_zero_weights_big_weights_and_out_bound(dj, orc):
    cases = [
        ("zero weights", graphgen.random_edges(2500, 12000, 0, 2, seed=83, directed=False), {}),
        ("weights beyond 16 bits", graphgen.random_edges(2000, 9000, 60000, 70000, seed=84, directed=True), {}),
        ("OUT bound only", graphgen.bernoulli(3000, 0.05, 1, 50, seed=85), {"settle": 1}),
        ("dense ties", graphgen.bernoulli(2048, 0.5, 1, 3, seed=86), {}),
    ]
    for what, e, kw in cases:
        G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
        W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
        srcs = [int(x) for x in graphgen.sources(e.n, 40, 87)]
        got, _ = run_batch(dj, G, e.n, srcs, engine=dj.DJ_BATCH_ENGINE_LOCKSTEP, **kw)
        check(orc, W, srcs, got, what)
        G.free()


def test_one_shot_batch_and_autotune(dj, orc):
    import torch
    e = graphgen.bernoulli(4000, 0.05, 1, 1000, seed=88)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
    srcs = [int(x) for x in graphgen.sources(e.n, 64, 89)]
    D = torch.full((64, e.n), -5, dtype=torch.int32, device="cuda")
    P = torch.full((64, e.n), -5, dtype=torch.int32, device="cuda")
    dj.dj_sssp_batch([G] * 64, srcs, list(D), list(P))  # untuned: the cluster engine
    dj.dj_sync()
    check(orc, W, srcs, (D.cpu().numpy(), P.cpu().numpy()), "one-shot batch")
    D.fill_(-5)
    b = dj.dj_batch_create([G] * 64, srcs, list(D), list(P))
    tune = dj.dj_batch_autotune(b)
    assert tune["engine"] in ("lockstep", "cluster") and tune["ms"] > 0
    D.fill_(-5)
    P.fill_(-5)
    dj.dj_batch_launch(b)
    dj.dj_sync()
    check(orc, W, srcs, (D.cpu().numpy(), P.cpu().numpy()), f"after autotune ({tune['engine']})")
    b.free()
    G.free()
    # a tuned entry that names the lockstep engine routes batches of that shape to it (a shape,
    # n in [1024, 2048) at density about 1/3, that no other batch test uses)
    import json
    import os
    import tempfile
    e = graphgen.bernoulli(1500, 0.3, 1, 1000, seed=90)
    G = dj.dj_load_edges(e.n, e.src, e.dst, e.w, False)
    W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
    srcs = [int(x) for x in graphgen.sources(e.n, 64, 91)]
    D = torch.full((64, e.n), -5, dtype=torch.int32, device="cuda")
    P = torch.full((64, e.n), -5, dtype=torch.int32, device="cuda")
    info = dj.dj_graph_get_info(G)
    nb = info["n"].bit_length() - 1
    db = 0
    while db < 20 and 2.0 ** (db + 1) <= info["n"] ** 2 / max(info["entries"], 1):
        db += 1
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.json")
        with open(path, "w") as f:
            json.dump({"version": 1, "entries": [{"n_bucket": nb, "density_bucket": db, "sms": sms,
                                                  "engine": "lockstep", "cluster_size": 0}]}, f)
        dj.dj_tune_load(path)
    assert dj.dj_tune_lookup(info["n"], info["entries"], sms)["engine"] == "lockstep"
    D.fill_(-5)
    P.fill_(-5)
    dj.dj_sssp_batch([G] * 64, srcs, list(D), list(P))
    dj.dj_sync()
    check(orc, W, srcs, (D.cpu().numpy(), P.cpu().numpy()), "one-shot batch, tuned to lockstep")
    b2 = dj.dj_batch_create([G] * 64, srcs, list(D), list(P))
    assert dj.dj_batch_get_engine(b2) == "lockstep"
    b2.free()
    G.free()
