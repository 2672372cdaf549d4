"""Serving: continuous batching returns, for every request, exactly the result of that solve alone.

Requests for graphs of different sizes arrive while others are running; they
are admitted as slots and budget free up and overlap on the device.  Each
result is compared element by element with dj_sssp on the same (graph, source)
and, for a sample, with the CPU oracle.
"""
import time

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


@pytest.fixture(scope="module")
def graphs(dj, orc):
    specs = [(600, 0.2, 11), (2500, 0.05, 12), (4100, 0.3, 13), (97, 0.5, 14), (9000, 0.02, 15)]
    out = []
    for n, p, seed in specs:
        e = graphgen.bernoulli(n, p, 1, 1000, seed)
        g = dj.dj_load_edges(n, e.src, e.dst, e.w, False)
        out.append((g, e))
    return out


def single(dj, g, s, n):
    import torch
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    dj.dj_sssp(g, s, d, p)
    dj.dj_sync()
    return d.cpu().numpy(), p.cpu().numpy()


def test_submit_poll_matches_single_solves(dj, orc, graphs):
    import torch
    srv = dj.dj_serve_create(dj.make_serve_opts(max_slots=16, idle_timeout_ns=50_000_000))
    gids = [dj.dj_serve_add_graph(srv, g) for g, _ in graphs]
    rng = np.random.default_rng(3)
    reqs, pooled = [], []
    for i in range(60):
        k = int(rng.integers(0, len(graphs)))
        n = graphs[k][1].n
        s = int(rng.integers(0, n))
        if i % 5 == 0:
            # server-owned result buffer: read it back before it can be reused
            t = dj.dj_serve_submit(srv, gids[k], s)
            while t is None:
                time.sleep(0.0005)
                t = dj.dj_serve_submit(srv, gids[k], s)
            dj.dj_serve_wait(srv, t)
            pooled.append((k, s, dj.dj_serve_result(srv, t, n)))
            continue
        d = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        p = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        t = dj.dj_serve_submit(srv, gids[k], s, d, p)
        while t is None:  # all slots busy: admitted once one frees up
            time.sleep(0.0005)
            t = dj.dj_serve_submit(srv, gids[k], s, d, p)
        reqs.append((t, k, s, d, p))
    for t, *_ in reqs:
        dj.dj_serve_wait(srv, t)
    st = dj.dj_serve_stats_get(srv)
    srv.destroy()  # the persistent kernel is gone before the reference solves run
    assert st["completed"] == 60 and st["submitted"] == 60
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
    assert st["kernel_launches"] >= 1
    for t, k, s, d, p in reqs:
        g, e = graphs[k]
        ref = single(dj, g, s, e.n)
        assert np.array_equal(d.cpu().numpy(), ref[0]) and np.array_equal(p.cpu().numpy(), ref[1]), (t, k, s)
    for k, s, got in pooled:
        g, e = graphs[k]
        ref = single(dj, g, s, e.n)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), ("pooled", k, s)
    for t, k, s, d, p in reqs[1:40:9]:  # and the CPU oracle on a few
        e = graphs[k][1]
        W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
        dr, pr = orc.dijkstra(W, s)
        assert np.array_equal(d.cpu().numpy(), dr) and np.array_equal(p.cpu().numpy(), pr)


def test_trace_continuous_batching(dj, graphs):
    """A Poisson trace faster than the GPU drains it with 6 slots: requests are deferred,
    admitted as slots free up, and every result equals its solve alone."""
    import torch
    R = 240
    rng = np.random.default_rng(9)
    req_g = rng.integers(0, len(graphs), R).astype(np.int32)
    req_s = np.array([rng.integers(0, graphs[k][1].n) for k in req_g], dtype=np.int32)
    arrival = np.cumsum(rng.exponential(1 / 20000.0, R))
    keep = set(range(0, R, 7))
    outs_d = [torch.empty(graphs[req_g[r]][1].n, dtype=torch.int32, device="cuda") if r in keep else None
              for r in range(R)]
    outs_p = [torch.empty(graphs[req_g[r]][1].n, dtype=torch.int32, device="cuda") if r in keep else None
              for r in range(R)]
    st = dj.dj_serve([g for g, _ in graphs], req_g, req_s, arrival, outs_d, outs_p,
                     dj.make_serve_opts(max_slots=6, idle_timeout_ns=50_000_000))
    assert st["completed"] == R
    assert st["rejected"] > 0  # some requests had to wait for a slot
    assert st["p99_us"] >= st["p50_us"] > 0 and st["solves_per_s"] > 0
    for r in sorted(keep):
        g, e = graphs[req_g[r]]
        ref = single(dj, g, int(req_s[r]), e.n)
        assert np.array_equal(outs_d[r].cpu().numpy(), ref[0]) and np.array_equal(outs_p[r].cpu().numpy(), ref[1])


def test_budget_admission(dj, graphs):
    g_small, e_small = graphs[3]
    g_big, _ = graphs[4]
    budget = int(dj.dj_graph_get_info(g_small)["bytes"]) + 8192
    srv = dj.dj_serve_create(dj.make_serve_opts(hbm_budget=budget, max_slots=4))
    gid = dj.dj_serve_add_graph(srv, g_small)
    with pytest.raises(dj.DjError) as ei:
        dj.dj_serve_add_graph(srv, g_big)
    assert ei.value.status == dj.DJ_ENOMEM
    t = dj.dj_serve_submit(srv, gid, 0)  # pooled result: fits the remaining budget
    assert t is not None
    dj.dj_serve_wait(srv, t)
    d, p = dj.dj_serve_result(srv, t, e_small.n)
    srv.destroy()
    ref = single(dj, g_small, 0, e_small.n)
    assert np.array_equal(d, ref[0]) and np.array_equal(p, ref[1])


def test_idle_exit_and_relaunch(dj, graphs):
    import torch
    g, e = graphs[1]
    srv = dj.dj_serve_create(dj.make_serve_opts(max_slots=4, idle_timeout_ns=20_000_000))
    gid = dj.dj_serve_add_graph(srv, g)
    d = torch.empty(e.n, dtype=torch.int32, device="cuda")
    p = torch.empty_like(d)
    t = dj.dj_serve_submit(srv, gid, 5, d, p)
    dj.dj_serve_wait(srv, t)
    time.sleep(0.2)  # the persistent kernel leaves after 20 ms without work
    d.fill_(-5)
    t = dj.dj_serve_submit(srv, gid, 6, d, p)
    dj.dj_serve_wait(srv, t)
    st = dj.dj_serve_stats_get(srv)
    srv.destroy()
    assert st["kernel_launches"] >= 2
    ref = single(dj, g, 6, e.n)
    assert np.array_equal(d.cpu().numpy(), ref[0]) and np.array_equal(p.cpu().numpy(), ref[1])


def test_bad_requests(dj, graphs):
    g, e = graphs[0]
    srv = dj.dj_serve_create(dj.make_serve_opts(max_slots=2))
    gid = dj.dj_serve_add_graph(srv, g)
    with pytest.raises(dj.DjError) as ei:
        dj.dj_serve_submit(srv, gid + 7, 0)
    assert ei.value.status == dj.DJ_EINVAL
    with pytest.raises(dj.DjError) as ei:
        dj.dj_serve_submit(srv, gid, e.n)
    assert ei.value.status == dj.DJ_EINVAL
    srv.destroy()


def test_bench_serving_mix_against_oracle(dj, orc):
    """The benchmark's own serving workload (64 resident graphs, n log-uniform in [512, 16384],
    p uniform in [0.01, 0.5], 10000 requests) run as the benchmark runs it (every request waiting
    at t = 0, 512 slots, default clusters): a seeded sample of about 1 in 50 results, covering every
    power-of-two n bucket and the largest graph, equals the CPU oracle element by element."""
    import torch
    spec = graphgen.WORKLOADS["serving_64graphs_10000req"]
    tr = graphgen.serving_trace(spec["graphs"], spec["requests"], 1.0, spec["seed"])
    graphs = []
    for gi in range(spec["graphs"]):
        e = graphgen.bernoulli(int(tr.graph_n[gi]), float(tr.graph_p[gi]), spec["wlo"], spec["whi"],
                               int(tr.graph_seed[gi]))
        graphs.append(dj.dj_load_edges(e.n, e.src, e.dst, e.w, False))
        del e
    R = spec["requests"]
    sample = set(range(0, R, 50))
    bucket = np.floor(np.log2(tr.graph_n[tr.req_graph])).astype(int)
    for b in np.unique(bucket):  # every n bucket, even if the stride missed it
        sample.add(int(np.nonzero(bucket == b)[0][0]))
    biggest = int(np.argmax(tr.graph_n))
    for gi in np.nonzero(tr.graph_n > 15000)[0]:  # the largest graphs (clusters of 16, wide copies)
        sample.update(int(r) for r in np.nonzero(tr.req_graph == gi)[0][:3])
    outs_d = [None] * R
    outs_p = [None] * R
    for r in sample:
        n = int(tr.graph_n[tr.req_graph[r]])
        outs_d[r] = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        outs_p[r] = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    st = dj.dj_serve(graphs, tr.req_graph, tr.req_source, np.zeros(R), outs_d, outs_p,
                     dj.make_serve_opts(max_slots=512))
    assert st["completed"] == R
    torch.cuda.synchronize()
    for g in graphs:
        g.free()
    assert int(tr.graph_n[biggest]) > 15000
    by_graph = {}
    for r in sorted(sample):
        by_graph.setdefault(int(tr.req_graph[r]), []).append(r)
    checked = set()
    for gi, rs in sorted(by_graph.items()):
        e = graphgen.bernoulli(int(tr.graph_n[gi]), float(tr.graph_p[gi]), spec["wlo"], spec["whi"],
                               int(tr.graph_seed[gi]))
        W = orc.build_matrix(e.n, e.src, e.dst, e.w, False)
        del e
        D, Pr, _ = orc.dijkstra_many_threads(W, np.array([tr.req_source[r] for r in rs], dtype=np.int32))
        for i, r in enumerate(rs):
            assert np.array_equal(outs_d[r].cpu().numpy(), D[i]), ("dist", r, gi)
            assert np.array_equal(outs_p[r].cpu().numpy(), Pr[i]), ("pred", r, gi)
            checked.add(int(bucket[r]))
        del W
    assert checked == set(int(b) for b in np.unique(bucket))
    assert len(sample) >= R // 50
