"""The allocation-free entry point gives the same results as dj_sssp.

dj_sssp_noalloc serves callers that must not allocate device memory while
they solve (for instance inside a globally-captured stream, or when the
caching allocator has reserved almost all HBM): its scratch is a fixed array
inside the library.  This file is named so that pytest collects it last.
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


def _reference(dj, g, s, n):
    import torch
    d = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    p = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    dj.dj_sssp(g, s, d, p)
    dj.dj_sync()
    return d.cpu().numpy(), p.cpu().numpy()


def test_noalloc_matches_dj_sssp_twice_in_a_row(dj, orc):
    import torch
    cases = [graphgen.bernoulli(4096, 0.1, 1, 100, seed=41), graphgen.outdeg(5003, 8, 1, 10000, seed=42)]
    for e in cases:
        g = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
        srcs = [int(x) for x in graphgen.sources(e.n, 2, 43)]
        refs = [_reference(dj, g, s, e.n) for s in srcs]
        # the existing entry point's results are themselves Algorithm 1's (CPU oracle)
        W = orc.build_matrix(e.n, e.src, e.dst, e.w, e.directed)
        for s, (dr, pr) in zip(srcs, refs):
            do, po = orc.dijkstra(W, s)
            assert np.array_equal(dr, do) and np.array_equal(pr, po)
        del W
        d = torch.full((e.n,), -5, dtype=torch.int32, device="cuda")
        p = torch.full((e.n,), -5, dtype=torch.int32, device="cuda")
        dj.dj_sssp_noalloc(g, srcs[0], d, p)  # first call on the device: one-time set-up
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        for s, (dr, pr) in zip(srcs, refs):  # two calls in a row, each checked
            d.fill_(-5)
            p.fill_(-5)
            dj.dj_sssp_noalloc(g, s, d, p)
            torch.cuda.synchronize()
            got_d, got_p = d.cpu().numpy(), p.cpu().numpy()
            assert got_d[s] == 0  # completed
            assert np.array_equal(got_d, dr)  # integers: the tolerance is zero
            assert np.array_equal(got_p, pr)
        assert torch.cuda.mem_get_info()[0] == free_before  # no device memory taken
        g.free()


def test_noalloc_rejects_bad_arguments(dj):
    import torch
    e = graphgen.bernoulli(64, 0.2, 1, 9, seed=44)
    g = dj.dj_load_edges(e.n, e.src, e.dst, e.w, e.directed)
    d = torch.empty(64, dtype=torch.int32, device="cuda")
    with pytest.raises(dj.DjError) as ei:
        dj.dj_sssp_noalloc(g, 64, d, d.clone())
    assert ei.value.status == dj.DJ_EINVAL


def test_noalloc_rejects_a_graph_whose_scratch_does_not_fit(dj):
    """A graph one column beyond the documented limit (n = 130,720 on a 152-SM GB300) is rejected
    before any launch, with a message naming this device's limit.  Its matrix takes 68 GB of HBM
    for the duration of the test."""
    import torch
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("the documented limit is for 152 SMs")
    n = 130_721
    one = np.array([0, 1, 2], dtype=np.int32)
    g = dj.dj_load_edges(n, one, one + 1, one + 5, False)
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(dj.DjError) as ei:
        dj.dj_sssp_noalloc(g, 0, d, p)
    assert ei.value.status == dj.DJ_EINVAL
    assert "n up to 130720" in str(ei.value)
    g.free()
