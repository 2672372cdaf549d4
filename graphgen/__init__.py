"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only draws random numbers and shapes them into edge lists, source
sets and request traces.  It contains no shortest-path arithmetic, and it
imports neither the CPU oracle nor the CUDA library.

Workload recipes (the paper's generator and weights are unstated; its graphs
are dense and 1:3-sparse int32 matrices, Section IV-A):
  * ``bernoulli``: undirected, each unordered pair is an edge with probability p,
    weight uniform in [wlo, whi].
  * ``outdeg``: directed (the paper's ``-w`` fill), each node draws d uniform
    targets; self-draws dropped, duplicates kept (the matrix keeps the minimum).
  * ``sources``: distinct seeded draws.
  * ``serving_trace``: per-graph sizes log-uniform in [nlo, nhi], densities
    uniform, and Poisson request arrivals.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

STREAM_USER = 16


def build(force: bool = False) -> str:
    """Compile the generator with the host C compiler (portable flags only)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC,
                    "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, i64, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32
        p = ctypes.c_void_p
        lib.gg_draw.restype = u64
        lib.gg_draw.argtypes = [u64, u64, u64]
        lib.gg_bounded.restype = u64
        lib.gg_bounded.argtypes = [u64, u64, u64, u64]
        lib.gg_fill_u64.restype = None
        lib.gg_fill_u64.argtypes = [u64, u64, u64, i64, p]
        lib.gg_fill_bounded.restype = None
        lib.gg_fill_bounded.argtypes = [u64, u64, u64, i64, u64, p]
        lib.gg_bernoulli_count.restype = i64
        lib.gg_bernoulli_count.argtypes = [i32, ctypes.c_double, u64, p]
        lib.gg_bernoulli_fill.restype = None
        lib.gg_bernoulli_fill.argtypes = [i32, ctypes.c_double, i32, i32, u64, p, p, p, p]
        lib.gg_outdeg_fill.restype = i64
        lib.gg_outdeg_fill.argtypes = [i32, i32, i32, i32, u64, p, p, p]
        lib.gg_distinct_sources.restype = None
        lib.gg_distinct_sources.argtypes = [i32, i32, u64, p, p]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class EdgeList:
    """An edge list in the layout the loader takes: three int32 arrays of length m."""
    n: int
    src: np.ndarray
    dst: np.ndarray
    w: np.ndarray
    directed: bool

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def bernoulli(n: int, p: float, wlo: int, whi: int, seed: int) -> EdgeList:
    """Undirected graph: each pair i<j is an edge with probability p."""
    lib = _load()
    counts = np.zeros(n, dtype=np.int64)
    m = lib.gg_bernoulli_count(n, float(p), seed, _ptr(counts))
    offsets = np.zeros(n, dtype=np.int64)
    if n > 1:
        np.cumsum(counts[:-1], out=offsets[1:])
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    w = np.empty(m, dtype=np.int32)
    if m:
        lib.gg_bernoulli_fill(n, float(p), wlo, whi, seed, _ptr(offsets), _ptr(src), _ptr(dst), _ptr(w))
    return EdgeList(n, src, dst, w, directed=False)


def outdeg(n: int, d: int, wlo: int, whi: int, seed: int) -> EdgeList:
    """Directed graph: each node draws d uniform out-targets (self-draws dropped)."""
    lib = _load()
    cap = n * d
    src = np.empty(cap, dtype=np.int32)
    dst = np.empty(cap, dtype=np.int32)
    w = np.empty(cap, dtype=np.int32)
    m = lib.gg_outdeg_fill(n, d, wlo, whi, seed, _ptr(src), _ptr(dst), _ptr(w))
    return EdgeList(n, src[:m].copy(), dst[:m].copy(), w[:m].copy(), directed=True)


def sources(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct source nodes of [0, n), in draw order."""
    if k > n:
        raise ValueError("k > n")
    lib = _load()
    out = np.empty(k, dtype=np.int32)
    seen = np.empty(n, dtype=np.uint8)
    lib.gg_distinct_sources(n, k, seed, _ptr(out), _ptr(seen))
    return out


def uniform01(seed: int, stream: int, count: int, ctr0: int = 0) -> np.ndarray:
    """count uniform doubles in [0, 1) (53-bit) from the counter-based stream."""
    lib = _load()
    raw = np.empty(count, dtype=np.uint64)
    if count:
        lib.gg_fill_u64(seed, STREAM_USER + stream, ctr0, count, _ptr(raw))
    return (raw >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def bounded(seed: int, stream: int, count: int, rng: int, ctr0: int = 0) -> np.ndarray:
    """count unbiased integers in [0, rng)."""
    lib = _load()
    out = np.empty(count, dtype=np.int64)
    if count:
        lib.gg_fill_bounded(seed, STREAM_USER + stream, ctr0, count, rng, _ptr(out))
    return out


def random_edges(n: int, m: int, wlo: int, whi: int, seed: int, directed: bool,
                 allow_self: bool = True) -> EdgeList:
    """m arbitrary (src, dst, w) triples: repeats and self-loops included, for edge-case tests."""
    s = bounded(seed, 1, m, n).astype(np.int32)
    d = bounded(seed, 2, m, n).astype(np.int32)
    w = (wlo + bounded(seed, 3, m, whi - wlo + 1)).astype(np.int32)
    if not allow_self:
        keep = s != d
        s, d, w = s[keep], d[keep], w[keep]
    return EdgeList(n, s, d, w, directed)


@dataclass
class ServingTrace:
    """Graph shapes and a request trace for the continuous-batching workload."""
    graph_n: np.ndarray        # int32 [G]
    graph_p: np.ndarray        # float64 [G]
    graph_seed: np.ndarray     # uint64 [G]
    req_graph: np.ndarray      # int32 [R]
    req_source: np.ndarray     # int32 [R]
    req_arrival_s: np.ndarray  # float64 [R], seconds from trace start


def serving_trace(num_graphs: int, num_requests: int, rate_per_s: float, seed: int,
                  nlo: int = 512, nhi: int = 16384, plo: float = 0.01, phi: float = 0.5) -> ServingTrace:
    """Log-uniform n in [nlo, nhi], uniform p in [plo, phi], Poisson arrivals at rate_per_s."""
    u_n = uniform01(seed, 1, num_graphs)
    u_p = uniform01(seed, 2, num_graphs)
    ratio = nhi / nlo
    graph_n = np.minimum(np.floor(nlo * np.power(ratio, u_n)), nhi).astype(np.int32)
    graph_p = plo + (phi - plo) * u_p
    graph_seed = np.array([_load().gg_draw(seed, STREAM_USER + 3, g) for g in range(num_graphs)],
                          dtype=np.uint64)
    req_graph = bounded(seed, 4, num_requests, num_graphs).astype(np.int32)
    u_src = uniform01(seed, 5, num_requests)
    req_source = np.minimum(np.floor(u_src * graph_n[req_graph]), graph_n[req_graph] - 1).astype(np.int32)
    u_t = uniform01(seed, 6, num_requests)
    gaps = -np.log1p(-u_t) / float(rate_per_s)
    req_arrival = np.cumsum(gaps)
    return ServingTrace(graph_n, graph_p, graph_seed, req_graph, req_source, req_arrival)


def single_source(n: int, seed: int) -> int:
    """The seed-derived source of a single-solve workload."""
    return int(sources(n, 1, seed)[0])


# The five workload shapes, by name (sizes, densities, weights and seeds).
WORKLOADS = {
    "dense_n1024_p0.1": dict(kind="bernoulli", n=1024, p=0.1, wlo=1, whi=100, seed=1, source=0),
    "dense_n16384_p0.5": dict(kind="bernoulli", n=16384, p=0.5, wlo=1, whi=1000, seed=2, source=None),
    "sparse_directed_n32768_deg8": dict(kind="outdeg", n=32768, d=8, wlo=1, whi=10000, seed=3, source=None),
    "multisource_n8192_p0.05_k256": dict(kind="bernoulli", n=8192, p=0.05, wlo=1, whi=1000, seed=4, k=256),
    "serving_64graphs_10000req": dict(kind="serving", graphs=64, requests=10000, wlo=1, whi=1000, seed=5),
    # a smaller dense case of the same shape for profiler captures (256 MiB matrix, still larger than L2)
    "dense_n8192_p0.5": dict(kind="bernoulli", n=8192, p=0.5, wlo=1, whi=1000, seed=6, source=None),
}


def make_graph(spec: dict) -> EdgeList:
    if spec["kind"] == "bernoulli":
        return bernoulli(spec["n"], spec["p"], spec["wlo"], spec["whi"], spec["seed"])
    if spec["kind"] == "outdeg":
        return outdeg(spec["n"], spec["d"], spec["wlo"], spec["whi"], spec["seed"])
    raise ValueError(spec["kind"])


def workload_source(spec: dict) -> int:
    if spec.get("source") is not None:
        return int(spec["source"])
    return single_source(spec["n"], spec["seed"])


__all__ = ["EdgeList", "ServingTrace", "WORKLOADS", "bernoulli", "outdeg", "sources", "uniform01",
           "bounded", "random_edges", "serving_trace", "single_source", "make_graph",
           "workload_source", "build"]
