"""CPU oracle for dense adjacency-matrix Dijkstra -- TEST INFRASTRUCTURE ONLY.

Plain serial C restatement of the paper's Algorithm 1 (Section III-A) and of
its edge-list-to-matrix input step, wrapped for numpy.  Only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference legs
may import this package.  It never imports the CUDA library, and the CUDA
library never calls it.

Every function here is pinned by the ``-m "not gpu"`` tests against things
other than itself: the paper's worked 4-node matrices, Floyd-Warshall and
Bellman-Ford brute force, a library shortest-path routine, the shortest-path
optimality invariants, and a closed form for the predecessor tree.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

INF = np.int32(2**31 - 1)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dijkstra_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no vector intrinsics)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-pthread", _SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            lib.orc_build_matrix.restype = ctypes.c_int
            lib.orc_build_matrix.argtypes = [i32, i64, p, p, p, ctypes.c_int, i64, p]
            lib.orc_dijkstra.restype = None
            lib.orc_dijkstra.argtypes = [i32, p, i64, i32, p, p]
            lib.orc_dijkstra_many.restype = None
            lib.orc_dijkstra_many.argtypes = [i32, p, i64, i32, p, p, p]
            lib.orc_dijkstra_many_mt.restype = ctypes.c_int32
            lib.orc_dijkstra_many_mt.argtypes = [i32, p, i64, i32, p, p, p, i32]
            _lib = lib
        return _lib


def _c(a: np.ndarray, dtype=np.int32) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def build_matrix(n: int, src, dst, w, directed: bool) -> np.ndarray:
    """Edge list -> n x n int32 matrix: INF = no edge, diagonal 0, repeats keep the minimum."""
    src, dst, w = _c(src), _c(dst), _c(w)
    m = src.shape[0]
    if dst.shape[0] != m or w.shape[0] != m:
        raise ValueError("edge arrays differ in length")
    G = np.empty((n, n), dtype=np.int32)
    rc = _load().orc_build_matrix(n, m, _ptr(src), _ptr(dst), _ptr(w), int(bool(directed)), n, _ptr(G))
    if rc != 0:
        raise ValueError("edge list holds an id outside [0, n) or an invalid weight")
    return G


def dijkstra(G: np.ndarray, s: int):
    """Algorithm 1 from source s; returns (dist, pred), int32 arrays of length n."""
    G = _c(G)
    n = G.shape[0]
    if G.ndim != 2 or G.shape[1] < n:
        raise ValueError("G must be n x ld with ld >= n")
    if not 0 <= s < n:
        raise ValueError("source out of range")
    dist = np.empty(n, dtype=np.int32)
    pred = np.empty(n, dtype=np.int32)
    _load().orc_dijkstra(n, _ptr(G), G.shape[1], int(s), _ptr(dist), _ptr(pred))
    return dist, pred


def dijkstra_many(G: np.ndarray, sources):
    """Algorithm 1 for each source in turn; returns (dist, pred) of shape (k, n)."""
    G = _c(G)
    n = G.shape[0]
    s = _c(sources)
    if s.size and (s.min() < 0 or s.max() >= n):
        raise ValueError("source out of range")
    k = s.shape[0]
    dist = np.empty((k, n), dtype=np.int32)
    pred = np.empty((k, n), dtype=np.int32)
    _load().orc_dijkstra_many(n, _ptr(G), G.shape[1], k, _ptr(s), _ptr(dist), _ptr(pred))
    return dist, pred


def dijkstra_many_threads(G: np.ndarray, sources, threads: int = 0):
    """dijkstra_many with the independent solves spread over host threads (0 = every core).
    Returns (dist, pred, threads_used); each solve is the same serial Algorithm 1."""
    G = _c(G)
    n = G.shape[0]
    s = _c(sources)
    if s.size and (s.min() < 0 or s.max() >= n):
        raise ValueError("source out of range")
    k = s.shape[0]
    if threads <= 0:
        threads = os.cpu_count() or 1
    dist = np.empty((k, n), dtype=np.int32)
    pred = np.empty((k, n), dtype=np.int32)
    used = _load().orc_dijkstra_many_mt(n, _ptr(G), G.shape[1], k, _ptr(s), _ptr(dist), _ptr(pred), int(threads))
    return dist, pred, int(used)


__all__ = ["INF", "build", "build_matrix", "dijkstra", "dijkstra_many", "dijkstra_many_threads"]
