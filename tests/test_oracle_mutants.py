"""The pins are strong enough: each plausible mistake planted in a copy of the oracle fails them.

Each mutant is a one-line textual change to oracle/dijkstra_oracle.c, compiled
on the CPU into a temporary library; the oracle itself is untouched.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import _pins as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dijkstra_oracle.c")

MUTANTS = {
    # relaxation keeps equal candidates (non-strict improvement)
    "relax_le": ("(int64_t)dist[u] + row[v] < (int64_t)dist[v]", "(int64_t)dist[u] + row[v] <= (int64_t)dist[v]"),
    # argmin takes the last index among equal distances
    "argmin_last": ("(u < 0 || dist[k] < dist[u])", "(u < 0 || dist[k] <= dist[u])"),
    # argmin forgets the visited mask
    "argmin_visited": ("if (!visited[k] && (u < 0", "if ((u < 0"),
    # 32-bit sum with the infinity guard dropped (wraps on INF + w)
    "no_inf_guard": ("row[v] != ORC_INF && (int64_t)dist[u] + row[v] < (int64_t)dist[v]",
                     "(int32_t)((uint32_t)dist[u] + (uint32_t)row[v]) < dist[v]"),
    # predecessor written with the wrong node
    "pred_v": ("pred[v] = u;", "pred[v] = v;"),
    # source distance never set
    "no_source": ("dist[s] = 0;", "dist[s] = dist[s];"),
    # weight added twice (a wrong term)
    "double_weight": ("dist[v] = (int32_t)((int64_t)dist[u] + row[v]);",
                      "dist[v] = (int32_t)((int64_t)dist[u] + 2 * (int64_t)row[v]);"),
    # fill: undirected input written one way only
    "fill_one_way": ("if (!directed && x < G[(int64_t)v * ld + u])", "if (0 && x < G[(int64_t)v * ld + u])"),
    # fill: repeated pairs keep the last weight instead of the minimum
    "fill_last": ("if (x < G[(int64_t)u * ld + v]) G[(int64_t)u * ld + v] = x;", "G[(int64_t)u * ld + v] = x;"),
    # fill: self-loops overwrite the diagonal
    "fill_selfloop": ("if (u == v) continue;", "if (u == v) { G[(int64_t)u * ld + v] = x; continue; }"),
    # transposed operand: relax reads column u instead of row u
    "transposed": ("const int32_t* row = G + (int64_t)u * ld;", "const int32_t* row = G + u; ld = ld;"),
}


def _compile(tmp_path, name, a, b):
    text = open(SRC).read()
    assert text.count(a) == 1, name
    text = text.replace(a, b)
    if name == "transposed":
        text = text.replace("row[v]", "row[(int64_t)v * ld]")
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(text)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", str(c), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.orc_build_matrix.restype = ctypes.c_int
    lib.orc_build_matrix.argtypes = [i32, i64, p, p, p, ctypes.c_int, i64, p]
    lib.orc_dijkstra.argtypes = [i32, p, i64, i32, p, p]
    return lib


def _wrap(lib):
    def build(n, src, dst, w, directed):
        src, dst, w = (np.ascontiguousarray(x, dtype=np.int32) for x in (src, dst, w))
        G = np.empty((n, n), dtype=np.int32)
        rc = lib.orc_build_matrix(n, src.size, src.ctypes.data, dst.ctypes.data, w.ctypes.data,
                                  int(directed), n, G.ctypes.data)
        if rc:
            raise ValueError
        return G

    def dijkstra(G, s):
        G = np.ascontiguousarray(G, dtype=np.int32)
        n = G.shape[0]
        d = np.empty(n, dtype=np.int32)
        p = np.empty(n, dtype=np.int32)
        lib.orc_dijkstra(n, G.ctypes.data, G.shape[1], s, d.ctypes.data, p.ctypes.data)
        return d, p

    return build, dijkstra


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    a, b = MUTANTS[name]
    build, dijkstra = _wrap(_compile(tmp_path, name, a, b))
    fails = P.run_pin_suite(build, dijkstra, quick=True)
    assert fails, f"mutant {name} passed every pin"
