"""Independent checks that pin the oracle, and property checks for any result.

Nothing here restates Algorithm 1's loop.  The references are:
  * Floyd-Warshall (all pairs, triple loop over intermediates) and Bellman-Ford
    (n-1 rounds of relaxing every edge): brute-force shortest distances.
  * scipy.sparse.csgraph.dijkstra: a library shortest-path routine.
  * BFS levels: the unit-weight special case.
  * The predecessor closed form.  With every off-diagonal weight >= 1,
    Algorithm 1 visits nodes in (final distance, index) order and sets pred[v]
    once, from the first visited u that reaches dist[v]; strict improvement
    keeps it.  So pred[v] is the u != v minimising (dist[u], u) among
    {u : dist[u] + G[u][v] == dist[v]}, and pred of the source and of
    unreachable nodes is -1.
  * The optimality invariants: dist[s] == 0; dist[v] <= dist[u] + G[u][v] on
    every edge out of a reachable u; each reachable v != s has
    dist[pred[v]] + G[pred[v]][v] == dist[v]; following pred reaches s.
"""
from __future__ import annotations

import os

import numpy as np

INF = 2**31 - 1
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------------------- golden files

def _tok(x: str) -> int:
    return INF if x == "inf" else int(x)


def parse_golden(name: str) -> dict:
    """Parse a fixture: 'edges' block, 'matrix <name>' blocks, 'expect' lines."""
    out = {"edges": None, "matrices": {}, "expect": []}
    lines = [ln.split("#", 1)[0].strip() for ln in open(os.path.join(GOLDEN, name))]
    lines = [ln for ln in lines if ln]
    i = 0
    while i < len(lines):
        ln = lines[i]
        if ln == "edges":
            rows = []
            i += 1
            while lines[i] != "end":
                rows.append([int(t) for t in lines[i].split()])
                i += 1
            out["edges"] = np.array(rows, dtype=np.int32)
        elif ln.startswith("matrix "):
            name_ = ln.split()[1]
            rows = []
            i += 1
            while lines[i] != "end":
                rows.append([_tok(t) for t in lines[i].split()])
                i += 1
            out["matrices"][name_] = np.array(rows, dtype=np.int64).astype(np.int32)
        elif ln.startswith("expect "):
            head, rest = ln[len("expect "):].split(":", 1)
            gname, src = head.split()
            d, p = rest.split("|")
            out["expect"].append((gname, int(src), np.array([_tok(t) for t in d.split()], dtype=np.int64).astype(np.int32),
                                  np.array([int(t) for t in p.split()], dtype=np.int32)))
        i += 1
    return out


# ----------------------------------------------------------------------------- brute force

def floyd_warshall(G: np.ndarray) -> np.ndarray:
    """All-pairs shortest distances by the triple loop over intermediates (int64, INF kept)."""
    n = G.shape[0]
    big = np.int64(1) << 50
    D = G.astype(np.int64)
    D[D == INF] = big
    np.fill_diagonal(D, np.minimum(np.diagonal(D), 0))
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    D[D >= big] = INF
    return D


def bellman_ford(G: np.ndarray, s: int) -> np.ndarray:
    """Single-source distances by n-1 rounds over every edge (plain Python)."""
    n = G.shape[0]
    edges = [(u, v, int(G[u, v])) for u in range(n) for v in range(n) if u != v and G[u, v] != INF]
    dist = [INF] * n
    dist[s] = 0
    for _ in range(max(n - 1, 1)):
        changed = False
        for u, v, w in edges:
            if dist[u] != INF and dist[u] + w < dist[v]:
                dist[v] = dist[u] + w
                changed = True
        if not changed:
            break
    return np.array(dist, dtype=np.int64)


def scipy_distances(G: np.ndarray, s: int) -> np.ndarray:
    """scipy's Dijkstra on the same matrix (INF = non-edge, diagonal dropped)."""
    from scipy.sparse.csgraph import csgraph_from_dense, dijkstra as sp_dijkstra
    H = G.astype(np.float64)
    H[G == INF] = np.inf
    np.fill_diagonal(H, np.inf)
    cs = csgraph_from_dense(H, null_value=np.inf)
    d = sp_dijkstra(cs, directed=True, indices=s)
    out = np.full(G.shape[0], INF, dtype=np.int64)
    fin = np.isfinite(d)
    out[fin] = np.rint(d[fin]).astype(np.int64)
    return out


def bfs_levels(G: np.ndarray, s: int) -> np.ndarray:
    """Hop counts from s over the finite off-diagonal entries (plain queue BFS)."""
    n = G.shape[0]
    lvl = np.full(n, INF, dtype=np.int64)
    lvl[s] = 0
    frontier = [s]
    while frontier:
        nxt = []
        for u in frontier:
            for v in np.nonzero((G[u] != INF))[0]:
                if v != u and lvl[v] == INF:
                    lvl[v] = lvl[u] + 1
                    nxt.append(int(v))
        frontier = nxt
    return lvl


def pred_closed_form(G: np.ndarray, s: int, dist: np.ndarray, chunk: int = 1024) -> np.ndarray:
    """pred[v] = argmin over (dist[u], u) of {u != v : dist[u] + G[u][v] == dist[v]} (weights >= 1)."""
    n = G.shape[0]
    d = dist.astype(np.int64)
    pred = np.full(n, -1, dtype=np.int32)
    # order the candidates by (dist[u], u) and keep the first hit per column
    order = np.lexsort((np.arange(n), d))
    order = order[d[order] != INF]
    best_rank = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
    for c0 in range(0, order.size, chunk):
        rows = order[c0:c0 + chunk]
        W = G[rows].astype(np.int64)
        cand = d[rows][:, None] + W
        hit = (W != INF) & (cand == d[None, :]) & (rows[:, None] != np.arange(n)[None, :])
        ranks = np.where(hit, (c0 + np.arange(rows.size))[:, None], np.iinfo(np.int64).max)
        best_rank = np.minimum(best_rank, ranks.min(axis=0))
    has = best_rank != np.iinfo(np.int64).max
    pred[has] = order[best_rank[has]]
    pred[s] = -1
    pred[d == INF] = -1
    return pred


# ----------------------------------------------------------------------------- invariants

def check_invariants(G: np.ndarray, s: int, dist: np.ndarray, pred: np.ndarray, chunk: int = 2048) -> list:
    """Return a list of violated properties (empty when the result is a shortest-path tree)."""
    errs = []
    n = G.shape[0]
    d = dist.astype(np.int64)
    p = pred.astype(np.int64)
    if d[s] != 0:
        errs.append("dist[s] != 0")
    if p[s] != -1:
        errs.append("pred[s] != -1")
    reach = d != INF
    # edge optimality, chunked over source rows
    for r0 in range(0, n, chunk):
        rows = np.arange(r0, min(n, r0 + chunk))
        rows = rows[reach[rows]]
        if rows.size == 0:
            continue
        W = G[rows].astype(np.int64)
        fin = W != INF
        viol = fin & (d[rows][:, None] + W < d[None, :])
        if viol.any():
            errs.append(f"edge optimality violated ({int(viol.sum())} edges)")
            break
    # predecessor consistency
    others = np.nonzero(reach & (np.arange(n) != s))[0]
    if others.size:
        pu = p[others]
        if (pu < 0).any() or (pu >= n).any():
            errs.append("reachable node without a valid pred")
        else:
            w = G[pu, others].astype(np.int64)
            if ((w == INF) | (d[pu] + w != d[others])).any():
                errs.append("pred edge does not attain dist")
    if (p[~reach] != -1).any():
        errs.append("unreachable node has a pred")
    # the pred graph reaches s from every reachable node (no cycles)
    if not errs and others.size:
        cur = others.copy()
        for _ in range(n):
            cur = cur[cur != s]
            if cur.size == 0:
                break
            cur = p[cur]
        if cur.size and (cur != s).any():
            errs.append("pred graph has a cycle")
    return errs


# ----------------------------------------------------------------------------- small random graphs

def random_matrix(rng: np.random.Generator, n: int, density: float, weights, directed: bool) -> np.ndarray:
    """A small dense-stored matrix with weights drawn from the given values (INF off-edges)."""
    G = np.full((n, n), INF, dtype=np.int64)
    mask = rng.random((n, n)) < density
    vals = rng.choice(np.asarray(weights, dtype=np.int64), size=(n, n))
    G[mask] = vals[mask]
    if not directed:
        iu = np.triu_indices(n, 1)
        G[(iu[1], iu[0])] = G[iu]
    np.fill_diagonal(G, 0)
    return G.astype(np.int32)


# ----------------------------------------------------------------------------- the pin suite

def run_pin_suite(build_matrix, dijkstra, quick: bool = False) -> list:
    """Run every pin against a (build_matrix, dijkstra) pair; return the failures.

    ``build_matrix(n, src, dst, w, directed) -> G`` and ``dijkstra(G, s) -> (dist, pred)``.
    Used on the oracle (expect no failures) and on deliberately broken copies of
    it (expect at least one failure each).
    """
    fails = []

    def eq(a, b):
        return np.array_equal(np.asarray(a, dtype=np.int64), np.asarray(b, dtype=np.int64))

    # 1. the paper's worked matrices: the fill step and every source
    g = parse_golden("worked_4node.txt")
    e = g["edges"]
    for kind, directed in (("undirected", False), ("directed", True)):
        G = build_matrix(4, e[:, 0], e[:, 1], e[:, 2], directed)
        if not eq(G, g["matrices"][kind]):
            fails.append(f"worked matrix fill ({kind})")
    for kind, s, dist, pred in g["expect"]:
        d, p = dijkstra(g["matrices"][kind], s)
        if not (eq(d, dist) and eq(p, pred)):
            fails.append(f"worked {kind} source {s}")
    # 2. the padded example
    g = parse_golden("padded_6node.txt")
    for kind, s, dist, pred in g["expect"]:
        d, p = dijkstra(g["matrices"][kind], s)
        if not (eq(d, dist) and eq(p, pred)):
            fails.append(f"padded source {s}")
    # 3. exhaustive: every directed 3-node graph with off-diagonal weights in {1, 2, inf}
    vals = (1, 2, INF)
    off = [(i, j) for i in range(3) for j in range(3) if i != j]
    import itertools
    for combo in itertools.product(vals, repeat=len(off)):
        G = np.zeros((3, 3), dtype=np.int32)
        for (i, j), w in zip(off, combo):
            G[i, j] = w
        D = floyd_warshall(G)
        for s in range(3):
            d, p = dijkstra(G, s)
            if not eq(d, D[s]) or not eq(p, pred_closed_form(G, s, D[s])):
                fails.append(f"exhaustive n=3 {combo} s={s}")
                break
        if len(fails) > 8:
            return fails
    # 4. random small graphs: ties, wide weights, directed and undirected, unreachable parts
    rng = np.random.default_rng(20250403)
    trials = 40 if quick else 160
    for t in range(trials):
        n = int(rng.integers(1, 41))
        directed = bool(t % 2)
        weights = (1, 2, 3) if t % 3 == 0 else tuple(range(1, 1000, 7))
        G = random_matrix(rng, n, float(rng.uniform(0.05, 0.6)), weights, directed)
        D = floyd_warshall(G)
        s = int(rng.integers(0, n))
        d, p = dijkstra(G, s)
        if not eq(d, D[s]):
            fails.append(f"random n={n} dist vs Floyd-Warshall")
        elif not eq(p, pred_closed_form(G, s, D[s])):
            fails.append(f"random n={n} pred vs closed form")
        elif check_invariants(G, s, d, p):
            fails.append(f"random n={n} invariants")
    # 5. zero weights allowed: distances and a valid tree
    for t in range(20):
        n = int(rng.integers(2, 25))
        G = random_matrix(rng, n, 0.3, (0, 0, 1, 2), bool(t % 2))
        D = floyd_warshall(G)
        d, p = dijkstra(G, 0)
        if not eq(d, D[0]) or check_invariants(G, 0, d, p):
            fails.append(f"zero-weight n={n}")
    # 6. Bellman-Ford on tiny graphs
    for t in range(20):
        n = int(rng.integers(2, 12))
        G = random_matrix(rng, n, 0.4, (1, 5, 9), True)
        s = int(rng.integers(0, n))
        if not eq(dijkstra(G, s)[0], bellman_ford(G, s)):
            fails.append(f"Bellman-Ford n={n}")
    # 7. library routine at a medium size
    for t in range(2 if quick else 4):
        n = 300
        G = random_matrix(rng, n, 0.05, tuple(range(1, 100)), bool(t % 2))
        s = int(rng.integers(0, n))
        d, p = dijkstra(G, s)
        if not eq(d, scipy_distances(G, s)):
            fails.append("scipy distances")
        elif not eq(p, pred_closed_form(G, s, d)):
            fails.append("scipy-size pred closed form")
    # 8. special cases
    G = random_matrix(rng, 60, 0.08, (1,), False)            # unit weights: BFS levels
    d, p = dijkstra(G, 0)
    if not eq(d, bfs_levels(G, 0)) or not eq(p, pred_closed_form(G, 0, d)):
        fails.append("unit weights vs BFS")
    n = 17
    G = np.full((n, n), 7, dtype=np.int32)                    # complete, equal weights
    np.fill_diagonal(G, 0)
    d, p = dijkstra(G, 5)
    if not (eq(np.delete(d, 5), np.full(n - 1, 7)) and eq(np.delete(p, 5), np.full(n - 1, 5))):
        fails.append("complete equal-weight graph")
    d, p = dijkstra(np.zeros((1, 1), dtype=np.int32), 0)       # single node
    if not (eq(d, [0]) and eq(p, [-1])):
        fails.append("single node")
    G = np.full((6, 6), INF, dtype=np.int32)                  # two components
    np.fill_diagonal(G, 0)
    G[0, 1] = G[1, 0] = 3
    G[1, 2] = G[2, 1] = 4
    G[3, 4] = G[4, 3] = 1
    d, p = dijkstra(G, 0)
    if not (eq(d, [0, 3, 7, INF, INF, INF]) and eq(p, [-1, 0, 1, -1, -1, -1])):
        fails.append("disconnected graph")
    # 9. the fill step: repeats keep the minimum, self-loops ignored, -w fills one direction
    src = np.array([0, 0, 2, 1, 1], dtype=np.int32)
    dst = np.array([1, 1, 2, 0, 2], dtype=np.int32)
    w = np.array([9, 4, 5, 6, 8], dtype=np.int32)
    G = build_matrix(3, src, dst, w, False)
    if not eq(G, [[0, 4, INF], [4, 0, 8], [INF, 8, 0]]):
        fails.append("undirected fill with repeats / self-loop")
    G = build_matrix(3, src, dst, w, True)
    if not eq(G, [[0, 4, INF], [6, 0, 8], [INF, INF, 0]]):
        fails.append("directed fill with repeats / self-loop")
    return fails
