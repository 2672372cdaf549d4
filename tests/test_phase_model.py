"""CPU model of the rules the GPU kernels use to settle many nodes per phase.

Not the oracle and not the product: a plain numpy restatement of the phase
logic, checked against the oracle's Algorithm 1 (Section III-A) on many small
random graphs full of equal weights.  Per phase it takes m = the smallest
unvisited dist (argmin a, smallest index), the OUT bound L = min over unvisited
u of dist[u] + minout[u] (capped at m + span), and -- when every off-diagonal
weight is >= 1 -- the IN bound dist[v] <= m + minin[v]; settles S; relaxes
every column with the lexicographic key (dist[u] + G[u][v], dist[u], u) over
u in S (the diagonal included, as the kernels read whole rows); and commits a
strictly smaller dist, or (IN bound on) an equal dist from a smaller (dist[u], u)
than the stored (dist[pred], pred).  It also checks, phase by phase, the
shortcuts the kernels take on top of that:
  - column filter: a column whose stored dist is below max(L, m + minin[v])
    never changes, and one equal to it changes only if its stored tie can be
    beaten;
  - tie sources: a tie-only column at m + minin[v] is decided by the rows u
    with G[u][v] == minin[v] and dist[u] == m alone (the smallest such u);
  - columns as rows: on an undirected graph column v of G is row v.
"""
import numpy as np
import pytest

INF = 2**31 - 1


def _bits(n: int) -> int:
    b = 1
    while b < 31 and (1 << b) < n:
        b += 1
    return b


def _span(n: int) -> int:
    return (1 << (32 - _bits(n))) - 1


def _best_keys(G, rows, du):
    """Per column, the lexicographic minimum of (du[i] + G[rows[i], v], du[i], rows[i])."""
    c = du[:, None] + G[rows, :]
    best_c = c.min(axis=0)
    at = c == best_c[None, :]
    best_d = np.where(at, du[:, None], np.iinfo(np.int64).max).min(axis=0)
    at &= du[:, None] == best_d[None, :]
    best_u = np.where(at, rows[:, None], np.iinfo(np.int64).max).min(axis=0)
    return best_c, best_d, best_u


K_LIST = 4  # in-/out-edges listed per node for the dynamic bounds


def _lists(off, axis):
    """Per node the K_LIST smallest finite off-diagonal weights (with the other endpoint) along
    `axis` (0: a column's in-edges, 1: a row's out-edges), ascending by (weight, endpoint), and the
    lower bound on the rest: the K_LIST-th weight if there are more, else INF."""
    n = off.shape[0]
    lw = np.full((n, K_LIST), INF, dtype=np.int64)
    lu = np.full((n, K_LIST), -1, dtype=np.int64)
    rest = np.full(n, INF, dtype=np.int64)
    for v in range(n):
        vals = off[:, v] if axis == 0 else off[v, :]
        ends = np.flatnonzero(vals < INF)
        order = np.lexsort((ends, vals[ends]))
        ends = ends[order]
        for i, u in enumerate(ends[:K_LIST]):
            lw[v, i], lu[v, i] = vals[u], u
        if ends.size > K_LIST:
            rest[v] = lw[v, K_LIST - 1]
    return lw, lu, rest


def phase_model(G, s, stats=None, dynamic=0):
    """dynamic: 0 static minima; 1 the IN bound from the smallest in-weight of rows not yet
    settled; 2 the OUT bound too from the smallest out-weight to columns not yet settled.  As in
    the kernel, a node counts as settled for these minima only from two phases on (the phase stamps
    of the previous phase are not yet visible to every CTA), the lists hold K_LIST entries and a
    cursor moves at most one entry per phase."""
    G = np.asarray(G, dtype=np.int64)
    n = G.shape[0]
    idx = np.arange(n)
    off = G.copy()
    off[idx, idx] = INF
    minout, minin = off.min(axis=1), off.min(axis=0)
    minin_static = minin.copy()
    fin = off[off < INF]
    use_in = fin.size == 0 or fin.min() >= 1
    span = _span(n)
    sym = bool((G == G.T).all())
    dist = np.full(n, INF, dtype=np.int64)
    pred = np.full(n, -1, dtype=np.int64)
    pdist = np.full(n, INF, dtype=np.int64)
    vis = np.zeros(n, dtype=bool)
    dist[s] = 0
    dyn = dynamic and use_in
    if dyn:
        ilw, ilu, irest = _lists(off, 0)
        olw, olu, orest = _lists(off, 1)
        k_in = np.zeros(n, dtype=np.int64)
        k_out = np.zeros(n, dtype=np.int64)
        stamp = np.full(n, INF, dtype=np.int64)  # phase + 1 of the node's settlement
        stamp[s] = 0
    phase = 0
    while True:
        U = ~vis
        if not U.any():
            break
        m = dist[U].min()
        if m >= INF:
            break
        a = np.flatnonzero(U & (dist == m))[0]
        L = min((dist[U] + minout[U]).min(), m + span, INF)
        ik = np.where(dist > minin, dist - minin, 0)
        S = U & ((dist < L) | (idx == a) | (use_in & (dist < INF) & (ik <= m) & (dist - m < span)))
        rows = np.flatnonzero(S)
        bc, bd, bu = _best_keys(G, rows, dist[rows])
        strict = bc < dist
        tie = (use_in & (bc == dist) & (dist < INF) & (pred >= 0) &
               ((bd < pdist) | ((bd == pdist) & (bu < pred))))
        commit = strict | tie

        # the dynamic minima really bound what the phase's rows offer: every row of S (unsettled at
        # the phase start) offers column v at least minin[v]; the OUT term bounds unsettled columns
        if dyn:
            assert (off[np.ix_(rows, idx)] >= minin[None, :]).all(), "an offer below the dynamic IN weight"
            if dynamic == 2:
                assert (off[np.ix_(rows, np.flatnonzero(U))] >= minout[rows][:, None]).all()

        # column filter: nothing outside the live columns can commit (with the dynamic OUT bound too:
        # a settled column can only take a tie, and no row whose out-minimum skips it can tie it)
        bound = np.maximum(L, m + minin) if use_in else np.full(n, L)
        stored_tie_beatable = use_in & (pred >= 0) & (pdist >= m) | (dist >= INF)
        live = ~(vis & (dist >= INF)) & ((dist > bound) | ((dist == bound) & stored_tie_beatable))
        assert not (commit & ~live).any(), "a column outside the filter changed"

        # tie sources: tie-only columns at m + minin[v] need only rows of weight minin[v] at dist m
        # (the kernels use them while the column's IN weight is still the static one)
        if use_in:
            tie_only = live & (dist == bound) & (dist < INF) & (dist == m + minin) & (minin == minin_static)
            for v in np.flatnonzero(tie_only):
                assert not strict[v]
                src = [u for u in range(n) if u != v and off[u, v] == minin[v]]
                at_m = [u for u in src if S[u] and dist[u] == m]
                got = min(at_m) if at_m else None
                if commit[v]:
                    assert got is not None and (bc[v], bd[v], bu[v]) == (dist[v], m, got)
                else:
                    assert got is None or (m, got) >= (pdist[v], pred[v])
                if stats is not None:
                    stats["tie_only"] += 1

        # columns as rows: an undirected graph's column v is its row v
        if sym:
            assert (G[:, rows].T == G[rows, :]).all()

        dist = np.where(commit, bc, dist)
        pdist = np.where(commit, bd, pdist)
        pred = np.where(commit, bu, pred)
        vis |= S
        if dyn:  # the kernel's per-phase update: one list entry checked per node
            stamp[S] = phase + 1
            for v in np.flatnonzero(~vis):
                k = k_in[v]
                if k < K_LIST and ilw[v, k] < INF and stamp[ilu[v, k]] <= phase:
                    k_in[v] = k + 1
                    minin[v] = ilw[v, k + 1] if k + 1 < K_LIST else irest[v]
                    if stats is not None:
                        stats["dyn_updates"] = stats.get("dyn_updates", 0) + 1
                if dynamic == 2:
                    k = k_out[v]
                    if k < K_LIST and olw[v, k] < INF and stamp[olu[v, k]] <= phase:
                        k_out[v] = k + 1
                        minout[v] = olw[v, k + 1] if k + 1 < K_LIST else orest[v]
                        if stats is not None:
                            stats["dyn_updates"] = stats.get("dyn_updates", 0) + 1
        phase += 1
        if stats is not None:
            stats["phases"] += 1
    return dist.astype(np.int32), pred.astype(np.int32)


def _random_graph(rng, n, p, wlo, whi, directed):
    G = np.full((n, n), INF, dtype=np.int64)
    mask = rng.random((n, n)) < p
    w = rng.integers(wlo, whi + 1, size=(n, n))
    G[mask] = w[mask]
    if not directed:
        G = np.minimum(G, G.T)
    np.fill_diagonal(G, 0)
    return G.astype(np.int32)


@pytest.mark.parametrize("dynamic", [0, 1, 2], ids=["static", "dynamic_in", "dynamic_in_out"])
@pytest.mark.parametrize("directed", [False, True], ids=["undirected", "directed"])
def test_phase_rules_match_algorithm_1(orc, directed, dynamic):
    rng = np.random.default_rng(20260504 + int(directed))
    stats = {"phases": 0, "tie_only": 0}
    nodes = 0
    ranges = [(1, 1), (1, 2), (1, 3), (0, 2), (1, 10), (5, 6), (1, 1000)]
    for trial in range(240):
        n = int(rng.integers(2, 48))
        p = float(rng.choice([0.05, 0.2, 0.5, 0.9, 1.0]))
        wlo, whi = ranges[trial % len(ranges)]
        G = _random_graph(rng, n, p, wlo, whi, directed)
        s = int(rng.integers(0, n))
        d_ref, p_ref = orc.dijkstra(G, s)
        nodes += int((d_ref < INF).sum())
        d, pr = phase_model(G, s, stats, dynamic)
        assert np.array_equal(d, d_ref), (trial, n, p, wlo, whi, s)
        assert np.array_equal(pr, p_ref), (trial, n, p, wlo, whi, s)
    # the shortcuts were exercised, and phases settled many nodes at once
    assert stats["tie_only"] > 30
    assert stats["phases"] < 0.75 * nodes
    if dynamic:
        assert stats.get("dyn_updates", 0) > 40  # the dynamic minima did move
