// Shared device routines of the solve engines.
//
// Every CTA owns a contiguous slice of columns (nodes) of one solve and keeps
// that slice's dist / pred / visited / row-minimum state in shared memory for
// the whole solve.  One *phase* is:
//
//   1. each CTA reduces its slice to a partial  (argmin key, L_c) and publishes
//      the candidates  {unvisited v : dist[v] < L_c} u {its argmin};
//   2. one barrier (grid-wide or cluster-wide);
//   3. every CTA combines the partials into the global  m = min dist,
//      a = argmin (smallest index on ties)  and  L;  the settled set is
//      S = {unvisited v : dist[v] < L} u {a};
//   4. every CTA streams the rows u in S over its own columns and keeps, per
//      column v, the smallest key  (dist[u] + G[u][v], dist[u] - m, u);
//      a strictly smaller candidate than dist[v] replaces dist[v], pred[v].
//
// Algorithm 1 (Section III-A) is the special case S = {a} (DJ_MODE_PLAIN).
// The phase mode settles more nodes per pass but gives the same dist and pred:
//   - L = min over unvisited u of (dist[u] + minout[u]) is the "OUT" bound of
//     Crauser, Mehlhorn, Meyer and Sanders (MFCS 1998).  Every unvisited v with
//     dist[v] < L already holds its final distance, and all of them precede
//     every other unvisited node in Algorithm 1's visit order, which is
//     (final dist, index) among them.
//   - Within S, the first node in visit order that offers the smallest
//     candidate to v is the one with the smallest (dist[u], u); the key above
//     orders exactly that way, so the fused pass picks Algorithm 1's pred.
//   - A final (visited or settled) node can never be strictly improved, so the
//     relaxation needs no visited test (it is kept in the selection only).
//   - L is capped at m + 2^(32 - bits(n)) - 1 so (dist[u] - m, u) packs into
//     32 bits below all ones (reserved for "none"); a smaller L only shrinks
//     S, and S always contains a.
//   - With every off-diagonal weight >= 1, the "IN" criterion of the same
//     paper also settles v when dist[v] <= m + minin[v] (minin: the smallest
//     weight into v): the last edge of a shorter path would have to leave an
//     unvisited node, whose distance is >= m.  Such nodes are final but may be
//     settled before Algorithm 1 would visit them, so commits compare the full
//     key (candidate, dist[u], u) with the stored (dist[v], dist[pred[v]],
//     pred[v]); the surviving pred is the u of smallest (dist[u], u) offering
//     dist[v], which is the one Algorithm 1 keeps when weights are >= 1.
//   - Column filter: every u in S was unvisited when the phase began, so it
//     offers v at least max(L, m + minin[v]).  Columns whose stored dist is
//     below that bound cannot change this phase, and one equal to it can only
//     take a tie, from a row whose tie word is below the column's stored one.
//     A CTA whose slice has no such "live" column skips the relaxation; one
//     with few live columns loads only their 16-byte groups, and only from
//     the rows that can still win there (relax_gather).
// All sums are unsigned 32-bit: dist <= INF and G <= INF, so dist + G never
// wraps, and an INF entry yields a candidate >= INF that never improves.
#pragma once

#include "dj_common.cuh"

namespace dj {

// Grid-wide barrier on a monotonic arrival counter (zeroed before launch):
// arrival is a release reduction, waiting an acquire load, so no separate
// fences are needed.
// Bounded: after timeout_ns it records kErrTimeout, raises the launch's abort
// flag and returns false; CTAs already waiting see the flag and leave too.
__device__ __forceinline__ bool grid_barrier(uint32_t* bar, uint32_t target, uint32_t* abort_flag, uint32_t* err,
                                             int64_t timeout_ns, uint32_t* s_flag, uint64_t* stamps = nullptr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: every write of this CTA ordered before the bar.sync above is
    // visible to a CTA whose acquire load observes the arrival
    red_add_release_gpu(bar, 1u);
    if (stamps) stamps[0] = global_ns();
    uint32_t ok = 1;
    if (static_cast<int32_t>(ld_acquire_gpu(bar) - target) < 0) {
      const uint64_t t0 = global_ns();
      uint32_t spins = 0;
      while (static_cast<int32_t>(ld_acquire_gpu(bar) - target) < 0) {
        if ((++spins & 63u) == 0) {
          if (ld_relaxed_gpu(abort_flag)) {
            ok = 0;
            break;
          }
          if (static_cast<int64_t>(global_ns() - t0) > timeout_ns) {
            atomicOr(err, kErrTimeout);
            atomicExch(abort_flag, 1u);
            ok = 0;
            break;
          }
        }
      }
    }
    if (ok && ld_relaxed_gpu(abort_flag)) ok = 0;
    if (stamps) stamps[1] = global_ns();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}


// The region (publishing CTA) of entry i of a phase's candidate list: the
// largest r with off[r] <= i < off[r + 1] (off: prefix of the regions'
// counts).  Branch-free fixed-depth search (nreg <= 512).
__device__ __forceinline__ int region_of(const uint32_t* off, int nreg, int i) {
  int lo = 0;
#pragma unroll
  for (int step = 256; step >= 1; step >>= 1) {
    const int c = lo + step;
    lo = (c < nreg && static_cast<int>(off[min(c, nreg - 1)]) <= i) ? c : lo;
  }
  return lo;
}

// region_of for a cluster's lists (nreg <= 16).
__device__ __forceinline__ int region_of16(const uint32_t* off, int nreg, int i) {
  int lo = 0;
#pragma unroll
  for (int step = 8; step >= 1; step >>= 1) {
    const int c = lo + step;
    lo = (c < nreg && static_cast<int>(off[min(c, nreg - 1)]) <= i) ? c : lo;
  }
  return lo;
}

// Chunk table of a candidate list: ctab[c] = region of entry 32 c.  Built by
// threads r < nreg in parallel from the prefix off; every chunk start lies in
// exactly one non-empty region.
__device__ __forceinline__ void build_chunk_table(const uint32_t* off, int nreg, uint32_t* ctab) {
  for (int r = threadIdx.x; r < nreg; r += blockDim.x) {
    const uint32_t a = off[r], b = off[r + 1];
    for (uint32_t c = (a + 31) >> 5; (c << 5) < b; ++c) ctab[c] = static_cast<uint32_t>(r);
  }
}

// region_of through the chunk table: a start region, then a walk past region
// ends (empty regions included) up to entry i.
__device__ __forceinline__ int region_at(const uint32_t* off, const uint32_t* ctab, int i) {
  int r = static_cast<int>(ctab[i >> 5]);
  while (static_cast<int>(off[r + 1]) <= i) ++r;
  return r;
}

struct BlockScratch {
  uint64_t r64[32];
  uint32_t r32[32];
  uint32_t r32b[32];
  uint32_t cnt[33];
  uint64_t b64;
  uint32_t b32;
  uint32_t pad;
};

// Column-slice state of one CTA (all shared memory).
struct Slice {
  uint32_t* dist;
  int32_t* pred;
  uint32_t* pdist;   // dist of pred[v] (the key's second field)
  uint32_t* minout;
  uint32_t* minin;   // the IN bound's in-weight of each column (dynamic: from rows still unsettled)
  uint8_t* vis;
  int c0;    // first column (node id) of the slice, a multiple of 4
  int sw;    // columns in the slice, a multiple of 4
  int nvec;  // sw / 4
};

// Global decision of one phase.
struct Decision {
  uint32_t m;     // smallest unvisited dist (kInf: done)
  uint32_t a;     // its node (smallest index on ties)
  uint32_t L;     // OUT bound: unvisited v with dist[v] < L are settled
  uint32_t span;  // packing span 2^(32 - bits(n)) - 1
  uint32_t use_in;
};

// IN key of a node: dist - minin (saturating); settled by IN when <= m.
__device__ __forceinline__ uint32_t in_key(uint32_t d, uint32_t minin) { return d > minin ? d - minin : 0u; }

__device__ __forceinline__ void slice_init(const Slice& s, int n, int source, const int32_t* minout_g,
                                           const int32_t* minin_g, bool need_minout, bool need_minin) {
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
    int v = s.c0 + j;
    bool real = v < n;
    s.dist[j] = (real && v == source) ? 0u : kInf;
    s.pdist[j] = (real && v == source) ? 0u : kInf;
    s.pred[j] = -1;
    s.vis[j] = real ? 0 : 1;  // padding columns never take part
    s.minout[j] = (real && need_minout) ? static_cast<uint32_t>(__ldg(minout_g + v)) : kInf;
    s.minin[j] = (real && need_minin) ? static_cast<uint32_t>(__ldg(minin_g + v)) : kInf;
  }
}

// slice_init with Algorithm 1's first step done at once: every node but the
// source is at INF, so the first pass settles exactly the source and relaxes
// its row -- dist[v] = G[s][v] with pred s wherever that is finite (the
// diagonal never improves the source's own 0).  The minima and the source
// row's entries are loaded together (one round trip instead of two); the
// caller synchronises the block before the state is used.
__device__ __forceinline__ void slice_init_source(const Slice& s, int n, int source, const int32_t* minout_g,
                                                  const int32_t* minin_g, bool need_minout, bool need_minin,
                                                  const int32_t* __restrict__ W, int64_t pitch) {
  const int32_t* row = W + static_cast<int64_t>(source) * pitch + s.c0;
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
    const int v = s.c0 + j;
    const bool real = v < n;
    const uint32_t mo = (real && need_minout) ? static_cast<uint32_t>(__ldg(minout_g + v)) : kInf;
    const uint32_t mi = (real && need_minin) ? static_cast<uint32_t>(__ldg(minin_g + v)) : kInf;
    const uint32_t w = (real && v != source) ? static_cast<uint32_t>(__ldg(row + j)) : kInf;
    const bool reached = w < kInf;
    s.dist[j] = (real && v == source) ? 0u : (reached ? w : kInf);
    s.pdist[j] = (real && (v == source || reached)) ? 0u : kInf;
    s.pred[j] = reached ? source : -1;
    s.vis[j] = (!real || v == source) ? 1 : 0;  // padding columns never take part; the source is settled
    s.minout[j] = mo;
    s.minin[j] = mi;
  }
}

// Block-wide min of (key64, val32); every thread gets the result.  Ends synced.
__device__ __forceinline__ void block_min2(uint64_t& k, uint32_t& l, BlockScratch* sc) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  k = warp_min_u64(k);
  l = warp_min_u32(l);
  if (lane == 0) {
    sc->r64[w] = k;
    sc->r32[w] = l;
  }
  __syncthreads();
  if (w == 0) {
    uint64_t kk = lane < nw ? sc->r64[lane] : kNoKey;
    uint32_t ll = lane < nw ? sc->r32[lane] : 0xFFFFFFFFu;
    kk = warp_min_u64(kk);
    ll = warp_min_u32(ll);
    if (lane == 0) {
      sc->b64 = kk;
      sc->b32 = ll;
    }
  }
  __syncthreads();
  k = sc->b64;
  l = sc->b32;
  __syncthreads();
}

// Settle bound of a CTA from its raw partial: no bound when nothing reachable
// is left; the argmin alone in plain mode; otherwise min(L_c, m + span, INF).
__device__ __forceinline__ uint32_t cap_bound(uint64_t key, uint32_t lc, uint32_t span, bool plain) {
  const uint32_t mc = static_cast<uint32_t>(key >> 32);
  if (mc >= kInf) return 0xFFFFFFFFu;
  if (plain) return mc;
  return min(min(lc, mc + span), kInf);
}

// Per-thread part of a slice's partial over the unvisited columns this thread
// visits: argmin key (dist << 32 | v), min(dist + minout), and their count.
struct Part {
  uint64_t key;
  uint32_t lc;
  uint32_t nu;
};

__device__ __forceinline__ void part_init(Part& pt) {
  pt.key = kNoKey;
  pt.lc = 0xFFFFFFFFu;
  pt.nu = 0;
}

__device__ __forceinline__ void column_partial(const Slice& s, int j, Part& pt) {
  if (!s.vis[j]) {
    const uint32_t d = s.dist[j];
    const uint64_t kj = (static_cast<uint64_t>(d) << 32) | static_cast<uint32_t>(s.c0 + j);
    pt.key = kj < pt.key ? kj : pt.key;
    pt.lc = min(pt.lc, d + s.minout[j]);  // <= 2^32 - 2: no wrap
    ++pt.nu;
  }
}

__device__ __forceinline__ void slice_partial(const Slice& s, Part& pt) {
  part_init(pt);
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) column_partial(s, j, pt);
}

// Step 1: reduce the per-thread partials to the slice's (key, L_c) and append
// the candidates {unvisited v : dist[v] < L_c} u {IN candidates} u {argmin} as
// (v, dist[v][, IN key]) to `out` (order irrelevant: the relaxation keys are order-free).  sc->cnt[32]
// must be zero on entry.  Returns the count; all threads get key, Lc, count.
__device__ __forceinline__ void put_entry(uint4* out, uint32_t v, uint32_t d, uint32_t ik, uint32_t, uint32_t) {
  *out = make_uint4(v, d, ik, 0u);
}
// 8-byte entry (cluster engine): v in the low bits_u bits, and above them v's
// smallest in-weight saturated to the field (all ones: look it up), so that a
// reader recomputes the IN key without a dependent global load.  Every finite
// weight fits: (n - 1) * max weight < 2^31 and n > 2^(bits_u - 1) give
// max weight < 2^(32 - bits_u).
__device__ __forceinline__ uint32_t minin_field_max(uint32_t bits_u) { return (1u << (32 - bits_u)) - 1u; }
__device__ __forceinline__ void put_entry(uint2* out, uint32_t v, uint32_t d, uint32_t, uint32_t minin,
                                          uint32_t bits_u) {
  *out = make_uint2(v | (min(minin, minin_field_max(bits_u)) << bits_u), d);
}
// The candidate (u, dist[u], IN key) of a packed 8-byte entry (IN key 0, unused,
// when the IN bound is off).
__device__ __forceinline__ uint4 unpack_entry(uint2 e, uint32_t bits_u, const int32_t* __restrict__ minin_g,
                                              bool use_in) {
  const uint32_t u = e.x & ((1u << bits_u) - 1u);
  if (!use_in) return make_uint4(u, e.y, 0u, 0u);
  uint32_t mi = e.x >> bits_u;
  if (mi == minin_field_max(bits_u)) mi = static_cast<uint32_t>(__ldg(minin_g + u));  // saturated: rare
  return make_uint4(u, e.y, in_key(e.y, mi), 0u);
}

template <class Entry>
__device__ __forceinline__ int publish_partial(const Slice& s, uint32_t span, bool plain, bool use_in,
                                               const Part& pt, Entry* out, BlockScratch* sc, uint64_t* key_out,
                                               uint32_t* Lc_out, uint32_t* unvis_out = nullptr,
                                               uint32_t bits_u = 0) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  uint64_t k = warp_min_u64(pt.key);
  uint32_t l = warp_min_u32(pt.lc);
  uint32_t nu = unvis_out ? warp_sum_u32(pt.nu) : 0u;
  if (lane == 0) {
    sc->r64[w] = k;
    sc->r32[w] = l;
    sc->r32b[w] = nu;
  }
  __syncthreads();
  k = kNoKey;
  l = 0xFFFFFFFFu;
  nu = 0;
  for (int i = 0; i < nw; ++i) {  // every thread reduces the warp results itself
    const uint64_t x = sc->r64[i];
    k = x < k ? x : k;
    l = min(l, sc->r32[i]);
    nu += sc->r32b[i];
  }
  if (unvis_out) *unvis_out = nu;
  const uint32_t Lc = cap_bound(k, l, span, plain);
  const uint32_t ac = static_cast<uint32_t>(k);
  const uint32_t mc = static_cast<uint32_t>(k >> 32);
  *key_out = k;
  *Lc_out = Lc;
  if (mc < kInf) {
    for (int j0 = 0; j0 < s.sw; j0 += blockDim.x) {
      const int j = j0 + threadIdx.x;
      bool p = false;
      uint32_t d = 0, ik = 0;
      if (j < s.sw && !s.vis[j]) {
        d = s.dist[j];
        ik = in_key(d, s.minin[j]);
        // a superset of this phase's settled nodes: the global m is <= mc
        p = d < Lc || static_cast<uint32_t>(s.c0 + j) == ac ||
            (use_in && !plain && d < kInf && ik <= mc && d - mc < span);
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, p);
      if (bal) {
        uint32_t pos = 0;
        if (lane == 0) pos = atomicAdd(&sc->cnt[32], static_cast<uint32_t>(__popc(bal)));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (p)
          put_entry(out + pos + __popc(bal & ((1u << lane) - 1u)), static_cast<uint32_t>(s.c0 + j), d, ik,
                    s.minin[j], bits_u);
      }
    }
  }
  __syncthreads();
  return static_cast<int>(sc->cnt[32]);
}

// Combine per-CTA partials (key, Lc) into the phase decision.
__device__ __forceinline__ Decision make_decision(uint64_t key, uint32_t Lc, uint32_t span, bool plain,
                                                 bool use_in) {
  Decision d;
  d.m = static_cast<uint32_t>(key >> 32);
  d.a = static_cast<uint32_t>(key);
  d.span = span;
  d.use_in = (use_in && !plain) ? 1u : 0u;
  if (d.m >= kInf) {
    d.m = kInf;
    d.L = 0;
  } else if (plain) {
    d.L = d.m;
  } else {
    d.L = min(min(Lc, d.m + span), kInf);
  }
  return d;
}

// Settled this phase: below the OUT bound, the argmin itself, or (weights >= 1)
// proven final by the IN bound while still packable.
__device__ __forceinline__ bool in_settled(uint32_t u, uint32_t du, uint32_t ik, const Decision& D) {
  return du < D.L || u == D.a || (D.use_in && du < kInf && ik <= D.m && du - D.m < D.span);
}

// Thread tile of the relaxation: warps split into `wpr` column chunks of
// 32*V vec4 each and `rgs` row groups; lane l of column chunk c owns the
// vec4 columns (c*V + k)*32 + l, k < V.
struct Tile {
  int rg, rgs, wc;
  bool active;
};

template <int V>
__device__ __forceinline__ Tile make_tile(int nvec, int rgs_cap) {
  Tile t;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int wpr = max(1, (nvec + 32 * V - 1) / (32 * V));
  t.rgs = max(1, min(nw / wpr, rgs_cap));
  t.rg = warp / wpr;
  t.wc = warp % wpr;
  t.active = t.rg < t.rgs;
  return t;
}

// A warp's ring of `depth` stages x U row slots in shared memory, filled by
// 1-D TMA bulk copies (one per row) that complete on the stage's mbarrier.
// Only this warp issues into and reads from its ring, so no other warp ever
// waits on it.  `gt` counts the warp's stages over the whole kernel: stage g
// uses slot g % depth and waits for parity (g / depth) & 1.
struct Ring {
  uint8_t* buf;
  uint64_t* bar;
  uint32_t depth;
  uint32_t srows;     // rows per stage (<= U)
  uint32_t rowbytes;  // bytes of this warp's column chunk of one row (0: idle warp)
  uint32_t gt;
};

// Per-column running best of one relaxation pass: candidate value bc and its
// tie-break word bt.  It starts at the column's stored key: (dist[v], the tie
// word of pred[v] relative to this phase), so a candidate commits only if it
// is lexicographically smaller -- a shorter distance, or the same distance
// offered by a node of smaller (dist, index).
template <int V>
struct Best {
  uint32_t bc[V][4];
  uint32_t bt[V][4];
};

// Tie word of column j's stored pred in this phase's packing: 0 when no
// candidate of the phase can tie-beat it (pred settled earlier, or the source),
// all ones when any can (unreached, or the pred's dist is beyond the span).
// Without the IN bound (some weight is 0, or plain mode) ties never commit:
// nodes are then settled in Algorithm 1's own order, where strict improvement
// is exactly its rule, while with zero weights a tie could even come from a
// node's own diagonal entry.
__device__ __forceinline__ uint32_t stored_tie(const Slice& s, int j, const Decision& D, uint32_t bits_u) {
  if (!D.use_in) return 0u;
  if (s.dist[j] >= kInf) return 0xFFFFFFFFu;
  const int32_t pr = s.pred[j];
  if (pr < 0) return 0u;
  const uint32_t pd = s.pdist[j];
  if (pd < D.m) return 0u;
  const uint32_t dd = pd - D.m;
  if (dd >= D.span) return 0xFFFFFFFFu;
  return (dd << bits_u) | static_cast<uint32_t>(pr);
}

template <int V>
__device__ __forceinline__ void best_init(Best<V>& b, const Slice& s, const Tile& t, const Decision& D,
                                          uint32_t bits_u) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const int jv = (t.wc * V + k) * 32 + lane;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const bool on = t.active && jv < s.nvec;
      b.bc[k][c] = on ? s.dist[4 * jv + c] : kInf;
      b.bt[k][c] = on ? stored_tie(s, 4 * jv + c, D, bits_u) : 0u;
    }
  }
}

__device__ __forceinline__ void best_update(uint32_t c, uint32_t tb, uint32_t& bc, uint32_t& bt) {
  if (c < bc || (c == bc && tb < bt)) {
    bc = c;
    bt = tb;
  }
}

// Commit the phase's best key of column `col` if it beats the stored one.
__device__ __forceinline__ void commit_key(const Slice& s, int col, uint64_t key, uint32_t tie0, const Decision& D,
                                           uint32_t bits_u) {
  const uint32_t c = static_cast<uint32_t>(key >> 32);
  const uint32_t tb = static_cast<uint32_t>(key);
  if (c < kInf && (c < s.dist[col] || (c == s.dist[col] && tb < tie0))) {
    s.dist[col] = c;
    s.pred[col] = static_cast<int32_t>(tb & ((1u << bits_u) - 1u));
    s.pdist[col] = D.m + (tb >> bits_u);
  }
}

// Whether a row of this phase's settled set S can still change column j.
// Every u in S was unvisited when the phase began, so it offers v at least
// max(L, m + minin[v]): L <= dist[u] + minout[u] <= dist[u] + G[u][v], and
// dist[u] >= m with G[u][v] >= minin[v] (that term only with the IN bound's
// data loaded).  A column whose stored dist is below the bound keeps both
// dist and pred this phase; one equal to it can only take a tie, which
// commits only when its stored pred can be tie-beaten (stored_tie != 0, never
// without the IN bound).  Padding columns (visited, INF) never take part.
// Returned as the row threshold of the column: 0 = not live; 2^32 = any
// settled row may strictly improve it; otherwise only a tie can commit, so
// only rows whose tie word is below this (stored_tie) matter.
__device__ __forceinline__ uint64_t column_live(const Slice& s, int j, const Decision& D, uint32_t bits_u) {
  const uint32_t d = s.dist[j];
  if (s.vis[j] && d >= kInf) return 0u;
  uint32_t bound = D.L;
  if (D.use_in) bound = max(bound, D.m + s.minin[j]);  // m < INF, minin <= INF: no wrap
  if (d != bound) return d > bound ? (1ull << 32) : 0u;
  return stored_tie(s, j, D, bits_u);
}

// The 4-column groups of this slice that hold a live column, into glist (any
// order), with the group's row threshold (the largest of its columns') in
// gthr.  Returns their count; ends synced.
// Also counts, for the choice of path, the groups the gather's column pass
// would leave to row items (sc->cnt[26]: a live column that is neither a
// tie-only column at m + minin[v] (with tie sources, `ties`) nor, on a
// symmetric matrix (`rows`), one any row may improve) and those improvable
// columns (sc->cnt[25]; beyond the pass's kMaxRowColumns their groups are
// gathered too).
__device__ __forceinline__ int live_groups(const Slice& s, const Decision& D, uint32_t bits_u, uint32_t* glist,
                                           uint64_t* gthr, BlockScratch* sc, bool ties = false, bool rows = false) {
  if (threadIdx.x == 0) {
    sc->cnt[30] = 0;
    sc->cnt[26] = 0;
    sc->cnt[25] = 0;
  }
  __syncthreads();
  if (!ties && !rows) {  // no column pass: only the groups and their thresholds
    for (int jv = threadIdx.x; jv < s.nvec; jv += blockDim.x) {
      uint64_t thr = column_live(s, 4 * jv, D, bits_u);
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        const uint64_t t = column_live(s, 4 * jv + c, D, bits_u);
        thr = t > thr ? t : thr;
      }
      if (thr) {
        const uint32_t i = atomicAdd(&sc->cnt[30], 1u);
        glist[i] = static_cast<uint32_t>(jv);
        gthr[i] = thr;
      }
    }
    __syncthreads();
    return static_cast<int>(sc->cnt[30]);
  }
  for (int jv = threadIdx.x; jv < s.nvec; jv += blockDim.x) {
    uint64_t thr = 0;
    bool hard = false;
    uint32_t nimp = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = 4 * jv + c;
      const uint64_t t = column_live(s, col, D, bits_u);
      thr = t > thr ? t : thr;
      if (t == 0) continue;
      const uint32_t d = s.dist[col];
      if (ties && t < (1ull << 32) && d < kInf && d == D.m + s.minin[col]) continue;
      if (rows && t == (1ull << 32)) {
        ++nimp;
        continue;
      }
      hard = true;
    }
    if (thr) {
      const uint32_t i = atomicAdd(&sc->cnt[30], 1u);
      glist[i] = static_cast<uint32_t>(jv);
      gthr[i] = thr;
      if (hard) atomicAdd(&sc->cnt[26], 1u);
      if (nimp) atomicAdd(&sc->cnt[25], nimp);
    }
  }
  __syncthreads();
  return static_cast<int>(sc->cnt[30]);
}

// Stage the settled entries among candidates [begin, end) of get(i) into the
// CTA's own shared-memory list as 32-bit tie words tb = ((dist[u] - m) << bits) | u
// (order irrelevant), so that warps read them locally afterwards.  All
// threads take part, K loads each in flight; returns the count; ends synced.
template <class Get>
__device__ __forceinline__ int stage_settled(const Get& get, int begin, int end, const Decision& D, uint32_t bits_u,
                                             uint32_t* list, BlockScratch* sc) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) sc->cnt[31] = 0;
  __syncthreads();
  constexpr int K = 8;
  const uint32_t lt = (1u << lane) - 1u;
  for (int i0 = begin; i0 < end; i0 += K * blockDim.x) {
    uint4 e[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = i0 + k * blockDim.x + threadIdx.x;
      e[k] = i < end ? get(i) : make_uint4(0xffffffffu, kInf, kInf, 0u);
    }
    // one reservation per warp for all K ballots
    uint32_t bal[K];
    uint32_t tot = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      bal[k] = __ballot_sync(0xffffffffu, e[k].x != 0xffffffffu && in_settled(e[k].x, e[k].y, e[k].z, D));
      tot += __popc(bal[k]);
    }
    if (tot) {
      uint32_t pos = 0;
      if (lane == 0) pos = atomicAdd(&sc->cnt[31], tot);
      pos = __shfl_sync(0xffffffffu, pos, 0);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if ((bal[k] >> lane) & 1u) list[pos + __popc(bal[k] & lt)] = ((e[k].y - D.m) << bits_u) | e[k].x;
        pos += __popc(bal[k]);
      }
    }
  }
  __syncthreads();
  return static_cast<int>(sc->cnt[31]);
}

// stage_settled for the grid's published candidate lists, read by bulk copies:
// candidates [begin, end) (entry i lies in region r with off[r] <= i <
// off[r + 1], at cl + r * swcap + i - off[r]) come into `buf` in chunks of
// buf_bytes / 16 entries, one copy per overlapping region (issued by thread r),
// all completing on one mbarrier of the pair rbar (gt counts their phases,
// the same in every thread); then the chunk is filtered from shared memory.
// Sets ok = false if a chunk did not arrive in time.  Returns the count; ends
// synced.
__device__ __forceinline__ int stage_settled_bulk(const uint32_t* off, int G, const uint4* cl, int swcap, int begin,
                                                  int end, const Decision& D, uint32_t bits_u, uint32_t* list,
                                                  uint8_t* buf, uint32_t buf_bytes, uint64_t* rbar, uint32_t& gt,
                                                  int64_t timeout_ns, BlockScratch* sc, bool& ok) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) sc->cnt[31] = 0;
  const int per = static_cast<int>(buf_bytes / 16);
  const uint4* b4 = reinterpret_cast<const uint4*>(buf);
  for (int c0 = begin; c0 < end; c0 += per) {
    const int c1 = min(end, c0 + per);
    const uint32_t g = gt++;
    uint64_t* bar = rbar + (g & 1u);
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, static_cast<uint32_t>(c1 - c0) * 16u);
    __syncthreads();  // the expectation precedes the copies; earlier reads of buf are done
    for (int r = threadIdx.x; r < G; r += blockDim.x) {
      const int lo = max(static_cast<int>(off[r]), c0), hi = min(static_cast<int>(off[r + 1]), c1);
      if (hi > lo) {
        fence_proxy_async_smem();  // earlier generic accesses of buf precede the copy
        bulk_g2s(buf + static_cast<size_t>(lo - c0) * 16, cl + static_cast<size_t>(r) * swcap + (lo - static_cast<int>(off[r])),
                 static_cast<uint32_t>(hi - lo) * 16u, bar);
      }
    }
    if (!mbar_wait_bounded(bar, (g >> 1) & 1u, timeout_ns)) {
      ok = false;
      mbar_wait_bounded(bar, (g >> 1) & 1u, timeout_ns);  // drain once more
    }
    constexpr int K = 4;
    for (int i0 = 0; i0 < c1 - c0; i0 += K * static_cast<int>(blockDim.x)) {
      uint4 e[K];
      uint32_t bal[K], tot = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = i0 + k * static_cast<int>(blockDim.x) + static_cast<int>(threadIdx.x);
        e[k] = i < c1 - c0 ? b4[i] : make_uint4(0xffffffffu, kInf, kInf, 0u);
        bal[k] = __ballot_sync(0xffffffffu, e[k].x != 0xffffffffu && in_settled(e[k].x, e[k].y, e[k].z, D));
        tot += __popc(bal[k]);
      }
      if (tot) {
        uint32_t pos = 0;
        if (lane == 0) pos = atomicAdd(&sc->cnt[31], tot);
        pos = __shfl_sync(0xffffffffu, pos, 0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if ((bal[k] >> lane) & 1u) list[pos + __popc(bal[k] & lt)] = ((e[k].y - D.m) << bits_u) | e[k].x;
          pos += __popc(bal[k]);
        }
      }
    }
    fence_proxy_async_smem();  // this thread's reads of buf precede the next copies into it
  }
  __syncthreads();
  return static_cast<int>(sc->cnt[31]);
}

// Entry i of a staged list, in the candidate form the relaxation takes.
__device__ __forceinline__ uint4 staged_entry(const uint32_t* list, int i, const Decision& D, uint32_t bits_u) {
  const uint32_t tb = list[i];
  return make_uint4(tb & ((1u << bits_u) - 1u), D.m + (tb >> bits_u), 0u, 0u);
}

// Relax the settled rows among `total` candidates (u, dist[u], IN key) given by
// get(i) over this CTA's slice.  Row group rg takes candidates rg, rg + rgs,
// ... (so every row group gets the same share): 32 at a time, one per lane,
// a ballot picks the settled ones, and their slices go through the warp's
// TMA ring in stages of up to U rows, `depth` stages ahead of the arithmetic.
// The common case (no lane improves or ties its column) costs four adds, four
// compares and one vote per row; the exact lexicographic update runs only
// otherwise.  No block-wide barrier is involved.
template <int V, int U, class Get>
__device__ __forceinline__ bool relax_pull(const Get& get, int total, const Slice& s, const Tile& t,
                                           const int32_t* __restrict__ W, int64_t pitch, const Decision& D,
                                           uint32_t bits_u, Ring& ring, uint32_t* slot_rows, uint32_t* slot_tb,
                                           int64_t timeout_ns, Best<V>& best) {
  if (!t.active || ring.rowbytes == 0 || t.rg >= total) return true;
  const int lane = threadIdx.x & 31;
  bool jok[V];
#pragma unroll
  for (int k = 0; k < V; ++k) jok[k] = (t.wc * V + k) * 32 + lane < s.nvec;
  const uint32_t umask = (1u << bits_u) - 1u;
  const uint32_t depth = ring.depth;
  const char* colbase = reinterpret_cast<const char*>(W + s.c0) + static_cast<size_t>(t.wc) * V * 32 * 16;
  const int64_t rowstride = pitch * 4;
  const uint32_t m = D.m;
  // stage counters, with their slot and parity kept incrementally
  uint32_t issued = ring.gt, consumed = ring.gt;
  uint32_t islot = ring.gt % depth;
  uint32_t cslot = islot, cpar = (ring.gt / depth) & 1u;
  bool ok = true;

  auto consume = [&]() {
    const uint32_t slot = cslot;
    if (!mbar_wait_bounded(ring.bar + slot, cpar, timeout_ns)) {
      ok = false;
      mbar_wait_bounded(ring.bar + slot, cpar, timeout_ns);  // drain once more
    }
    const int rows = static_cast<int>(slot_rows[slot]);
    const uint8_t* sb = ring.buf + static_cast<size_t>(slot) * ring.srows * ring.rowbytes + 16 * lane;
    const uint32_t* tbs = slot_tb + slot * U;
#pragma unroll
    for (int uu = 0; uu < U; ++uu) {
      if (uu < rows) {
        const uint32_t tb = tbs[uu];
        const uint32_t du = m + (tb >> bits_u);
        uint32_t c[V][4];
        bool hit = false;
#pragma unroll
        for (int k = 0; k < V; ++k) {
          if (jok[k]) {
            const int4 x = *reinterpret_cast<const int4*>(sb + static_cast<size_t>(uu) * ring.rowbytes + 512 * k);
            c[k][0] = du + static_cast<uint32_t>(x.x);
            c[k][1] = du + static_cast<uint32_t>(x.y);
            c[k][2] = du + static_cast<uint32_t>(x.z);
            c[k][3] = du + static_cast<uint32_t>(x.w);
            hit |= (c[k][0] <= best.bc[k][0]) | (c[k][1] <= best.bc[k][1]) | (c[k][2] <= best.bc[k][2]) |
                   (c[k][3] <= best.bc[k][3]);
          } else {
            c[k][0] = c[k][1] = c[k][2] = c[k][3] = 0xFFFFFFFFu;
          }
        }
        if (__any_sync(0xffffffffu, hit)) {
#pragma unroll
          for (int k = 0; k < V; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q) best_update(c[k][q], tb, best.bc[k][q], best.bt[k][q]);
        }
      }
    }
    __syncwarp();
    fence_proxy_async_smem();  // this slot's reads are done before its next TMA write
    ++consumed;
    if (++cslot == depth) {
      cslot = 0;
      cpar ^= 1u;
    }
  };

  // candidate k of this row group is get(rg + rgs * k); lane l takes k = 32 j + l
  const int K = (total - t.rg + t.rgs - 1) / t.rgs;
  auto fetch = [&](int j) -> uint4 {
    const int k = 32 * j + lane;
    return k < K ? get(t.rg + t.rgs * k) : make_uint4(0xffffffffu, kInf, kInf, 0u);
  };
  uint4 nxt = fetch(0), nxt2 = fetch(1);  // two chunks of candidates in flight
  for (int j = 0; 32 * j < K; ++j) {
    const uint4 e = nxt;
    nxt = nxt2;
    nxt2 = fetch(j + 2);
    const bool settled = e.x != 0xffffffffu && in_settled(e.x, e.y, e.z, D);
    const uint32_t mask = __ballot_sync(0xffffffffu, settled);
    const int nrows = __popc(mask);
    const int rank = __popc(mask & ((1u << lane) - 1u));
    const int srows = static_cast<int>(ring.srows);
    for (int k0 = 0; k0 < nrows; k0 += srows) {
      if (issued - consumed == depth) consume();
      const uint32_t slot = islot;
      const int rows = min(srows, nrows - k0);
      const bool mine = settled && rank >= k0 && rank < k0 + rows;
      if (lane == 0) {
        slot_rows[slot] = static_cast<uint32_t>(rows);
        mbar_arrive_expect_tx(ring.bar + slot, static_cast<uint32_t>(rows) * ring.rowbytes);
      }
      if (mine) slot_tb[slot * U + (rank - k0)] = ((e.y - m) << bits_u) | e.x;
      __syncwarp();
      if (mine) {
        bulk_g2s(ring.buf + (static_cast<size_t>(slot) * ring.srows + (rank - k0)) * ring.rowbytes,
                 colbase + static_cast<int64_t>(e.x & umask) * rowstride, ring.rowbytes, ring.bar + slot);
      }
      ++issued;
      if (++islot == depth) islot = 0;
    }
  }
  while (consumed != issued) consume();
  ring.gt = issued;
  return ok;
}

// Relax only the live groups glist[0, nlg) of this slice: the settled rows
// among `total` candidates are staged into `list` (list_cap at a time, by
// stage(begin, end), which returns their count and ends synced) and cut into
// chunks of kGatherChunk rows; work item (chunk c, group g) goes
// to thread (c * nlg + g) mod blockDim, so a group that needs every row is
// spread over the whole block.  An item loads the group's 16 bytes of each of
// its rows whose tie word is below the group's threshold gthr[g] (all of them
// in flight at once), keeps the running best of the group's 4 columns, and merges it
// into bkey (64-bit keys (candidate << 32) | tie word, shared-memory
// atomicMin).  On entry bkey[j] must hold (dist[j] << 32) | ~0 for every
// column.  Ends synced.
// With `colpass` (the whole list in one segment, room in `bm`), a column pass
// (gather_column_pass) first decides the columns that can only take a tie at
// the IN bound from their tie sources and, on a symmetric matrix (sym), the
// columns any row may improve from their own row; groups left with no other
// live column drop out of the gather.
constexpr int kGatherChunk = 16;
constexpr int kMaxRowColumns = 4;  // whole-row reads of the gather's column pass per CTA (one after another)

// Tie sources of the columns: src[v * cap + k], k < cnt[v], are the u != v
// with G[u][v] == minin[v] (cnt[v] > cap: too many to list).
struct TieSources {
  const int32_t* src;
  const int32_t* cnt;
  int32_t cap;  // 0: none
};

// Column pass of the gather path, before its row items.  `tab` (pitch 16-bit
// entries, in shared memory) holds dist[u] - m for the settled rows of the
// phase (0xFFFF: not settled); it is exact unless `exact` is false (some
// settled row lies 0xFFFF or more above m).  Two kinds of live column leave
// the group gather:
//   - A column whose stored dist equals its bound m + minin[v] (>= L) can
//     only take a tie, and only from a settled u with dist[u] = m and G[u][v]
//     = minin[v]: every settled u has dist[u] >= m, and G[u][v] >= minin[v]
//     off the diagonal (v's own zero diagonal offers v its dist with a tie
//     word above the stored one, so it never commits).  Such a u is one of
//     v's tie sources, and among those with dist[u] = m the smallest index has
//     the smallest tie word.  One warp per column checks its listed sources.
//   - On a symmetric matrix, a column any settled row may improve (dist above
//     its bound) reads row v whole -- it is column v -- once, coalesced,
//     against the table, instead of one 16-byte piece per settled row.
// The groups' row thresholds are recomputed from their remaining columns and
// glist / gthr compacted.  clist (2 * sw entries of shared memory) holds the
// two column lists.  Returns the new group count; ends synced.
__device__ __forceinline__ int gather_column_pass(const Slice& s, const int32_t* __restrict__ W, int64_t pitch,
                                                  const Decision& D, uint32_t bits_u, const TieSources& ts,
                                                  bool rows_ok, const uint16_t* tab, uint32_t* clist,
                                                  uint32_t* glist, uint64_t* gthr, int nlg, uint64_t* bkey,
                                                  BlockScratch* sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = static_cast<int>(blockDim.x >> 5);
  uint32_t* tl = clist;          // tie-source columns
  uint32_t* rl = clist + s.sw;   // whole-row columns
  if (threadIdx.x == 0) {
    sc->cnt[28] = 0;
    sc->cnt[29] = 0;
  }
  __syncthreads();
  for (int gi = threadIdx.x; gi < nlg; gi += blockDim.x) {
    const int jv = static_cast<int>(glist[gi]);
    uint64_t thr = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = 4 * jv + q;
      const uint64_t t = column_live(s, col, D, bits_u);
      if (t == 0) continue;
      const uint32_t d = s.dist[col];
      if (ts.cap > 0 && t < (1ull << 32) && D.use_in && d < kInf && d == D.m + s.minin[col]) {
        tl[atomicAdd(&sc->cnt[28], 1u)] = static_cast<uint32_t>(col);
        continue;
      }
      if (rows_ok && t == (1ull << 32)) {
        const uint32_t k = atomicAdd(&sc->cnt[29], 1u);
        if (k < static_cast<uint32_t>(kMaxRowColumns)) {  // at most this many rows; the rest stay gathered
          rl[k] = static_cast<uint32_t>(col);
          continue;
        }
      }
      thr = t > thr ? t : thr;
    }
    gthr[gi] = thr;
  }
  __syncthreads();
  const int ntl = static_cast<int>(sc->cnt[28]), nrl = min(static_cast<int>(sc->cnt[29]), kMaxRowColumns);
  // tie-source columns, one warp each (a column with more sources than listed keeps its group)
  for (int k = warp; k < ntl; k += nwarps) {
    const int col = static_cast<int>(tl[k]);
    const int v = s.c0 + col;
    const int nsrc = ts.cnt[v];
    uint32_t best = 0xFFFFFFFFu;
    if (nsrc <= ts.cap && lane < nsrc) {
      const uint32_t u = static_cast<uint32_t>(ts.src[static_cast<int64_t>(v) * ts.cap + lane]);
      if (tab[u] == 0) best = u;
    }
    best = warp_min_u32(best);
    if (nsrc > ts.cap) {  // back to the gather: fold the column's threshold into its group
      if (lane == 0) {
        const uint64_t t = column_live(s, col, D, bits_u);
        for (int gi = 0; gi < nlg; ++gi)
          if (static_cast<int>(glist[gi]) == col / 4) {
            atomicMax(reinterpret_cast<unsigned long long*>(gthr + gi), static_cast<unsigned long long>(t));
            break;
          }
      }
    } else if (lane == 0 && best != 0xFFFFFFFFu) {
      const uint64_t key = (static_cast<uint64_t>(s.dist[col]) << 32) | best;  // tie word (0 << bits) | u
      atomicMin(reinterpret_cast<unsigned long long*>(bkey + col), static_cast<unsigned long long>(key));
    }
  }
  // whole-row columns: the block reads row v (= column v) once, coalesced
  const int nvec = static_cast<int>(pitch / 4);
  const uint2* tab4 = reinterpret_cast<const uint2*>(tab);
  for (int k = 0; k < nrl; ++k) {
    const int col = static_cast<int>(rl[k]);
    const int4* row = reinterpret_cast<const int4*>(W + static_cast<int64_t>(s.c0 + col) * pitch);
    uint32_t bc = 0xFFFFFFFFu, bt = 0xFFFFFFFFu;
    constexpr int R = 8;
    for (int g0 = 0; g0 < nvec; g0 += R * static_cast<int>(blockDim.x)) {
      int4 x[R];
      uint2 t2[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int gv = g0 + r * static_cast<int>(blockDim.x) + static_cast<int>(threadIdx.x);
        t2[r] = gv < nvec ? tab4[gv] : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
        x[r] = (t2[r].x & t2[r].y) != 0xFFFFFFFFu ? __ldg(row + gv) : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int gv = g0 + r * static_cast<int>(blockDim.x) + static_cast<int>(threadIdx.x);
        const uint32_t t4[4] = {t2[r].x & 0xFFFFu, t2[r].x >> 16, t2[r].y & 0xFFFFu, t2[r].y >> 16};
        const uint32_t w4[4] = {static_cast<uint32_t>(x[r].x), static_cast<uint32_t>(x[r].y),
                                static_cast<uint32_t>(x[r].z), static_cast<uint32_t>(x[r].w)};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (t4[q] != 0xFFFFu)
            best_update(D.m + t4[q] + w4[q], (t4[q] << bits_u) | static_cast<uint32_t>(4 * gv + q), bc, bt);
      }
    }
    const uint64_t key = warp_min_u64((static_cast<uint64_t>(bc) << 32) | bt);
    if (lane == 0 && static_cast<uint32_t>(key) != 0xFFFFFFFFu)
      atomicMin(reinterpret_cast<unsigned long long*>(bkey + col), static_cast<unsigned long long>(key));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int gi = 0; gi < nlg; ++gi)
      if (gthr[gi]) {
        glist[k] = glist[gi];
        gthr[k] = gthr[gi];
        ++k;
      }
    sc->cnt[28] = static_cast<uint32_t>(k);
  }
  __syncthreads();
  return static_cast<int>(sc->cnt[28]);
}

template <class Stage>
__device__ __forceinline__ void relax_gather(const Stage& stage, int total, const Slice& s,
                                             const int32_t* __restrict__ W, int64_t pitch, const Decision& D,
                                             uint32_t bits_u, uint32_t* glist, uint64_t* gthr, int nlg,
                                             uint32_t* list, int list_cap, uint64_t* bkey, const TieSources& ts,
                                             bool sym, bool colpass, uint32_t* bm, BlockScratch* sc) {
  const uint32_t umask = (1u << bits_u) - 1u;
  constexpr int K = kGatherChunk;
  for (int seg = 0; seg < total; seg += list_cap) {
    const int cnt = stage(seg, min(total, seg + list_cap));  // settled rows of [seg, ...) into list; synced
    // the column pass (the caller checked that it applies: the whole list in one segment, room in
    // bm for the table (2 bytes per column) plus two column lists)
    if (colpass) {
      uint16_t* tab = reinterpret_cast<uint16_t*>(bm);
      if (threadIdx.x == 0) sc->cnt[27] = 0;
      for (int i = threadIdx.x; i < static_cast<int>(pitch / 2); i += blockDim.x) bm[i] = 0xFFFFFFFFu;
      __syncthreads();
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t tb = list[i];
        const uint32_t dd = tb >> bits_u;
        tab[tb & umask] = static_cast<uint16_t>(min(dd, 0xFFFEu));
        if (dd >= 0xFFFEu) sc->cnt[27] = 1;  // the table is not exact
      }
      __syncthreads();
      nlg = gather_column_pass(s, W, pitch, D, bits_u, ts, sym && sc->cnt[27] == 0, tab, bm + pitch / 2, glist, gthr,
                               nlg, bkey, sc);
      fence_proxy_async_smem();  // the scratch's generic accesses precede later copies into its bytes
    }
    const int items = nlg * ((cnt + kGatherChunk - 1) / kGatherChunk);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int c = it / nlg, g = it - c * nlg;
      const uint64_t thr = gthr[g];
      const int col = 4 * static_cast<int>(glist[g]);
      const int32_t* base = W + s.c0 + col;
      uint32_t bc[4], bt[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bc[q] = s.dist[col + q];
        bt[q] = 0xFFFFFFFFu;
      }
      const int r1 = min(cnt, (c + 1) * kGatherChunk);
      for (int r0 = c * kGatherChunk; r0 < r1; r0 += K) {
        int4 x[K];
        uint32_t tbk[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int r = r0 + k;
          tbk[k] = r < r1 ? list[r] : 0u;
          const bool need = r < r1 && tbk[k] < thr;
          x[k] = need ? __ldg(reinterpret_cast<const int4*>(base + static_cast<int64_t>(tbk[k] & umask) * pitch))
                      : make_int4(0, 0, 0, 0);
          if (!need) tbk[k] = 0xFFFFFFFFu;  // marks the slot unused
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (tbk[k] == 0xFFFFFFFFu) continue;
          const uint32_t du = D.m + (tbk[k] >> bits_u);
          best_update(du + static_cast<uint32_t>(x[k].x), tbk[k], bc[0], bt[0]);
          best_update(du + static_cast<uint32_t>(x[k].y), tbk[k], bc[1], bt[1]);
          best_update(du + static_cast<uint32_t>(x[k].z), tbk[k], bc[2], bt[2]);
          best_update(du + static_cast<uint32_t>(x[k].w), tbk[k], bc[3], bt[3]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (bt[q] == 0xFFFFFFFFu) continue;  // nothing offered
        const uint64_t key = (static_cast<uint64_t>(bc[q]) << 32) | bt[q];
        unsigned long long* slot = reinterpret_cast<unsigned long long*>(bkey + col + q);
        if (key < *slot) atomicMin(slot, static_cast<unsigned long long>(key));
      }
    }
    __syncthreads();  // bkey complete; the list is rewritten by the next segment
  }
}

// Row-split relaxation (grid engine, phases with many settled rows).  Reading
// a whole row per CTA streams HBM faster than every CTA reading its slice of
// every row, at the price of a merge: CTA b takes the settled rows among
// candidates b, b + G, b + 2G, ... and streams each row over all columns in
// chunks of 4 T CPT columns.  Thread 0 copies a row's chunk with one TMA bulk
// copy into shared buffer (g & 1), g counting the CTA's buffered rows over the
// kernel (rs_gt), so two rows are in flight; thread t keeps the running bests
// of the chunk's 4-column groups t + T j (j < CPT) in registers.  A best that
// can commit -- below the column's dist in the snapshot `gsnap` the owners
// wrote when this phase began, or equal to it where the snapshot's top bit
// says a tie can still win -- is merged into gkey (64-bit keys
// (candidate << 32) | tie word, global atomicMin); the owners read their
// slice of gkey after a grid barrier and commit from it.  The owners announce
// their snapshots on *snap_count (one release increment per CTA); the first
// merge waits, bounded, for snap_target of them -- long done by then, since
// the snapshots are written before the rows are streamed.  Returns false if a
// copy or that wait did not complete in time.  Ends synced.
template <int CPT, class Get>
__device__ __forceinline__ bool relax_rows(const Get& get, int total, int b, int G, const int32_t* __restrict__ W,
                                           int64_t pitch, const Decision& D, uint32_t bits_u,
                                           const uint32_t* __restrict__ gsnap, unsigned long long* gkey,
                                           uint32_t* list, int list_cap, uint8_t* rbuf, uint64_t* rbar,
                                           uint32_t& rs_gt, int64_t timeout_ns, const uint32_t* snap_count,
                                           uint32_t snap_target, uint32_t* abort_flag, BlockScratch* sc) {
  const uint32_t umask = (1u << bits_u) - 1u;
  if (threadIdx.x == 0) sc->cnt[31] = 0;
  __syncthreads();
  // this CTA's share (at most ceil(total / G) <= the slice width <= list_cap rows)
  for (int k = threadIdx.x; b + G * k < total; k += blockDim.x) {
    const uint4 e = get(b + G * k);
    if (in_settled(e.x, e.y, e.z, D)) {
      const uint32_t at = atomicAdd(&sc->cnt[31], 1u);
      if (at < static_cast<uint32_t>(list_cap)) list[at] = ((e.y - D.m) << bits_u) | e.x;
    }
  }
  __syncthreads();
  const int nrows = min(static_cast<int>(sc->cnt[31]), list_cap);
  const int T = static_cast<int>(blockDim.x);
  const int nvec = static_cast<int>(pitch / 4);
  const int chunkv = T * CPT;
  const size_t bufbytes = static_cast<size_t>(min(chunkv, nvec)) * 16;
  bool ok = true;
  for (int c0 = 0; c0 < nvec; c0 += chunkv) {
    const int cv = min(chunkv, nvec - c0);
    const uint32_t bytes = static_cast<uint32_t>(cv) * 16u;
    auto issue = [&](int r) {  // thread 0
      const uint32_t g = rs_gt + static_cast<uint32_t>(r);
      const uint32_t u = list[r] & umask;
      fence_proxy_async_smem();  // earlier generic reads of the buffer precede the copy
      mbar_arrive_expect_tx(rbar + (g & 1u), bytes);
      bulk_g2s(rbuf + (g & 1u) * bufbytes, W + static_cast<int64_t>(u) * pitch + 4 * static_cast<int64_t>(c0), bytes,
               rbar + (g & 1u));
    };
    if (threadIdx.x == 0) {
      if (nrows > 0) issue(0);
      if (nrows > 1) issue(1);
    }
    uint32_t bc[CPT][4], bt[CPT][4];
#pragma unroll
    for (int j = 0; j < CPT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bc[j][q] = 0xFFFFFFFFu;
        bt[j][q] = 0xFFFFFFFFu;
      }
    for (int r = 0; r < nrows; ++r) {
      const uint32_t g = rs_gt + static_cast<uint32_t>(r);
      if (!mbar_wait_bounded(rbar + (g & 1u), (g >> 1) & 1u, timeout_ns)) {
        ok = false;
        mbar_wait_bounded(rbar + (g & 1u), (g >> 1) & 1u, timeout_ns);  // drain once more
      }
      const uint32_t tb = list[r];
      const uint32_t du = D.m + (tb >> bits_u);
      const int4* buf = reinterpret_cast<const int4*>(rbuf + (g & 1u) * bufbytes);
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int gv = static_cast<int>(threadIdx.x) + T * j;
        if (gv < cv) {
          const int4 x = buf[gv];
          best_update(du + static_cast<uint32_t>(x.x), tb, bc[j][0], bt[j][0]);
          best_update(du + static_cast<uint32_t>(x.y), tb, bc[j][1], bt[j][1]);
          best_update(du + static_cast<uint32_t>(x.z), tb, bc[j][2], bt[j][2]);
          best_update(du + static_cast<uint32_t>(x.w), tb, bc[j][3], bt[j][3]);
        }
      }
      __syncthreads();  // buffer (g & 1) is free again
      if (threadIdx.x == 0 && r + 2 < nrows) issue(r + 2);
    }
    rs_gt += static_cast<uint32_t>(nrows);
    if (c0 == 0) {  // every owner's snapshot is visible before the first merge
      __shared__ uint32_t s_snap_ok;
      if (threadIdx.x == 0) {
        uint32_t okw = 1;
        if (static_cast<int32_t>(ld_acquire_gpu(snap_count) - snap_target) < 0) {
          const uint64_t t0 = global_ns();
          while (static_cast<int32_t>(ld_acquire_gpu(snap_count) - snap_target) < 0) {
            if (ld_relaxed_gpu(abort_flag) || static_cast<int64_t>(global_ns() - t0) > timeout_ns) {
              okw = 0;
              break;
            }
          }
        }
        s_snap_ok = okw;
      }
      __syncthreads();
      if (!s_snap_ok) {
        fence_proxy_async_smem();
        return false;
      }
    }
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int gv = static_cast<int>(threadIdx.x) + T * j;
      if (gv >= cv || (bt[j][0] & bt[j][1] & bt[j][2] & bt[j][3]) == 0xFFFFFFFFu) continue;  // nothing offered
      const uint4 sn = __ldcg(reinterpret_cast<const uint4*>(gsnap) + c0 + gv);
      const uint32_t s4[4] = {sn.x, sn.y, sn.z, sn.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t d = s4[q] & 0x7FFFFFFFu;
        if (bc[j][q] < d || (bc[j][q] == d && (s4[q] >> 31) && bt[j][q] != 0xFFFFFFFFu))
          atomicMin(gkey + 4 * (c0 + gv) + q, (static_cast<unsigned long long>(bc[j][q]) << 32) | bt[j][q]);
      }
    }
  }
  fence_proxy_async_smem();  // this thread's reads of the buffers precede later copies into them
  return ok;
}

// Row-push relaxation (grid engine, phases of graphs that are not dense).
// Work items are (candidate k, column chunk c) pairs, k < total, chunks of
// kPushChunk columns; item it = k * chunks + c goes to warp it mod (G * warps)
// of the grid, so one settled row's chunks are read side by side by the warps
// of one CTA.  A warp skips a candidate that is not settled; otherwise every
// lane loads its 16-byte pieces of the chunk (kPushLoads in flight) and pushes
// each finite entry w into gkey[v] as the 64-bit key ((dist[u] + w) << 32) |
// tie word with atomicMin, so that after a grid barrier gkey[v] holds the
// smallest (candidate, dist[u] - m, u) any settled row offers v -- the key the
// other paths reduce per column -- and the owners commit from it.  Rows are
// read whole and contiguously: large coalesced requests instead of every
// CTA's narrow slice of every row.  No barrier inside.
constexpr int kPushChunk = 2048;  // columns per work item (8 KB)
constexpr int kPushLoads = 16;    // 16-byte loads in flight per lane (one round per item)

// The settled entries among candidates [begin, end) of get(i), as tie words
// ((dist[u] - m) << bits) | u, into list: every CTA derives the same list from
// the same published candidates (a block-wide scan, no atomics; thread t's
// entries i0 + j * T + t in order of t, then j), so work items indexed by list
// position mean the same row in every CTA.  Each load instruction of a warp
// reads 32 consecutive entries: every CTA reads the whole list at once, and
// 16-byte pieces at a 64-byte stride doubled the L2 requests on its few
// hundred lines (2.1-3.1 us for one round of ~2000 candidates).  At most
// end - begin entries; returns the count; ends synced.
template <class Get>
__device__ __forceinline__ int compact_settled(const Get& get, int begin, int end, const Decision& D,
                                               uint32_t bits_u, uint32_t* list, BlockScratch* sc) {
  constexpr int K = 4;  // candidates per thread (loads in flight)
  const int T = static_cast<int>(blockDim.x), lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  int out = 0;
  for (int i0 = begin; i0 < end; i0 += K * T) {
    uint4 e[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int i = i0 + j * T + static_cast<int>(threadIdx.x);
      e[j] = i < end ? get(i) : make_uint4(0xffffffffu, kInf, kInf, 0u);
    }
    uint32_t flags = 0, cnt = 0;
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (e[j].x != 0xffffffffu && in_settled(e[j].x, e[j].y, e[j].z, D)) {
        flags |= 1u << j;
        ++cnt;
      }
    uint32_t incl = cnt;  // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) sc->r32[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t wsum = lane < nw ? sc->r32[lane] : 0u;
      uint32_t wi = wsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      if (lane < nw) sc->r32b[lane] = wi - wsum;  // exclusive prefix of the warps
      if (lane == 31) sc->b32 = wi;
    }
    __syncthreads();
    uint32_t pos = static_cast<uint32_t>(out) + sc->r32b[warp] + incl - cnt;
#pragma unroll
    for (int j = 0; j < K; ++j)
      if ((flags >> j) & 1u) list[pos++] = ((e[j].y - D.m) << bits_u) | e[j].x;
    out += static_cast<int>(sc->b32);
    __syncthreads();  // sc is rewritten by the next round
  }
  return out;
}

// Push the rows of the cnt settled tie words in list (the same list in every
// CTA) as work items (row k, chunk c) spread over every warp of the grid.
__device__ __forceinline__ void relax_push(const uint32_t* list, int cnt, int G, const int32_t* __restrict__ W,
                                           int64_t pitch, const Decision& D, uint32_t bits_u,
                                           unsigned long long* gkey) {
  const int lane = threadIdx.x & 31, nw = static_cast<int>(blockDim.x >> 5);
  const uint32_t umask = (1u << bits_u) - 1u;
  const int chunks = static_cast<int>((pitch + kPushChunk - 1) / kPushChunk);
  const int64_t items = static_cast<int64_t>(cnt) * chunks;
  const int64_t stride = static_cast<int64_t>(G) * nw;
  for (int64_t it = static_cast<int64_t>(blockIdx.x) * nw + (threadIdx.x >> 5); it < items; it += stride) {
    const int k = static_cast<int>(it / chunks);
    const int c = static_cast<int>(it - static_cast<int64_t>(k) * chunks);
    const uint32_t tb32 = list[k];
    const uint32_t u = tb32 & umask;
    const uint32_t du = D.m + (tb32 >> bits_u);
    const uint64_t tb = static_cast<uint64_t>(tb32);
    const int64_t col0 = static_cast<int64_t>(c) * kPushChunk;
    const int nv = static_cast<int>(min(static_cast<int64_t>(kPushChunk), pitch - col0) / 4);
    const int32_t* row = W + static_cast<int64_t>(u) * pitch + col0;
    for (int v0 = 0; v0 < nv; v0 += 32 * kPushLoads) {
      int4 x[kPushLoads];
#pragma unroll
      for (int r = 0; r < kPushLoads; ++r) {
        const int iv = v0 + 32 * r + lane;
        x[r] = iv < nv ? ld_stream16(row + 4 * iv) : make_int4(int(kInf), int(kInf), int(kInf), int(kInf));
      }
#pragma unroll
      for (int r = 0; r < kPushLoads; ++r) {
        const uint32_t w4[4] = {static_cast<uint32_t>(x[r].x), static_cast<uint32_t>(x[r].y),
                                static_cast<uint32_t>(x[r].z), static_cast<uint32_t>(x[r].w)};
        if ((w4[0] & w4[1] & w4[2] & w4[3]) == kInf) continue;  // all four INF (entries are <= INF)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (w4[q] < kInf)
            atomicMin(gkey + col0 + 4 * (v0 + 32 * r + lane) + q,
                      (static_cast<unsigned long long>(du + w4[q]) << 32) | tb);
      }
    }
  }
}

// Snapshot word of column j for relax_rows: dist, with the top bit set when
// a tie can still replace pred (IN bound on, pred's dist >= this phase's m).
__device__ __forceinline__ uint32_t snapshot_word(const Slice& s, int j, const Decision& D) {
  const bool tie = D.use_in && s.pred[j] >= 0 && s.pdist[j] >= D.m && s.dist[j] < kInf;
  return s.dist[j] | (tie ? 0x80000000u : 0u);
}

// One column of a commit: mark it visited if it was settled this phase
// (judged on its state before the commit), commit a lexicographically
// smaller key b, and fold the column into this thread's next partial.
__device__ __forceinline__ void commit_column(const Slice& s, int col, uint64_t b, const Decision& D,
                                              uint32_t bits_u, Part& pt) {
  const uint32_t d = s.dist[col];
  const uint32_t tie0 = stored_tie(s, col, D, bits_u);
  if (!s.vis[col] && in_settled(static_cast<uint32_t>(s.c0 + col), d, in_key(d, s.minin[col]), D)) s.vis[col] = 1;
  commit_key(s, col, b, tie0, D, bits_u);
  column_partial(s, col, pt);
}

// Commit from the per-column keys of relax_gather, or from none (bkey null:
// no live column in the slice).
__device__ __forceinline__ void commit_keys(const Slice& s, const Decision& D, uint32_t bits_u, const uint64_t* bkey,
                                            Part& pt) {
  part_init(pt);
  for (int col = threadIdx.x; col < s.sw; col += blockDim.x)
    commit_column(s, col, bkey ? bkey[col] : kNoKey, D, bits_u, pt);
}

// Merge the row groups' bests, then for every column: mark it visited if it
// was settled this phase (judged on its state before this phase's commit),
// commit a lexicographically smaller key, and fold the column into this
// thread's part of the next partial.  Starts with a barrier when row groups
// must be merged.
// With `amerge` the row groups' bests meet in merge[col] (one key per column,
// kNoKey between phases) by shared-memory atomicMin instead of one merge row
// per row group.
template <int V>
__device__ __forceinline__ void commit_partial(const Slice& s, const Tile& t, const Decision& D, uint64_t* merge,
                                               uint32_t bits_u, const Best<V>& best, Part& pt, bool amerge = false) {
  const int lane = threadIdx.x & 31;
  part_init(pt);
  auto one = [&](int col, uint64_t b) { commit_column(s, col, b, D, bits_u, pt); };
  if (amerge && t.rgs > 1) {
    if (t.active) {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int jv = (t.wc * V + k) * 32 + lane;
        if (jv < s.nvec) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint64_t key = (static_cast<uint64_t>(best.bc[k][c]) << 32) | best.bt[k][c];
            unsigned long long* slot = reinterpret_cast<unsigned long long*>(merge + 4 * jv + c);
            if (key < *slot) atomicMin(slot, static_cast<unsigned long long>(key));
          }
        }
      }
    }
    __syncthreads();
    for (int col = threadIdx.x; col < s.sw; col += blockDim.x) {
      const uint64_t b = merge[col];
      merge[col] = kNoKey;  // ready for the next phase (several barriers away)
      one(col, b);
    }
    return;
  }
  if (t.rgs == 1) {
    if (t.active) {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int jv = (t.wc * V + k) * 32 + lane;
        if (jv < s.nvec) {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            one(4 * jv + c, (static_cast<uint64_t>(best.bc[k][c]) << 32) | best.bt[k][c]);
        }
      }
    }
    return;
  }
  if (t.active) {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int jv = (t.wc * V + k) * 32 + lane;
      if (jv < s.nvec) {
        uint64_t* dst = merge + static_cast<size_t>(t.rg) * s.sw + 4 * jv;
#pragma unroll
        for (int c = 0; c < 4; ++c) dst[c] = (static_cast<uint64_t>(best.bc[k][c]) << 32) | best.bt[k][c];
      }
    }
  }
  __syncthreads();
  for (int col = threadIdx.x; col < s.sw; col += blockDim.x) {
    uint64_t b = kNoKey;
    for (int r = 0; r < t.rgs; ++r) {
      const uint64_t x = merge[static_cast<size_t>(r) * s.sw + col];
      b = x < b ? x : b;
    }
    one(col, b);
  }
}

// Dynamic IN bound, after a commit: every unsettled node u has W[u][v] >= the smallest
// in-weight of column v from rows still unsettled, so that weight may replace minin[v] in the IN
// criterion and the column filter (a shorter path to v must enter it from an unsettled u, whose
// dist is at least m).  Column v lists its kInLists smallest in-weights with their rows
// (ascending) and a lower bound on the rest; cursor k0 skips listed rows known settled.  A row
// counts as settled only once its phase stamp (phase + 1; 0 for the source) is at most `phase`,
// i.e. it settled in an earlier phase: every CTA's commit of those phases precedes the barrier
// this one passed, so the bound is the same in every run.  Rows settled since are treated as
// unsettled, which only makes the bound smaller.  One row is checked per column and phase.
// The same for the OUT bound (dynamic OUT): every unsettled u and unsettled w != u have
// W[u][w] >= the smallest out-weight of row u to columns still unsettled, which may replace
// minout[u] in L = min over unsettled u of dist[u] + minout[u].  If an unsettled x with dist[x] < L
// were not final, take on a shortest path to x the first unsettled node y whose successor z is
// unsettled (one exists: otherwise x's predecessor is settled and dist[x] is exact); y's
// predecessor is settled, so dist[y] is exact and the path is at least dist[y] + W[y][z] >= L.
// L also still bounds every offer that could change a settled column v (the column filter's use
// of it): only a tie can, from a row u unsettled now; a column settled in the previous phase is
// not yet excluded from u's minimum, and one settled earlier cannot be tied by such a u at all
// (had v been settled by the IN bound, u would have been at dist m then and settled with it; by
// the OUT bound, every u with dist[u] < dist[v] was final then and settled with it).
struct DynIn {
  const uint2* list;   // shared: [sw][kList] (weight, row) of the columns' in-edges
  const uint32_t* rest;
  uint8_t* k0;
  const uint2* olist;  // shared: [sw][kList] (weight, column) of the slice's nodes' out-edges
  const uint32_t* orest;
  uint8_t* ok0;
  uint32_t* sph;        // global phase stamps (phase + 1 of each node's settlement; the source's 0)
  uint32_t* pre;        // shared: [sw][2] the stamps the next update checks, fetched ahead
  uint8_t* stamped;     // shared: [sw] the column's own stamp is written
};
// Start fetching (cp.async) the stamps the next dyn_in_update checks, one or two per unsettled
// column, right after a phase's decision: they arrive while the phase relaxes.  A stamp read this
// early may miss a settlement of the running phase, which the update's rule ignores anyway.
template <int kList>
__device__ __forceinline__ void dyn_in_prefetch(const Slice& s, const DynIn& dy) {
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
    const bool open = !s.vis[j];
    const int k = dy.k0[j], ko = dy.olist ? dy.ok0[j] : kList;
    // each slot is written once: by the copy, or (nothing to check) with all ones
    if (open && k < kList && dy.list[j * kList + k].x < kInf)
      cp_async4(dy.pre + 2 * j, dy.sph + dy.list[j * kList + k].y);
    else
      dy.pre[2 * j] = 0xFFFFFFFFu;
    if (open && ko < kList && dy.olist[j * kList + ko].x < kInf)
      cp_async4(dy.pre + 2 * j + 1, dy.sph + dy.olist[j * kList + ko].y);
    else
      dy.pre[2 * j + 1] = 0xFFFFFFFFu;
  }
  cp_async_commit();
}
// After the commit of phase `phase`: stamp the columns this phase settled (phase + 1), then move
// the cursors of the unsettled ones.
template <int kList>
__device__ __forceinline__ void dyn_in_update(const Slice& s, const DynIn& dy, uint32_t phase) {
  cp_async_wait_all();  // this thread's prefetches (the same columns it checks below)
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
    if (s.vis[j]) {
      if (!dy.stamped[j]) {
        dy.sph[s.c0 + j] = phase + 1;
        dy.stamped[j] = 1;
      }
      continue;
    }
    const int k = dy.k0[j], ko = dy.olist ? dy.ok0[j] : kList;
    // an exhausted list (INF entry) keeps its bound: its stamp slot holds all ones
    const uint32_t sp = k < kList ? dy.pre[2 * j] : 0xFFFFFFFFu;
    const uint32_t spo = ko < kList ? dy.pre[2 * j + 1] : 0xFFFFFFFFu;
    if (sp <= phase) {
      dy.k0[j] = static_cast<uint8_t>(k + 1);
      s.minin[j] = k + 1 < kList ? dy.list[j * kList + k + 1].x : dy.rest[j];
    }
    if (spo <= phase) {
      dy.ok0[j] = static_cast<uint8_t>(ko + 1);
      s.minout[j] = ko + 1 < kList ? dy.olist[j * kList + ko + 1].x : dy.orest[j];
    }
  }
}

__device__ __forceinline__ void slice_write_out(const Slice& s, int n, int32_t* dist_out, int32_t* pred_out) {
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
    const int v = s.c0 + j;
    if (v < n) {
      dist_out[v] = static_cast<int32_t>(s.dist[j]);
      pred_out[v] = s.pred[j];
    }
  }
}

}  // namespace dj
