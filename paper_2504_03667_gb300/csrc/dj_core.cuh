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
//   - L is capped at m + 2^(32 - bits(n)) so (dist[u] - m, u) packs into 32
//     bits; a smaller L only shrinks S, and S always contains a.
// All sums are unsigned 32-bit: dist <= INF and G <= INF, so dist + G never
// wraps, and an INF entry yields a candidate >= INF that never improves.
#pragma once

#include "dj_common.cuh"

namespace dj {

struct BlockScratch {
  uint64_t r64[32];
  uint32_t r32[32];
  uint32_t cnt[33];
  uint64_t b64;
  uint32_t b32;
  uint32_t pad;
};

// Column-slice state of one CTA (all shared memory).
struct Slice {
  uint32_t* dist;
  int32_t* pred;
  uint32_t* minout;
  uint8_t* vis;
  int c0;    // first column (node id) of the slice, a multiple of 4
  int sw;    // columns in the slice, a multiple of 4
  int nvec;  // sw / 4
};

// Global decision of one phase.
struct Decision {
  uint32_t m;  // smallest unvisited dist (kInf: done)
  uint32_t a;  // its node (smallest index on ties)
  uint32_t L;  // settle bound: S = {unvisited v : dist[v] < L} u {a}
};

__device__ __forceinline__ void slice_init(const Slice& s, int n, int source, const int32_t* minout_g,
                                           bool need_minout) {
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
    int v = s.c0 + j;
    bool real = v < n;
    s.dist[j] = (real && v == source) ? 0u : kInf;
    s.pred[j] = -1;
    s.vis[j] = real ? 0 : 1;  // padding columns never take part
    s.minout[j] = (real && need_minout) ? static_cast<uint32_t>(__ldg(minout_g + v)) : kInf;
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

// Local partial of step 1: returns the slice's argmin key (dist << 32 | v) and
// its settle bound L_c (already capped), and writes the candidates
// {unvisited v : dist[v] < L_c} u {argmin} as (v, dist[v]) to `out`
// (compacted, increasing v).  Returns the candidate count.  `plain` publishes
// the argmin only.
__device__ __forceinline__ int slice_publish(const Slice& s, uint32_t span, bool plain, uint2* out,
                                             uint64_t* key_out, uint32_t* Lc_out, BlockScratch* sc) {
  uint64_t key = kNoKey;
  uint32_t lc = 0xFFFFFFFFu;
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
    if (!s.vis[j]) {
      uint32_t d = s.dist[j];
      uint64_t kj = (static_cast<uint64_t>(d) << 32) | static_cast<uint32_t>(s.c0 + j);
      key = kj < key ? kj : key;
      lc = min(lc, d + s.minout[j]);  // <= 2^32 - 2: no wrap
    }
  }
  block_min2(key, lc, sc);
  const uint32_t mc = static_cast<uint32_t>(key >> 32);
  const uint32_t ac = static_cast<uint32_t>(key);
  uint32_t Lc;
  if (mc >= kInf) {
    Lc = 0xFFFFFFFFu;  // nothing reachable left in this slice: no bound
  } else if (plain) {
    Lc = mc;  // only the argmin itself
  } else {
    Lc = min(min(lc, mc + span), kInf);
  }
  *key_out = key;
  *Lc_out = Lc;
  if (mc >= kInf) return 0;
  // compaction of {unvisited, dist < Lc} u {argmin}
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int base = 0;
  for (int j0 = 0; j0 < s.sw; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    bool p = false;
    uint32_t d = 0;
    if (j < s.sw && !s.vis[j]) {
      d = s.dist[j];
      p = d < Lc || static_cast<uint32_t>(s.c0 + j) == ac;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, p);
    if (lane == 0) sc->cnt[w] = __popc(bal);
    __syncthreads();
    if (w == 0) {
      uint32_t c = lane < nw ? sc->cnt[lane] : 0;
      uint32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (lane < nw) sc->cnt[lane] = incl - c;
      if (lane == 31) sc->cnt[32] = incl;
    }
    __syncthreads();
    if (p) out[base + sc->cnt[w] + __popc(bal & ((1u << lane) - 1u))] =
        make_uint2(static_cast<uint32_t>(s.c0 + j), d);
    base += sc->cnt[32];
    __syncthreads();
  }
  return base;
}

// Combine per-CTA partials (key, Lc) into the phase decision.
__device__ __forceinline__ Decision make_decision(uint64_t key, uint32_t Lc, uint32_t span, bool plain) {
  Decision d;
  d.m = static_cast<uint32_t>(key >> 32);
  d.a = static_cast<uint32_t>(key);
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

__device__ __forceinline__ bool in_settled(uint32_t u, uint32_t du, const Decision& D) {
  return du < D.L || u == D.a;
}

// Step 3 for the CTA's own nodes: mark the settled ones visited.
__device__ __forceinline__ void slice_mark(const Slice& s, const Decision& D) {
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
    if (!s.vis[j] && in_settled(static_cast<uint32_t>(s.c0 + j), s.dist[j], D)) s.vis[j] = 1;
  }
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

template <int V>
__device__ __forceinline__ void best_reset(uint64_t (&best)[V][4]) {
#pragma unroll
  for (int k = 0; k < V; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) best[k][c] = kNoKey;
}

// Apply U rows (entries e[], already filtered: e.x == 0xffffffff marks an
// empty slot) to the lane's columns.
template <int V, int U>
__device__ __forceinline__ void relax_rows(const uint2 (&e)[U], const int32_t* __restrict__ Wc0, int64_t pitch,
                                           const int (&jv)[V], const bool (&jok)[V], uint32_t m,
                                           uint32_t bits_u, uint64_t (&best)[V][4]) {
  int4 x[U][V];
#pragma unroll
  for (int uu = 0; uu < U; ++uu) {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      if (e[uu].x != 0xffffffffu && jok[k]) {
        x[uu][k] = ld_stream16(Wc0 + static_cast<int64_t>(e[uu].x) * pitch + 4 * jv[k]);
      } else {
        x[uu][k] = make_int4(int(kInf), int(kInf), int(kInf), int(kInf));
      }
    }
  }
#pragma unroll
  for (int uu = 0; uu < U; ++uu) {
    const uint32_t du = e[uu].x != 0xffffffffu ? e[uu].y : kInf;
    const uint32_t tb = ((du - m) << bits_u) | (e[uu].x & ((1u << bits_u) - 1u));
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const uint32_t c0 = du + static_cast<uint32_t>(x[uu][k].x);
      const uint32_t c1 = du + static_cast<uint32_t>(x[uu][k].y);
      const uint32_t c2 = du + static_cast<uint32_t>(x[uu][k].z);
      const uint32_t c3 = du + static_cast<uint32_t>(x[uu][k].w);
      const uint64_t k0 = (static_cast<uint64_t>(c0) << 32) | tb;
      const uint64_t k1 = (static_cast<uint64_t>(c1) << 32) | tb;
      const uint64_t k2 = (static_cast<uint64_t>(c2) << 32) | tb;
      const uint64_t k3 = (static_cast<uint64_t>(c3) << 32) | tb;
      best[k][0] = k0 < best[k][0] ? k0 : best[k][0];
      best[k][1] = k1 < best[k][1] ? k1 : best[k][1];
      best[k][2] = k2 < best[k][2] ? k2 : best[k][2];
      best[k][3] = k3 < best[k][3] ? k3 : best[k][3];
    }
  }
}

// Relaxation over `cnt` entries produced by `get(i)` (entries are (u, dist[u])
// candidates; the ones outside the settled set are skipped).  Entries of the
// next iteration are fetched before the current rows are consumed.
template <int V, int U, class Get>
__device__ __forceinline__ void relax_entries(const Get& get, int cnt, const Slice& s, const Tile& t,
                                              const int32_t* __restrict__ W, int64_t pitch, const Decision& D,
                                              uint32_t bits_u, uint64_t (&best)[V][4]) {
  if (!t.active) return;
  const int lane = threadIdx.x & 31;
  int jv[V];
  bool jok[V];
#pragma unroll
  for (int k = 0; k < V; ++k) {
    jv[k] = (t.wc * V + k) * 32 + lane;
    jok[k] = jv[k] < s.nvec;
  }
  const int32_t* Wc0 = W + s.c0;
  const int step = t.rgs * U;
  uint2 nxt[U];
#pragma unroll
  for (int uu = 0; uu < U; ++uu) {
    const int idx = t.rg + uu * t.rgs;
    nxt[uu] = idx < cnt ? get(idx) : make_uint2(0xffffffffu, kInf);
  }
  for (int i = t.rg; i < cnt; i += step) {
    uint2 e[U];
#pragma unroll
    for (int uu = 0; uu < U; ++uu) {
      e[uu] = nxt[uu];
      if (e[uu].x != 0xffffffffu && !in_settled(e[uu].x, e[uu].y, D)) e[uu].x = 0xffffffffu;
    }
#pragma unroll
    for (int uu = 0; uu < U; ++uu) {
      const int idx = i + step + uu * t.rgs;
      nxt[uu] = idx < cnt ? get(idx) : make_uint2(0xffffffffu, kInf);
    }
    relax_rows<V, U>(e, Wc0, pitch, jv, jok, D.m, bits_u, best);
  }
}

__device__ __forceinline__ void commit_key(const Slice& s, int col, uint64_t key, uint32_t bits_u) {
  const uint32_t c = static_cast<uint32_t>(key >> 32);
  if (c < s.dist[col]) {
    s.dist[col] = c;
    s.pred[col] = static_cast<int32_t>(static_cast<uint32_t>(key) & ((1u << bits_u) - 1u));
  }
}

// Merge the row groups' keys and commit.  Ends synced.
template <int V>
__device__ __forceinline__ void merge_commit(const Slice& s, const Tile& t, uint64_t* merge, uint32_t bits_u,
                                             uint64_t (&best)[V][4]) {
  const int lane = threadIdx.x & 31;
  if (t.rgs == 1) {
    if (t.active) {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int jv = (t.wc * V + k) * 32 + lane;
        if (jv < s.nvec) {
#pragma unroll
          for (int c = 0; c < 4; ++c) commit_key(s, 4 * jv + c, best[k][c], bits_u);
        }
      }
    }
    __syncthreads();
    return;
  }
  if (t.active) {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int jv = (t.wc * V + k) * 32 + lane;
      if (jv < s.nvec) {
        uint64_t* dst = merge + static_cast<size_t>(t.rg) * s.sw + 4 * jv;
#pragma unroll
        for (int c = 0; c < 4; ++c) dst[c] = best[k][c];
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
    commit_key(s, col, b, bits_u);
  }
  __syncthreads();
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
