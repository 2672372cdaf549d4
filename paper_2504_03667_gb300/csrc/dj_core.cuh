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
// (compacted, in no particular order).  Returns the candidate count.  `plain` publishes
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
  // append {unvisited, dist < Lc} u {argmin}: one shared-memory atomic per warp
  // (the order of the list is irrelevant: the relaxation keys are order-free)
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) sc->cnt[32] = 0;
  __syncthreads();
  for (int j0 = 0; j0 < s.sw; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    bool p = false;
    uint32_t d = 0;
    if (j < s.sw && !s.vis[j]) {
      d = s.dist[j];
      p = d < Lc || static_cast<uint32_t>(s.c0 + j) == ac;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, p);
    if (bal) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&sc->cnt[32], static_cast<uint32_t>(__popc(bal)));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (p) out[base + __popc(bal & ((1u << lane) - 1u))] = make_uint2(static_cast<uint32_t>(s.c0 + j), d);
    }
  }
  __syncthreads();
  const int total = static_cast<int>(sc->cnt[32]);
  __syncthreads();
  return total;
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

// Settled rows are staged in shared memory as their 32-bit tie-break word
// tb = ((dist[u] - m) << bits_u) | u  (dist[u] = m + (tb >> bits_u)).
// stage_list appends the settled entries among candidates [begin, end) of
// `get` to `list` (order irrelevant) and returns the new count.  Ends synced.
template <class Get>
__device__ __forceinline__ int stage_list(const Get& get, int begin, int end, const Decision& D, uint32_t bits_u,
                                          uint32_t* list, int base, BlockScratch* sc) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) sc->cnt[32] = static_cast<uint32_t>(base);
  __syncthreads();
  constexpr int K = 4;
  for (int i0 = begin; i0 < end; i0 += K * blockDim.x) {
    uint2 e[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = i0 + k * blockDim.x + threadIdx.x;
      e[k] = i < end ? get(i) : make_uint2(0xffffffffu, kInf);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool p = e[k].x != 0xffffffffu && in_settled(e[k].x, e[k].y, D);
      const uint32_t bal = __ballot_sync(0xffffffffu, p);
      if (bal) {
        uint32_t pos = 0;
        if (lane == 0) pos = atomicAdd(&sc->cnt[32], static_cast<uint32_t>(__popc(bal)));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (p) list[pos + __popc(bal & ((1u << lane) - 1u))] = ((e[k].y - D.m) << bits_u) | e[k].x;
      }
    }
  }
  __syncthreads();
  const int total = static_cast<int>(sc->cnt[32]);
  __syncthreads();
  return total;
}

// A warp's ring of `depth` stages x U row slots in shared memory, filled by
// 1-D TMA bulk copies (one per row) that complete on the stage's mbarrier.
// Only this warp issues into and reads from its ring, so no other warp ever
// waits on it.  `gt` counts the warp's stages over the whole kernel: stage g
// uses slot g % depth and waits for parity (g / depth) & 1 (depth = 2^lg).
struct Ring {
  uint8_t* buf;
  uint64_t* bar;
  uint32_t lg;        // log2(depth)
  uint32_t rowbytes;  // bytes of this warp's column chunk of one row (0: idle warp)
  uint32_t gt;
};

// Per-column running best of one relaxation pass: candidate value bc and its
// tie-break word bt.  It starts at (dist[v], 0): a candidate that does not beat
// the current dist can never be committed, and a tie with it never wins.
template <int V>
struct Best {
  uint32_t bc[V][4];
  uint32_t bt[V][4];
};

template <int V>
__device__ __forceinline__ void best_init(Best<V>& b, const Slice& s, const Tile& t) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const int jv = (t.wc * V + k) * 32 + lane;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      b.bc[k][c] = (t.active && jv < s.nvec) ? s.dist[4 * jv + c] : kInf;
      b.bt[k][c] = 0;
    }
  }
}

__device__ __forceinline__ void best_update(uint32_t c, uint32_t tb, uint32_t& bc, uint32_t& bt) {
  if (c < bc || (c == bc && tb < bt)) {
    bc = c;
    bt = tb;
  }
}

// Relax the `cnt` staged rows over this CTA's slice.  Row group rg takes
// list entries rg, rg + rgs, ...; its column-chunk warp streams those rows'
// slices through its ring `depth` stages ahead of the arithmetic.  The common
// case (no lane improves or ties its column) costs four adds, four compares
// and one vote per row; the exact lexicographic update runs only otherwise.
template <int V, int U>
__device__ __forceinline__ bool relax_list(const uint32_t* __restrict__ list, int cnt, const Slice& s, const Tile& t,
                                           const int32_t* __restrict__ W, int64_t pitch, uint32_t m, uint32_t bits_u,
                                           Ring& ring, int64_t timeout_ns, Best<V>& best) {
  if (!t.active || ring.rowbytes == 0) return true;
  const int lane = threadIdx.x & 31;
  bool jok[V];
#pragma unroll
  for (int k = 0; k < V; ++k) jok[k] = (t.wc * V + k) * 32 + lane < s.nvec;
  const uint32_t umask = (1u << bits_u) - 1u;
  const uint32_t dmask = (1u << ring.lg) - 1u;
  const int J = t.rg < cnt ? (cnt - t.rg + t.rgs - 1) / t.rgs : 0;
  const int nst = (J + U - 1) / U;
  const char* colbase = reinterpret_cast<const char*>(W + s.c0) + static_cast<size_t>(t.wc) * V * 32 * 16;
  const int64_t rowstride = pitch * 4;
  const uint32_t* mylist = list + t.rg;
  const int rgs = t.rgs;
  auto issue = [&](int st) {
    const uint32_t slot = (ring.gt + static_cast<uint32_t>(st)) & dmask;
    const int rows = min(U, J - st * U);
    uint64_t* bar = ring.bar + slot;
    if (lane == 0) mbar_arrive_expect_tx(bar, static_cast<uint32_t>(rows) * ring.rowbytes);
    __syncwarp();
    if (lane < rows) {
      const uint32_t u = mylist[(st * U + lane) * rgs] & umask;
      bulk_g2s(ring.buf + (static_cast<size_t>(slot) * U + lane) * ring.rowbytes,
               colbase + static_cast<int64_t>(u) * rowstride, ring.rowbytes, bar);
    }
  };
  const int depth = 1 << ring.lg;
  const int pre = min(depth, nst);
  for (int st = 0; st < pre; ++st) issue(st);
  bool ok = true;
  for (int st = 0; st < nst; ++st) {
    const uint32_t g = ring.gt + static_cast<uint32_t>(st);
    const uint32_t slot = g & dmask;
    const uint32_t parity = (g >> ring.lg) & 1u;
    if (!mbar_wait_bounded(ring.bar + slot, parity, timeout_ns)) {
      ok = false;
      mbar_wait_bounded(ring.bar + slot, parity, timeout_ns);  // drain once more
    }
    const int rows = min(U, J - st * U);
    const uint8_t* sb = ring.buf + static_cast<size_t>(slot) * U * ring.rowbytes + 16 * lane;
    const uint32_t* lrow = mylist + st * U * rgs;
#pragma unroll
    for (int uu = 0; uu < U; ++uu) {
      if (uu < rows) {
        const uint32_t tb = lrow[uu * rgs];
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
    if (st + depth < nst) issue(st + depth);
  }
  ring.gt += static_cast<uint32_t>(nst);
  return ok;
}

__device__ __forceinline__ void commit_key(const Slice& s, int col, uint64_t key, uint32_t bits_u) {
  const uint32_t c = static_cast<uint32_t>(key >> 32);
  if (c < s.dist[col]) {
    s.dist[col] = c;
    s.pred[col] = static_cast<int32_t>(static_cast<uint32_t>(key) & ((1u << bits_u) - 1u));
  }
}

// Merge the row groups' bests and commit.  Ends synced.
template <int V>
__device__ __forceinline__ void merge_commit(const Slice& s, const Tile& t, uint64_t* merge, uint32_t bits_u,
                                             const Best<V>& best) {
  const int lane = threadIdx.x & 31;
  if (t.rgs == 1) {
    if (t.active) {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const int jv = (t.wc * V + k) * 32 + lane;
        if (jv < s.nvec) {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            commit_key(s, 4 * jv + c, (static_cast<uint64_t>(best.bc[k][c]) << 32) | best.bt[k][c], bits_u);
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
