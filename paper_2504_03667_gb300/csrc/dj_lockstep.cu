// Lockstep multi-source engine: many sources of ONE graph advance together,
// phase by phase, so that each matrix row a phase needs is read from HBM once
// and applied to every source that settles it in that phase.
//
// Every source runs the phase logic of dj_core.cuh (Algorithm 1 of Section
// III-A with the exact OUT and IN settle bounds and the lexicographic pred
// key), so its dist and pred are the ones Algorithm 1 gives.  What is shared
// is the streaming: a phase settles, for each source s, a set S_s of rows;
// every CTA owns a column slice, and for each "row block" (the rows whose
// nodes another CTA owns) it reads its slice of those rows once, in one bulk
// copy from a column-tiled copy of the matrix, and applies every row of the
// block to every source whose S_s contains it.  With k sources in the group
// the HBM bytes of a phase are at most one matrix (all row blocks) instead of
// sum_s |S_s| rows.
//
// Layout.  Thread t of a CTA serves source s = t / TPS and columns
// [28 (t % TPS), 28 (t % TPS) + 28) of the CTA's slice: the 28 cells' dist
// live in registers; the phase's best tie word of each cell (read only when a
// candidate ties its dist), its pred and the weight of the edge from pred (for
// the IN bound's tie rule) in shared memory.
// One phase:
//   1. each thread reduces its cells to (argmin key, dist + minout) and the
//      TPS threads of a source combine them: one partial per (source, CTA);
//   2. grid barrier; CTA b reduces the G partials of sources b, b + G, ...
//      into that source's decision (m, a, L);
//   3. grid barrier; every CTA reads all decisions, finds its settled cells,
//      and publishes them per source as tie words ((dist - m_s) << bits) | v,
//      with a prefix over the sources (a block scan, in source order);
//   4. grid barrier; every CTA streams the row blocks that hold a settled
//      cell (published list + its slice of the block's rows, one TMA bulk
//      copy each, four stages in flight) and each thread applies its
//      source's entries of the block to its 28 cells;
//   5. commit (per cell, in registers) and mark the settled cells visited.
// The loop ends when no source has a reachable unvisited node.
#include <algorithm>
#include <string>
#include <vector>

#include "dj_common.cuh"
#include "dj_core.cuh"
#include "dj_internal.h"

namespace dj {

namespace {

constexpr int kLsCols = 28;     // columns (cells) per thread
constexpr int kLsVec = kLsCols / 4;
constexpr int kLsThreads = 512;
constexpr int kLsStages = 4;    // row blocks in flight per CTA
constexpr int kLsEcap = 2560;   // published entries of a row block staged in shared memory (the rest: L2)
constexpr uint16_t kNoPred = 0xFFFF;
constexpr int kLsMinGroup = 32;  // sources per launch at least

// Control words of a lockstep launch (zero when it starts; the last CTA to
// leave zeroes them again, as in the grid engine).
constexpr int kLsBar = 0, kLsAbort = 5, kLsExit = 12, kLsCtlWords = 16;

struct LsParams {
  const int32_t* W;       // the matrix: n rows x pitch
  const int32_t* T;       // column-tiled copy: [G][n][swmax], entries of columns >= the slice width INF
  const int32_t* minout;  // n
  const int32_t* minin;   // n
  const LsSource* src;    // S sources of this launch
  uint32_t* ctl;          // control words
  uint4* partials;        // [2][S][G]  (key lo, key hi, L_c, 0)
  uint4* dec;             // [2][S]     (m, a, L, 0)
  uint32_t* regions;      // [2][G][rstride]: prefix[S + 1], then the tie words in source order
  uint32_t* totals;       // [2][G]
  uint32_t* words;        // per-device words: [0] error bits, [1] phases
  int64_t pitch;
  int64_t timeout_ns;
  int32_t n, S, TPS, swmax, rstride, nvec_total;
  uint32_t bits_u, span;
  int32_t use_in;
};

__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Tie word of a cell's stored pred relative to this phase (as stored_tie in dj_core.cuh):
// 0 = no candidate of the phase can tie-beat it, all ones = any can.
__device__ __forceinline__ uint32_t ls_stored_tie(uint32_t d, uint16_t pr, uint16_t pw, uint32_t m, uint32_t span,
                                                  uint32_t bits_u, bool use_in) {
  if (!use_in) return 0u;
  if (d >= kInf) return 0xFFFFFFFFu;
  if (pr == kNoPred) return 0u;
  const uint32_t pd = d - pw;
  if (pd < m) return 0u;
  const uint32_t dd = pd - m;
  if (dd >= span) return 0xFFFFFFFFu;
  return (dd << bits_u) | pr;
}

__device__ __forceinline__ void ls_exit(uint32_t* ctl) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctl + kLsExit, 1u) == gridDim.x - 1) {
      __threadfence();
#pragma unroll
      for (int i = 0; i < kLsCtlWords; ++i) ctl[i] = 0u;
    }
  }
}

__device__ __forceinline__ void ls_solve(const LsParams& p, uint8_t* smem, BlockScratch& sc, uint32_t& s_flag) {
  const int G = gridDim.x, b = blockIdx.x;
  const int T = static_cast<int>(blockDim.x), t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int nwarps = T >> 5;
  const int TPS = p.TPS, S = p.S;
  const int s = t / TPS, part = t - s * TPS;
  const bool active = s < S;
  const uint32_t bits_u = p.bits_u, umask = (1u << bits_u) - 1u;
  const bool use_in = p.use_in != 0;
  // this CTA's slice (as the grid engine)
  const int v0 = static_cast<int>(static_cast<int64_t>(b) * p.nvec_total / G);
  const int v1 = static_cast<int>(static_cast<int64_t>(b + 1) * p.nvec_total / G);
  const int c0 = 4 * v0, sw = 4 * (v1 - v0);
  const int swmax = p.swmax;

  // shared memory
  uint8_t* q = smem;
  uint16_t* pred16 = reinterpret_cast<uint16_t*>(q);  // [S][swmax]
  q += static_cast<size_t>(S) * swmax * 2;
  uint16_t* pw16 = reinterpret_cast<uint16_t*>(q);  // [S][swmax] weight of the edge from pred (IN tie rule)
  q += static_cast<size_t>(S) * swmax * 2;
  q = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(q) + 15) & ~uintptr_t(15));
  uint32_t* tb32 = reinterpret_cast<uint32_t*>(q);  // [S][swmax] the phase's best tie word of each cell
  q += static_cast<size_t>(S) * swmax * 4;
  uint32_t* mo = reinterpret_cast<uint32_t*>(q);  // [swmax] minout of the slice's columns
  q += static_cast<size_t>(swmax) * 4;
  uint32_t* mi = reinterpret_cast<uint32_t*>(q);  // [swmax] minin
  q += static_cast<size_t>(swmax) * 4;
  uint4* sdec = reinterpret_cast<uint4*>(q);  // [S] decisions of this phase
  q += static_cast<size_t>(S) * 16;
  uint32_t* stot = reinterpret_cast<uint32_t*>(q);  // [G] published entries per row block
  q += (static_cast<size_t>(G) + 3) / 4 * 16;
  uint64_t* bars = reinterpret_cast<uint64_t*>(q);  // [kLsStages]
  q += kLsStages * 8;
  uint32_t* sdone = reinterpret_cast<uint32_t*>(q);  // [kLsStages] warps done with each stage
  q += 16;
  int32_t* blist = reinterpret_cast<int32_t*>(q);  // [G] the phase's non-empty row blocks
  q += (static_cast<size_t>(G) + 3) / 4 * 16;
  q = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(q) + 127) & ~uintptr_t(127));
  const size_t pre_bytes = (static_cast<size_t>(S) + 1 + 3) / 4 * 16;  // prefix, padded to 16 bytes
  const size_t ent_bytes = static_cast<size_t>(kLsEcap) * 4;
  const size_t row_bytes = static_cast<size_t>(swmax) * swmax * 4;
  const size_t stage_bytes = (pre_bytes + ent_bytes + row_bytes + 127) & ~size_t(127);
  uint8_t* stages = q;

  for (int j = t; j < swmax; j += T) {
    const int v = c0 + j;
    const bool real = j < sw && v < p.n;
    mo[j] = real ? static_cast<uint32_t>(__ldg(p.minout + v)) : kInf;
    mi[j] = real ? static_cast<uint32_t>(__ldg(p.minin + v)) : kInf;
  }
  if (t < kLsStages) {
    mbar_init(bars + t, 1);
    sdone[t] = 0u;
  }
  fence_mbar_init();

  // cells: Algorithm 1's first step (the source's own row) done at initialisation
  uint32_t dist[kLsCols];
  uint32_t vis = 0, chg = 0;
  uint32_t* const tbs = tb32 + static_cast<size_t>(active ? s : 0) * swmax + part * kLsCols;  // this thread's cells
  const int jbase = part * kLsCols;
  int32_t src = -1;
  if (active) {
    src = p.src[s].source;
    const int32_t* srow = p.W + static_cast<int64_t>(src) * p.pitch + c0;
#pragma unroll
    for (int i = 0; i < kLsCols; ++i) {
      const int j = jbase + i;
      const int v = c0 + j;
      dist[i] = kInf;
      uint16_t pr = kNoPred, pw = 0;
      if (j >= sw || v >= p.n) {
        vis |= 1u << i;  // padding: never takes part
      } else if (v == src) {
        dist[i] = 0;
        vis |= 1u << i;
      } else {
        const uint32_t w = static_cast<uint32_t>(__ldg(srow + j));
        if (w < kInf) {
          dist[i] = w;
          pr = static_cast<uint16_t>(src);
          pw = static_cast<uint16_t>(min(w, 0xFFFFu));
        }
      }
      if (j < swmax) {
        pred16[static_cast<size_t>(s) * swmax + j] = pr;
        pw16[static_cast<size_t>(s) * swmax + j] = pw;
      }
    }
  }
  __syncthreads();

  uint32_t* bar = p.ctl + kLsBar;
  uint32_t* abort_flag = p.ctl + kLsAbort;
  uint32_t nbar = 0, phase = 0, gt = 0;
  __shared__ int s_nb;  // non-empty row blocks of the phase
  for (;; ++phase) {
    const uint32_t par = phase & 1u;
    // 1. partial of this thread's cells, combined over the source's TPS threads
    uint64_t key = kNoKey;
    uint32_t lc = 0xFFFFFFFFu;
    if (active) {
#pragma unroll
      for (int i = 0; i < kLsCols; ++i) {
        if ((vis >> i) & 1u) continue;
        const uint64_t kk = (static_cast<uint64_t>(dist[i]) << 32) | static_cast<uint32_t>(c0 + jbase + i);
        key = kk < key ? kk : key;
        lc = min(lc, dist[i] + mo[jbase + i]);  // <= 2^32 - 2: no wrap
      }
    }
    for (int o = 1; o < TPS; o <<= 1) {
      const uint64_t k2 = __shfl_xor_sync(0xffffffffu, key, o);
      key = k2 < key ? k2 : key;
      lc = min(lc, __shfl_xor_sync(0xffffffffu, lc, o));
    }
    if (active && part == 0)
      p.partials[(static_cast<size_t>(par) * S + s) * G + b] =
          make_uint4(static_cast<uint32_t>(key), static_cast<uint32_t>(key >> 32), lc, 0u);
    if (!grid_barrier(bar, ++nbar * static_cast<uint32_t>(G), abort_flag, p.words, p.timeout_ns, &s_flag)) return;
    // 2. decisions of the sources this CTA reduces (one warp per source)
    for (int s2 = b + G * warp; s2 < S; s2 += G * nwarps) {
      uint64_t k = kNoKey;
      uint32_t l = 0xFFFFFFFFu;
      const uint4* pp = p.partials + (static_cast<size_t>(par) * S + s2) * G;
      for (int i = lane; i < G; i += 32) {
        const uint4 x = __ldcg(pp + i);
        const uint64_t kk = (static_cast<uint64_t>(x.y) << 32) | x.x;
        k = kk < k ? kk : k;
        l = min(l, x.z);
      }
      k = warp_min_u64(k);
      l = warp_min_u32(l);
      if (lane == 0) {
        const Decision D = make_decision(k, l, p.span, false, use_in);
        p.dec[static_cast<size_t>(par) * S + s2] = make_uint4(D.m, D.a, D.L, 0u);
      }
    }
    if (!grid_barrier(bar, ++nbar * static_cast<uint32_t>(G), abort_flag, p.words, p.timeout_ns, &s_flag)) return;
    // 3. every decision; this CTA's settled cells, published per source in source order
    uint32_t any = 0;
    for (int i = t; i < S; i += T) {
      const uint4 d = __ldcg(p.dec + static_cast<size_t>(par) * S + i);
      sdec[i] = d;
      any |= d.x < kInf ? 1u : 0u;
    }
    if (__syncthreads_or(any) == 0) break;
    Decision D;
    D.m = kInf;
    D.a = 0;
    D.L = 0;
    D.span = p.span;
    D.use_in = use_in ? 1u : 0u;
    if (active) {
      const uint4 d = sdec[s];
      D.m = d.x;
      D.a = d.y;
      D.L = d.z;
    }
    uint32_t smask = 0;
    if (active && D.m < kInf) {
#pragma unroll
      for (int i = 0; i < kLsCols; ++i) {
        if ((vis >> i) & 1u) continue;
        const uint32_t d = dist[i];
        if (d < kInf && in_settled(static_cast<uint32_t>(c0 + jbase + i), d, in_key(d, mi[jbase + i]), D))
          smask |= 1u << i;
      }
    }
    const uint32_t cnt = __popc(smask);
    uint32_t incl = cnt;  // exclusive block scan in thread (= source) order
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    if (lane == 31) sc.r32[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t ws = lane < nwarps ? sc.r32[lane] : 0u;
      uint32_t wi = ws;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += x;
      }
      if (lane < nwarps) sc.r32b[lane] = wi - ws;
      if (lane == 31) sc.b32 = wi;
    }
    __syncthreads();
    const uint32_t off = sc.r32b[warp] + incl - cnt;
    const uint32_t total = sc.b32;
    uint32_t* reg = p.regions + (static_cast<size_t>(par) * G + b) * p.rstride;
    if (active && part == 0) reg[s] = off;  // the source's first entry (its threads are consecutive)
    if (t == 0) {
      reg[S] = total;
      p.totals[static_cast<size_t>(par) * G + b] = total;
    }
    if (smask) {
      uint32_t w = off;
#pragma unroll
      for (int i = 0; i < kLsCols; ++i)
        if ((smask >> i) & 1u) reg[S + 1 + w++] = ((dist[i] - D.m) << bits_u) | static_cast<uint32_t>(c0 + jbase + i);
    }
    fence_proxy_async_global();  // the lists are read by bulk copies after the barrier
    // the phase's starting key of every cell: (dist, the stored pred's tie word)
    if (active) {
#pragma unroll
      for (int i = 0; i < kLsCols; ++i) {
        if (jbase + i >= swmax) break;
        const size_t at = static_cast<size_t>(s) * swmax + jbase + i;
        tbs[i] = ls_stored_tie(dist[i], pred16[at], pw16[at], D.m, p.span, bits_u, use_in);
      }
    }
    if (!grid_barrier(bar, ++nbar * static_cast<uint32_t>(G), abort_flag, p.words, p.timeout_ns, &s_flag)) return;
    // 4. stream the row blocks holding settled cells and relax.  Warps run decoupled: each waits
    //    only for a block's copies, and the last warp done with a stage issues the copies of the
    //    block kLsStages further on, so warps with more entries in one block catch up in the next.
    for (int i = t; i < G; i += T) stot[i] = __ldcg(p.totals + static_cast<size_t>(par) * G + i);
    __syncthreads();
    if (t == 0) {  // the non-empty blocks, in order (the same list in every thread)
      int nb = 0;
      for (int rb = 0; rb < G; ++rb)
        if (stot[rb] != 0) blist[nb++] = rb;
      s_nb = nb;
    }
    __syncthreads();
    const int nb = s_nb;
    auto block_rows = [&](int rb, int* rc0) {
      const int a0 = static_cast<int>(static_cast<int64_t>(rb) * p.nvec_total / G);
      const int a1 = static_cast<int>(static_cast<int64_t>(rb + 1) * p.nvec_total / G);
      *rc0 = 4 * a0;
      return max(0, min(4 * (a1 - a0), p.n - 4 * a0));
    };
    auto issue = [&](int rb, uint32_t g) {  // one thread
      uint8_t* st = stages + static_cast<size_t>(g % kLsStages) * stage_bytes;
      int rc0 = 0;
      const int rows = block_rows(rb, &rc0);
      const uint32_t ne = min(stot[rb], static_cast<uint32_t>(kLsEcap));
      const uint32_t lbytes = ((static_cast<uint32_t>(S) + 1u + ne) * 4u + 15u) & ~15u;
      const uint32_t rbytes = static_cast<uint32_t>(rows) * static_cast<uint32_t>(swmax) * 4u;
      uint64_t* bq = bars + (g % kLsStages);
      fence_proxy_async_global();  // the lists other CTAs published before the barrier
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bq, lbytes + rbytes);
      bulk_g2s(st, p.regions + (static_cast<size_t>(par) * G + rb) * p.rstride, lbytes, bq);
      if (rbytes)
        bulk_g2s(st + pre_bytes + ent_bytes,
                 p.T + (static_cast<size_t>(b) * p.n + static_cast<size_t>(rc0)) * static_cast<size_t>(swmax), rbytes, bq);
    };
    if (t == 0)
      for (int i = 0; i < min(nb, kLsStages); ++i) issue(blist[i], gt + static_cast<uint32_t>(i));
    const uint32_t m = D.m;
    bool ok = true;
    for (int idx = 0; idx < nb; ++idx) {
      const int rb = blist[idx];
      const uint32_t g = gt + static_cast<uint32_t>(idx);
      const uint32_t slot = g % kLsStages;
      uint8_t* st = stages + static_cast<size_t>(slot) * stage_bytes;
      if (!mbar_wait_bounded(bars + slot, (g / kLsStages) & 1u, p.timeout_ns)) {
        ok = false;
        mbar_wait_bounded(bars + slot, (g / kLsStages) & 1u, p.timeout_ns);  // drain once more
      }
      int rc0 = 0;
      block_rows(rb, &rc0);
      const uint32_t* pre = reinterpret_cast<const uint32_t*>(st);
      const uint32_t* ent = pre + S + 1;
      const uint32_t* gent = p.regions + (static_cast<size_t>(par) * G + rb) * p.rstride + S + 1;
      const int4* rowsm = reinterpret_cast<const int4*>(st + pre_bytes + ent_bytes);
      if (active && m < kInf) {
        const uint32_t e0 = pre[s], e1 = pre[s + 1];
        for (uint32_t e = e0; e < e1; ++e) {
          const uint32_t tw = e < static_cast<uint32_t>(kLsEcap) ? ent[e] : __ldcg(gent + e);
          const uint32_t u = tw & umask;
          const uint32_t du = m + (tw >> bits_u);
          const int4* rv = rowsm + (static_cast<size_t>(u - rc0) * swmax + jbase) / 4;
#pragma unroll
          for (int k = 0; k < kLsVec; ++k) {
            if (jbase + 4 * k >= swmax) break;
            const int4 x = rv[k];
            const uint32_t c4[4] = {du + static_cast<uint32_t>(x.x), du + static_cast<uint32_t>(x.y),
                                    du + static_cast<uint32_t>(x.z), du + static_cast<uint32_t>(x.w)};
            // common case: no candidate reaches its cell's dist (four compares); the exact rule
            // (strict improvement, or a tie won by a smaller tie word) only otherwise
            const bool hit = (c4[0] <= dist[4 * k]) | (c4[1] <= dist[4 * k + 1]) | (c4[2] <= dist[4 * k + 2]) |
                             (c4[3] <= dist[4 * k + 3]);
            if (hit) {
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const int i = 4 * k + qq;
                const uint32_t c = c4[qq];
                if (c >= kInf) continue;  // an INF entry from a row at dist 0 never commits
                if (c < dist[i]) {
                  dist[i] = c;
                  tbs[i] = tw;
                  chg |= 1u << i;
                } else if (c == dist[i] && tw < tbs[i]) {
                  tbs[i] = tw;
                  chg |= 1u << i;
                }
              }
            }
          }
        }
      }
      // this warp is done with the stage; the last warp to finish it issues the copies of the
      // block kLsStages further on into it
      fence_proxy_async_smem();  // this thread's reads of the stage precede the next copy into it
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        if (atomicAdd(&sdone[slot], 1u) == static_cast<uint32_t>(nwarps) - 1u) {
          sdone[slot] = 0u;
          __threadfence_block();
          if (idx + kLsStages < nb) issue(blist[idx + kLsStages], g + kLsStages);
        }
      }
    }
    gt += static_cast<uint32_t>(nb);
    __syncthreads();  // every warp is past this phase's stages
    if (!ok) {
      atomicOr(p.words, kErrTimeout);
      atomicExch(abort_flag, 1u);
    }
    // 5. commit: a cell whose key changed took a strictly smaller one; mark the settled cells visited
    if (active && chg) {
#pragma unroll
      for (int i = 0; i < kLsCols; ++i) {
        if (!((chg >> i) & 1u)) continue;
        const size_t at = static_cast<size_t>(s) * swmax + jbase + i;
        const uint32_t tw = tbs[i];
        pred16[at] = static_cast<uint16_t>(tw & umask);
        pw16[at] = static_cast<uint16_t>(min(dist[i] - (m + (tw >> bits_u)), 0xFFFFu));
      }
    }
    chg = 0;
    vis |= smask;
  }
  // results
  if (active) {
    int32_t* dout = p.src[s].dist;
    int32_t* pout = p.src[s].pred;
#pragma unroll
    for (int i = 0; i < kLsCols; ++i) {
      const int j = jbase + i;
      const int v = c0 + j;
      if (j < sw && v < p.n) {
        const uint16_t pr = pred16[static_cast<size_t>(s) * swmax + j];
        dout[v] = static_cast<int32_t>(dist[i]);
        pout[v] = pr == kNoPred ? -1 : static_cast<int32_t>(pr);
      }
    }
  }
  if (b == 0 && t == 0) p.words[1] = phase;
}

__global__ void __launch_bounds__(kLsThreads, 1) k_sssp_lockstep(const LsParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ BlockScratch sc;
  __shared__ uint32_t s_flag;
  pdl_launch_dependents();
  pdl_wait();
  ls_solve(p, smem, sc, s_flag);  // returns early (uniformly per CTA) on a timeout
  ls_exit(p.ctl);
}

// T[b][r][c] = W[r][c0_b + c] for c < the width of slice b, INF beyond (c < swmax).
__global__ void k_tile_columns(const int32_t* __restrict__ W, int64_t pitch, int32_t n, int32_t G, int32_t nvec_total,
                               int32_t swmax, int32_t* __restrict__ T) {
  const int64_t per_b = static_cast<int64_t>(n) * (swmax / 4);
  const int64_t total = per_b * G;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(i / per_b);
    const int64_t rem = i - static_cast<int64_t>(b) * per_b;
    const int64_t r = rem / (swmax / 4);
    const int cv = static_cast<int>(rem - r * (swmax / 4));
    const int a0 = static_cast<int>(static_cast<int64_t>(b) * nvec_total / G);
    const int a1 = static_cast<int>(static_cast<int64_t>(b + 1) * nvec_total / G);
    int4 x = make_int4(int(kInf), int(kInf), int(kInf), int(kInf));
    if (cv < a1 - a0) x = *reinterpret_cast<const int4*>(W + r * pitch + 4 * (a0 + cv));
    reinterpret_cast<int4*>(T)[i] = x;
  }
}

}  // namespace

// Shared memory of one lockstep CTA (must match the carving in ls_solve).
static size_t ls_smem_bytes(int S, int swmax, int G) {
  size_t b = static_cast<size_t>(S) * swmax * 4;  // pred16 + pw16
  b = (b + 15) & ~size_t(15);
  b += static_cast<size_t>(S) * swmax * 4;        // tie words
  b += static_cast<size_t>(swmax) * 8;            // minout, minin
  b += static_cast<size_t>(S) * 16;               // decisions
  b += (static_cast<size_t>(G) + 3) / 4 * 16;     // per-block totals
  b += kLsStages * 8 + 16;                        // mbarriers, stage done counters
  b += (static_cast<size_t>(G) + 3) / 4 * 16;     // non-empty block list
  b += 128;                                       // stage alignment
  const size_t pre = (static_cast<size_t>(S) + 1 + 3) / 4 * 16;
  const size_t stage = (pre + static_cast<size_t>(kLsEcap) * 4 + static_cast<size_t>(swmax) * swmax * 4 + 127) & ~size_t(127);
  return b + kLsStages * stage;
}

int plan_lockstep(const dj_graph* g, int32_t k, LockstepPlan* plan) {
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  if (!ctx->coop) return set_error(DJ_EUNSUPPORTED, "device lacks cooperative launch");
  if (g->format != DJ_FORMAT_DENSE) return set_error(DJ_EUNSUPPORTED, "lockstep batches need the dense matrix");
  if (g->n > 65535) return set_error(DJ_EUNSUPPORTED, "lockstep batches keep 16-bit predecessors (n <= 65535)");
  const int nvec_total = g->pitch / 4;
  const int G = std::min(ctx->num_sms, nvec_total);
  const int nvec_cta = (nvec_total + G - 1) / G;
  const int swmax = 4 * nvec_cta;
  int TPS = 1;
  while (TPS * kLsCols < swmax) TPS *= 2;
  if (TPS > 32) return set_error(DJ_EUNSUPPORTED, "slices too wide for the lockstep engine");
  int S = std::min(kLsThreads / TPS, 256);
  const size_t budget = static_cast<size_t>(ctx->max_smem_optin) - 1024;
  while (S > 1 && ls_smem_bytes(S, swmax, G) > budget) S /= 2;
  // groups of fewer sources share too little to pay for three grid barriers per phase
  if (S < kLsMinGroup || ls_smem_bytes(S, swmax, G) > budget)
    return set_error(DJ_EUNSUPPORTED, "lockstep layout holds fewer than 32 sources per group at this n");
  plan->G = G;
  plan->TPS = TPS;
  plan->swmax = swmax;
  plan->S_max = S;
  plan->nvec_total = nvec_total;
  plan->groups = k > 0 ? (k + S - 1) / S : 0;
  plan->S = plan->groups > 0 ? (k + plan->groups - 1) / plan->groups : 0;  // balanced groups
  plan->smem = ls_smem_bytes(plan->S > 0 ? plan->S : 1, swmax, G);
  plan->rstride = static_cast<int>(((static_cast<size_t>(plan->S) + 1 + static_cast<size_t>(plan->S) * swmax + 3) / 4) * 4);
  plan->k = k;
  const void* fn = reinterpret_cast<const void*>(&k_sssp_lockstep);
  if (int rc = prepare_function(ctx, fn, plan->smem, false)) return rc;
  int occ = 0;
  if (int rc = function_occupancy(ctx, fn, kLsThreads, plan->smem, &occ)) return rc;
  cudaError_t e = cudaSuccess;
  if (occ < 1) return set_error(DJ_EUNSUPPORTED, "lockstep engine cannot be resident");
  // workspace: control words, partials, decisions, per-block totals and published lists
  const size_t ctl = 256;
  const size_t part = static_cast<size_t>(2) * plan->S * G * 16;
  const size_t dec = static_cast<size_t>(2) * plan->S * 16;
  const size_t tot = (static_cast<size_t>(2) * G * 4 + 15) & ~size_t(15);
  const size_t regs = static_cast<size_t>(2) * G * plan->rstride * 4 + 64;  // + slack for 16-byte copy rounding
  plan->off_part = ctl;
  plan->off_dec = ctl + part;
  plan->off_tot = plan->off_dec + dec;
  plan->off_reg = plan->off_tot + tot;
  plan->ws_bytes = plan->off_reg + regs;
  return DJ_OK;
}

// The column-tiled copy of g's matrix for G slices (kept with the graph until it is freed).
int lockstep_tiles(dj_graph* g, const LockstepPlan& plan, cudaStream_t st, const int32_t** out) {
  if (g->tiled && g->tiled_G == plan.G) {
    *out = g->tiled;
    return DJ_OK;
  }
  if (g->tiled) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize(tiled copy)");
    cudaFree(g->tiled);
    g->bytes -= g->tiled_bytes;
    g->tiled = nullptr;
  }
  const size_t bytes = static_cast<size_t>(plan.G) * g->n * plan.swmax * 4;
  cudaError_t e = cudaMalloc(&g->tiled, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g->tiled = nullptr;
    return set_error(DJ_ENOMEM, "cudaMalloc of the column-tiled matrix failed (" + std::to_string(bytes) + " bytes)");
  }
  g->tiled_G = plan.G;
  g->tiled_bytes = bytes;
  g->bytes += bytes;
  const int64_t work = static_cast<int64_t>(plan.G) * g->n * (plan.swmax / 4);
  const int blocks = static_cast<int>(std::min<int64_t>((work + 255) / 256, 152 * 32));
  k_tile_columns<<<std::max(blocks, 1), 256, 0, st>>>(g->W, g->pitch, g->n, plan.G, plan.nvec_total, plan.swmax, g->tiled);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "k_tile_columns");
  *out = g->tiled;
  return DJ_OK;
}

int run_lockstep(const dj_graph* g, const LockstepPlan& plan, const int32_t* tiled, const LsSource* src_dev,
                 uint8_t* ws, uint32_t* words, int64_t timeout_ns, int allow_in, cudaStream_t st) {
  for (int gi = 0; gi < plan.groups; ++gi) {
    const int first = gi * plan.S;
    const int S = std::min(plan.S, plan.k - first);
    LsParams p;
    p.W = g->W;
    p.T = tiled;
    p.minout = g->minout;
    p.minin = g->minin;
    p.src = src_dev + first;
    p.ctl = reinterpret_cast<uint32_t*>(ws);
    p.partials = reinterpret_cast<uint4*>(ws + plan.off_part);
    p.dec = reinterpret_cast<uint4*>(ws + plan.off_dec);
    p.totals = reinterpret_cast<uint32_t*>(ws + plan.off_tot);
    p.regions = reinterpret_cast<uint32_t*>(ws + plan.off_reg);
    p.words = words;
    p.pitch = g->pitch;
    p.timeout_ns = timeout_ns > 0 ? timeout_ns : 2000000000LL;
    p.n = g->n;
    p.S = S;
    p.TPS = plan.TPS;
    p.swmax = plan.swmax;
    p.rstride = plan.rstride;
    p.nvec_total = plan.nvec_total;
    p.bits_u = host_bits_for(static_cast<uint32_t>(g->n));
    p.span = host_span_for(static_cast<uint32_t>(g->n));
    // the IN bound's tie rule keeps the pred edge's weight in 16 bits
    p.use_in = (allow_in && g->wmin >= 1 && g->wmax < 0xFFFF) ? 1 : 0;
    void* args[] = {&p};
    cudaError_t e = launch_cooperative(reinterpret_cast<void*>(&k_sssp_lockstep), plan.G, kLsThreads, args, plan.smem,
                                       st, true);
    if (e != cudaSuccess) return cuda_error(e, "cooperative launch (lockstep engine)");
  }
  return DJ_OK;
}

}  // namespace dj
