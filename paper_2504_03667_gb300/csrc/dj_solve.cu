// Solve engines for Algorithm 1 (Section III-A), both persistent:
//
//  * Grid engine: one cooperative launch with every SM's CTA(s) resident.  Each
//    CTA owns a contiguous column slice (its nodes' dist / pred / visited /
//    minout live in its shared memory for the whole solve); the only global
//    traffic besides the matrix rows is one 16-byte partial per CTA and the
//    candidate list per phase, exchanged through L2 around ONE grid barrier per
//    phase.  This is the in-kernel form of the paper's MPI Allreduce step
//    (Algorithm 2, Section III-B), with the 1-D column partition of
//    Section III-B applied to CTAs instead of processes.
//
//  * Cluster engine: one thread-block cluster per solve; the slices live in
//    the cluster's distributed shared memory and the per-phase exchange is a
//    DSMEM read of the other CTAs' partials and candidate lists around one
//    cluster barrier.  Clusters pull solves from a device queue, so one launch
//    runs many solves (batches, serving) and small single solves.
//
// The phase logic (what is settled per pass and why it equals Algorithm 1) is
// in dj_core.cuh.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>

#include "dj_common.cuh"
#include "dj_core.cuh"
#include "dj_internal.h"
#include "dj_noalloc_size.h"

namespace dj {

// ============================================================ grid engine

struct GridParams {
  const int32_t* W;
  const int32_t* minout;
  int32_t* dist_out;
  int32_t* pred_out;
  uint32_t* ctl;  // [0] barrier arrivals, [5] abort flag, [8] row-split snapshots published
  uint4* partials;  // [2][G]: (key lo, key hi, L_c, count)
  uint4* cand;      // [2][cand_cap] candidates (u, dist[u], IN key, 0)
  uint32_t* words;  // per-device words: [0] error bits, [1] phases
  int64_t pitch;
  int64_t timeout_ns;
  int32_t n;
  int32_t nvec_total;
  int32_t source;
  int32_t plain;
  int32_t use_in;
  uint32_t bits_u;
  uint32_t span;
  uint32_t cand_cap;
  int32_t swcap;
  int32_t rgs_cap;
  int32_t skip_cta;
  int32_t depth;     // ring stages per warp
  int32_t srows;     // rows per ring stage
  int32_t rowcap;    // bytes of one ring row slot
  int32_t trace_cap;
  uint64_t* trace;   // optional per-phase timeline (CTA 0)
  int32_t list_cap;    // staged settled rows per segment (column-filtered relaxation)
  int32_t gather_max;  // load only the live columns when at most this many groups are live (-1: never filter)
  int32_t rs_min;      // row-split relaxation for phases with at least this many candidates (0: never)
  int32_t rp_min;      // row-push relaxation (graphs that are not dense) from this many candidates (0: never)
  int32_t ring_bytes;  // bytes of the ring region (also the row-split buffers)
  uint32_t* gsnap;     // [pitch] column snapshots at the start of a row-split phase
  unsigned long long* gkey;  // [2][pitch] merged row-split keys per phase parity, all ones between uses
  TieSources ts;       // the columns' tie sources (cap 0: not used)
  int32_t sym;         // the matrix is symmetric (undirected graph): column v is row v
  // dynamic IN bound (dyn_in != 0): the columns' in-lists and the per-node settle-phase stamps
  const uint2* inlist;
  const uint32_t* inrest;
  const uint2* outlist;
  const uint32_t* outrest;
  uint32_t* sph;
  int32_t dyn_in;
};

constexpr int kMaxPartialsPerLane = 10;  // the decision warp reads up to 320 CTA partials
constexpr int kRowSplitCpt = 8;          // row split: 4-column groups per thread per column chunk
constexpr int kColPassMin = 1024;        // gather column pass: phases with at least this many candidates

// Control words of a grid launch (the first 16 words of its workspace): the
// barrier's arrival counter, the abort flag, the row split's snapshot counter
// and the exit counter.  They are zero when a launch starts: zeroed once when
// the workspace is created, and put back to zero by the last CTA to leave
// each launch (grid_exit), so back-to-back solves on one stream need no
// memset between them.
constexpr int kCtlBarrier = 0;
constexpr int kCtlAbort = 5;
constexpr int kCtlSnapshots = 8;
constexpr int kCtlExit = 12;
constexpr int kCtlWords = 16;

// Every CTA calls this once, after its last access of the control words (all
// threads, uniform control flow).  The CTA that arrives last zeroes them for
// the next launch on the stream, which starts only after this one has ended.
__device__ __forceinline__ void grid_exit(uint32_t* ctl) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's barrier arrivals precede its exit count
    if (atomicAdd(ctl + kCtlExit, 1u) == gridDim.x - 1) {
      __threadfence();
#pragma unroll
      for (int i = 0; i < kCtlWords; ++i) ctl[i] = 0u;
    }
  }
}

// DYN: the dynamic IN (and OUT) bound; a separate instantiation, so that the kernels of other
// graphs compile without its code.
template <int V, int U, bool DYN>
__device__ __forceinline__ void grid_solve(const GridParams& p, uint8_t* smem, BlockScratch& sc, Decision& s_dec,
                                           uint32_t& s_flag, uint32_t& s_rem) {
  const int G = gridDim.x, b = blockIdx.x;
  if (p.trace && b == 0 && threadIdx.x == 0 && p.trace_cap >= 10) p.trace[p.trace_cap - 2] = global_ns();  // entry
  Slice s;
  const int v0 = static_cast<int>(static_cast<int64_t>(b) * p.nvec_total / G);
  const int v1 = static_cast<int>(static_cast<int64_t>(b + 1) * p.nvec_total / G);
  s.c0 = 4 * v0;
  s.nvec = v1 - v0;
  s.sw = 4 * s.nvec;
  const int nwarps = static_cast<int>(blockDim.x >> 5);
  uint8_t* q = smem;
  uint64_t* merge = reinterpret_cast<uint64_t*>(q);
  q += p.rgs_cap > 1 ? static_cast<size_t>(p.rgs_cap) * p.swcap * 8 : 0;
  uint32_t* s_off = reinterpret_cast<uint32_t*>(q);  // [G + 1] prefix of the CTAs' candidate counts
  q += (static_cast<size_t>(G) + 1 + 3) / 4 * 16;
  uint32_t* ctab = reinterpret_cast<uint32_t*>(q);  // [G * swcap / 32 + 1] region of every 32nd candidate
  q += (static_cast<size_t>(G) * p.swcap / 32 + 1 + 3) / 4 * 16;
  s.dist = reinterpret_cast<uint32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.pred = reinterpret_cast<int32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.pdist = reinterpret_cast<uint32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.minout = reinterpret_cast<uint32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.minin = reinterpret_cast<uint32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.vis = q;
  q += (static_cast<size_t>(p.swcap) + 15) / 16 * 16;
  uint64_t* bkey = reinterpret_cast<uint64_t*>(q);  // per-column keys of the filtered relaxation
  q += static_cast<size_t>(p.swcap) * 8;
  uint64_t* gthr = reinterpret_cast<uint64_t*>(q);  // their row thresholds
  q += static_cast<size_t>(p.swcap) / 4 * 8;
  uint32_t* glist = reinterpret_cast<uint32_t*>(q);  // live 4-column groups
  q += (static_cast<size_t>(p.swcap) / 4 + 3) / 4 * 16;
  uint32_t* list = reinterpret_cast<uint32_t*>(q);  // staged settled rows
  q += static_cast<size_t>(p.list_cap) * 4;
  DynIn dy{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, p.sph, nullptr, nullptr};
  if (DYN) {  // in- (and out-) lists of the slice's nodes, rest bounds, cursors, prefetched stamps
    const bool dout = (p.dyn_in & 2) != 0;
    uint2* il = reinterpret_cast<uint2*>(q);
    q += static_cast<size_t>(p.swcap) * kInLists * 8;
    uint2* ol = reinterpret_cast<uint2*>(q);
    if (dout) q += static_cast<size_t>(p.swcap) * kInLists * 8;
    uint32_t* ir = reinterpret_cast<uint32_t*>(q);
    q += static_cast<size_t>(p.swcap) * 4;
    uint32_t* orr = reinterpret_cast<uint32_t*>(q);
    if (dout) q += static_cast<size_t>(p.swcap) * 4;
    uint8_t* stamped = q;
    q += static_cast<size_t>(p.swcap) * 4;
    uint8_t* k0 = q;
    q += (static_cast<size_t>(p.swcap) + 15) / 16 * 16;
    uint8_t* ok0 = q;
    if (dout) q += (static_cast<size_t>(p.swcap) + 15) / 16 * 16;
    dy.pre = reinterpret_cast<uint32_t*>(q);
    q += static_cast<size_t>(p.swcap) * 8;
    for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
      const int v = s.c0 + j;
      const bool real = v < p.n;
#pragma unroll
      for (int i = 0; i < kInLists; ++i) {
        il[j * kInLists + i] = real ? __ldg(p.inlist + static_cast<size_t>(v) * kInLists + i) : make_uint2(kInf, ~0u);
        if (dout)
          ol[j * kInLists + i] = real ? __ldg(p.outlist + static_cast<size_t>(v) * kInLists + i) : make_uint2(kInf, ~0u);
      }
      ir[j] = real ? __ldg(p.inrest + v) : kInf;
      if (dout) {
        orr[j] = real ? __ldg(p.outrest + v) : kInf;
        ok0[j] = 0;
      }
      k0[j] = 0;
      stamped[j] = (real && v == p.source) ? 1 : 0;
      if (real) p.sph[v] = v == p.source ? 0u : 0xFFFFFFFFu;  // ordered before use by the first barrier
    }
    dy.list = il;
    dy.rest = ir;
    dy.k0 = k0;
    dy.stamped = stamped;
    if (dout) {
      dy.olist = ol;
      dy.orest = orr;
      dy.ok0 = ok0;
    }
  }
  q = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(q) + 127) & ~uintptr_t(127));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* rings = q;  // the warps' TMA rings; in row-split phases the two row buffers
  q += static_cast<size_t>(p.ring_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(q);
  q += static_cast<size_t>(nwarps) * p.depth * 8;
  uint64_t* rbar = reinterpret_cast<uint64_t*>(q);  // the row buffers' mbarriers
  q += 16;
  uint32_t* slot_rows = reinterpret_cast<uint32_t*>(q) + static_cast<size_t>(warp) * p.depth;
  q += static_cast<size_t>(nwarps) * p.depth * 4;
  uint32_t* slot_tb = reinterpret_cast<uint32_t*>(q) + static_cast<size_t>(warp) * p.depth * U;

  if (p.plain)
    slice_init(s, p.n, p.source, p.minout, p.minout + p.n, false, false);
  else
    slice_init_source(s, p.n, p.source, p.minout, p.minout + p.n, true, p.use_in != 0, p.W, p.pitch);
  const Tile t = make_tile<V>(s.nvec, p.rgs_cap);
  Ring ring;
  ring.buf = rings + static_cast<size_t>(warp) * p.depth * p.srows * p.rowcap;
  ring.srows = static_cast<uint32_t>(p.srows);
  ring.bar = bars + static_cast<size_t>(warp) * p.depth;
  ring.depth = static_cast<uint32_t>(p.depth);
  ring.gt = 0;
  ring.rowbytes = t.active ? static_cast<uint32_t>(max(0, min(32 * V, s.nvec - t.wc * 32 * V)) * 16) : 0u;
  if (lane == 0)
    for (int i = 0; i < p.depth; ++i) mbar_init(ring.bar + i, 1);
  if (threadIdx.x == 0) {
    sc.cnt[32] = 0;
    mbar_init(rbar, 1);
    mbar_init(rbar + 1, 1);
  }
  fence_mbar_init();
  __syncthreads();

  uint32_t* bar = p.ctl + kCtlBarrier;
  uint32_t* abort_flag = p.ctl + kCtlAbort;
  if (p.gkey) {  // row-split / row-push merge keys of this slice, ordered before use by the first barrier
    for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
      p.gkey[s.c0 + j] = ~0ull;
      p.gkey[static_cast<size_t>(p.pitch) + s.c0 + j] = ~0ull;
    }
  }
  Part part;
  slice_partial(s, part);
  uint32_t phase = 0, nbar = 0, rs_gt = 0, rs_phases = 0;
  for (;;) {
    // per-phase timeline of CTA 0 (profiling only): 8 stamps per phase
    uint64_t* tr = (p.trace && b == 0 && static_cast<int>(8 * phase + 7) < p.trace_cap - 2) ? p.trace + 8 * phase
                                                                                           : nullptr;
    if (tr && threadIdx.x == 0) tr[0] = global_ns();
    // 1. publish this slice's partial and its candidates (into its own region)
    uint4* out = p.cand + (static_cast<size_t>(phase & 1) * G + b) * p.swcap;
    uint64_t key;
    uint32_t Lc;
    uint32_t unvis = 0;
    const bool packed = p.rs_min > 0 || p.rp_min > 0;
    const int c = publish_partial(s, p.span, p.plain != 0, p.use_in != 0, part, out, &sc, &key, &Lc,
                                  packed ? &unvis : nullptr);
    // with row split or row push on (slices < 2^16 columns): count | (unvisited non-candidates << 16)
    const uint32_t w4 = packed ? static_cast<uint32_t>(c) | ((unvis - static_cast<uint32_t>(c)) << 16)
                               : static_cast<uint32_t>(c);
    if (threadIdx.x == 0)
      p.partials[static_cast<size_t>(phase & 1) * G + b] =
          make_uint4(static_cast<uint32_t>(key), static_cast<uint32_t>(key >> 32), Lc, w4);
    // 2. one grid barrier per phase
    if (tr && threadIdx.x == 0) tr[1] = global_ns();
    if (b == p.skip_cta) return;  // testing: this CTA never arrives
    if (!grid_barrier(bar, ++nbar * static_cast<uint32_t>(G), abort_flag, p.words, p.timeout_ns, &s_flag,
                      tr ? tr + 2 : nullptr))
      return;
    // 3. global decision and the prefix of candidate counts, from the G partials
    if (warp == 0) {
      // lane l reads partials l, l + 32, ... (<= kMaxPartialsPerLane each, G <= 320): every load
      // instruction covers 32 consecutive partials
      uint64_t k = kNoKey;
      uint32_t l = 0xFFFFFFFFu, rem = 0, carry = 0;
      const uint4* part = p.partials + static_cast<size_t>(phase & 1) * G;
      uint4 xs[kMaxPartialsPerLane];
#pragma unroll
      for (int r = 0; r < kMaxPartialsPerLane; ++r)  // all loads in flight at once
        xs[r] = 32 * r + lane < G ? __ldcg(part + 32 * r + lane)
                                  : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u);
#pragma unroll
      for (int r = 0; r < kMaxPartialsPerLane; ++r) {
        if (32 * r >= G) break;
        const uint4 x = xs[r];
        const uint64_t kk = (static_cast<uint64_t>(x.y) << 32) | x.x;
        k = kk < k ? kk : k;
        l = min(l, x.z);
        const uint32_t cnt = packed ? (x.w & 0xFFFFu) : x.w;
        rem += packed ? (x.w >> 16) : 0u;
        uint32_t incl = cnt;  // prefix of the counts over this row of 32 partials
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t tt = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += tt;
        }
        if (32 * r + lane < G) s_off[32 * r + lane] = carry + incl - cnt;
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) s_off[G] = carry;
      k = warp_min_u64(k);
      l = warp_min_u32(l);
      rem = warp_sum_u32(rem);
      if (lane == 0) {
        s_rem = rem;
        s_dec = make_decision(k, l, p.span, p.plain != 0, p.use_in != 0);
        sc.cnt[32] = 0;  // next publication's counter (every thread has read this one)
      }
    }
    __syncthreads();
    const Decision D = s_dec;
    const int total = static_cast<int>(s_off[G]);
    build_chunk_table(s_off, G, ctab);
    __syncthreads();
    if (tr && threadIdx.x == 0) {
      tr[4] = global_ns();
      tr[7] = static_cast<uint64_t>(total);
    }
    if (D.m >= kInf) break;
    // 4. relax this slice with the settled rows: only columns a settled row can
    //    still change take part.  None: nothing to read; a few: load just those
    //    groups; otherwise stream the whole slice through the warps' rings.
    const uint4* cl = p.cand + static_cast<size_t>(phase & 1) * G * p.swcap;
    const int swcap = p.swcap;
    const uint4 one = make_uint4(D.a, D.m, 0u, 0u);  // plain mode: Algorithm 1's single row a
    auto get = [cl, swcap, s_off, ctab](int i) {
      const int r = region_at(s_off, ctab, i);
      return __ldcg(cl + static_cast<size_t>(r) * swcap + (i - static_cast<int>(s_off[r])));
    };
    // row split for a big phase after which a fair share of the nodes stays unsettled (otherwise
    // few columns are live and the filtered paths read less); the same decision in every CTA
    const bool rowsplit = p.rs_min > 0 && !p.plain && total >= p.rs_min && 16ull * s_rem >= static_cast<uint64_t>(p.n);
    // row push (graphs that are not dense): phases with enough candidates to occupy the grid's
    // warps, while a fair share of the nodes stays unsettled (otherwise the filtered paths read less)
    const bool rowpush = !rowsplit && p.rp_min > 0 && !p.plain && total >= p.rp_min &&
                         16ull * s_rem >= static_cast<uint64_t>(p.n);
    // the gather's column pass: on undirected graphs (measured: it costs the sparse directed graph
    // more than it saves), for phases with enough settled rows to pay for it, the whole list in one
    // segment, room for its table and lists
    const bool colpass = !p.plain && p.sym && total >= kColPassMin && total <= p.list_cap &&
                         p.ring_bytes / 4 >= static_cast<int>(p.pitch / 2) + 2 * s.sw;
    const int nlg = (rowsplit || rowpush) ? 0
                    : p.gather_max >= 0 ? live_groups(s, D, p.bits_u, glist, gthr, &sc, colpass && p.ts.cap > 0,
                                                      colpass && p.sym != 0)
                                        : s.nvec;
    // gather when few groups are live, or when the column pass leaves few to row items and few
    // whole rows to read
    const bool gather =
        p.gather_max >= 0 &&
        (nlg <= p.gather_max ||
         (colpass && static_cast<int>(sc.cnt[26]) + max(0, static_cast<int>(sc.cnt[25]) - kMaxRowColumns) <= p.gather_max));
    if (tr && threadIdx.x == 0) tr[7] |= static_cast<uint64_t>(rowsplit ? 0xFFFFu : rowpush ? 0xFFFEu : nlg) << 32;
    // the stamps the post-commit update needs (a row-push phase fetches them after its compaction,
    // whose loads of the published lists would otherwise wait behind them)
    if (DYN && !rowpush) dyn_in_prefetch<kInLists>(s, dy);
    if (rowpush) {
      unsigned long long* gk = p.gkey + static_cast<size_t>(phase & 1) * p.pitch;
      for (int seg = 0; seg < total; seg += p.list_cap) {  // the same segments and lists in every CTA
        const int cnt = compact_settled(get, seg, min(total, seg + p.list_cap), D, p.bits_u, list, &sc);
        if (DYN && seg == 0) dyn_in_prefetch<kInLists>(s, dy);
        relax_push(list, cnt, G, p.W, p.pitch, D, p.bits_u, gk);
        __syncthreads();  // the list is rewritten by the next segment
      }
      // every CTA's pushes are in gkey before the owners read their slices
      if (!grid_barrier(bar, ++nbar * static_cast<uint32_t>(G), abort_flag, p.words, p.timeout_ns, &s_flag))
        return;
      for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
        bkey[j] = __ldcg(gk + s.c0 + j);
        gk[s.c0 + j] = ~0ull;  // reused two phases later, after at least one more barrier
      }
      __syncthreads();
      if (tr && threadIdx.x == 0) tr[5] = global_ns();
      commit_keys(s, D, p.bits_u, bkey, part);
    } else if (rowsplit) {
      unsigned long long* gk = p.gkey + static_cast<size_t>(phase & 1) * p.pitch;
      // this slice's snapshot for the other CTAs' merges, announced without waiting
      for (int j = threadIdx.x; j < s.sw; j += blockDim.x) p.gsnap[s.c0 + j] = snapshot_word(s, j, D);
      __syncthreads();
      if (threadIdx.x == 0) red_add_release_gpu(p.ctl + kCtlSnapshots, 1u);
      ++rs_phases;
      if (!relax_rows<kRowSplitCpt>(get, total, b, G, p.W, p.pitch, D, p.bits_u, p.gsnap, gk, list, p.list_cap,
                                    rings, rbar, rs_gt, p.timeout_ns, p.ctl + kCtlSnapshots,
                                    rs_phases * static_cast<uint32_t>(G),
                                    abort_flag, &sc)) {
        atomicOr(p.words, kErrTimeout);
        atomicExch(abort_flag, 1u);
      }
      // every CTA's merges are in gkey before the owners read their slices
      if (!grid_barrier(bar, ++nbar * static_cast<uint32_t>(G), abort_flag, p.words, p.timeout_ns, &s_flag))
        return;
      for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
        bkey[j] = __ldcg(gk + s.c0 + j);
        gk[s.c0 + j] = ~0ull;  // reused two phases later, after at least one more barrier
      }
      __syncthreads();
      if (tr && threadIdx.x == 0) tr[5] = global_ns();
      commit_keys(s, D, p.bits_u, bkey, part);
    } else if (gather) {
      if (nlg > 0) {
        for (int j = threadIdx.x; j < s.sw; j += blockDim.x) bkey[j] = (static_cast<uint64_t>(s.dist[j]) << 32) | 0xFFFFFFFFu;
        if (p.plain) {
          auto stage = [&](int b0, int b1) {
            return stage_settled([one](int) { return one; }, b0, b1, D, p.bits_u, list, &sc);
          };
          relax_gather(stage, 1, s, p.W, p.pitch, D, p.bits_u, glist, gthr, nlg, list, p.list_cap, bkey,
                       TieSources{nullptr, nullptr, 0}, false, false, nullptr, &sc);
        } else {
          // the published lists come in by bulk copies through the (idle) ring region
          bool ok = true;
          auto stage = [&](int b0, int b1) {
            return stage_settled_bulk(s_off, G, cl, swcap, b0, b1, D, p.bits_u, list, rings,
                                      static_cast<uint32_t>(p.ring_bytes), rbar, rs_gt, p.timeout_ns, &sc, ok);
          };
          relax_gather(stage, total, s, p.W, p.pitch, D, p.bits_u, glist, gthr, nlg, list, p.list_cap, bkey, p.ts,
                       p.sym != 0, colpass, reinterpret_cast<uint32_t*>(rings), &sc);
          if (!ok) {
            atomicOr(p.words, kErrTimeout);
            atomicExch(abort_flag, 1u);
          }
        }
      }
      if (tr && threadIdx.x == 0) tr[5] = global_ns();
      // 5. mark, commit, and the next partial
      commit_keys(s, D, p.bits_u, nlg > 0 ? bkey : nullptr, part);
    } else {
      Best<V> best;
      best_init<V>(best, s, t, D, p.bits_u);
      bool ok;
      if (p.plain)
        ok = relax_pull<V, U>([one](int) { return one; }, 1, s, t, p.W, p.pitch, D, p.bits_u, ring, slot_rows,
                              slot_tb, p.timeout_ns, best);
      else
        ok = relax_pull<V, U>(get, total, s, t, p.W, p.pitch, D, p.bits_u, ring, slot_rows, slot_tb, p.timeout_ns,
                              best);
      if (!ok) {
        atomicOr(p.words, kErrTimeout);
        atomicExch(abort_flag, 1u);
      }
      if (tr && threadIdx.x == 0) tr[5] = global_ns();
      // 5. merge, mark, commit, and the next partial
      commit_partial<V>(s, t, D, merge, p.bits_u, best, part);
    }
    if (DYN) {  // stamp this phase's settled columns; the next phase's IN weights: rows settled earlier drop out
      __syncthreads();
      dyn_in_update<kInLists>(s, dy, phase);
    }
    if (tr && threadIdx.x == 0) tr[6] = global_ns();
    ++phase;
  }
  slice_write_out(s, p.n, p.dist_out, p.pred_out);
  if (b == 0 && threadIdx.x == 0) {
    p.words[1] = phase;
    if (p.trace && p.trace_cap >= 10) p.trace[p.trace_cap - 1] = global_ns();  // exit
  }
}

template <int V, int U, int THREADS, bool DYN>
__global__ void __launch_bounds__(THREADS, 1) k_sssp_grid(const GridParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ BlockScratch sc;
  __shared__ Decision s_dec;
  __shared__ uint32_t s_flag;
  __shared__ uint32_t s_rem;  // unvisited columns that are no candidates, summed over the CTAs
  // launched as a programmatic dependent of the previous kernel on the stream: its launch overlaps
  // that kernel's end, but nothing (graph, workspace, outputs) is touched before it has completed
  pdl_launch_dependents();
  pdl_wait();
  grid_solve<V, U, DYN>(p, smem, sc, s_dec, s_flag, s_rem);  // returns early (uniformly per CTA) on a timeout
  grid_exit(p.ctl);
}

// ============================================================ cluster engine

// Where the cluster engine gets its solves.  fetch() and complete() run on
// thread 0 of cluster rank 0 only.
struct BatchJobs {
  const SolveDesc* descs;
  uint32_t* queue;  // [0] next solve index, [1] exit count: both zero when a launch starts
  int32_t k;
  __device__ bool fetch(uint32_t* job, uint32_t) const {
    *job = atomicAdd(queue, 1u);
    return *job < static_cast<uint32_t>(k);
  }
  __device__ SolveDesc desc(uint32_t job) const { return descs[job]; }
  __device__ void complete(uint32_t, uint32_t) const {}
  static constexpr bool kTrace = false;
  __device__ bool early() const { return true; }  // launched the ordinary way: nothing to wait for
  __device__ void before_write() const {}
  // once per cluster, by rank 0, after its last fetch: the last cluster to leave zeroes the
  // queue for the next launch (the stream starts it only after this one has ended)
  __device__ void leave() const {
    __threadfence();
    if (atomicAdd(queue + 1, 1u) == nclusters_x() - 1) {
      __threadfence();
      queue[0] = 0u;
      queue[1] = 0u;
    }
  }
};

// One solve whose descriptor travels in the kernel's parameters: no table,
// queue or memset on the device.  Launched as a single cluster; its rank 0
// records the phase count in the per-device word.  It is launched as a
// programmatic dependent of the kernel before it on the stream: it starts
// while that kernel is still running (every CTA lets its own dependents start
// at once), solves from the graph, which no kernel writes meanwhile (unless
// `early_ok` is 0, after an upload: then it waits first), and waits for its
// predecessor to complete only before it writes dist, pred and the phase
// count.  So results reach memory in stream order, and back-to-back solves of
// small graphs overlap on the GPU's idle SMs.
struct SingleJob {
  SolveDesc d;
  uint32_t* phases_out;
  int32_t early_ok;
  __device__ bool fetch(uint32_t* job, uint32_t iter) const {
    *job = 0;
    return iter == 0 && cluster_id_x() == 0;
  }
  __device__ SolveDesc desc(uint32_t) const { return d; }
  __device__ void complete(uint32_t, uint32_t phases) const {
    if (phases_out) *phases_out = phases;
  }
  static constexpr bool kTrace = true;  // the per-phase timeline is compiled into this kernel only
  __device__ bool early() const { return early_ok != 0; }
  __device__ void before_write() const { pdl_wait(); }
  __device__ void leave() const {}
};

// Serving: requests arrive in a ring of descriptors in mapped pinned host
// memory.  The host publishes request r by writing ring[r % cap] and then
// tail = r + 1 (release); a cluster claims r by advancing the device-side head
// with a CAS, and reports completion with done[r % cap] = r + 1 (release,
// system scope).  Waiting for work is bounded: after idle_ns without a
// request, or once the host sets *stop, fetch() returns false and the kernel
// exits (the host relaunches it when requests come again).
struct ServeJobs {
  const SolveDesc* ring;  // mapped host memory, cap entries
  const uint32_t* tail;   // mapped host memory
  const uint32_t* stop;   // mapped host memory
  uint32_t* done;         // mapped host memory, cap entries
  uint32_t* head;         // device memory
  uint32_t cap_mask;
  int64_t idle_ns;
  __device__ bool fetch(uint32_t* job, uint32_t) const {
    uint64_t t0 = global_ns();
    for (;;) {
      if (ld_acquire_sys(stop)) return false;
      const uint32_t h = ld_relaxed_gpu(head);
      const uint32_t t = ld_acquire_sys(tail);
      if (static_cast<int32_t>(t - h) > 0) {
        if (atomicCAS(head, h, h + 1) == h) {
          *job = h;
          return true;
        }
        continue;
      }
      if (static_cast<int64_t>(global_ns() - t0) > idle_ns) return false;
      __nanosleep(256);
    }
  }
  __device__ SolveDesc desc(uint32_t job) const {
    const SolveDesc* src = ring + (job & cap_mask);
    SolveDesc d;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(&d);
#pragma unroll
    for (int i = 0; i < 4; ++i) d4[i] = __ldcv(s4 + i);
    return d;
  }
  __device__ void complete(uint32_t job, uint32_t) const {
    __threadfence_system();
    st_release_sys(done + (job & cap_mask), job + 1);
  }
  static constexpr bool kTrace = false;
  __device__ bool early() const { return true; }
  __device__ void before_write() const {}
  __device__ void leave() const {}
};

struct ClusterParams {
  uint32_t* words;  // per-device words: [0] error bits
  uint64_t* trace;  // optional per-phase timeline of the first solve (rank 0), as the grid engine's
  int32_t trace_cap;
  int64_t timeout_ns;
  int32_t swcap;
  int32_t rgs_cap;
  int32_t depth;
  int32_t srows;
  int32_t rowcap;
  int32_t list_cap;  // staged settled rows per segment
  int32_t amerge;    // row groups merge through atomicMin into one key per column
};

template <int V, int U, int THREADS, class Jobs>
__global__ void __launch_bounds__(THREADS, 2) k_sssp_cluster(const ClusterParams p, const Jobs jobs) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ BlockScratch sc;
  __shared__ __align__(16) uint4 s_part[2];  // this CTA's published partial, per phase parity
  __shared__ uint32_t s_job;                 // rank 0: the solve index it fetched
  __shared__ uint32_t s_jobl;                // local copy
  __shared__ Decision s_dec;
  __shared__ uint32_t s_off[17];   // candidate offsets of the ranks (prefix)
  __shared__ uint32_t s_addr[16];  // DSMEM address of each rank's candidate list

  const uint32_t rank = cluster_rank(), C = cluster_size();
  const int nwarps = static_cast<int>(blockDim.x >> 5);
  uint8_t* q = smem;
  uint64_t* merge = reinterpret_cast<uint64_t*>(q);
  q += p.rgs_cap > 1 ? static_cast<size_t>(p.amerge ? 1 : p.rgs_cap) * p.swcap * 8 : 0;
  uint2* own = reinterpret_cast<uint2*>(q);  // [2][swcap] (v, dist[v]), read by the other CTAs of the cluster
  q += static_cast<size_t>(p.swcap) * 16;
  Slice s;
  s.dist = reinterpret_cast<uint32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.pred = reinterpret_cast<int32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.pdist = reinterpret_cast<uint32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.minout = reinterpret_cast<uint32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.minin = reinterpret_cast<uint32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  s.vis = q;
  q += (static_cast<size_t>(p.swcap) + 15) / 16 * 16;
  uint32_t* list = reinterpret_cast<uint32_t*>(q);  // staged settled rows of the cluster
  q += static_cast<size_t>(p.list_cap) * 4;
  q = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(q) + 127) & ~uintptr_t(127));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* rings = q;
  q += static_cast<size_t>(nwarps) * p.depth * p.srows * p.rowcap;
  uint64_t* bars = reinterpret_cast<uint64_t*>(q);
  q += static_cast<size_t>(nwarps) * p.depth * 8;
  uint32_t* slot_rows = reinterpret_cast<uint32_t*>(q) + static_cast<size_t>(warp) * p.depth;
  q += static_cast<size_t>(nwarps) * p.depth * 4;
  uint32_t* slot_tb = reinterpret_cast<uint32_t*>(q) + static_cast<size_t>(warp) * p.depth * U;
  Ring ring;
  ring.buf = rings + static_cast<size_t>(warp) * p.depth * p.srows * p.rowcap;
  ring.srows = static_cast<uint32_t>(p.srows);
  ring.bar = bars + static_cast<size_t>(warp) * p.depth;
  ring.depth = static_cast<uint32_t>(p.depth);
  ring.gt = 0;
  if (lane == 0)
    for (int i = 0; i < p.depth; ++i) mbar_init(ring.bar + i, 1);
  if (p.amerge && p.rgs_cap > 1)
    for (int j = threadIdx.x; j < p.swcap; j += blockDim.x) merge[j] = kNoKey;
  fence_mbar_init();
  __syncthreads();
  pdl_launch_dependents();  // the next kernel on the stream may start (it waits where it must)

  for (uint32_t iter = 0;; ++iter) {
    // next solve: rank 0 takes it from the job source, every CTA reads it through DSMEM
    if (rank == 0 && threadIdx.x == 0) {
      uint32_t j = 0;
      s_job = jobs.fetch(&j, iter) ? j : 0xFFFFFFFFu;
      if (s_job == 0xFFFFFFFFu) jobs.leave();
    }
    cluster_sync_all();
    if (threadIdx.x == 0) s_jobl = (rank == 0) ? s_job : ld_dsmem_u32(dsmem_addr(&s_job, 0));
    __syncthreads();
    const uint32_t job = s_jobl;
    if (job == 0xFFFFFFFFu) {
      cluster_sync_all();  // rank 0's s_job stays readable until everyone has it
      return;
    }
    // per-phase timeline of the first solve (rank 0, thread 0; profiling only)
    uint64_t* const trace = (Jobs::kTrace && p.trace && iter == 0 && rank == 0 && threadIdx.x == 0) ? p.trace : nullptr;
    if (trace && p.trace_cap >= 10) trace[p.trace_cap - 2] = global_ns();
    const SolveDesc d = jobs.desc(job);
    if (!jobs.early()) pdl_wait();  // the kernel before may still be writing the graph
    const int nvec_total = static_cast<int>(d.pitch / 4);
    const int v0 = static_cast<int>(static_cast<int64_t>(rank) * nvec_total / C);
    const int v1 = static_cast<int>(static_cast<int64_t>(rank + 1) * nvec_total / C);
    s.c0 = 4 * v0;
    s.nvec = v1 - v0;
    s.sw = 4 * s.nvec;
    if (d.plain)
      slice_init(s, d.n, d.source, d.minout, d.minout + d.n, false, false);
    else
      slice_init_source(s, d.n, d.source, d.minout, d.minout + d.n, true, d.use_in != 0, d.W, d.pitch);
    const Tile t = make_tile<V>(s.nvec, p.rgs_cap);
    ring.rowbytes = t.active ? static_cast<uint32_t>(max(0, min(32 * V, s.nvec - t.wc * 32 * V)) * 16) : 0u;
    if (threadIdx.x == 0) sc.cnt[32] = 0;
    __syncthreads();

    Part part;
    slice_partial(s, part);
    uint32_t phase = 0;
    for (;;) {
      uint64_t* tr = (Jobs::kTrace && trace && static_cast<int>(8 * phase + 7) < p.trace_cap - 2) ? trace + 8 * phase
                                                                                                 : nullptr;
      if (tr) tr[0] = global_ns();
      uint2* mine = own + static_cast<size_t>(phase & 1) * p.swcap;
      uint64_t key;
      uint32_t Lc;
      const int c = publish_partial(s, d.span, d.plain != 0, d.use_in != 0, part, mine, &sc, &key, &Lc, nullptr,
                                    d.bits_u);
      if (threadIdx.x == 0)
        s_part[phase & 1] =
            make_uint4(static_cast<uint32_t>(key), static_cast<uint32_t>(key >> 32), Lc, static_cast<uint32_t>(c));
      if (tr) tr[1] = global_ns();
      cluster_sync_all();
      if (tr) tr[2] = global_ns();
      if (warp == 0) {
        uint4 x = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u);
        if (static_cast<uint32_t>(lane) < C) x = ld_dsmem_u32x4(dsmem_addr(&s_part[phase & 1], lane));
        uint64_t k = (static_cast<uint64_t>(x.y) << 32) | x.x;
        uint32_t l = x.z;
        k = warp_min_u64(k);
        l = warp_min_u32(l);
        const uint32_t cntv = x.w;
        uint32_t incl = cntv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t tt = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += tt;
        }
        if (static_cast<uint32_t>(lane) < C) {
          s_off[lane] = incl - cntv;
          s_addr[lane] = dsmem_addr(own + static_cast<size_t>(phase & 1) * p.swcap, lane);
        }
        if (static_cast<uint32_t>(lane) == C - 1) s_off[C] = incl;
        if (lane == 0) {
          s_dec = make_decision(k, l, d.span, d.plain != 0, d.use_in != 0);
          sc.cnt[32] = 0;
        }
      }
      __syncthreads();
      const Decision D = s_dec;
      const int total = static_cast<int>(s_off[C]);
      if (tr) {
        tr[3] = global_ns();
        tr[7] = static_cast<uint64_t>(total);
      }
      if (D.m >= kInf) break;
      Best<V> best;
      best_init<V>(best, s, t, D, d.bits_u);
      const int Cn = static_cast<int>(C);
      bool ok;
      if (d.plain) {  // Algorithm 1's single row a: no candidate list to read
        const uint4 one = make_uint4(D.a, D.m, 0u, 0u);
        ok = relax_pull<V, U>([one](int) { return one; }, 1, s, t, d.W, d.pitch, D, d.bits_u, ring, slot_rows,
                              slot_tb, p.timeout_ns, best);
      } else {
        // stage the cluster's settled rows locally (one pass of remote reads by
        // all threads), then every warp pulls them from its own shared memory
        ok = true;
        const uint32_t bu = d.bits_u;
        for (int seg = 0; seg < total; seg += p.list_cap) {
          const int32_t* minin_g = d.minout + d.n;
          const int cnt = stage_settled(
              [Cn, minin_g, bu, D](int i) {
                const int r = region_of16(s_off, Cn, i);
                const uint2 e = ld_dsmem_u32x2(s_addr[r] + 8u * static_cast<uint32_t>(i - static_cast<int>(s_off[r])));
                return unpack_entry(e, bu, minin_g, D.use_in != 0);
              },
              seg, min(total, seg + p.list_cap), D, bu, list, &sc);
          if (tr && seg == 0) tr[4] = global_ns();
          ok = relax_pull<V, U>([list, D, bu](int i) { return staged_entry(list, i, D, bu); }, cnt, s, t, d.W,
                                d.pitch, D, bu, ring, slot_rows, slot_tb, p.timeout_ns, best) &&
               ok;
          __syncthreads();  // the list is rewritten by the next segment
        }
      }
      if (tr) tr[5] = global_ns();
      if (!ok) atomicOr(p.words, kErrTimeout);
      commit_partial<V>(s, t, D, merge, d.bits_u, best, part, p.amerge != 0);
      if (tr) tr[6] = global_ns();
      ++phase;
    }
    jobs.before_write();  // results reach memory in stream order
    slice_write_out(s, d.n, d.dist, d.pred);
    // every CTA's outputs are visible system-wide before rank 0 reports completion
    __syncthreads();
    if (threadIdx.x == 0) __threadfence_system();
    cluster_sync_all();
    if (rank == 0 && threadIdx.x == 0) {
      jobs.complete(job, phase);
      if (trace && p.trace_cap >= 10) trace[p.trace_cap - 1] = global_ns();
    }
  }
}

// ============================================================ host launchers

namespace {

constexpr int kRowsPerStage = 8;  // U: rows per ring stage
constexpr int kGridListCap = 8192;  // grid engine: staged settled rows per segment
// Grid engine: a phase takes the row split once n / 8 nodes are its candidates, within
// [512, 2048]: the split saves time in proportion to rows x row bytes and costs a fixed
// barrier and merge, so smaller graphs profit from smaller phases (measured on GB300, p = 0.5:
// n = 4096 fastest near 512, n = 8192 near 700..1100, n = 16384 flat from 1100 to 2048, and
// p = 0.1 at n = 16384 slower below 2048).
int auto_rowsplit_min(int32_t n) { return std::min(2048, std::max(512, static_cast<int>(n / 8))); }

constexpr int kGridThreads = 512;
constexpr int kClusterThreads = 256;

// Column filter default: load only the live groups when at most a quarter of a
// slice's 4-column groups (and at least 2) are live.
int auto_gather_max(int nvec_cta) { return std::min(kGridThreads, std::max(2, nvec_cta / 4)); }

// Shared-memory layout of one CTA (must match the carving in the kernels).
struct Layout {
  int V = 0;
  int swcap = 0;    // columns of the widest slice
  int rgs_cap = 0;  // row groups (merge buffer rows)
  int depth = 0;    // ring stages per warp
  int srows = 0;    // rows per stage (<= kRowsPerStage)
  int list_cap = 0; // staged settled rows per segment
  bool filter = false;  // grid engine: per-column keys and live groups of the filtered relaxation
  int dyn = 0;          // grid engine: 1 in-lists (dynamic IN), 2 also out-lists (dynamic OUT), with rests and cursors
  bool amerge = false;  // row groups merge by atomicMin into one key per column (no merge rows)
  size_t rs_bytes = 0;  // grid engine: the two row-split buffers (share the ring region)
  int rowcap = 0;   // bytes of one ring row slot
  size_t smem = 0;
};

size_t ring_region(const Layout& L, int nwarps) {
  return std::max(static_cast<size_t>(nwarps) * L.depth * L.srows * L.rowcap, L.rs_bytes);
}

// own_copies: published candidate lists kept in shared memory (cluster: 2);
// offs: prefix entries of the grid engine's candidate counts (grid: G + 1).
size_t layout_bytes(const Layout& L, int nwarps, int own_copies, int offs) {
  size_t b = L.rgs_cap > 1 ? static_cast<size_t>(L.amerge ? 1 : L.rgs_cap) * L.swcap * 8 : 0;  // merge
  b += static_cast<size_t>(L.swcap) * 16 * own_copies;                           // published candidates
  b += (static_cast<size_t>(offs) + 3) / 4 * 16;                                 // candidate-count prefix
  if (offs) b += (static_cast<size_t>(offs - 1) * L.swcap / 32 + 1 + 3) / 4 * 16;  // its chunk table
  b += static_cast<size_t>(L.swcap) * 20;                                        // dist, pred, pdist, minout, minin
  b += (static_cast<size_t>(L.swcap) + 15) / 16 * 16;                            // visited
  b += static_cast<size_t>(L.list_cap) * 4;                                      // staged rows
  if (L.dyn)  // lists, rests and cursors (one or two sets), stamped flags, prefetched stamps
    b += static_cast<size_t>(L.dyn) * (static_cast<size_t>(L.swcap) * (kInLists * 8 + 4) +
                                       (static_cast<size_t>(L.swcap) + 15) / 16 * 16) +
         static_cast<size_t>(L.swcap) * 12;
  if (L.filter)  // per-column keys, group thresholds, live groups
    b += static_cast<size_t>(L.swcap) * 8 + static_cast<size_t>(L.swcap) / 4 * 8 +
         (static_cast<size_t>(L.swcap) / 4 + 3) / 4 * 16;
  b += 128;                                                                      // ring alignment
  b += ring_region(L, nwarps);                                                   // TMA rings / row buffers
  b += static_cast<size_t>(nwarps) * L.depth * 8 + 16;                           // mbarriers
  b += static_cast<size_t>(nwarps) * L.depth * (kRowsPerStage + 1) * 4;          // stage row counts + keys
  return b;
}

// V (vec4 per lane): the smallest that lets one warp cover the whole slice, so
// every warp is its own row group (most rows in flight); else the smallest
// whose column chunks fit the warps.
int pick_v(int nvec_cta, int nwarps) {
  for (int v : {1, 2, 4})
    if (nvec_cta <= 32 * v) return v;
  for (int v : {1, 2, 4})
    if ((nvec_cta + 32 * v - 1) / (32 * v) <= nwarps) return v;
  return 0;
}

// Fit the layout into `budget` bytes: the deepest ring up to want_depth stages,
// with the longest stages (up to kRowsPerStage rows) that fit at that depth.
int make_layout(int nvec_cta, int nwarps, int own_copies, int offs, int want_depth, size_t budget, Layout* L,
                int force_v = 0) {
  L->V = force_v ? force_v : pick_v(nvec_cta, nwarps);
  if (!L->V) return set_error(DJ_EUNSUPPORTED, "graph too large for this engine configuration");
  L->swcap = 4 * std::max(nvec_cta, 1);
  const int wpr = std::max(1, (nvec_cta + 32 * L->V - 1) / (32 * L->V));
  L->rgs_cap = std::max(1, nwarps / wpr);
  L->rowcap = std::min(32 * L->V, std::max(nvec_cta, 1)) * 16;
  for (int depth = want_depth; depth >= 1; --depth) {
    for (int srows = kRowsPerStage; srows >= 1; srows /= 2) {
      L->depth = depth;
      L->srows = srows;
      L->smem = layout_bytes(*L, nwarps, own_copies, offs);
      if (L->smem <= budget) return DJ_OK;
    }
  }
  return set_error(DJ_EUNSUPPORTED, "slice state exceeds shared memory");
}

template <int V, bool DYN>
void* grid_kernel() {
  return reinterpret_cast<void*>(&k_sssp_grid<V, kRowsPerStage, kGridThreads, DYN>);
}
template <int V, class Jobs>
void* cluster_kernel() {
  return reinterpret_cast<void*>(&k_sssp_cluster<V, kRowsPerStage, kClusterThreads, Jobs>);
}
void* grid_kernel_for(int v, bool dyn = false) {
  switch (v) {
    case 1: return dyn ? grid_kernel<1, true>() : grid_kernel<1, false>();
    case 2: return dyn ? grid_kernel<2, true>() : grid_kernel<2, false>();
    case 4: return dyn ? grid_kernel<4, true>() : grid_kernel<4, false>();
  }
  return nullptr;
}
template <class Jobs>
void* cluster_kernel_v(int v) {
  switch (v) {
    case 1: return cluster_kernel<1, Jobs>();
    case 2: return cluster_kernel<2, Jobs>();
    case 4: return cluster_kernel<4, Jobs>();
  }
  return nullptr;
}
void* cluster_kernel_for(int v, int kind = kJobsBatch) {
  if (kind == kJobsServe) return cluster_kernel_v<ServeJobs>(v);
  if (kind == kJobsSingle) return cluster_kernel_v<SingleJob>(v);
  return cluster_kernel_v<BatchJobs>(v);
}


}  // namespace

// A cooperative launch (every CTA resident at once), as a programmatic dependent of the
// previous kernel on the stream when `pdl` (the kernel waits for it before touching memory;
// only the launch itself overlaps).  If the runtime rejects that pairing, the plain cooperative
// launch is used from then on.
static std::atomic<int> g_coop_pdl_ok{1};
cudaError_t launch_cooperative(void* fn, int G, int threads, void** args, size_t smem, cudaStream_t st, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(G));
  cfg.blockDim = dim3(static_cast<unsigned>(threads));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (pdl && g_coop_pdl_ok.load()) ? 2 : 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
  if (e != cudaSuccess && cfg.numAttrs == 2) {
    cudaGetLastError();
    g_coop_pdl_ok.store(0);
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, fn, args);
  }
  return e;
}

int launch_grid(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, const dj_solve_opts& o,
                cudaStream_t st) {
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  if (!ctx->coop) return set_error(DJ_EUNSUPPORTED, "device lacks cooperative launch");
  const int nvec_total = g->pitch / 4;
  const int per_sm = o.ctas_per_sm > 0 ? o.ctas_per_sm : 1;
  int G = std::min({ctx->num_sms * per_sm, nvec_total, 32 * kMaxPartialsPerLane});
  const int nwarps = kGridThreads / 32;
  const int nvec_cta = (nvec_total + G - 1) / G;
  const int want_depth = o.unroll > 0 ? std::min(o.unroll, 8) : 2;
  const size_t budget = static_cast<size_t>(ctx->max_smem_optin) / per_sm - 1024;
  Layout L;
  L.filter = true;
  L.list_cap = std::min(nvec_total * 4, kGridListCap);
  // row split pays on dense graphs (few phases, thousands of rows each); auto: density >= 1/32
  const bool dense = g->entries * 32 >= static_cast<uint64_t>(g->n) * static_cast<uint64_t>(g->n);
  // the dynamic IN bound, and with DJ_SETTLE_DYN also the dynamic OUT bound (graphs that keep
  // in-lists: not dense, every weight >= 1)
  const bool dyn_ok = o.mode != DJ_MODE_PLAIN && g->inlist && g->wmin >= 1;
  const int dyn = !dyn_ok ? 0
                  : (o.settle == DJ_SETTLE_AUTO || o.settle == DJ_SETTLE_OUT_DYN_IN) ? 1
                  : o.settle == DJ_SETTLE_DYN                                         ? 2
                                                                                      : 0;
  const bool dyn_in = dyn > 0;
  L.dyn = dyn;
  const bool want_rs = o.mode != DJ_MODE_PLAIN && (o.rowsplit > 0 || (o.rowsplit == 0 && dense));
  L.rs_bytes = want_rs ? static_cast<size_t>(2) * std::min(nvec_total, kGridThreads * kRowSplitCpt) * 16 : 0;
  if (make_layout(nvec_cta, nwarps, 0, G + 1, want_depth, budget, &L) != DJ_OK) {
    clear_error();
    L.rs_bytes = 0;  // no room for the row buffers: no row split
    if (int rc = make_layout(nvec_cta, nwarps, 0, G + 1, want_depth, budget, &L)) return rc;
  }
  void* fn = grid_kernel_for(L.V, dyn_in && g->wmin >= 1 && o.settle != DJ_SETTLE_OUT);
  if (int rc = prepare_function(ctx, fn, L.smem, false)) return rc;
  int occ = 0;
  if (int rc = function_occupancy(ctx, fn, kGridThreads, L.smem, &occ)) return rc;
  cudaError_t e = cudaSuccess;
  if (occ < 1) return set_error(DJ_EUNSUPPORTED, "grid engine cannot be resident");
  if (occ < per_sm) return set_error(DJ_EUNSUPPORTED, "requested CTAs per SM cannot be resident");

  const size_t ctl_bytes = 256;
  const size_t part_bytes = static_cast<size_t>(2) * G * sizeof(uint4);
  const uint32_t cand_cap = static_cast<uint32_t>(G) * static_cast<uint32_t>(L.swcap);  // one region per CTA
  const size_t cand_bytes = static_cast<size_t>(2) * cand_cap * sizeof(uint4);
  // row split needs its buffers, a CTA's share of the candidates (<= the slice width) in the
  // staged list, and slices below 2^16 columns (packed counts in the partials)
  const int rs_min = (!want_rs || L.rs_bytes == 0 || L.swcap > L.list_cap || L.swcap >= 65536) ? 0
                     : o.rowsplit > 0                                                         ? o.rowsplit
                                                                                              : auto_rowsplit_min(g->n);
  // row push on graphs that are not dense (or forced while the row split is off); packed partial
  // counts need slices below 2^16 columns
  // (auto: phases of at least 4 candidates per CTA; measured on the sparse directed n = 32768
  // graph: 2298 us per solve without, 2244 from G, 2220 from 2 G, 2200 from 4 G candidates)
  const int rp_min = (o.mode == DJ_MODE_PLAIN || o.rowpush < 0 || rs_min > 0 || L.swcap >= 65536) ? 0
                     : o.rowpush > 0                                                       ? o.rowpush
                     : !dense                                                              ? 4 * G
                                                                                           : 0;
  const size_t snap_bytes = rs_min > 0 ? static_cast<size_t>(g->pitch) * 4 : 0;  // pitch is a multiple of 4
  const size_t gkey_bytes = (rs_min > 0 || rp_min > 0) ? static_cast<size_t>(2) * g->pitch * 8 : 0;
  const size_t sph_bytes = dyn_in ? static_cast<size_t>(g->pitch) * 4 : 0;
  // the stream's kept workspace (its control words are zero between launches: see grid_exit),
  // or one allocated for this call
  const size_t ws_bytes = ctl_bytes + part_bytes + cand_bytes + snap_bytes + gkey_bytes + sph_bytes;
  uint8_t* ws = nullptr;
  if (int rc = stream_workspace(ctx, st, ws_bytes, ctl_bytes, &ws)) return rc;
  const bool own_ws = ws == nullptr;
  if (own_ws) {
    e = cudaMallocAsync(&ws, ws_bytes, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(grid workspace)");
    cudaMemsetAsync(ws, 0, ctl_bytes, st);
  }

  GridParams p;
  p.W = g->W;
  p.minout = g->minout;
  p.dist_out = dist;
  p.pred_out = pred;
  p.ctl = reinterpret_cast<uint32_t*>(ws);
  p.partials = reinterpret_cast<uint4*>(ws + ctl_bytes);
  p.cand = reinterpret_cast<uint4*>(ws + ctl_bytes + part_bytes);
  p.words = ctx->words;
  p.pitch = g->pitch;
  p.timeout_ns = o.timeout_ns > 0 ? o.timeout_ns : 2000000000LL;
  p.n = g->n;
  p.nvec_total = nvec_total;
  p.source = source;
  p.plain = o.mode == DJ_MODE_PLAIN ? 1 : 0;
  p.use_in = (g->wmin >= 1 && o.settle != DJ_SETTLE_OUT) ? 1 : 0;
  p.bits_u = host_bits_for(static_cast<uint32_t>(g->n));
  p.span = host_span_for(static_cast<uint32_t>(g->n));
  p.cand_cap = cand_cap;
  p.swcap = L.swcap;
  p.rgs_cap = L.rgs_cap;
  p.skip_cta = o.debug_skip_cta;
  p.depth = L.depth;
  p.srows = L.srows;
  p.rowcap = L.rowcap;
  p.trace_cap = o.trace ? o.trace_cap : 0;
  p.trace = o.trace;
  p.list_cap = L.list_cap;
  // plain mode relaxes one row per phase: the filter's per-phase pass would cost more than it saves
  p.gather_max = (o.live < 0 || (o.live == 0 && o.mode == DJ_MODE_PLAIN)) ? -1
                 : o.live > 0                                              ? std::min(o.live, kGridThreads)
                                                                           : auto_gather_max(nvec_cta);
  p.rs_min = rs_min;
  p.rp_min = rp_min;
  p.ring_bytes = static_cast<int32_t>(ring_region(L, nwarps));
  p.gsnap = rs_min > 0 ? reinterpret_cast<uint32_t*>(ws + ctl_bytes + part_bytes + cand_bytes) : nullptr;
  p.gkey = (rs_min > 0 || rp_min > 0)
               ? reinterpret_cast<unsigned long long*>(ws + ctl_bytes + part_bytes + cand_bytes + snap_bytes)
               : nullptr;
  p.sym = g->directed ? 0 : 1;
  p.dyn_in = dyn_in && p.use_in ? (dyn == 2 ? 3 : 1) : 0;  // bit 0: IN lists, bit 1: OUT lists
  // the tie sources belong to the static minimum in-weight: not used with the dynamic bound
  p.ts = p.use_in && !p.plain && g->tsrc && !p.dyn_in ? TieSources{g->tsrc, g->tcnt, g->tcap}
                                                      : TieSources{nullptr, nullptr, 0};
  p.inlist = g->inlist;
  p.inrest = g->inrest;
  p.outlist = g->outlist;
  p.outrest = g->outrest;
  p.sph = dyn_in ? reinterpret_cast<uint32_t*>(ws + ctl_bytes + part_bytes + cand_bytes + snap_bytes + gkey_bytes)
                 : nullptr;
  void* args[] = {&p};
  e = launch_cooperative(fn, G, kGridThreads, args, L.smem, st, true);
  if (own_ws) cudaFreeAsync(ws, st);
  if (e != cudaSuccess) return cuda_error(e, "cooperative launch (grid engine)");
  return DJ_OK;
}

static int cluster_layout(int32_t max_pitch, const ClusterLaunch& cl, Layout* L) {
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  const int C = cl.cluster_size;
  const int nvec_total = max_pitch / 4;
  const int nvec_cta = (nvec_total + C - 1) / C;
  const int nwarps = kClusterThreads / 32;
  // two CTAs per SM when they fit, so clusters of different solves share SMs
  const size_t half = static_cast<size_t>(ctx->max_smem_optin) / 2 - 1024;
  L->list_cap = std::min(max_pitch, 512);
  // wide copies: four 4-column groups per lane, so a warp copies 2 KB of each of its rows (larger
  // TMA copies stream faster per SM); its row groups merge by atomicMin, two CTAs per SM
  const bool wide = cl.copies == DJ_COPIES_WIDE || (cl.copies == DJ_COPIES_AUTO && nvec_cta >= 256);
  if (wide && nvec_cta >= 128 && (nvec_cta + 127) / 128 < nwarps) {
    Layout W = *L;
    W.amerge = true;
    if (make_layout(nvec_cta, nwarps, 1, 0, 2, half, &W, 4) == DJ_OK && W.srows >= 2) {
      *L = W;
      return DJ_OK;
    }
    clear_error();
  }
  // full 8-row stages first (short stages stream markedly slower); two CTAs per SM if that still fits
  // two 8-byte candidate lists = one 16-byte "copy" in the layout arithmetic
  if (make_layout(nvec_cta, nwarps, 1, 0, 2, half, L) == DJ_OK && L->srows == kRowsPerStage) return DJ_OK;
  clear_error();
  return make_layout(nvec_cta, nwarps, 1, 0, 2, static_cast<size_t>(ctx->max_smem_optin) - 1024, L);
}

static int prepare_cluster(void* fn, const ClusterLaunch& cl, size_t smem) {
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  return prepare_function(ctx, fn, smem, cl.cluster_size > 8);
}

int cluster_max_clusters(int32_t max_pitch, const ClusterLaunch& cl, int* clusters) {
  Layout L;
  if (int rc = cluster_layout(max_pitch, cl, &L)) return rc;
  void* fn = cluster_kernel_for(L.V);
  if (int rc = prepare_cluster(fn, cl, L.smem)) return rc;
  cudaLaunchConfig_t cfg = {};
  DevCtx* ctx = nullptr;
  get_ctx(&ctx);
  cfg.gridDim = dim3(cl.cluster_size * ctx->num_sms);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = L.smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl.cluster_size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
  if (e != cudaSuccess) return cuda_error(e, "cudaOccupancyMaxActiveClusters");
  if (n < 1) return set_error(DJ_EUNSUPPORTED, "cluster configuration cannot be resident");
  *clusters = n;
  return DJ_OK;
}

bool cluster_config_ok(int32_t max_pitch, const ClusterLaunch& cl) {
  int n = 0;
  const bool ok = cluster_max_clusters(max_pitch, cl, &n) == DJ_OK && n >= 1;
  if (!ok) clear_error();
  return ok;
}

int plan_cluster(int32_t max_pitch, const ClusterLaunch& cl, int32_t k, ClusterPlan* plan, int kind) {
  if (cl.cluster_size < 1 || cl.cluster_size > 16) return set_error(DJ_EINVAL, "cluster size must be 1..16");
  const bool serve = kind == kJobsServe;
  Layout L;
  if (int rc = cluster_layout(max_pitch, cl, &L)) return rc;
  void* fn = cluster_kernel_for(L.V, kind);
  if (int rc = prepare_cluster(fn, cl, L.smem)) return rc;
  int Q = cl.clusters;
  if (Q <= 0) {
    if (int rc = cluster_max_clusters(max_pitch, cl, &Q)) return rc;
  }
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  plan->fn = fn;
  plan->clusters = serve ? std::max(1, Q) : std::max(1, std::min(Q, std::max(k, 1)));
  plan->cluster_size = cl.cluster_size;
  plan->threads = kClusterThreads;
  plan->smem = L.smem;
  plan->swcap = L.swcap;
  plan->rgs_cap = L.rgs_cap;
  plan->depth = L.depth;
  plan->srows = L.srows;
  plan->rowcap = L.rowcap;
  plan->list_cap = L.list_cap;
  plan->amerge = L.amerge ? 1 : 0;
  plan->words = ctx->words;
  return DJ_OK;
}

static int launch_plan(const ClusterPlan& plan, void** args, cudaStream_t st, bool pdl = false) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(plan.clusters * plan.cluster_size));
  cfg.blockDim = dim3(static_cast<unsigned>(plan.threads));
  cfg.dynamicSmemBytes = plan.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = plan.cluster_size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, plan.fn, args);
  if (e != cudaSuccess && pdl) {  // not accepted here: the ordinary launch gives the same results
    cudaGetLastError();
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, plan.fn, args);
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaLaunchKernelEx(cluster engine)");
  return DJ_OK;
}

static ClusterParams params_of(const ClusterPlan& plan) {
  ClusterParams p;
  p.words = plan.words;
  p.trace = nullptr;
  p.trace_cap = 0;
  p.timeout_ns = 2000000000LL;
  p.swcap = plan.swcap;
  p.rgs_cap = plan.rgs_cap;
  p.depth = plan.depth;
  p.srows = plan.srows;
  p.rowcap = plan.rowcap;
  p.list_cap = plan.list_cap;
  p.amerge = plan.amerge;
  return p;
}

int run_cluster(const ClusterPlan& plan, const SolveDesc* descs_dev, int32_t k, uint32_t* queue, cudaStream_t st,
                bool zero_queue) {
  if (zero_queue) {  // a fresh queue; a prepared batch's is zeroed once and reset by each launch's last cluster
    cudaError_t e = cudaMemsetAsync(queue, 0, 2 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(queue)");
  }
  ClusterParams p = params_of(plan);
  BatchJobs jobs;
  jobs.descs = descs_dev;
  jobs.queue = queue;
  jobs.k = k;
  void* args[] = {&p, &jobs};
  return launch_plan(plan, args, st);
}

int run_serve_kernel(const ClusterPlan& plan, const ServeRing& r, cudaStream_t st) {
  ClusterParams p = params_of(plan);
  ServeJobs jobs;
  jobs.ring = r.ring;
  jobs.tail = r.tail;
  jobs.stop = r.stop;
  jobs.done = r.done;
  jobs.head = r.head;
  jobs.cap_mask = r.cap_mask;
  jobs.idle_ns = r.idle_ns;
  void* args[] = {&p, &jobs};
  return launch_plan(plan, args, st);
}

int launch_cluster(const SolveDesc* descs_dev, int32_t k, int32_t /*max_n*/, int32_t max_pitch, uint32_t* queue,
                   const ClusterLaunch& cl, cudaStream_t st) {
  ClusterPlan plan;
  if (int rc = plan_cluster(max_pitch, cl, k, &plan)) return rc;
  return run_cluster(plan, descs_dev, k, queue, st, true);
}

int run_cluster_single(const ClusterPlan& plan, const SolveDesc& d, uint32_t* phases_out, uint64_t* trace,
                       int32_t trace_cap, bool early, cudaStream_t st) {
  ClusterParams p = params_of(plan);
  p.trace = trace;
  p.trace_cap = trace ? trace_cap : 0;
  SingleJob job;
  job.d = d;
  job.phases_out = phases_out;
  job.early_ok = early ? 1 : 0;
  void* args[] = {&p, &job};
  return launch_plan(plan, args, st, true);
}

SolveDesc make_desc(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, int plain) {
  SolveDesc d;
  d.W = g->W;
  d.minout = g->minout;
  d.dist = dist;
  d.pred = pred;
  d.pitch = g->pitch;
  d.n = g->n;
  d.source = source;
  d.bits_u = host_bits_for(static_cast<uint32_t>(g->n));
  d.span = host_span_for(static_cast<uint32_t>(g->n));
  d.plain = plain;
  d.use_in = g->wmin >= 1 ? 1 : 0;
  return d;
}

}  // namespace dj

// ============================================================ allocation-free single solve

// Scratch of dj_sssp_noalloc: the grid engine's control words, per-CTA
// partials and candidate lists, in a fixed array that exists on every GPU
// that loads this library (until the process exits).  In host code the name
// `g_noalloc_scratch` is only a stand-in for the device object; its device
// address is looked up once per device with cudaGetSymbolAddress.
namespace dj {
namespace {

static_assert(kNoAllocMaxCtas == 32 * kMaxPartialsPerLane, "scratch arithmetic and the decision warp agree");

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
  bool ready = false;
  uint8_t* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int num_sms = 0;
  int max_smem_optin = 0;
  int coop = 0;
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

// One-time set-up for the current device: device attributes and the scratch
// array's device address.  Neither allocates device memory.
int noalloc_setup(NoAllocDevice** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(DJ_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch array)");
    int major = 0;
    if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&d.coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess)
      return cuda_error(e, "cudaDeviceGetAttribute");
    if (major < 10) return set_error(DJ_EUNSUPPORTED, "this library targets sm_103a (Blackwell) devices");
    d.scratch = static_cast<uint8_t*>(ptr);
    d.ready = true;
  }
  *out = &d;
  return DJ_OK;
}

}  // namespace

}  // namespace dj

using namespace dj;

// One solve on the grid engine without any device allocation: see dj.h.
extern "C" int dj_sssp_noalloc(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, uint64_t stream) {
  clear_error();
  if (!g || !dist || !pred) return set_error(DJ_EINVAL, "NULL argument");
  if (source < 0 || source >= g->n) return set_error(DJ_EINVAL, "source outside [0, n)");
  if (int rc = require_dense(g)) return rc;
  NoAllocDevice* dv = nullptr;
  if (int rc = noalloc_setup(&dv)) return rc;
  if (!dv->coop) return set_error(DJ_EUNSUPPORTED, "device lacks cooperative launch");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  const int nvec_total = g->pitch / 4;
  const int G = noalloc_ctas(g->pitch, dv->num_sms);
  const int nwarps = kGridThreads / 32;
  const int nvec_cta = (nvec_total + G - 1) / G;
  const size_t need = noalloc_scratch_bytes(g->pitch, dv->num_sms);
  if (need > kNoAllocScratchBytes)
    return set_error(DJ_EINVAL, "graph too large for dj_sssp_noalloc: it needs " + std::to_string(need) +
                                    " bytes of scratch and the fixed array holds " +
                                    std::to_string(kNoAllocScratchBytes) + " (n up to " +
                                    std::to_string(noalloc_max_pitch(dv->num_sms)) + " on this device)");
  Layout L;
  L.filter = true;
  L.list_cap = std::min(nvec_total * 4, kGridListCap);
  if (int rc = make_layout(nvec_cta, nwarps, 0, G + 1, 2, static_cast<size_t>(dv->max_smem_optin) - 1024, &L))
    return rc;
  const size_t part_bytes = static_cast<size_t>(2) * G * sizeof(uint4);
  if (static_cast<size_t>(L.swcap) != static_cast<size_t>(noalloc_slice_cap(g->pitch, dv->num_sms)) ||
      sizeof(uint4) != kNoAllocEntryBytes)
    return set_error(DJ_EUNSUPPORTED, "internal: scratch layout disagrees with the slice layout");
  void* fn = grid_kernel_for(L.V);
  const int dyn = raise_smem_limit(fn, dv->max_smem_optin);  // as the other entry points: never lowered
  if (dyn < 0) return dyn;
  if (L.smem > static_cast<size_t>(dyn)) return set_error(DJ_EUNSUPPORTED, "slice state exceeds shared memory");
  // every CTA must be resident at once (cooperative launch); the query allocates nothing
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kGridThreads, L.smem);
  if (e != cudaSuccess) return cuda_error(e, "occupancy query");
  if (occ < 1) return set_error(DJ_EUNSUPPORTED, "grid engine cannot be resident");

  uint8_t* ws = dv->scratch;
  // the counters and status words must start at zero; dist[source] = -1 until the solve completes
  e = cudaMemsetAsync(ws, 0, kNoAllocCtlBytes + kNoAllocWordBytes, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(scratch)");
  e = cudaMemsetAsync(dist + source, 0xFF, sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(dist[source])");

  GridParams p;
  p.W = g->W;
  p.minout = g->minout;
  p.dist_out = dist;
  p.pred_out = pred;
  p.ctl = reinterpret_cast<uint32_t*>(ws);
  p.words = reinterpret_cast<uint32_t*>(ws + kNoAllocCtlBytes);
  p.partials = reinterpret_cast<uint4*>(ws + kNoAllocCtlBytes + kNoAllocWordBytes);
  p.cand = reinterpret_cast<uint4*>(ws + kNoAllocCtlBytes + kNoAllocWordBytes + part_bytes);
  p.pitch = g->pitch;
  p.timeout_ns = 2000000000LL;
  p.n = g->n;
  p.nvec_total = nvec_total;
  p.source = source;
  p.plain = 0;
  p.use_in = g->wmin >= 1 ? 1 : 0;
  p.bits_u = host_bits_for(static_cast<uint32_t>(g->n));
  p.span = host_span_for(static_cast<uint32_t>(g->n));
  p.cand_cap = static_cast<uint32_t>(G * L.swcap);
  p.swcap = L.swcap;
  p.rgs_cap = L.rgs_cap;
  p.skip_cta = -1;
  p.depth = L.depth;
  p.srows = L.srows;
  p.rowcap = L.rowcap;
  p.trace_cap = 0;
  p.trace = nullptr;
  p.list_cap = L.list_cap;
  p.gather_max = auto_gather_max(nvec_cta);
  p.rs_min = 0;  // no row-split or row-push state in the fixed scratch
  p.rp_min = 0;
  p.ring_bytes = static_cast<int32_t>(ring_region(L, nwarps));
  p.gsnap = nullptr;
  p.gkey = nullptr;
  p.ts = p.use_in && g->tsrc ? TieSources{g->tsrc, g->tcnt, g->tcap} : TieSources{nullptr, nullptr, 0};
  p.sym = g->directed ? 0 : 1;
  p.dyn_in = 0;  // no room for the phase stamps in the fixed scratch
  p.inlist = nullptr;
  p.inrest = nullptr;
  p.outlist = nullptr;
  p.outrest = nullptr;
  p.sph = nullptr;
  void* args[] = {&p};
  e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kGridThreads), args, L.smem, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaLaunchCooperativeKernel(grid engine)");
  return DJ_OK;
}
