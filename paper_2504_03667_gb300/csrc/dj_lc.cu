// Label-correcting solve: the paper's CUDA variant (Algorithms 3 and 4,
// Section III-C) rebuilt for this GPU as a comparison point.
//
// The paper's kernel gives each thread a row u and, sweep after sweep, lowers
// dist[v] with atomicMin(dist[u] + G[u][v]) for every v until a Thrust
// reduction over an `updated` array finds no change; the host drives the
// sweeps.  That is a Bellman-Ford fixed point: its dist are the exact shortest
// distances, its pred is whichever improving write landed (nondeterministic,
// and not Algorithm 1's in general).
//
// Here one cooperative persistent kernel runs every sweep: each CTA owns a
// column slice (dist, pred in shared memory), a sweep relaxes only the rows
// whose dist changed in the previous sweep (the frontier, published by the
// rows' owners as (u, dist[u]) around one grid barrier), every warp reads its
// frontier rows' slices with 16-byte loads (lane l: columns 4 l .. 4 l + 3 of
// each 128-column chunk, several rows in flight), and the per-column minimum of (dist[u] + G[u][v], u)
// over the sweep is committed on strict improvement.  The sweep loop ends on
// the device when the frontier is empty.  dist equals Algorithm 1's; pred is a
// shortest-path tree (dist[pred[v]] + G[pred[v]][v] == dist[v]) with the
// smallest improving u of the last improving sweep, not Algorithm 1's choice
// among equal paths.
#include <algorithm>

#include "dj_common.cuh"
#include "dj_core.cuh"
#include "dj_internal.h"

namespace dj {

struct LcParams {
  const int32_t* W;
  int32_t* dist_out;
  int32_t* pred_out;
  uint32_t* ctl;       // [0] barrier arrivals, [5] abort flag
  uint32_t* counts;    // [2][G] frontier entries per CTA, by sweep parity
  uint2* front;        // [2][G][swcap] (u, dist[u]) by sweep parity
  uint32_t* words;     // per-device words: [0] error bits, [1] sweeps
  int64_t pitch;
  int64_t timeout_ns;
  int32_t n;
  int32_t nvec_total;
  int32_t source;
  int32_t swcap;
};

constexpr int kLcThreads = 512;
constexpr int kLcLoads = 8;  // 16-byte loads in flight per lane (rows x column groups)

template <int V>
__global__ void __launch_bounds__(kLcThreads, 1) k_sssp_lc(const LcParams p) {
  constexpr int kLcRows = kLcLoads / V;  // frontier rows in flight per warp
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ uint32_t s_flag;
  __shared__ uint32_t s_cnt;
  const int G = gridDim.x, b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int v0 = static_cast<int>(static_cast<int64_t>(b) * p.nvec_total / G);
  const int v1 = static_cast<int>(static_cast<int64_t>(b + 1) * p.nvec_total / G);
  const int c0 = 4 * v0, nvec = v1 - v0, sw = 4 * nvec;
  uint8_t* q = smem;
  uint64_t* merge = reinterpret_cast<uint64_t*>(q);  // [nw][swcap] per-warp bests
  q += static_cast<size_t>(nw) * p.swcap * 8;
  uint32_t* dist = reinterpret_cast<uint32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  int32_t* pred = reinterpret_cast<int32_t*>(q);
  q += static_cast<size_t>(p.swcap) * 4;
  uint32_t* s_off = reinterpret_cast<uint32_t*>(q);  // [G + 1]
  q += (static_cast<size_t>(G) + 1 + 3) / 4 * 16;
  uint32_t* ctab = reinterpret_cast<uint32_t*>(q);  // region of every 32nd frontier entry
  q += (static_cast<size_t>(G) * p.swcap / 32 + 1 + 3) / 4 * 16;
  uint8_t* changed = q;

  for (int j = threadIdx.x; j < sw; j += blockDim.x) {
    const int v = c0 + j;
    dist[j] = (v < p.n && v == p.source) ? 0u : kInf;
    pred[j] = -1;
    changed[j] = (v < p.n && v == p.source) ? 1 : 0;  // sweep 0 relaxes the source's row
  }
  __syncthreads();
  uint32_t* bar = p.ctl;
  uint32_t* abort_flag = p.ctl + 5;
  uint32_t sweep = 0;
  for (;; ++sweep) {
    // 1. publish this slice's changed columns as frontier entries
    const uint32_t par = sweep & 1u;
    uint2* out = p.front + (static_cast<size_t>(par) * G + b) * p.swcap;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int j0 = 0; j0 < sw; j0 += blockDim.x) {
      const int j = j0 + threadIdx.x;
      const bool c = j < sw && changed[j];
      const uint32_t bal = __ballot_sync(0xffffffffu, c);
      if (bal) {
        uint32_t pos = 0;
        if (lane == 0) pos = atomicAdd(&s_cnt, static_cast<uint32_t>(__popc(bal)));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (c) out[pos + __popc(bal & ((1u << lane) - 1u))] = make_uint2(static_cast<uint32_t>(c0 + j), dist[j]);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) p.counts[static_cast<size_t>(par) * G + b] = s_cnt;
    if (!grid_barrier(bar, (sweep + 1) * static_cast<uint32_t>(G), abort_flag, p.words, p.timeout_ns, &s_flag)) return;
    // 2. the frontier: prefix of the CTAs' counts (warp 0), chunk table
    if (warp == 0) {
      const uint32_t* cnt = p.counts + static_cast<size_t>(par) * G;
      uint32_t sum = 0;
      const int per = (G + 31) / 32;
      const int i0 = min(G, lane * per), i1 = min(G, i0 + per);
      for (int i = i0; i < i1; ++i) {
        s_off[i] = sum;
        sum += __ldcg(cnt + i);
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      for (int i = i0; i < i1; ++i) s_off[i] += incl - sum;
      if (lane == 31) s_off[G] = incl;
    }
    __syncthreads();
    const int total = static_cast<int>(s_off[G]);
    if (total == 0) break;  // nothing changed in the last sweep: the fixed point
    if (sweep >= static_cast<uint32_t>(p.n)) {  // non-negative weights converge within n sweeps
      if (threadIdx.x == 0) atomicOr(p.words, kErrTimeout);
      break;
    }
    build_chunk_table(s_off, G, ctab);
    __syncthreads();
    // 3. relax: warp w takes frontier entries w, w + nw, ...; lane l owns columns
    //    4 (l + 32 k) .. + 3 of the slice; kLcRows rows in flight
    const uint2* fl = p.front + static_cast<size_t>(par) * G * p.swcap;
    const int swcap = p.swcap;
    auto entry = [fl, swcap, s_off, ctab](int i) {
      const int r = region_at(s_off, ctab, i);
      return __ldcg(fl + static_cast<size_t>(r) * swcap + (i - static_cast<int>(s_off[r])));
    };
    uint32_t bc[V][4], bt[V][4];
#pragma unroll
    for (int k = 0; k < V; ++k)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        bc[k][c] = 0xFFFFFFFFu;
        bt[k][c] = 0xFFFFFFFFu;
      }
    const int4* W4 = reinterpret_cast<const int4*>(p.W);
    const int64_t rowvec = p.pitch / 4;
    const int K = (total - warp + nw - 1) / nw;  // this warp's entries
    uint2 nxt = lane < K ? entry(warp + nw * lane) : make_uint2(0u, kInf);
    for (int j = 0; 32 * j < K; ++j) {
      const uint2 cur = nxt;
      const int kk = 32 * (j + 1) + lane;
      nxt = kk < K ? entry(warp + nw * kk) : make_uint2(0u, kInf);
      const int cnt = min(32, K - 32 * j);
      for (int r0 = 0; r0 < cnt; r0 += kLcRows) {
        int4 x[kLcRows][V];
        uint32_t du[kLcRows], uu[kLcRows];
#pragma unroll
        for (int r = 0; r < kLcRows; ++r) {
          uu[r] = __shfl_sync(0xffffffffu, cur.x, (r0 + r) & 31);
          du[r] = __shfl_sync(0xffffffffu, cur.y, (r0 + r) & 31);
          const bool on = r0 + r < cnt;
#pragma unroll
          for (int k = 0; k < V; ++k) {
            const int g = lane + 32 * k;
            x[r][k] = (on && g < nvec) ? __ldcs(W4 + static_cast<int64_t>(uu[r]) * rowvec + v0 + g)
                                       : make_int4(kInf, kInf, kInf, kInf);
          }
          if (!on) du[r] = 0u;
        }
#pragma unroll
        for (int r = 0; r < kLcRows; ++r)
#pragma unroll
          for (int k = 0; k < V; ++k) {
            best_update(du[r] + static_cast<uint32_t>(x[r][k].x), uu[r], bc[k][0], bt[k][0]);
            best_update(du[r] + static_cast<uint32_t>(x[r][k].y), uu[r], bc[k][1], bt[k][1]);
            best_update(du[r] + static_cast<uint32_t>(x[r][k].z), uu[r], bc[k][2], bt[k][2]);
            best_update(du[r] + static_cast<uint32_t>(x[r][k].w), uu[r], bc[k][3], bt[k][3]);
          }
      }
    }
    // 4. merge the warps' bests and commit strict improvements
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int g = lane + 32 * k;
      if (g < nvec)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          merge[static_cast<size_t>(warp) * p.swcap + 4 * g + c] = (static_cast<uint64_t>(bc[k][c]) << 32) | bt[k][c];
    }
    __syncthreads();
    for (int col = threadIdx.x; col < sw; col += blockDim.x) {
      uint64_t best = kNoKey;
      for (int w = 0; w < nw; ++w) {
        const uint64_t x = merge[static_cast<size_t>(w) * p.swcap + col];
        best = x < best ? x : best;
      }
      const uint32_t c = static_cast<uint32_t>(best >> 32);
      const bool imp = c < kInf && c < dist[col];  // padding columns hold INF weights: never
      if (imp) {
        dist[col] = c;
        pred[col] = static_cast<int32_t>(static_cast<uint32_t>(best));
      }
      changed[col] = imp ? 1 : 0;
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < sw; j += blockDim.x) {
    const int v = c0 + j;
    if (v < p.n) {
      p.dist_out[v] = static_cast<int32_t>(dist[j]);
      p.pred_out[v] = pred[j];
    }
  }
  if (b == 0 && threadIdx.x == 0) p.words[1] = sweep;
}

namespace {

void* lc_kernel_for(int v) {
  switch (v) {
    case 1: return reinterpret_cast<void*>(&k_sssp_lc<1>);
    case 2: return reinterpret_cast<void*>(&k_sssp_lc<2>);
    case 4: return reinterpret_cast<void*>(&k_sssp_lc<4>);
  }
  return nullptr;
}

}  // namespace

}  // namespace dj

using namespace dj;

extern "C" int dj_sssp_lc(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, uint64_t stream) {
  clear_error();
  if (!g || !dist || !pred) return set_error(DJ_EINVAL, "NULL argument");
  if (source < 0 || source >= g->n) return set_error(DJ_EINVAL, "source outside [0, n)");
  if (int rc = require_dense(g)) return rc;
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  if (!ctx->coop) return set_error(DJ_EUNSUPPORTED, "device lacks cooperative launch");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nvec_total = g->pitch / 4;
  const int G = std::min({ctx->num_sms, nvec_total, 1024});
  const int nvec_cta = (nvec_total + G - 1) / G;
  int V = 0;
  for (int v : {1, 2, 4})
    if (nvec_cta <= 32 * v) {
      V = v;
      break;
    }
  if (!V) return set_error(DJ_EUNSUPPORTED, "graph too large for the label-correcting solve");
  const int swcap = 4 * nvec_cta;
  const int nw = kLcThreads / 32;
  const size_t smem = static_cast<size_t>(nw) * swcap * 8 + static_cast<size_t>(swcap) * 8 +
                      (static_cast<size_t>(G) + 1 + 3) / 4 * 16 +
                      (static_cast<size_t>(G) * swcap / 32 + 1 + 3) / 4 * 16 + (static_cast<size_t>(swcap) + 15) / 16 * 16;
  if (smem > static_cast<size_t>(ctx->max_smem_optin)) return set_error(DJ_EUNSUPPORTED, "slice state exceeds shared memory");
  void* fn = lc_kernel_for(V);
  if (int rc = prepare_function(ctx, fn, smem, false)) return rc;
  int occ = 0;
  if (int rc = function_occupancy(ctx, fn, kLcThreads, smem, &occ)) return rc;
  cudaError_t e = cudaSuccess;
  if (occ < 1) return set_error(DJ_EUNSUPPORTED, "label-correcting solve cannot be resident");

  const size_t ctl_bytes = 256;
  const size_t cnt_bytes = (static_cast<size_t>(2) * G * 4 + 15) / 16 * 16;
  const size_t front_bytes = static_cast<size_t>(2) * G * swcap * sizeof(uint2);
  uint8_t* ws = nullptr;
  e = cudaMallocAsync(&ws, ctl_bytes + cnt_bytes + front_bytes, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(label-correcting workspace)");
  cudaMemsetAsync(ws, 0, ctl_bytes, st);
  LcParams p;
  p.W = g->W;
  p.dist_out = dist;
  p.pred_out = pred;
  p.ctl = reinterpret_cast<uint32_t*>(ws);
  p.counts = reinterpret_cast<uint32_t*>(ws + ctl_bytes);
  p.front = reinterpret_cast<uint2*>(ws + ctl_bytes + cnt_bytes);
  p.words = ctx->words;
  p.pitch = g->pitch;
  p.timeout_ns = 2000000000LL;
  p.n = g->n;
  p.nvec_total = nvec_total;
  p.source = source;
  p.swcap = swcap;
  void* args[] = {&p};
  e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kLcThreads), args, smem, st);
  cudaFreeAsync(ws, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaLaunchCooperativeKernel(label-correcting)");
  return DJ_OK;
}
