// Compressed-row graphs: the same Algorithm 1 solve without the n x n matrix.
//
// The paper stores every graph as a dense adjacency matrix and concludes that
// its n^2 memory is what limits sparse graphs (Section IV, Conclusion).  A
// graph loaded with dj_load_edges_csr keeps only its edges (row offsets,
// columns, weights: 8 bytes per directed edge), and dj_sssp runs it on a
// cooperative kernel that keeps the grid engine's phase logic -- per-CTA
// column slices, one exchange of partials and candidates per phase, the OUT
// and IN settle bounds, lexicographic keys -- and replaces the row streaming:
// each CTA takes every G-th settled candidate and pushes its row's edges as
// 64-bit keys (candidate << 32) | tie word into a global per-node key array
// with atomicMin; after a second grid barrier the owners commit their slices
// from it exactly as the row-split phases of the dense engine do.
#include <algorithm>
#include <string>
#include <vector>

#include "dj_common.cuh"
#include "dj_core.cuh"
#include "dj_internal.h"

namespace dj {

struct CsrParams {
  const int64_t* row_ptr;  // n + 1
  const int32_t* col;      // nnz
  const int32_t* wt;       // nnz
  const int32_t* minout;   // n
  const int32_t* minin;    // n
  int32_t* dist_out;
  int32_t* pred_out;
  uint32_t* ctl;           // [0] barrier arrivals, [5] abort flag
  uint4* partials;         // [2][G]
  uint4* cand;             // [2][G][swcap]
  unsigned long long* gkey;  // [2][pitch], all ones between uses
  uint32_t* words;         // per-device words: [0] error bits, [1] phases
  int64_t pitch;
  int64_t timeout_ns;
  int32_t n;
  int32_t nvec_total;
  int32_t source;
  int32_t plain;
  int32_t use_in;
  uint32_t bits_u;
  uint32_t span;
  int32_t swcap;
  int32_t list_cap;
};

constexpr int kCsrThreads = 512;
constexpr int kCsrMaxPartials = 10;  // the decision warp reads up to 320 CTA partials

__global__ void __launch_bounds__(kCsrThreads, 1) k_sssp_csr(const CsrParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ BlockScratch sc;
  __shared__ Decision s_dec;
  __shared__ uint32_t s_flag;
  const int G = gridDim.x, b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  Slice s;
  const int v0 = static_cast<int>(static_cast<int64_t>(b) * p.nvec_total / G);
  const int v1 = static_cast<int>(static_cast<int64_t>(b + 1) * p.nvec_total / G);
  s.c0 = 4 * v0;
  s.nvec = v1 - v0;
  s.sw = 4 * s.nvec;
  uint8_t* q = smem;
  uint64_t* bkey = reinterpret_cast<uint64_t*>(q);  // this slice's merged keys
  q += static_cast<size_t>(p.swcap) * 8;
  uint32_t* s_off = reinterpret_cast<uint32_t*>(q);  // [G + 1] prefix of the candidate counts
  q += (static_cast<size_t>(G) + 1 + 3) / 4 * 16;
  uint32_t* ctab = reinterpret_cast<uint32_t*>(q);
  q += (static_cast<size_t>(G) * p.swcap / 32 + 1 + 3) / 4 * 16;
  uint32_t* list = reinterpret_cast<uint32_t*>(q);  // this CTA's settled rows (tie words)
  q += static_cast<size_t>(p.list_cap) * 4;
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

  slice_init(s, p.n, p.source, p.minout, p.minin, !p.plain, p.use_in && !p.plain);
  for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {  // merge keys, ordered by the first barrier
    p.gkey[s.c0 + j] = ~0ull;
    p.gkey[static_cast<size_t>(p.pitch) + s.c0 + j] = ~0ull;
  }
  if (threadIdx.x == 0) sc.cnt[32] = 0;
  __syncthreads();
  if (!p.plain) {  // the first step settles only the source: apply its edges that land in this slice
    const int64_t e0 = p.row_ptr[p.source], e1 = p.row_ptr[p.source + 1];
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int v = __ldg(p.col + e);
      if (v >= s.c0 && v < s.c0 + s.sw) {
        s.dist[v - s.c0] = static_cast<uint32_t>(__ldg(p.wt + e));
        s.pred[v - s.c0] = p.source;
        s.pdist[v - s.c0] = 0u;
      }
    }
    if (p.source >= s.c0 && p.source < s.c0 + s.sw && threadIdx.x == 0) s.vis[p.source - s.c0] = 1;
    __syncthreads();
  }
  uint32_t* bar = p.ctl;
  uint32_t* abort_flag = p.ctl + 5;
  const uint32_t umask = (1u << p.bits_u) - 1u;
  Part part;
  slice_partial(s, part);
  uint32_t phase = 0, nbar = 0;
  for (;;) {
    // 1. publish the slice's partial and candidates
    uint4* out = p.cand + (static_cast<size_t>(phase & 1) * G + b) * p.swcap;
    uint64_t key;
    uint32_t Lc;
    const int c = publish_partial(s, p.span, p.plain != 0, p.use_in != 0, part, out, &sc, &key, &Lc);
    if (threadIdx.x == 0)
      p.partials[static_cast<size_t>(phase & 1) * G + b] =
          make_uint4(static_cast<uint32_t>(key), static_cast<uint32_t>(key >> 32), Lc, static_cast<uint32_t>(c));
    if (!grid_barrier(bar, ++nbar * static_cast<uint32_t>(G), abort_flag, p.words, p.timeout_ns, &s_flag)) return;
    // 2. decision and the candidate prefix
    if (warp == 0) {
      const int per = (G + 31) / 32;
      const int i0 = min(G, lane * per), i1 = min(G, i0 + per);
      uint64_t k = kNoKey;
      uint32_t l = 0xFFFFFFFFu, sum = 0;
      const uint4* pt = p.partials + static_cast<size_t>(phase & 1) * G;
      uint4 xs[kCsrMaxPartials];
#pragma unroll
      for (int r = 0; r < kCsrMaxPartials; ++r)
        xs[r] = (i0 + r < i1) ? __ldcg(pt + i0 + r) : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u);
#pragma unroll
      for (int r = 0; r < kCsrMaxPartials; ++r) {
        const uint4 x = xs[r];
        const uint64_t kk = (static_cast<uint64_t>(x.y) << 32) | x.x;
        k = kk < k ? kk : k;
        l = min(l, x.z);
        if (i0 + r < i1) s_off[i0 + r] = sum;
        sum += x.w;
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      for (int i = i0; i < i1; ++i) s_off[i] += incl - sum;
      if (lane == 31) s_off[G] = incl;
      k = warp_min_u64(k);
      l = warp_min_u32(l);
      if (lane == 0) {
        s_dec = make_decision(k, l, p.span, p.plain != 0, p.use_in != 0);
        sc.cnt[32] = 0;
      }
    }
    __syncthreads();
    const Decision D = s_dec;
    const int total = static_cast<int>(s_off[G]);
    if (D.m >= kInf) break;
    build_chunk_table(s_off, G, ctab);
    if (threadIdx.x == 0) sc.cnt[31] = 0;
    __syncthreads();
    // 3. this CTA's share of the settled rows: candidates b, b + G, ... (plain mode: the argmin's owner)
    const uint4* cl = p.cand + static_cast<size_t>(phase & 1) * G * p.swcap;
    if (p.plain) {
      if (D.a >= static_cast<uint32_t>(s.c0) && D.a < static_cast<uint32_t>(s.c0 + s.sw) && threadIdx.x == 0) {
        list[0] = D.a;  // dist[a] - m = 0
        sc.cnt[31] = 1;
      }
    } else {
      for (int k = threadIdx.x; b + G * k < total; k += blockDim.x) {
        const int i = b + G * k;
        const int r = region_at(s_off, ctab, i);
        const uint4 e = __ldcg(cl + static_cast<size_t>(r) * p.swcap + (i - static_cast<int>(s_off[r])));
        if (in_settled(e.x, e.y, e.z, D)) {
          const uint32_t at = atomicAdd(&sc.cnt[31], 1u);
          if (at < static_cast<uint32_t>(p.list_cap)) list[at] = ((e.y - D.m) << p.bits_u) | e.x;
        }
      }
    }
    __syncthreads();
    const int nrows = min(static_cast<int>(sc.cnt[31]), p.list_cap);
    // 4. push every edge of those rows: warp w takes rows w, w + nw, ...; lanes take the edges
    unsigned long long* gk = p.gkey + static_cast<size_t>(phase & 1) * p.pitch;
    for (int r = warp; r < nrows; r += nw) {
      const uint32_t tb = list[r];
      const uint32_t u = tb & umask;
      const uint32_t du = D.m + (tb >> p.bits_u);
      const int64_t e0 = p.row_ptr[u], e1 = p.row_ptr[u + 1];
      for (int64_t e = e0 + lane; e < e1; e += 32) {
        const int v = __ldg(p.col + e);
        const unsigned long long kk =
            (static_cast<unsigned long long>(du + static_cast<uint32_t>(__ldg(p.wt + e))) << 32) | tb;
        if (kk < *reinterpret_cast<volatile unsigned long long*>(gk + v)) atomicMin(gk + v, kk);
      }
    }
    // every CTA's pushes are in gkey before the owners read their slices
    if (!grid_barrier(bar, ++nbar * static_cast<uint32_t>(G), abort_flag, p.words, p.timeout_ns, &s_flag)) return;
    for (int j = threadIdx.x; j < s.sw; j += blockDim.x) {
      bkey[j] = __ldcg(gk + s.c0 + j);
      gk[s.c0 + j] = ~0ull;  // reused two phases later, after at least one more barrier
    }
    __syncthreads();
    // 5. mark, commit, and the next partial
    commit_keys(s, D, p.bits_u, bkey, part);
    ++phase;
  }
  slice_write_out(s, p.n, p.dist_out, p.pred_out);
  if (b == 0 && threadIdx.x == 0) p.words[1] = phase;
}

}  // namespace dj

using namespace dj;

// ------------------------------------------------------------------ loading

extern "C" int dj_load_edges_csr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int32_t* w,
                                 int directed, uint64_t stream, dj_graph** out) {
  clear_error();
  if (!out) return set_error(DJ_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1) return set_error(DJ_EINVAL, "n must be >= 1");
  if (m < 0) return set_error(DJ_EINVAL, "m must be >= 0");
  if (m > 0 && (!src || !dst || !w)) return set_error(DJ_EINVAL, "edge arrays are NULL");
  // validation and the kept (u, v, w) triples, both directions for undirected graphs
  struct Edge {
    uint64_t key;  // (u << 32) | v
    int32_t w;
  };
  std::vector<Edge> es;
  es.reserve(static_cast<size_t>(directed ? m : 2 * m));
  int64_t wmax = 0;
  for (int64_t e = 0; e < m; ++e) {
    const int32_t u = src[e], v = dst[e], x = w[e];
    if (u < 0 || u >= n || v < 0 || v >= n)
      return set_error(DJ_EINVAL, "edge " + std::to_string(e) + " has a node id outside [0, n)");
    if (x < 0 || x == DJ_INF)
      return set_error(DJ_EINVAL, "edge " + std::to_string(e) + " has a weight outside [0, INT32_MAX)");
    if (u == v) continue;  // self-loops never shorten a path
    if (x > wmax) wmax = x;
    es.push_back({(static_cast<uint64_t>(u) << 32) | static_cast<uint32_t>(v), x});
    if (!directed) es.push_back({(static_cast<uint64_t>(v) << 32) | static_cast<uint32_t>(u), x});
  }
  if (n > 1 && static_cast<int64_t>(n - 1) * wmax >= static_cast<int64_t>(DJ_INF))
    return set_error(DJ_EOVERFLOW, "(n-1) * max weight >= INT32_MAX: path lengths could overflow int32");
  // sort by (u, v, w); a repeated pair keeps its smallest weight
  std::sort(es.begin(), es.end(), [](const Edge& a, const Edge& b) { return a.key != b.key ? a.key < b.key : a.w < b.w; });
  std::vector<int64_t> row_ptr(static_cast<size_t>(n) + 1, 0);
  std::vector<int32_t> col, wt;
  col.reserve(es.size());
  wt.reserve(es.size());
  std::vector<int32_t> minout(static_cast<size_t>(n), DJ_INF), minin(static_cast<size_t>(n), DJ_INF);
  int32_t wmin = DJ_INF;
  for (size_t i = 0; i < es.size(); ++i) {
    if (i > 0 && es[i].key == es[i - 1].key) continue;
    const int32_t u = static_cast<int32_t>(es[i].key >> 32), v = static_cast<int32_t>(es[i].key & 0xFFFFFFFFu);
    col.push_back(v);
    wt.push_back(es[i].w);
    ++row_ptr[static_cast<size_t>(u) + 1];
    minout[u] = std::min(minout[u], es[i].w);
    minin[v] = std::min(minin[v], es[i].w);
    wmin = std::min(wmin, es[i].w);
  }
  for (int32_t u = 0; u < n; ++u) row_ptr[static_cast<size_t>(u) + 1] += row_ptr[u];
  const int64_t nnz = static_cast<int64_t>(col.size());

  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  auto* g = new dj_graph();
  g->n = n;
  g->pitch = (n + 31) / 32 * 32;
  g->directed = directed ? 1 : 0;
  g->format = DJ_FORMAT_CSR;
  cudaGetDevice(&g->device);
  g->wmin = wmin;
  g->wmax = static_cast<int32_t>(wmax);
  g->entries = static_cast<uint64_t>(nnz);
  g->nnz = nnz;
  const size_t rp_bytes = (static_cast<size_t>(n) + 1) * sizeof(int64_t);
  const size_t e_bytes = static_cast<size_t>(std::max<int64_t>(nnz, 1)) * sizeof(int32_t);
  const size_t m_bytes = 2 * static_cast<size_t>(n) * sizeof(int32_t);
  if (cudaMalloc(&g->row_ptr, rp_bytes) != cudaSuccess || cudaMalloc(&g->col, e_bytes) != cudaSuccess ||
      cudaMalloc(&g->wt, e_bytes) != cudaSuccess || cudaMalloc(&g->minout, m_bytes) != cudaSuccess) {
    cudaGetLastError();
    dj_graph_free(g);
    return set_error(DJ_ENOMEM, "cudaMalloc of the compressed-row arrays failed");
  }
  g->minin = g->minout + n;
  g->bytes = rp_bytes + 2 * e_bytes + m_bytes;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(g->row_ptr, row_ptr.data(), rp_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nnz > 0)
    e = cudaMemcpyAsync(g->col, col.data(), static_cast<size_t>(nnz) * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nnz > 0)
    e = cudaMemcpyAsync(g->wt, wt.data(), static_cast<size_t>(nnz) * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->minout, minout.data(), static_cast<size_t>(n) * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->minin, minin.data(), static_cast<size_t>(n) * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
  if (e != cudaSuccess) {
    dj_graph_free(g);
    return cuda_error(e, "uploading the compressed-row arrays");
  }
  *out = g;
  return DJ_OK;
}

// ------------------------------------------------------------------ solving

namespace dj {

int launch_csr(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, const dj_solve_opts& o,
               cudaStream_t st) {
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  if (!ctx->coop) return set_error(DJ_EUNSUPPORTED, "device lacks cooperative launch");
  const int nvec_total = g->pitch / 4;
  const int G = std::min({ctx->num_sms, nvec_total, 32 * kCsrMaxPartials});
  const int nvec_cta = (nvec_total + G - 1) / G;
  const int swcap = 4 * nvec_cta;
  const int list_cap = swcap;  // a CTA's share of the candidates is at most one slice wide
  const size_t smem = static_cast<size_t>(swcap) * 8 + (static_cast<size_t>(G) + 1 + 3) / 4 * 16 +
                      (static_cast<size_t>(G) * swcap / 32 + 1 + 3) / 4 * 16 + static_cast<size_t>(list_cap) * 4 +
                      static_cast<size_t>(swcap) * 20 + (static_cast<size_t>(swcap) + 15) / 16 * 16;
  if (smem > static_cast<size_t>(ctx->max_smem_optin) - 1024)
    return set_error(DJ_EUNSUPPORTED, "slice state exceeds shared memory");
  void* fn = reinterpret_cast<void*>(&k_sssp_csr);
  if (int rc = prepare_function(ctx, fn, smem, false)) return rc;
  int occ = 0;
  if (int rc = function_occupancy(ctx, fn, kCsrThreads, smem, &occ)) return rc;
  cudaError_t e = cudaSuccess;
  if (occ < 1) return set_error(DJ_EUNSUPPORTED, "compressed-row solve cannot be resident");

  const size_t ctl_bytes = 256;
  const size_t part_bytes = static_cast<size_t>(2) * G * sizeof(uint4);
  const size_t cand_bytes = static_cast<size_t>(2) * G * swcap * sizeof(uint4);
  const size_t gkey_bytes = static_cast<size_t>(2) * g->pitch * 8;
  uint8_t* ws = nullptr;
  e = cudaMallocAsync(&ws, ctl_bytes + part_bytes + cand_bytes + gkey_bytes, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(csr workspace)");
  cudaMemsetAsync(ws, 0, ctl_bytes, st);
  CsrParams p;
  p.row_ptr = g->row_ptr;
  p.col = g->col;
  p.wt = g->wt;
  p.minout = g->minout;
  p.minin = g->minin;
  p.dist_out = dist;
  p.pred_out = pred;
  p.ctl = reinterpret_cast<uint32_t*>(ws);
  p.partials = reinterpret_cast<uint4*>(ws + ctl_bytes);
  p.cand = reinterpret_cast<uint4*>(ws + ctl_bytes + part_bytes);
  p.gkey = reinterpret_cast<unsigned long long*>(ws + ctl_bytes + part_bytes + cand_bytes);
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
  p.swcap = swcap;
  p.list_cap = list_cap;
  void* args[] = {&p};
  e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kCsrThreads), args, smem, st);
  cudaFreeAsync(ws, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaLaunchCooperativeKernel(csr)");
  return DJ_OK;
}

}  // namespace dj
