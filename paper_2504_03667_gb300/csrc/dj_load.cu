// Graph construction: edge list (or dense matrix) -> device adjacency matrix.
//
// Section III of the paper: the input is an edge list that each program
// writes into an n x n adjacency matrix (not timed); Section III-A: the -w
// flag fills a directed graph, otherwise undirected.  Here the matrix is
// built directly in HBM: a vectorised INF fill with a zero diagonal, a scatter
// of the edges with atomicMin (so a repeated pair keeps its smallest weight,
// independent of order), and one pass computing each row's smallest finite
// off-diagonal weight (minout) and each column's (minin), both used by the
// phase-batched solve to prove nodes final.  Rows are
// padded to a multiple of 32 int32 (128 bytes) with INF, the device analogue
// of the paper's INF padding of Section III-B.
#include <algorithm>
#include <string>

#include "dj_common.cuh"
#include "dj_internal.h"

namespace dj {

__global__ void k_fill(int32_t* __restrict__ W, int64_t pitch, int32_t n) {
  const int64_t nv = static_cast<int64_t>(n) * pitch / 4;
  int4* W4 = reinterpret_cast<int4*>(W);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < nv;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t e = i * 4;
    const int64_t r = e / pitch;
    const int64_t c = e - r * pitch;
    int4 v = make_int4(int(kInf), int(kInf), int(kInf), int(kInf));
    if (r >= c && r < c + 4) (&v.x)[r - c] = 0;
    W4[i] = v;
  }
}

__global__ void k_scatter(int32_t* __restrict__ W, int64_t pitch, const int32_t* __restrict__ src,
                          const int32_t* __restrict__ dst, const int32_t* __restrict__ w, int64_t m,
                          int directed) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t u = src[e], v = dst[e], x = w[e];
    if (u == v) continue;  // self-loops ignored: the diagonal stays 0
    atomicMin(W + static_cast<int64_t>(u) * pitch + v, x);
    if (!directed) atomicMin(W + static_cast<int64_t>(v) * pitch + u, x);
  }
}

// Copy a dense matrix with row stride ld into the padded layout, checking every
// entry lies in [0, INF]; bad entries set flags[0].
__global__ void k_copy_dense(int32_t* __restrict__ W, int64_t pitch, const int32_t* __restrict__ A, int64_t ld,
                             int32_t n, uint32_t* flags) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < static_cast<int64_t>(n) * n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = i / n, c = i - r * n;
    const int32_t x = A[r * ld + c];
    if (x < 0 && flags) atomicOr(flags, 1u);
    W[r * pitch + c] = x;
  }
}

// One warp per row: minout[u] = min finite W[u][v], v != u; plus the global
// finite min / max and the number of finite entries (stats[0] = min,
// stats[1] = max, stats[2..3] = count as a 64-bit word).
__global__ void k_rowmin(const int32_t* __restrict__ W, int64_t pitch, int32_t n, int32_t* __restrict__ minout,
                         uint32_t* stats) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  uint32_t gmin = kInf, gmax = 0;
  unsigned long long cnt = 0;
  for (int64_t u = warp; u < n; u += nwarps) {
    const int32_t* row = W + u * pitch;
    uint32_t mn = kInf, mx = 0;
    for (int64_t v = lane; v < n; v += 32) {
      const uint32_t x = static_cast<uint32_t>(row[v]);
      if (v != u && x < kInf) {
        mn = min(mn, x);
        mx = max(mx, x);
        ++cnt;
      }
    }
    mn = warp_min_u32(mn);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) minout[u] = static_cast<int32_t>(mn);
    gmin = min(gmin, mn);
    gmax = max(gmax, mx);
  }
  if (stats) {
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) {
      atomicMin(stats, gmin);
      atomicMax(stats + 1, gmax);
      atomicAdd(reinterpret_cast<unsigned long long*>(stats + 2), cnt);
    }
  }
}

// Upload from pinned host memory (device-accessible through unified addressing):
// each warp copies one row at a time from `src` (row stride ld) into the
// graph's row and takes the row's minimum finite off-diagonal entry on the
// way, so the matrix crosses the host link once and is not read again for
// its row minima.  With `vec` (ld a multiple of 4, src 16-byte aligned) the
// row moves in 16-byte pieces, four in flight per lane, and its last n mod 4
// entries one by one.  Padding columns are left as they are (INF).  With
// `ties` (a symmetric matrix, whose column v is row v and whose minin is
// minout) the warp also lists column u's tie sources as k_tiesrc would: the
// entries of row u other than the diagonal equal to its minimum, up to cap of
// them, and their count.
constexpr int kTieSourceCap = 32;
__global__ void k_upload_rows(const int32_t* __restrict__ src, int64_t ld, int32_t* __restrict__ W, int64_t pitch,
                              int32_t n, int32_t* __restrict__ minout, int vec, int ties,
                              int32_t* __restrict__ tsrc, int32_t* __restrict__ tcnt, int32_t cap) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nwarps) {
    const int32_t* s = src + u * ld;
    int32_t* d = W + u * pitch;
    uint32_t mn = kInf;
    auto take = [&](int64_t c, int32_t x) {
      if (c != u && static_cast<uint32_t>(x) < kInf) mn = min(mn, static_cast<uint32_t>(x));
    };
    int64_t done = 0;
    if (vec) {
      const int64_t nq = n / 4;
      const int4* s4 = reinterpret_cast<const int4*>(s);
      int4* d4 = reinterpret_cast<int4*>(d);
      for (int64_t q0 = 0; q0 < nq; q0 += 4 * 32) {
        int4 x[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int64_t q = q0 + 32 * r + lane;
          x[r] = q < nq ? s4[q] : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int64_t q = q0 + 32 * r + lane;
          if (q < nq) {
            d4[q] = x[r];
            take(4 * q, x[r].x);
            take(4 * q + 1, x[r].y);
            take(4 * q + 2, x[r].z);
            take(4 * q + 3, x[r].w);
          }
        }
      }
      done = 4 * nq;
    }
    for (int64_t c = done + lane; c < n; c += 32) {
      const int32_t x = s[c];
      d[c] = x;
      take(c, x);
    }
    mn = warp_min_u32(mn);
    if (lane == 0) minout[u] = static_cast<int32_t>(mn);
    if (ties) {
      __syncwarp();  // the row as every lane wrote it (now in L2)
      int32_t cnt = 0;
      const uint32_t lt = (1u << lane) - 1u;
      auto one = [&](int64_t c, int32_t x) {  // every lane calls it together
        const bool hit = c < n && c != u && static_cast<uint32_t>(x) == mn;
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int32_t pos = cnt + __popc(bal & lt);
          if (pos < cap) tsrc[u * cap + pos] = static_cast<int32_t>(c);
        }
        cnt += __popc(bal);
      };
      if (mn < kInf) {
        // the row's (device, pitch-aligned) 16-byte pieces, 4 per lane in flight; the list order
        // is fixed by the loop but immaterial to its users
        const int64_t nq = (n + 3) / 4;  // pieces covering the row (the last may hold padding: INF)
        const int4* d4 = reinterpret_cast<const int4*>(d);
        for (int64_t q0 = 0; q0 < nq; q0 += 4 * 32) {
          int4 x[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int64_t q = q0 + 32 * r + lane;
            x[r] = q < nq ? d4[q] : make_int4(int(kInf), int(kInf), int(kInf), int(kInf));
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int64_t c = 4 * (q0 + 32 * r + lane);
            one(c, x[r].x);
            one(c + 1, x[r].y);
            one(c + 2, x[r].z);
            one(c + 3, x[r].w);
          }
        }
      }
      if (lane == 0) tcnt[u] = cnt;
    }
  }
}

// minin[v] = min finite W[u][v], u != v.  A block covers 256 columns x kColRows
// rows (coalesced row reads), keeps a per-column minimum in registers and
// folds it into minin with one atomicMin per column.  minin starts at INF.
constexpr int kColRows = 256;
__global__ void k_colmin(const int32_t* __restrict__ W, int64_t pitch, int32_t n, int32_t* __restrict__ minin) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * kColRows;
  if (v >= n) return;
  uint32_t mn = kInf;
  const int64_t r1 = min(static_cast<int64_t>(n), r0 + kColRows);
  for (int64_t u = r0; u < r1; ++u) {
    const uint32_t x = static_cast<uint32_t>(W[u * pitch + v]);
    if (u != v) mn = min(mn, x);
  }
  if (mn < kInf) atomicMin(minin + v, static_cast<int32_t>(mn));
}

// Tie sources: for every column v, the rows u != v with W[u][v] == minin[v],
// up to cap per column; tcnt[v] counts them all (starts at 0).  A column whose
// stored dist equals m + minin[v] can only be tied by one of these rows.  A
// block covers 256 columns x kColRows rows like k_colmin: each thread keeps
// its column's minin in a register and reads the rows coalesced.
__global__ void k_tiesrc(const int32_t* __restrict__ W, int64_t pitch, int32_t n, const int32_t* __restrict__ minin,
                         int32_t* __restrict__ tsrc, int32_t* __restrict__ tcnt, int32_t cap) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * kColRows;
  if (v >= n) return;
  const int32_t mv = minin[v];
  if (static_cast<uint32_t>(mv) >= kInf) return;  // no finite weight into v
  const int64_t r1 = min(static_cast<int64_t>(n), r0 + kColRows);
#pragma unroll 8
  for (int64_t u = r0; u < r1; ++u) {
    if (W[u * pitch + v] == mv && u != v) {
      const int32_t pos = atomicAdd(tcnt + v, 1);
      if (pos < cap) tsrc[v * cap + pos] = static_cast<int32_t>(u);
    }
  }
}

// In-lists: for every column v the kInLists smallest finite off-diagonal weights W[u][v] with
// their rows u, ascending by (weight, row), and a lower bound on every other in-weight (the
// kInLists-th weight when the column has more in-edges, INF otherwise).  One thread per column
// reads its column top to bottom (a warp reads 128 contiguous bytes per row).
__global__ void k_inlist(const int32_t* __restrict__ W, int64_t pitch, int32_t n, uint2* __restrict__ inlist,
                         uint32_t* __restrict__ inrest) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint64_t k[kInLists];
#pragma unroll
  for (int i = 0; i < kInLists; ++i) k[i] = ~0ull;
  uint32_t cnt = 0;
  const int32_t* col = W + v;
  for (int64_t u0 = 0; u0 < n; u0 += 8) {
    uint32_t w8[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) w8[r] = u0 + r < n ? static_cast<uint32_t>(__ldg(col + (u0 + r) * pitch)) : kInf;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t u = u0 + r;
      if (w8[r] >= kInf || u == v) continue;
      ++cnt;
      uint64_t key = (static_cast<uint64_t>(w8[r]) << 32) | static_cast<uint32_t>(u);
#pragma unroll
      for (int i = 0; i < kInLists; ++i)  // insertion into the sorted list
        if (key < k[i]) {
          const uint64_t t = k[i];
          k[i] = key;
          key = t;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < kInLists; ++i)
    inlist[v * kInLists + i] = k[i] == ~0ull ? make_uint2(kInf, 0xFFFFFFFFu)
                                             : make_uint2(static_cast<uint32_t>(k[i] >> 32), static_cast<uint32_t>(k[i]));
  inrest[v] = cnt > static_cast<uint32_t>(kInLists) ? static_cast<uint32_t>(k[kInLists - 1] >> 32) : kInf;
}

// Out-lists: for every row u the kInLists smallest finite off-diagonal weights W[u][v] with their
// columns, ascending by (weight, column), and the lower bound on the others (as k_inlist).  One
// warp per row: each lane keeps the smallest of its columns, then the warp takes the list's
// entries one by one as the minimum of the lanes' heads.
__global__ void k_outlist(const int32_t* __restrict__ W, int64_t pitch, int32_t n, uint2* __restrict__ outlist,
                          uint32_t* __restrict__ outrest) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nwarps) {
    const int32_t* row = W + u * pitch;
    uint64_t k[kInLists];
#pragma unroll
    for (int i = 0; i < kInLists; ++i) k[i] = ~0ull;
    uint32_t cnt = 0;
    for (int64_t v = lane; v < n; v += 32) {
      const uint32_t w = static_cast<uint32_t>(__ldg(row + v));
      if (w >= kInf || v == u) continue;
      ++cnt;
      uint64_t key = (static_cast<uint64_t>(w) << 32) | static_cast<uint32_t>(v);
#pragma unroll
      for (int i = 0; i < kInLists; ++i)
        if (key < k[i]) {
          const uint64_t t = k[i];
          k[i] = key;
          key = t;
        }
    }
    cnt = warp_sum_u32(cnt);
    uint64_t out[kInLists];
#pragma unroll
    for (int i = 0; i < kInLists; ++i) {  // the warp's i-th smallest: the minimum of the lanes' heads
      const uint64_t mn = warp_min_u64(k[0]);
      out[i] = mn;
      if (k[0] == mn && mn != ~0ull) {  // keys are distinct (the column is in the key): one lane pops
#pragma unroll
        for (int j = 0; j + 1 < kInLists; ++j) k[j] = k[j + 1];
        k[kInLists - 1] = ~0ull;
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < kInLists; ++i)
        outlist[u * kInLists + i] = out[i] == ~0ull ? make_uint2(kInf, 0xFFFFFFFFu)
                                                    : make_uint2(static_cast<uint32_t>(out[i] >> 32),
                                                                 static_cast<uint32_t>(out[i]));
      outrest[u] = cnt > static_cast<uint32_t>(kInLists) ? static_cast<uint32_t>(out[kInLists - 1] >> 32) : kInf;
    }
  }
}

__global__ void k_fill_i32(int32_t* __restrict__ p, int64_t count, int32_t value) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    p[i] = value;
}

// Columns [n, pitch) of every row hold INF.
__global__ void k_pad_cols(int32_t* __restrict__ W, int64_t pitch, int32_t n) {
  const int64_t padw = pitch - n;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < padw * n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = i / padw;
    W[r * pitch + n + (i - r * padw)] = static_cast<int32_t>(kInf);
  }
}

// flags[0] |= 1 if any of the n x n entries is negative.
__global__ void k_check_nonneg(const int32_t* __restrict__ W, int64_t pitch, int32_t n, uint32_t* flags) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < static_cast<int64_t>(n) * n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = i / n;
    if (W[r * pitch + (i - r * n)] < 0) atomicOr(flags, 1u);
  }
}

}  // namespace dj

using namespace dj;

static int grid_for(int64_t work, int threads = 256) {
  int64_t b = (work + threads - 1) / threads;
  return static_cast<int>(std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 32));
}

static int alloc_graph(int32_t n, int directed, dj_graph** out) {
  auto* g = new dj_graph();
  g->n = n;
  g->pitch = (n + 31) / 32 * 32;
  g->directed = directed ? 1 : 0;
  cudaGetDevice(&g->device);
  const size_t mbytes = static_cast<size_t>(n) * g->pitch * sizeof(int32_t);
  cudaError_t e = cudaMalloc(&g->W, mbytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return set_error(DJ_ENOMEM, "cudaMalloc of the adjacency matrix failed (" + std::to_string(mbytes) + " bytes)");
  }
  e = cudaMalloc(&g->minout, 2 * static_cast<size_t>(n) * sizeof(int32_t));
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g->W);
    delete g;
    return set_error(DJ_ENOMEM, "cudaMalloc of the row / column minima failed");
  }
  g->minin = g->minout + n;
  g->tcap = kTieSourceCap;
  e = cudaMalloc(&g->tsrc, static_cast<size_t>(n) * (kTieSourceCap + 1) * sizeof(int32_t));
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g->W);
    cudaFree(g->minout);
    delete g;
    return set_error(DJ_ENOMEM, "cudaMalloc of the tie sources failed");
  }
  g->tcnt = g->tsrc + static_cast<size_t>(n) * kTieSourceCap;
  g->bytes = mbytes + static_cast<size_t>(n) * (kTieSourceCap + 3) * sizeof(int32_t);
  *out = g;
  return DJ_OK;
}

static void launch_inlists(dj_graph* g, cudaStream_t st) {
  k_inlist<<<static_cast<unsigned>((g->n + 127) / 128), 128, 0, st>>>(g->W, g->pitch, g->n, g->inlist, g->inrest);
  if (g->outlist != g->inlist)
    k_outlist<<<grid_for(static_cast<int64_t>(g->n) * 32), 256, 0, st>>>(g->W, g->pitch, g->n, g->outlist, g->outrest);
}

// Column minima (a copy of the row minima for undirected graphs, else
// k_colmin), then the columns' tie sources (and in-lists, where the graph keeps them).
// Row minima (unless `have_rows`: the upload kernel took them, and on a symmetric matrix the tie
// sources too), column minima, tie sources and, for graphs that keep them, the in- and out-lists.
static void launch_minima(dj_graph* g, uint32_t* stats, cudaStream_t st, bool have_rows = false) {
  if (!have_rows)
    k_rowmin<<<grid_for(static_cast<int64_t>(g->n) * 32), 256, 0, st>>>(g->W, g->pitch, g->n, g->minout, stats);
  if (!g->directed) {
    cudaMemcpyAsync(g->minin, g->minout, static_cast<size_t>(g->n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  } else {
    k_fill_i32<<<grid_for(g->n), 256, 0, st>>>(g->minin, g->n, static_cast<int32_t>(kInf));
    dim3 grid(static_cast<unsigned>((g->n + 255) / 256), static_cast<unsigned>((g->n + kColRows - 1) / kColRows));
    k_colmin<<<grid, 256, 0, st>>>(g->W, g->pitch, g->n, g->minin);
  }
  if (!(have_rows && !g->directed)) {
    cudaMemsetAsync(g->tcnt, 0, static_cast<size_t>(g->n) * sizeof(int32_t), st);
    dim3 tgrid(static_cast<unsigned>((g->n + 255) / 256), static_cast<unsigned>((g->n + kColRows - 1) / kColRows));
    k_tiesrc<<<tgrid, 256, 0, st>>>(g->W, g->pitch, g->n, g->minin, g->tsrc, g->tcnt, g->tcap);
  }
  if (g->inlist) launch_inlists(g, st);
}

// Row and column minima + global weight range, then the overflow rule (n-1) * wmax < INT32_MAX.
static int finish_graph(dj_graph* g, cudaStream_t st) {
  uint32_t* stats = nullptr;
  cudaError_t e = cudaMallocAsync(&stats, 4 * sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(stats)");
  uint32_t init[4] = {kInf, 0, 0, 0};
  cudaMemcpyAsync(stats, init, sizeof(init), cudaMemcpyHostToDevice, st);
  launch_minima(g, stats, st);
  uint32_t res[4];
  cudaMemcpyAsync(res, stats, sizeof(res), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(stats, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "building the row minima");
  g->wmin = static_cast<int32_t>(res[0]);
  g->wmax = static_cast<int32_t>(res[1]);
  g->entries = static_cast<uint64_t>(res[2]) | (static_cast<uint64_t>(res[3]) << 32);
  if (g->n > 1 && static_cast<int64_t>(g->n - 1) * g->wmax >= static_cast<int64_t>(DJ_INF))
    return set_error(DJ_EOVERFLOW, "(n-1) * max weight >= INT32_MAX: path lengths could overflow int32");
  // graphs that are not dense keep in-lists for the grid engine's dynamic IN bound
  const uint64_t nn = static_cast<uint64_t>(g->n) * static_cast<uint64_t>(g->n);
  if (g->entries * 32 < nn && g->wmin >= 1 && !g->inlist) {
    const size_t lb = static_cast<size_t>(g->n) * kInLists * sizeof(uint2), rb = static_cast<size_t>(g->n) * 4;
    const int lists = g->directed ? 2 : 1;  // a symmetric matrix's out-lists are its in-lists
    uint8_t* buf = nullptr;
    // [in-lists][out-lists][in rests][out rests]: the 8-byte entries first, at multiples of 32 n bytes
    if (cudaMalloc(&buf, lists * (lb + rb)) == cudaSuccess) {
      g->inlist = reinterpret_cast<uint2*>(buf);
      g->outlist = lists == 2 ? reinterpret_cast<uint2*>(buf + lb) : g->inlist;
      g->inrest = reinterpret_cast<uint32_t*>(buf + lists * lb);
      g->outrest = lists == 2 ? reinterpret_cast<uint32_t*>(buf + 2 * lb + rb) : g->inrest;
      g->bytes += lists * (lb + rb);
      launch_inlists(g, st);
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_error(e, "building the in-lists");
    } else {
      cudaGetLastError();  // no room: the static IN bound only
    }
  }
  return DJ_OK;
}

extern "C" int dj_load_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int32_t* w,
                             int directed, uint64_t stream, dj_graph** out) {
  clear_error();
  if (!out) return set_error(DJ_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1) return set_error(DJ_EINVAL, "n must be >= 1");
  if (m < 0) return set_error(DJ_EINVAL, "m must be >= 0");
  if (m > 0 && (!src || !dst || !w)) return set_error(DJ_EINVAL, "edge arrays are NULL");
  // host-side validation and the weight range of the kept (non-self-loop) edges
  int64_t wmax = 0;
  for (int64_t e = 0; e < m; ++e) {
    const int32_t u = src[e], v = dst[e], x = w[e];
    if (u < 0 || u >= n || v < 0 || v >= n)
      return set_error(DJ_EINVAL, "edge " + std::to_string(e) + " has a node id outside [0, n)");
    if (x < 0 || x == DJ_INF)
      return set_error(DJ_EINVAL, "edge " + std::to_string(e) + " has a weight outside [0, INT32_MAX)");
    if (u != v && x > wmax) wmax = x;
  }
  if (n > 1 && static_cast<int64_t>(n - 1) * wmax >= static_cast<int64_t>(DJ_INF))
    return set_error(DJ_EOVERFLOW, "(n-1) * max weight >= INT32_MAX: path lengths could overflow int32");
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dj_graph* g = nullptr;
  if (int rc = alloc_graph(n, directed, &g)) return rc;
  k_fill<<<grid_for(static_cast<int64_t>(n) * g->pitch / 4), 256, 0, st>>>(g->W, g->pitch, n);
  if (m > 0) {
    const int64_t chunk = std::min<int64_t>(m, int64_t(1) << 24);  // 16 Mi edges (192 MiB) per stage
    int32_t* stage = nullptr;
    cudaError_t e = cudaMallocAsync(&stage, static_cast<size_t>(chunk) * 3 * sizeof(int32_t), st);
    if (e != cudaSuccess) {
      dj_graph_free(g);
      return cuda_error(e, "cudaMallocAsync(edge staging)");
    }
    for (int64_t off = 0; off < m; off += chunk) {
      const int64_t c = std::min(chunk, m - off);
      cudaMemcpyAsync(stage, src + off, c * sizeof(int32_t), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(stage + chunk, dst + off, c * sizeof(int32_t), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(stage + 2 * chunk, w + off, c * sizeof(int32_t), cudaMemcpyHostToDevice, st);
      k_scatter<<<grid_for(c), 256, 0, st>>>(g->W, g->pitch, stage, stage + chunk, stage + 2 * chunk, c, directed);
      // the host arrays may be pageable: finish this stage before reusing the buffer
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        dj_graph_free(g);
        return cuda_error(e, "scattering edges");
      }
    }
    cudaFreeAsync(stage, st);
  }
  if (int rc = finish_graph(g, st)) {
    dj_graph_free(g);
    return rc;
  }
  *out = g;
  return DJ_OK;
}

static int copy_dense_in(dj_graph* g, const int32_t* W, int64_t ld, int w_on_device, bool check, cudaStream_t st) {
  const int32_t n = g->n;
  uint32_t* flags = nullptr;
  cudaError_t e;
  if (check) {
    e = cudaMallocAsync(&flags, sizeof(uint32_t), st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(flags)");
    cudaMemsetAsync(flags, 0, sizeof(uint32_t), st);
  }
  if (w_on_device) {
    k_copy_dense<<<grid_for(static_cast<int64_t>(n) * n), 256, 0, st>>>(g->W, g->pitch, W, ld, n,
                                                                         flags ? flags : nullptr);
  } else {
    e = cudaMemcpy2DAsync(g->W, static_cast<size_t>(g->pitch) * sizeof(int32_t), W,
                          static_cast<size_t>(ld) * sizeof(int32_t), static_cast<size_t>(n) * sizeof(int32_t),
                          static_cast<size_t>(n), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy2DAsync(host matrix)");
    if (check) k_check_nonneg<<<grid_for(static_cast<int64_t>(n) * n), 256, 0, st>>>(g->W, g->pitch, n, flags);
  }
  if (g->pitch > n)
    k_pad_cols<<<grid_for(static_cast<int64_t>(g->pitch - n) * n), 256, 0, st>>>(g->W, g->pitch, n);
  if (!check) return DJ_OK;
  uint32_t bad = 0;
  cudaMemcpyAsync(&bad, flags, sizeof(bad), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(flags, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "copying the dense matrix");
  if (bad) return set_error(DJ_EINVAL, "matrix holds a negative entry");
  return DJ_OK;
}

extern "C" int dj_load_dense(int32_t n, const int32_t* W, int64_t ld, int w_on_device, uint64_t stream,
                             dj_graph** out) {
  clear_error();
  if (!out) return set_error(DJ_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !W || ld < n) return set_error(DJ_EINVAL, "need n >= 1, W != NULL and ld >= n");
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dj_graph* g = nullptr;
  if (int rc = alloc_graph(n, 1, &g)) return rc;
  if (int rc = copy_dense_in(g, W, ld, w_on_device, true, st)) {
    dj_graph_free(g);
    return rc;
  }
  if (int rc = finish_graph(g, st)) {
    dj_graph_free(g);
    return rc;
  }
  *out = g;
  return DJ_OK;
}

extern "C" int dj_graph_upload(dj_graph* g, const int32_t* W, int64_t ld, uint64_t stream) {
  clear_error();
  if (int rc = require_dense(g)) return rc;
  if (!g || !W || ld < g->n) return set_error(DJ_EINVAL, "need g, W != NULL and ld >= n");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  // pinned host memory the device can address: one kernel copies the rows and takes their minima
  cudaPointerAttributes pa;
  const cudaError_t pe = cudaPointerGetAttributes(&pa, W);
  if (pe != cudaSuccess) cudaGetLastError();  // clear that query's own status only
  const bool zero_copy = pe == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr;
  if (zero_copy) {
    const int32_t* src = static_cast<const int32_t*>(pa.devicePointer);
    const int vec = (ld % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0) ? 1 : 0;
    k_upload_rows<<<grid_for(static_cast<int64_t>(g->n) * 32), 256, 0, st>>>(
        src, ld, g->W, g->pitch, g->n, g->minout, vec, g->directed ? 0 : 1, g->tsrc, g->tcnt, g->tcap);
    e = cudaGetLastError();
  } else if (ld == g->n && g->n == g->pitch) {  // no padding columns on either side: one contiguous copy
    e = cudaMemcpyAsync(g->W, W, static_cast<size_t>(g->n) * g->pitch * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  } else {
    e = cudaMemcpy2DAsync(g->W, static_cast<size_t>(g->pitch) * sizeof(int32_t), W,
                          static_cast<size_t>(ld) * sizeof(int32_t), static_cast<size_t>(g->n) * sizeof(int32_t),
                          static_cast<size_t>(g->n), cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return cuda_error(e, "host-to-device matrix copy (upload)");
  g->upload_pending = 1;
  launch_minima(g, nullptr, st, zero_copy);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "row minima");
  return DJ_OK;
}

extern "C" int dj_graph_download(const dj_graph* g, int32_t* W, int64_t ld, uint64_t stream) {
  clear_error();
  if (int rc = require_dense(g)) return rc;
  if (!g || !W || ld < g->n) return set_error(DJ_EINVAL, "need g, W != NULL and ld >= n");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpy2DAsync(W, static_cast<size_t>(ld) * sizeof(int32_t), g->W,
                                    static_cast<size_t>(g->pitch) * sizeof(int32_t), static_cast<size_t>(g->n) * sizeof(int32_t),
                                    static_cast<size_t>(g->n), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy2DAsync(download)");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "download");
  return DJ_OK;
}

extern "C" int dj_graph_get_info(const dj_graph* g, dj_graph_info* info) {
  clear_error();
  if (!g || !info) return set_error(DJ_EINVAL, "NULL argument");
  info->n = g->n;
  info->pitch = g->pitch;
  info->directed = g->directed;
  info->min_weight = g->wmin;
  info->max_weight = g->wmax;
  info->device = g->device;
  info->matrix = g->W;
  info->minout = g->minout;
  info->minin = g->minin;
  info->bytes = g->bytes;
  info->entries = g->entries;
  info->format = g->format;
  return DJ_OK;
}

extern "C" int dj_graph_free(dj_graph* g) {
  clear_error();
  if (!g) return DJ_OK;
  cudaFree(g->W);
  cudaFree(g->minout);  // minin shares this allocation
  cudaFree(g->tsrc);    // tcnt shares this allocation
  cudaFree(g->inlist);  // inrest shares this allocation
  cudaFree(g->row_ptr);
  cudaFree(g->col);
  cudaFree(g->wt);
  cudaFree(g->tiled);
  delete g;
  return DJ_OK;
}

namespace dj {
int require_dense(const dj_graph* g) {
  if (g && g->format != DJ_FORMAT_DENSE)
    return set_error(DJ_EUNSUPPORTED, "this call needs the dense matrix; the graph was loaded in compressed-row form");
  return DJ_OK;
}
}  // namespace dj
