// Serving: continuous batching of single-source solves on resident graphs.
//
// The paper times one solve per program run (Section IV); serving is the
// deployment form of the same Algorithm 1 solve.  Design:
//   * graphs stay resident in HBM; the server admits them against a byte budget;
//   * requests are descriptors in a ring of mapped pinned host memory; the host
//     publishes them one by one (tail, release) and never waits for the GPU;
//   * one persistent cluster-engine kernel keeps every cluster busy: each
//     cluster claims the next published request, solves it in distributed
//     shared memory and raises the request's done word; requests that arrive
//     while others are running are picked up by whichever cluster frees first,
//     so solves of different graphs and sizes overlap on the device;
//   * the kernel leaves after an idle timeout and is relaunched on demand;
//   * latency is measured on the host from submission (or scheduled arrival,
//     for traces) to the moment the done word is seen.
// All calls on one server must come from one host thread.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "dj_internal.h"

using namespace dj;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct PoolBuf {
  int32_t* ptr = nullptr;  // dist (n) then pred (n)
  size_t bytes = 0;
  int64_t owner = -1;  // ticket whose result it holds
  bool busy = false;   // reserved by an in-flight request
};

struct Slot {
  uint64_t ticket = 0;
  double t_ref = 0;  // latency reference: submit time or scheduled arrival
  int pool = -1;
  bool done = false;
};

// Slices of about 1024 columns: wide ring copies, and clusters small enough to keep
// many requests in flight (measured on the 64-graph serving mix: cluster size 16
// for the n=16384 graphs raised saturation by 10 % and cut p99 by 15 % against 8).
int heuristic_cluster(int32_t pitch) {
  int c = 2;
  while (c < 16 && c * 1024 < pitch) c *= 2;  // a power of two: slices of at most ~1024 columns
  return c;
}

}  // namespace

struct dj_server {
  int device = 0;
  dj_serve_opts opts{};
  cudaStream_t stream = nullptr;
  cudaEvent_t kernel_end = nullptr;
  bool kernel_live = false;
  int launches = 0;
  // mapped pinned host memory
  SolveDesc* ring_h = nullptr;
  SolveDesc* ring_d = nullptr;
  uint32_t* ctl_h = nullptr;  // [0] tail, [16] stop (separate cache lines)
  uint32_t* ctl_d = nullptr;
  uint32_t* done_h = nullptr;
  uint32_t* done_d = nullptr;
  uint32_t* head_d = nullptr;  // device memory
  uint32_t cap = 0;
  uint64_t next_ticket = 0;
  std::vector<Slot> slots;     // by ticket % cap
  std::deque<uint64_t> order;  // in submission order; the front is the oldest not yet reaped
  size_t inflight = 0;
  // graphs and budget
  std::vector<const dj_graph*> graphs;
  uint64_t graph_bytes = 0;
  uint64_t pool_bytes = 0;
  uint64_t fixed_bytes = 0;
  std::vector<PoolBuf> pool;
  int32_t plan_pitch = 0;
  ClusterPlan plan;
  bool plan_valid = false;
  // statistics
  std::vector<double> lat_us;
  double first_ref = -1, last_done = -1;
  uint64_t submitted = 0, completed = 0, rejected = 0;
};

namespace {

int stop_kernel(dj_server* s) {
  if (!s->kernel_live) return DJ_OK;
  __atomic_store_n(s->ctl_h + 16, 1u, __ATOMIC_RELEASE);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  __atomic_store_n(s->ctl_h + 16, 0u, __ATOMIC_RELEASE);
  s->kernel_live = false;
  if (e != cudaSuccess) return cuda_error(e, "serving kernel");
  return DJ_OK;
}

int ensure_plan(dj_server* s) {
  int32_t pitch = 32;
  for (auto* g : s->graphs) pitch = std::max(pitch, g->pitch);
  if (s->plan_valid && pitch <= s->plan_pitch) return DJ_OK;
  if (int rc = stop_kernel(s)) return rc;
  ClusterLaunch cl;
  cl.cluster_size = s->opts.cluster_size > 0 ? s->opts.cluster_size : heuristic_cluster(pitch);
  cl.clusters = s->opts.clusters;
  if (int rc = plan_cluster(pitch, cl, 0, &s->plan, kJobsServe)) return rc;
  s->plan_pitch = pitch;
  s->plan_valid = true;
  return DJ_OK;
}

// (Re)launch the persistent kernel if requests wait and it is not running.
int ensure_kernel(dj_server* s) {
  if (s->kernel_live) {
    cudaError_t q = cudaEventQuery(s->kernel_end);
    if (q == cudaErrorNotReady) return DJ_OK;
    s->kernel_live = false;
    if (q != cudaSuccess) return cuda_error(q, "serving kernel");
  }
  if (s->inflight == 0) return DJ_OK;
  if (int rc = ensure_plan(s)) return rc;
  ServeRing r;
  r.ring = s->ring_d;
  r.tail = s->ctl_d;
  r.stop = s->ctl_d + 16;
  r.done = s->done_d;
  r.head = s->head_d;
  r.cap_mask = s->cap - 1;
  r.idle_ns = s->opts.idle_timeout_ns > 0 ? s->opts.idle_timeout_ns : 200000000LL;
  if (int rc = run_serve_kernel(s->plan, r, s->stream)) return rc;
  cudaError_t e = cudaEventRecord(s->kernel_end, s->stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
  s->kernel_live = true;
  ++s->launches;
  return DJ_OK;
}

// Collect completed requests (done word == ticket + 1) and record their latency.
void reap(dj_server* s) {
  if (s->inflight == 0) return;
  const double t = now_s();
  for (uint64_t tk : s->order) {
    Slot& sl = s->slots[tk & (s->cap - 1)];
    if (sl.done || sl.ticket != tk) continue;
    const uint32_t w = __atomic_load_n(s->done_h + (tk & (s->cap - 1)), __ATOMIC_ACQUIRE);
    if (w != static_cast<uint32_t>(tk + 1)) continue;
    sl.done = true;
    --s->inflight;
    ++s->completed;
    s->lat_us.push_back((t - sl.t_ref) * 1e6);
    s->last_done = t;
    if (sl.pool >= 0) s->pool[sl.pool].busy = false;
  }
  while (!s->order.empty() && s->slots[s->order.front() & (s->cap - 1)].done) s->order.pop_front();
}

// A pooled result buffer of at least `bytes`, within the budget; -1 if none.
int take_pool(dj_server* s, size_t bytes) {
  int best = -1;
  for (size_t i = 0; i < s->pool.size(); ++i)
    if (!s->pool[i].busy && s->pool[i].bytes >= bytes && (best < 0 || s->pool[i].bytes < s->pool[best].bytes))
      best = static_cast<int>(i);
  if (best >= 0) return best;
  size_t want = 4096;
  while (want < bytes) want *= 2;
  if (s->graph_bytes + s->pool_bytes + s->fixed_bytes + want > s->opts.hbm_budget) return -1;
  PoolBuf b;
  if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  b.bytes = want;
  s->pool_bytes += want;
  s->pool.push_back(b);
  return static_cast<int>(s->pool.size() - 1);
}

int submit(dj_server* s, int32_t gid, int32_t source, int32_t* dist, int32_t* pred, double t_ref, uint64_t* ticket) {
  if (gid < 0 || gid >= static_cast<int32_t>(s->graphs.size())) return set_error(DJ_EINVAL, "unknown graph id");
  const dj_graph* g = s->graphs[gid];
  if (source < 0 || source >= g->n) return set_error(DJ_EINVAL, "source outside [0, n)");
  if ((dist == nullptr) != (pred == nullptr)) return set_error(DJ_EINVAL, "pass both dist and pred, or neither");
  reap(s);
  // a slot is free when fewer than max_slots are in flight and the ring entry's
  // previous occupant (ticket - cap) has completed
  if (s->inflight >= static_cast<size_t>(s->opts.max_slots) ||
      (!s->order.empty() && s->next_ticket - s->order.front() >= s->cap)) {
    ++s->rejected;
    return set_error(DJ_EBUSY, "every serving slot is in flight");
  }
  int pool = -1;
  if (!dist) {
    pool = take_pool(s, static_cast<size_t>(g->n) * 8);
    if (pool < 0) {
      ++s->rejected;
      return set_error(DJ_EBUSY, "no result memory left in the HBM budget");
    }
    s->pool[pool].busy = true;
    dist = s->pool[pool].ptr;
    pred = s->pool[pool].ptr + g->n;
  }
  const uint64_t tk = s->next_ticket;
  const uint32_t slot = static_cast<uint32_t>(tk & (s->cap - 1));
  s->ring_h[slot] = make_desc(g, source, dist, pred, 0);
  Slot& sl = s->slots[slot];
  sl.ticket = tk;
  sl.t_ref = t_ref;
  sl.pool = pool;
  sl.done = false;
  if (pool >= 0) s->pool[pool].owner = static_cast<int64_t>(tk);
  __atomic_store_n(s->ctl_h, static_cast<uint32_t>(tk + 1), __ATOMIC_RELEASE);  // publish
  s->next_ticket = tk + 1;
  s->order.push_back(tk);
  ++s->inflight;
  ++s->submitted;
  if (s->first_ref < 0 || t_ref < s->first_ref) s->first_ref = t_ref;
  if (int rc = ensure_kernel(s)) return rc;
  if (ticket) *ticket = tk;
  return DJ_OK;
}

void free_server(dj_server* s) {
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& b : s->pool) cudaFree(b.ptr);
  if (s->head_d) cudaFree(s->head_d);
  if (s->ring_h) cudaFreeHost(s->ring_h);
  if (s->ctl_h) cudaFreeHost(s->ctl_h);
  if (s->done_h) cudaFreeHost(s->done_h);
  if (s->kernel_end) cudaEventDestroy(s->kernel_end);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // namespace

extern "C" void dj_serve_opts_init(dj_serve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
}

extern "C" int dj_serve_create(const dj_serve_opts* opts, dj_server** out) {
  clear_error();
  if (!out) return set_error(DJ_EINVAL, "out is NULL");
  *out = nullptr;
  dj_serve_opts o;
  dj_serve_opts_init(&o);
  if (opts) o = *opts;
  if (o.max_slots < 0 || o.max_slots > 4096) return set_error(DJ_EINVAL, "max_slots must be in [0, 4096]");
  if (o.cluster_size < 0 || o.cluster_size > 16) return set_error(DJ_EINVAL, "cluster_size must be in [0, 16]");
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  if (o.max_slots == 0) o.max_slots = 512;
  if (o.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    o.hbm_budget = static_cast<uint64_t>(0.9 * static_cast<double>(fr));
  }
  auto* s = new dj_server();
  s->device = ctx->device;
  s->opts = o;
  uint32_t cap = 1;
  while (cap < 2u * static_cast<uint32_t>(o.max_slots)) cap *= 2;
  s->cap = cap;
  s->slots.resize(cap);
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->kernel_end, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaHostAlloc(&s->ring_h, cap * sizeof(SolveDesc), cudaHostAllocMapped)) != cudaSuccess ||
      (e = cudaHostAlloc(&s->ctl_h, 256, cudaHostAllocMapped)) != cudaSuccess ||
      (e = cudaHostAlloc(&s->done_h, cap * sizeof(uint32_t), cudaHostAllocMapped)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&s->ring_d, s->ring_h, 0)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&s->ctl_d, s->ctl_h, 0)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&s->done_d, s->done_h, 0)) != cudaSuccess ||
      (e = cudaMalloc(&s->head_d, 256)) != cudaSuccess || (e = cudaMemset(s->head_d, 0, 256)) != cudaSuccess) {
    int rc = cuda_error(e, "creating the server");
    free_server(s);
    return rc;
  }
  std::memset(s->ctl_h, 0, 256);
  std::memset(s->done_h, 0, cap * sizeof(uint32_t));
  s->fixed_bytes = 256;
  *out = s;
  return DJ_OK;
}

extern "C" int dj_serve_add_graph(dj_server* s, const dj_graph* g, int32_t* graph_id) {
  clear_error();
  if (!s || !g || !graph_id) return set_error(DJ_EINVAL, "NULL argument");
  if (g->device != s->device) return set_error(DJ_EINVAL, "graph on another device");
  if (int rc = require_dense(g)) return rc;
  if (s->graph_bytes + s->pool_bytes + s->fixed_bytes + g->bytes > s->opts.hbm_budget)
    return set_error(DJ_ENOMEM, "graph does not fit the serving HBM budget");
  s->graphs.push_back(g);
  s->graph_bytes += g->bytes;
  *graph_id = static_cast<int32_t>(s->graphs.size() - 1);
  return DJ_OK;
}

extern "C" int dj_serve_submit(dj_server* s, int32_t graph_id, int32_t source, int32_t* dist, int32_t* pred,
                               uint64_t* ticket) {
  clear_error();
  if (!s) return set_error(DJ_EINVAL, "NULL server");
  return submit(s, graph_id, source, dist, pred, now_s(), ticket);
}

extern "C" int dj_serve_poll(dj_server* s, uint64_t ticket, int* done) {
  clear_error();
  if (!s || !done) return set_error(DJ_EINVAL, "NULL argument");
  if (ticket >= s->next_ticket) return set_error(DJ_EINVAL, "unknown ticket");
  reap(s);
  if (int rc = ensure_kernel(s)) return rc;
  const Slot& sl = s->slots[ticket & (s->cap - 1)];
  *done = (sl.ticket != ticket || sl.done) ? 1 : 0;
  return DJ_OK;
}

extern "C" int dj_serve_wait(dj_server* s, uint64_t ticket, int64_t timeout_ns) {
  clear_error();
  const double t_end = now_s() + static_cast<double>(timeout_ns) * 1e-9;
  for (;;) {
    int done = 0;
    if (int rc = dj_serve_poll(s, ticket, &done)) return rc;
    if (done) return DJ_OK;
    if (now_s() > t_end) return set_error(DJ_ETIMEOUT, "request not completed within the timeout");
  }
}

extern "C" int dj_serve_result(dj_server* s, uint64_t ticket, int32_t* dist_host, int32_t* pred_host) {
  clear_error();
  if (!s || !dist_host || !pred_host) return set_error(DJ_EINVAL, "NULL argument");
  int done = 0;
  if (int rc = dj_serve_poll(s, ticket, &done)) return rc;
  if (!done) return set_error(DJ_EBUSY, "request still in flight");
  for (auto& b : s->pool) {
    if (b.owner == static_cast<int64_t>(ticket) && !b.busy) {
      const Slot& sl = s->slots[ticket & (s->cap - 1)];
      (void)sl;
      // the descriptor ring still holds the request's n when the slot was not reused
      const SolveDesc& d = s->ring_h[ticket & (s->cap - 1)];
      if (d.dist != b.ptr) break;
      const size_t bytes = static_cast<size_t>(d.n) * sizeof(int32_t);
      cudaError_t e = cudaMemcpy(dist_host, b.ptr, bytes, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(pred_host, b.ptr + d.n, bytes, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_error(e, "copying a pooled result");
      return DJ_OK;
    }
  }
  return set_error(DJ_EINVAL, "no pooled result for this ticket (caller-owned outputs, or the buffer was reused)");
}

static double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * static_cast<double>(v.size() - 1);
  const size_t i = static_cast<size_t>(std::floor(pos));
  const size_t j = std::min(i + 1, v.size() - 1);
  return v[i] + (v[j] - v[i]) * (pos - static_cast<double>(i));
}

extern "C" int dj_serve_stats_get(dj_server* s, dj_serve_stats* st) {
  clear_error();
  if (!s || !st) return set_error(DJ_EINVAL, "NULL argument");
  reap(s);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->rejected = s->rejected;
  st->p50_us = percentile(s->lat_us, 0.50);
  st->p90_us = percentile(s->lat_us, 0.90);
  st->p99_us = percentile(s->lat_us, 0.99);
  st->max_us = s->lat_us.empty() ? 0.0 : *std::max_element(s->lat_us.begin(), s->lat_us.end());
  double sum = 0;
  for (double x : s->lat_us) sum += x;
  st->mean_us = s->lat_us.empty() ? 0.0 : sum / static_cast<double>(s->lat_us.size());
  const double span = s->last_done - s->first_ref;
  st->solves_per_s = (s->completed > 0 && span > 0) ? static_cast<double>(s->completed) / span : 0.0;
  st->resident_bytes = s->graph_bytes + s->pool_bytes + s->fixed_bytes;
  st->kernel_launches = s->launches;
  return DJ_OK;
}

extern "C" int dj_serve_destroy(dj_server* s) {
  clear_error();
  if (!s) return DJ_OK;
  // finish in-flight work (bounded), then stop the kernel and release everything
  const double t_end = now_s() + 60.0;
  while (s->inflight > 0 && now_s() < t_end) {
    reap(s);
    if (ensure_kernel(s) != DJ_OK) break;
  }
  int rc = stop_kernel(s);
  free_server(s);
  return rc;
}

extern "C" int dj_serve(const dj_graph* const* graphs, int32_t num_graphs, int64_t R, const int32_t* req_graph,
                        const int32_t* req_source, const double* arrival_s, int32_t* const* out_dist,
                        int32_t* const* out_pred, const dj_serve_opts* opts, dj_serve_stats* st) {
  clear_error();
  if (!graphs || num_graphs < 1 || R < 0 || (R > 0 && (!req_graph || !req_source || !arrival_s)) || !st)
    return set_error(DJ_EINVAL, "NULL or empty argument");
  dj_server* s = nullptr;
  if (int rc = dj_serve_create(opts, &s)) return rc;
  for (int32_t i = 0; i < num_graphs; ++i) {
    int32_t gid = 0;
    if (int rc = dj_serve_add_graph(s, graphs[i], &gid)) {
      dj_serve_destroy(s);
      return rc;
    }
  }
  if (int rc = ensure_plan(s)) {
    dj_serve_destroy(s);
    return rc;
  }
  const double t0 = now_s();
  int64_t r = 0, deferred = 0, last_deferred = -1;
  uint64_t last_completed = 0;
  double t_progress = t0;
  int rc = DJ_OK;
  while (r < R || s->inflight > 0) {
    const double t = now_s();
    while (r < R && t >= t0 + arrival_s[r]) {
      int32_t* d = out_dist ? out_dist[r] : nullptr;
      int32_t* p = out_pred ? out_pred[r] : nullptr;
      const int x = submit(s, req_graph[r], req_source[r], d, p, t0 + arrival_s[r], nullptr);
      if (x == DJ_EBUSY) {  // admitted later, when a slot and memory free up
        if (last_deferred != r) {
          ++deferred;
          last_deferred = r;
        }
        break;
      }
      if (x != DJ_OK) {
        rc = x;
        r = R;
        break;
      }
      ++r;
    }
    reap(s);
    if (int e = ensure_kernel(s)) {
      rc = e;
      break;
    }
    if (s->completed != last_completed) {
      last_completed = s->completed;
      t_progress = t;
    } else if (s->inflight > 0 && t - t_progress > 30.0) {
      rc = set_error(DJ_ETIMEOUT, "no request completed for 30 s");
      break;
    }
  }
  if (rc == DJ_OK) {
    dj_serve_stats_get(s, st);
    st->rejected = static_cast<uint64_t>(deferred);  // requests admitted later than they arrived
  }
  const std::string err = dj_last_error();
  const int drc = dj_serve_destroy(s);
  if (rc != DJ_OK) return set_error(rc, err);
  if (drc != DJ_OK) return drc;
  // rejected counts admission retries, not lost requests
  return DJ_OK;
}
