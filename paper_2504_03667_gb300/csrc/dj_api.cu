// C ABI glue: error reporting, the per-device context, single solves and
// batched solves.  Every entry point validates its arguments on the host and
// only then enqueues device work.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "dj_common.cuh"
#include "dj_internal.h"

namespace dj {

static thread_local std::string g_last_error;

int set_error(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}
int cuda_error(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return DJ_ECUDA;
}
void clear_error() { g_last_error.clear(); }

static std::mutex g_ctx_mu;
static DevCtx g_ctx[64];

int get_ctx(DevCtx** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice (is a CUDA GPU present?)");
  if (dev < 0 || dev >= 64) return set_error(DJ_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  DevCtx& c = g_ctx[dev];
  if (c.device != dev) {
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceProperties");
    if (prop.major < 10) return set_error(DJ_EUNSUPPORTED, "this library targets sm_103a (Blackwell) devices");
    c.num_sms = prop.multiProcessorCount;
    c.max_smem_optin = static_cast<int>(prop.sharedMemPerBlockOptin);
    c.coop = prop.cooperativeLaunch;
    int cl = 0;
    cudaDeviceGetAttribute(&cl, cudaDevAttrClusterLaunch, dev);
    c.cluster_launch = cl;
    e = cudaMalloc(&c.words, 64 * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(device words)");
    e = cudaMemset(c.words, 0, 64 * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_error(e, "cudaMemset(device words)");
    c.device = dev;
  }
  *out = &c;
  return DJ_OK;
}

static std::mutex g_ws_mu;
constexpr size_t kMaxStreamWorkspaces = 64;

int stream_workspace(DevCtx* ctx, cudaStream_t st, size_t bytes, size_t zero_bytes, uint8_t** out) {
  *out = nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamIsCapturing");
  // a captured graph may be replayed on any stream, alongside other solves: it gets its own
  // stream-ordered allocation instead of this stream's buffer
  if (cap != cudaStreamCaptureStatusNone) return DJ_OK;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  StreamWs* w = nullptr;
  for (auto& x : ctx->ws)
    if (x.stream == st) w = &x;
  if (w && w->bytes >= bytes) {
    *out = w->ptr;
    return DJ_OK;
  }
  if (!w) {
    if (ctx->ws.size() >= kMaxStreamWorkspaces) return DJ_OK;
    ctx->ws.push_back(StreamWs{st, nullptr, 0});
    w = &ctx->ws.back();
  } else {
    e = cudaStreamSynchronize(st);  // earlier solves on st may still use the old buffer
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize(workspace growth)");
    cudaFree(w->ptr);
    w->ptr = nullptr;
    w->bytes = 0;
  }
  const size_t want = std::max(bytes, size_t(1) << 20);
  e = cudaMalloc(&w->ptr, want);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(stream workspace)");
  e = cudaMemsetAsync(w->ptr, 0, std::min(zero_bytes, want), st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(stream workspace)");
  w->bytes = want;
  *out = w->ptr;
  return DJ_OK;
}

}  // namespace dj

using namespace dj;

extern "C" const char* dj_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* dj_status_string(int status) {
  switch (status) {
    case DJ_OK: return "ok";
    case DJ_EINVAL: return "invalid argument";
    case DJ_ENOMEM: return "out of memory";
    case DJ_EOVERFLOW: return "path lengths could overflow int32";
    case DJ_ECUDA: return "CUDA error";
    case DJ_ETIMEOUT: return "in-kernel wait timed out";
    case DJ_EBUSY: return "busy";
    case DJ_EUNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

extern "C" int dj_version(void) { return 10000; }

extern "C" void dj_solve_opts_init(dj_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->debug_skip_cta = -1;
}

extern "C" void dj_batch_opts_init(dj_batch_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
}

// ------------------------------------------------------------------ single solves

// Size below which one cluster beats the whole-GPU grid engine (fewer, cheaper barriers), and
// the lower one for graphs with at least n^2/4 finite entries, whose few phases each move much
// of the matrix (GB300, single solves, w 1..1000: p = 0.5 grid 134 / cluster 214 us at n = 3072,
// 148 / 138 at n = 2048; p = 0.05 grid 459 / cluster 433 at n = 3072, 431 / 463 at n = 4096).
static constexpr int32_t kGridMinN = 4096;
static constexpr int32_t kGridMinNDense = 2560;

static bool auto_grid(const dj_graph* g) {
  const uint64_t n = static_cast<uint64_t>(g->n);
  return g->n >= kGridMinN || (g->n >= kGridMinNDense && g->entries * 4 >= n * n);
}

static int default_cluster_size(int32_t n) {
  (void)n;
  return 8;
}

static int solve_cluster_single(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred,
                                const dj_solve_opts& o, cudaStream_t st) {
  ClusterLaunch cl;
  cl.cluster_size = o.cluster_size > 0 ? o.cluster_size : default_cluster_size(g->n);
  cl.clusters = 1;
  SolveDesc d = make_desc(g, source, dist, pred, o.mode == DJ_MODE_PLAIN ? 1 : 0);
  if (o.settle == DJ_SETTLE_OUT) d.use_in = 0;
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  // one cluster, the descriptor in the kernel's parameters: a single launch, no device memory
  ClusterPlan plan;
  if (int rc = plan_cluster(g->pitch, cl, 1, &plan, kJobsSingle)) return rc;
  // right after an upload the solve waits for the kernels before it before reading the graph
  const bool early = g->upload_pending == 0;
  const_cast<dj_graph*>(g)->upload_pending = 0;
  return run_cluster_single(plan, d, ctx->words + 1, o.trace, o.trace ? o.trace_cap : 0, early, st);
}

extern "C" int dj_sssp_ex(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, const dj_solve_opts* opts,
                          uint64_t stream) {
  clear_error();
  if (!g || !dist || !pred) return set_error(DJ_EINVAL, "NULL argument");
  if (source < 0 || source >= g->n) return set_error(DJ_EINVAL, "source outside [0, n)");
  dj_solve_opts o;
  dj_solve_opts_init(&o);
  if (opts) o = *opts;
  if (o.mode < DJ_MODE_AUTO || o.mode > DJ_MODE_PLAIN) return set_error(DJ_EINVAL, "unknown mode");
  if (o.settle < DJ_SETTLE_AUTO || o.settle > DJ_SETTLE_OUT_IN) return set_error(DJ_EINVAL, "unknown settle bounds");
  if (o.live < -1) return set_error(DJ_EINVAL, "live must be -1, 0 or a group count");
  if (o.rowsplit < -1) return set_error(DJ_EINVAL, "rowsplit must be -1, 0 or a candidate count");
  if (o.rowpush < -1) return set_error(DJ_EINVAL, "rowpush must be -1, 0 or a candidate count");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (g->format == DJ_FORMAT_CSR) return launch_csr(g, source, dist, pred, o, st);
  int engine = o.engine;
  if (engine == DJ_ENGINE_AUTO) engine = auto_grid(g) ? DJ_ENGINE_GRID : DJ_ENGINE_CLUSTER;
  if (engine == DJ_ENGINE_GRID) return launch_grid(g, source, dist, pred, o, st);
  if (engine == DJ_ENGINE_CLUSTER) return solve_cluster_single(g, source, dist, pred, o, st);
  return set_error(DJ_EINVAL, "unknown engine");
}

extern "C" int dj_sssp(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, uint64_t stream) {
  return dj_sssp_ex(g, source, dist, pred, nullptr, stream);
}

extern "C" int dj_sync(uint64_t stream) {
  clear_error();
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  uint32_t bits = 0;
  e = cudaMemcpy(&bits, ctx->words, sizeof(bits), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "reading the device error word");
  if (bits) {
    cudaMemset(ctx->words, 0, sizeof(uint32_t));
    if (bits & kErrTimeout) return set_error(DJ_ETIMEOUT, "a bounded in-kernel wait ran out; the kernel returned early");
    return set_error(DJ_ECUDA, "device reported error bits " + std::to_string(bits));
  }
  return DJ_OK;
}

extern "C" int dj_last_phases(void) {
  DevCtx* ctx = nullptr;
  if (get_ctx(&ctx)) return -1;
  uint32_t v = 0;
  if (cudaMemcpy(&v, ctx->words + 1, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return v == 0xFFFFFFFFu ? -1 : static_cast<int>(v);
}

extern "C" int dj_sssp_host(const dj_graph* g, int32_t source, int32_t* dist_host, int32_t* pred_host,
                            uint64_t stream) {
  clear_error();
  if (!g || !dist_host || !pred_host) return set_error(DJ_EINVAL, "NULL argument");
  if (source < 0 || source >= g->n) return set_error(DJ_EINVAL, "source outside [0, n)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int32_t* buf = nullptr;
  const size_t bytes = static_cast<size_t>(g->n) * sizeof(int32_t);
  cudaError_t e = cudaMallocAsync(&buf, 2 * bytes, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(results)");
  int rc = dj_sssp(g, source, buf, buf + g->n, stream);
  if (rc == DJ_OK) {
    cudaMemcpyAsync(dist_host, buf, bytes, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(pred_host, buf + g->n, bytes, cudaMemcpyDeviceToHost, st);
  }
  cudaFreeAsync(buf, st);
  if (rc != DJ_OK) return rc;
  return dj_sync(stream);
}

// ------------------------------------------------------------------ batches

struct dj_batch {
  int device = 0;
  int32_t k = 0;
  int32_t max_n = 0;
  int32_t max_pitch = 0;
  SolveDesc* descs = nullptr;  // device, sorted by decreasing n
  uint32_t* queue = nullptr;   // device word
  ClusterLaunch cl;
  ClusterPlan plan;
  bool tuned = false;
};

// Autotuned choices per (n bucket, density bucket, SM count), process-wide.
struct TuneKey {
  int nb, db, sms;
  bool operator==(const TuneKey& o) const { return nb == o.nb && db == o.db && sms == o.sms; }
};
struct TuneVal {
  int cluster_size, threads;
};
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, TuneVal>> g_tune;

static int n_bucket(int32_t n) {
  int b = 0;
  while ((1 << (b + 1)) <= n && b < 30) ++b;
  return b;
}

static int heuristic_cluster_size(int32_t max_pitch) {
  // slices of about 1024 columns: long row segments copied wide, yet many solves in flight
  int c = 2;
  while (c < 16 && c * 1024 < max_pitch) c *= 2;  // a power of two
  return c;
}

static int batch_descs(const dj_graph* const* graphs, const int32_t* sources, int32_t k, int32_t* const* dist,
                       int32_t* const* pred, int plain, int device, std::vector<SolveDesc>* h, int32_t* max_n,
                       int32_t* max_pitch);

extern "C" int dj_batch_create(const dj_graph* const* graphs, const int32_t* sources, int32_t k,
                               int32_t* const* dist, int32_t* const* pred, const dj_batch_opts* opts, dj_batch** out) {
  clear_error();
  if (!out) return set_error(DJ_EINVAL, "out is NULL");
  *out = nullptr;
  if (k < 0 || (k > 0 && (!graphs || !sources || !dist || !pred))) return set_error(DJ_EINVAL, "NULL argument");
  dj_batch_opts o;
  dj_batch_opts_init(&o);
  if (opts) o = *opts;
  if (o.copies < DJ_COPIES_AUTO || o.copies > DJ_COPIES_WIDE) return set_error(DJ_EINVAL, "unknown copies");
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  std::vector<SolveDesc> h;
  int32_t max_n, max_pitch;
  if (int rc = batch_descs(graphs, sources, k, dist, pred, o.mode == DJ_MODE_PLAIN ? 1 : 0, ctx->device, &h, &max_n,
                           &max_pitch))
    return rc;
  if (o.settle == DJ_SETTLE_OUT)
    for (auto& d : h) d.use_in = 0;
  auto* b = new dj_batch();
  b->device = ctx->device;
  b->k = k;
  b->max_n = max_n;
  b->max_pitch = max_pitch;
  const size_t bytes = static_cast<size_t>(std::max(k, 1)) * sizeof(SolveDesc) + 64;
  cudaError_t e = cudaMalloc(&b->descs, bytes);
  if (e != cudaSuccess) {
    delete b;
    return set_error(DJ_ENOMEM, "cudaMalloc(batch descriptors)");
  }
  b->queue = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(b->descs) + static_cast<size_t>(std::max(k, 1)) * sizeof(SolveDesc));
  // the queue words start at zero; every launch's last cluster puts them back (no memset per launch)
  e = cudaMemset(b->queue, 0, 64);
  if (e != cudaSuccess) {
    cudaFree(b->descs);
    delete b;
    return cuda_error(e, "cudaMemset(batch queue)");
  }
  if (k > 0) {
    e = cudaMemcpy(b->descs, h.data(), static_cast<size_t>(k) * sizeof(SolveDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(b->descs);
      delete b;
      return cuda_error(e, "descriptor upload");
    }
  }
  b->cl.cluster_size = o.cluster_size > 0 ? o.cluster_size : 0;
  b->cl.threads = 256;
  b->cl.clusters = o.clusters;
  b->cl.copies = o.copies;
  if (b->cl.cluster_size == 0) {
    TuneKey key{n_bucket(max_n), 0, ctx->num_sms};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& kv : g_tune)
      if (kv.first == key) b->cl.cluster_size = kv.second.cluster_size;
  }
  if (b->cl.cluster_size == 0) b->cl.cluster_size = heuristic_cluster_size(max_pitch);
  if (int rc = plan_cluster(b->max_pitch, b->cl, b->k, &b->plan)) {
    cudaFree(b->descs);
    delete b;
    return rc;
  }
  *out = b;
  return DJ_OK;
}

extern "C" int dj_batch_launch(dj_batch* b, uint64_t stream) {
  clear_error();
  if (!b) return set_error(DJ_EINVAL, "NULL batch");
  if (b->k == 0) return DJ_OK;
  return run_cluster(b->plan, b->descs, b->k, b->queue, reinterpret_cast<cudaStream_t>(stream), false);
}

extern "C" int dj_batch_free(dj_batch* b) {
  clear_error();
  if (!b) return DJ_OK;
  cudaFree(b->descs);
  delete b;
  return DJ_OK;
}

extern "C" int dj_batch_autotune(dj_batch* b, uint64_t stream, int32_t* cluster_size, int32_t* threads,
                                 float* best_ms) {
  clear_error();
  if (!b) return set_error(DJ_EINVAL, "NULL batch");
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  ClusterLaunch best_cl = b->cl;
  const ClusterLaunch saved = b->cl;
  for (int c : {2, 4, 8, 16}) {
    ClusterLaunch cl = saved;
    cl.cluster_size = c;
    if (!cluster_config_ok(b->max_pitch, cl)) continue;
    b->cl = cl;
    if (plan_cluster(b->max_pitch, b->cl, b->k, &b->plan) != DJ_OK) {
      clear_error();
      continue;
    }
    float ms_sum = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      cudaEventRecord(e0, st);
      if (dj_batch_launch(b, stream) != DJ_OK) ok = false;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) ms_sum += ms;  // first run warms up
    }
    if (!ok) {
      clear_error();
      cudaGetLastError();
      continue;
    }
    const float ms = ms_sum / 2.f;
    if (ms < best) {
      best = ms;
      best_cl = cl;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cl = best_cl;
  if (int rc = plan_cluster(b->max_pitch, b->cl, b->k, &b->plan)) return rc;
  b->tuned = true;
  {
    TuneKey key{n_bucket(b->max_n), 0, ctx->num_sms};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    bool found = false;
    for (auto& kv : g_tune)
      if (kv.first == key) {
        kv.second = TuneVal{best_cl.cluster_size, best_cl.threads};
        found = true;
      }
    if (!found) g_tune.push_back({key, TuneVal{best_cl.cluster_size, best_cl.threads}});
  }
  if (cluster_size) *cluster_size = best_cl.cluster_size;
  if (threads) *threads = best_cl.threads;
  if (best_ms) *best_ms = best;
  if (best >= 1e29f) return set_error(DJ_EUNSUPPORTED, "no cluster configuration could run");
  return DJ_OK;
}

// Build the sorted descriptor table of a batch on the host.
static int batch_descs(const dj_graph* const* graphs, const int32_t* sources, int32_t k, int32_t* const* dist,
                       int32_t* const* pred, int plain, int device, std::vector<SolveDesc>* h, int32_t* max_n,
                       int32_t* max_pitch) {
  h->resize(static_cast<size_t>(k));
  *max_n = 1;
  *max_pitch = 32;
  for (int32_t i = 0; i < k; ++i) {
    const dj_graph* g = graphs[i];
    if (!g || !dist[i] || !pred[i]) return set_error(DJ_EINVAL, "NULL graph or result pointer at " + std::to_string(i));
    if (g->device != device) return set_error(DJ_EINVAL, "graph on another device");
    if (sources[i] < 0 || sources[i] >= g->n) return set_error(DJ_EINVAL, "source outside [0, n) at " + std::to_string(i));
    if (int rc = require_dense(g)) return rc;
    (*h)[i] = make_desc(g, sources[i], dist[i], pred[i], plain);
    *max_n = std::max(*max_n, g->n);
    *max_pitch = std::max(*max_pitch, g->pitch);
  }
  std::stable_sort(h->begin(), h->end(), [](const SolveDesc& a, const SolveDesc& b) { return a.n > b.n; });
  return DJ_OK;
}

extern "C" int dj_sssp_batch(const dj_graph* const* graphs, const int32_t* sources, int32_t k, int32_t* const* dist,
                             int32_t* const* pred, uint64_t stream) {
  clear_error();
  if (k < 0 || (k > 0 && (!graphs || !sources || !dist || !pred))) return set_error(DJ_EINVAL, "NULL argument");
  if (k == 0) return DJ_OK;
  DevCtx* ctx = nullptr;
  if (int rc = get_ctx(&ctx)) return rc;
  std::vector<SolveDesc> h;
  int32_t max_n, max_pitch;
  if (int rc = batch_descs(graphs, sources, k, dist, pred, 0, ctx->device, &h, &max_n, &max_pitch)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // stream-ordered table: allocated, filled, used and freed in stream order
  uint8_t* ws = nullptr;
  const size_t tbytes = static_cast<size_t>(k) * sizeof(SolveDesc);
  cudaError_t e = cudaMallocAsync(&ws, tbytes + 64, st);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(batch descriptors)");
  e = cudaMemcpyAsync(ws, h.data(), tbytes, cudaMemcpyHostToDevice, st);  // pageable: staged before return
  if (e != cudaSuccess) {
    cudaFreeAsync(ws, st);
    return cuda_error(e, "descriptor upload");
  }
  ClusterLaunch cl;
  cl.cluster_size = heuristic_cluster_size(max_pitch);
  {
    TuneKey key{n_bucket(max_n), 0, ctx->num_sms};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& kv : g_tune)
      if (kv.first == key) cl.cluster_size = kv.second.cluster_size;
  }
  int rc = launch_cluster(reinterpret_cast<SolveDesc*>(ws), k, max_n, max_pitch,
                          reinterpret_cast<uint32_t*>(ws + tbytes), cl, st);
  cudaFreeAsync(ws, st);
  return rc;
}
