// C ABI glue: error reporting, the per-device context, single solves and
// batched solves.  Every entry point validates its arguments on the host and
// only then enqueues device work.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
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

static std::mutex g_fn_mu;

static FnSetup* fn_setup(DevCtx* ctx, const void* fn) {  // g_fn_mu held
  for (auto& f : ctx->fns)
    if (f.fn == fn) return &f;
  ctx->fns.push_back(FnSetup{});
  ctx->fns.back().fn = fn;
  return &ctx->fns.back();
}

int raise_smem_limit(const void* fn, int max_smem_optin) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, fn);
  if (e != cudaSuccess) return cuda_error(e, "cudaFuncGetAttributes");
  const int dyn = max_smem_optin - static_cast<int>(a.sharedSizeBytes);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(dynamic shared memory)");
  return dyn;
}

int prepare_function(DevCtx* ctx, const void* fn, size_t smem, bool nonportable) {
  std::lock_guard<std::mutex> lk(g_fn_mu);
  FnSetup* f = fn_setup(ctx, fn);
  if (f->smem == 0) {
    const int dyn = raise_smem_limit(fn, ctx->max_smem_optin);
    if (dyn < 0) return dyn;  // an error status
    f->smem = static_cast<size_t>(dyn);
  }
  if (smem > f->smem) return set_error(DJ_EUNSUPPORTED, "slice state exceeds shared memory");
  if (nonportable && !f->nonportable) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return cuda_error(e, "non-portable cluster size");
    f->nonportable = true;
  }
  return DJ_OK;
}

int function_occupancy(DevCtx* ctx, const void* fn, int threads, size_t smem, int* occ) {
  std::lock_guard<std::mutex> lk(g_fn_mu);
  FnSetup* f = fn_setup(ctx, fn);
  if (f->occ < 0 || f->occ_smem != smem || f->occ_threads != threads) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    f->occ = n;
    f->occ_smem = smem;
    f->occ_threads = threads;
  }
  *occ = f->occ;
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
  if (o.settle < DJ_SETTLE_AUTO || o.settle > DJ_SETTLE_DYN) return set_error(DJ_EINVAL, "unknown settle bounds");
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
  // lockstep engine (every solve on one graph)
  dj_graph* graph = nullptr;   // the shared graph, or nullptr
  bool lockstep = false;       // launches run the lockstep engine
  bool ls_ok = false;          // the lockstep engine can run this batch
  LockstepPlan ls;
  LsSource* ls_src = nullptr;  // device: the k sources in the caller's order
  uint8_t* ls_ws = nullptr;    // device workspace (first 256 bytes zero between launches)
  int ls_use_in = 1;
  bool ls_possible = false;    // one graph, phase mode: the autotuner may try the lockstep engine
  std::vector<LsSource> ls_host;
};

// ---- autotuned choices per (n bucket, density bucket, SM count), process-wide, optionally
// kept in a JSON file (DJ_TUNE_FILE, or dj_tune_load / dj_tune_save)
struct TuneKey {
  int nb, db, sms;
  bool operator==(const TuneKey& o) const { return nb == o.nb && db == o.db && sms == o.sms; }
};
struct TuneVal {
  int engine;  // DJ_BATCH_ENGINE_CLUSTER or DJ_BATCH_ENGINE_LOCKSTEP
  int cluster_size, threads;
  double ms;
};
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, TuneVal>> g_tune;
static bool g_tune_env_loaded = false;

static int n_bucket(int32_t n) {
  int b = 0;
  while ((1 << (b + 1)) <= n && b < 30) ++b;
  return b;
}
// floor(log2(n^2 / finite entries)), at most 20: 0 for complete graphs, 1 at density 1/2, 4 at 1/20
static int density_bucket(int32_t n, uint64_t entries) {
  const double ratio = static_cast<double>(n) * static_cast<double>(n) / static_cast<double>(std::max<uint64_t>(entries, 1));
  int b = 0;
  while (b < 20 && std::ldexp(1.0, b + 1) <= ratio) ++b;
  return b;
}
static TuneKey tune_key(int32_t n, uint64_t entries, int sms) { return TuneKey{n_bucket(n), density_bucket(n, entries), sms}; }

static int tune_load_locked(const char* path);
static void tune_env_load_locked() {
  if (g_tune_env_loaded) return;
  g_tune_env_loaded = true;
  const char* f = std::getenv("DJ_TUNE_FILE");
  if (f && *f) {
    tune_load_locked(f);
    clear_error();
  }
}
static bool tune_find(const TuneKey& key, TuneVal* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_env_load_locked();
  for (auto& kv : g_tune)
    if (kv.first == key) {
      *out = kv.second;
      return true;
    }
  return false;
}
static void tune_put_locked(const TuneKey& key, const TuneVal& v) {
  for (auto& kv : g_tune)
    if (kv.first == key) {
      kv.second = v;
      return;
    }
  g_tune.push_back({key, v});
}

// The table as JSON: {"version": 1, "entries": [{"n_bucket": .., "density_bucket": .., "sms": ..,
// "engine": "cluster"|"lockstep", "cluster_size": .., "threads": .., "ms": ..}, ...]}
static int tune_save_locked(const char* path) {
  std::string out = "{\"version\": 1, \"entries\": [";
  for (size_t i = 0; i < g_tune.size(); ++i) {
    const auto& k = g_tune[i].first;
    const auto& v = g_tune[i].second;
    char buf[256];
    std::snprintf(buf, sizeof(buf),
                  "%s\n  {\"n_bucket\": %d, \"density_bucket\": %d, \"sms\": %d, \"engine\": \"%s\", "
                  "\"cluster_size\": %d, \"threads\": %d, \"ms\": %.6g}",
                  i ? "," : "", k.nb, k.db, k.sms, v.engine == DJ_BATCH_ENGINE_LOCKSTEP ? "lockstep" : "cluster",
                  v.cluster_size, v.threads, v.ms);
    out += buf;
  }
  out += "\n]}\n";
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return set_error(DJ_EINVAL, std::string("cannot write ") + tmp);
  const bool ok = std::fwrite(out.data(), 1, out.size(), f) == out.size();
  std::fclose(f);
  if (!ok || std::rename(tmp.c_str(), path) != 0) return set_error(DJ_EINVAL, std::string("cannot write ") + path);
  return DJ_OK;
}

// Minimal reader for the format above: every {...} object inside "entries" with integer fields
// and an "engine" string.  Entries with missing fields are skipped; later entries of a key win.
static bool json_int(const std::string& obj, const char* name, long* out) {
  const std::string key = std::string("\"") + name + "\"";
  size_t p = obj.find(key);
  if (p == std::string::npos) return false;
  p = obj.find(':', p + key.size());
  if (p == std::string::npos) return false;
  char* end = nullptr;
  const long v = std::strtol(obj.c_str() + p + 1, &end, 10);
  if (end == obj.c_str() + p + 1) return false;
  *out = v;
  return true;
}
static bool json_num(const std::string& obj, const char* name, double* out) {
  const std::string key = std::string("\"") + name + "\"";
  size_t p = obj.find(key);
  if (p == std::string::npos) return false;
  p = obj.find(':', p + key.size());
  if (p == std::string::npos) return false;
  char* end = nullptr;
  const double v = std::strtod(obj.c_str() + p + 1, &end);
  if (end == obj.c_str() + p + 1) return false;
  *out = v;
  return true;
}
static int tune_load_locked(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return set_error(DJ_EINVAL, std::string("cannot read ") + path);
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  std::fclose(f);
  size_t p = text.find("\"entries\"");
  if (p == std::string::npos) return set_error(DJ_EINVAL, std::string("no \"entries\" in ") + path);
  p = text.find('[', p);
  int loaded = 0;
  while (p != std::string::npos) {
    const size_t a = text.find('{', p);
    const size_t close = text.find(']', p);
    if (a == std::string::npos || (close != std::string::npos && close < a)) break;
    const size_t z = text.find('}', a);
    if (z == std::string::npos) break;
    const std::string obj = text.substr(a, z - a + 1);
    p = z + 1;
    long nb, db, sms, cs = 0, th = 0;
    double ms = 0.0;
    if (!json_int(obj, "n_bucket", &nb) || !json_int(obj, "density_bucket", &db) || !json_int(obj, "sms", &sms))
      continue;
    json_int(obj, "cluster_size", &cs);
    json_int(obj, "threads", &th);
    json_num(obj, "ms", &ms);
    const int engine = obj.find("\"lockstep\"") != std::string::npos ? DJ_BATCH_ENGINE_LOCKSTEP : DJ_BATCH_ENGINE_CLUSTER;
    if (engine == DJ_BATCH_ENGINE_CLUSTER && (cs < 1 || cs > 16)) continue;
    tune_put_locked(TuneKey{static_cast<int>(nb), static_cast<int>(db), static_cast<int>(sms)},
                    TuneVal{engine, static_cast<int>(cs), static_cast<int>(th), ms});
    ++loaded;
  }
  return DJ_OK;
}

extern "C" int dj_tune_load(const char* path) {
  clear_error();
  if (!path) return set_error(DJ_EINVAL, "NULL path");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_env_loaded = true;
  return tune_load_locked(path);
}

extern "C" int dj_tune_save(const char* path) {
  clear_error();
  if (!path) return set_error(DJ_EINVAL, "NULL path");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return tune_save_locked(path);
}

extern "C" int dj_tune_lookup(int32_t n, uint64_t entries, int32_t num_sms, int32_t* engine, int32_t* cluster_size) {
  clear_error();
  if (n < 1 || num_sms < 1) return set_error(DJ_EINVAL, "need n >= 1 and num_sms >= 1");
  TuneVal v;
  if (!tune_find(tune_key(n, entries, num_sms), &v)) return set_error(DJ_EINVAL, "no tuned entry for this key");
  if (engine) *engine = v.engine;
  if (cluster_size) *cluster_size = v.cluster_size;
  return DJ_OK;
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

// The one graph every solve of the batch uses, or nullptr.
static dj_graph* shared_graph(const dj_graph* const* graphs, int32_t k) {
  if (k < 1) return nullptr;
  for (int32_t i = 1; i < k; ++i)
    if (graphs[i] != graphs[0]) return nullptr;
  return const_cast<dj_graph*>(graphs[0]);
}

// Auto never picks the lockstep engine without a tuned entry that does: measured on GB300 it is
// slower than the cluster engine on every shape tried (256 sources of n = 8192, p = 0.05:
// 18.7 against 10.1 ms; n = 4096, p = 0.5: 7.9 against 2.4 ms), being bound by instruction
// issue where the cluster engine is bound by streaming.

static void free_batch(dj_batch* b) {
  if (!b) return;
  cudaFree(b->descs);
  cudaFree(b->ls_src);
  cudaFree(b->ls_ws);
  delete b;
}

// Sizes, source table, workspace and tiled matrix of the lockstep engine for batch b (once).
static int prepare_lockstep(dj_batch* b) {
  if (b->ls_ok) return DJ_OK;
  if (int rc = plan_lockstep(b->graph, b->k, &b->ls)) return rc;
  const std::vector<LsSource>& hs = b->ls_host;
  cudaError_t e = cudaMalloc(&b->ls_src, hs.size() * sizeof(LsSource));
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(lockstep sources)");
  e = cudaMemcpy(b->ls_src, hs.data(), hs.size() * sizeof(LsSource), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "lockstep source upload");
  e = cudaMalloc(&b->ls_ws, b->ls.ws_bytes);
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(lockstep workspace)");
  e = cudaMemset(b->ls_ws, 0, 256);
  if (e != cudaSuccess) return cuda_error(e, "cudaMemset(lockstep workspace)");
  const int32_t* tiled = nullptr;
  if (int rc = lockstep_tiles(b->graph, b->ls, nullptr, &tiled)) return rc;
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "building the column-tiled matrix");
  b->ls_ok = true;
  return DJ_OK;
}

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
  if (o.engine < DJ_BATCH_ENGINE_AUTO || o.engine > DJ_BATCH_ENGINE_LOCKSTEP) return set_error(DJ_EINVAL, "unknown engine");
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
    free_batch(b);
    return cuda_error(e, "cudaMemset(batch queue)");
  }
  if (k > 0) {
    e = cudaMemcpy(b->descs, h.data(), static_cast<size_t>(k) * sizeof(SolveDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_batch(b);
      return cuda_error(e, "descriptor upload");
    }
  }
  b->graph = shared_graph(graphs, k);
  TuneVal tv{};
  const bool have_tune = b->graph && tune_find(tune_key(b->graph->n, b->graph->entries, ctx->num_sms), &tv);
  b->cl.cluster_size = o.cluster_size > 0 ? o.cluster_size : 0;
  b->cl.threads = 256;
  b->cl.clusters = o.clusters;
  b->cl.copies = o.copies;
  if (b->cl.cluster_size == 0 && have_tune && tv.engine == DJ_BATCH_ENGINE_CLUSTER) b->cl.cluster_size = tv.cluster_size;
  if (b->cl.cluster_size == 0) b->cl.cluster_size = heuristic_cluster_size(max_pitch);
  if (int rc = plan_cluster(b->max_pitch, b->cl, b->k, &b->plan)) {
    free_batch(b);
    return rc;
  }
  // the lockstep engine: forced, or auto for enough solves of one graph (a tuned entry decides)
  const bool want_ls = o.mode != DJ_MODE_PLAIN && b->graph &&
                       (o.engine == DJ_BATCH_ENGINE_LOCKSTEP ||
                        (o.engine == DJ_BATCH_ENGINE_AUTO && o.cluster_size == 0 && have_tune &&
                         tv.engine == DJ_BATCH_ENGINE_LOCKSTEP));
  b->ls_use_in = o.settle == DJ_SETTLE_OUT ? 0 : 1;
  b->ls_possible = b->graph && o.mode != DJ_MODE_PLAIN && o.engine != DJ_BATCH_ENGINE_CLUSTER && k > 0;
  if (o.engine == DJ_BATCH_ENGINE_LOCKSTEP && !b->ls_possible) {
    free_batch(b);
    return set_error(DJ_EUNSUPPORTED, "the lockstep engine needs every solve on one graph, in phase mode");
  }
  if (b->ls_possible) {
    b->ls_host.resize(static_cast<size_t>(k));
    for (int32_t i = 0; i < k; ++i) b->ls_host[i] = LsSource{dist[i], pred[i], sources[i], 0};
  }
  if (want_ls) {
    const int rc = prepare_lockstep(b);
    if (rc != DJ_OK && o.engine == DJ_BATCH_ENGINE_LOCKSTEP) {
      free_batch(b);
      return rc;
    }
    if (rc != DJ_OK) clear_error();
  }
  b->lockstep = want_ls && b->ls_ok;
  *out = b;
  return DJ_OK;
}

static int launch_batch(dj_batch* b, cudaStream_t st) {
  if (b->k == 0) return DJ_OK;
  if (b->lockstep) {
    DevCtx* ctx = nullptr;
    if (int rc = get_ctx(&ctx)) return rc;
    const int32_t* tiled = nullptr;
    if (int rc = lockstep_tiles(b->graph, b->ls, st, &tiled)) return rc;
    return run_lockstep(b->graph, b->ls, tiled, b->ls_src, b->ls_ws, ctx->words, 0, b->ls_use_in, st);
  }
  return run_cluster(b->plan, b->descs, b->k, b->queue, st, false);
}

extern "C" int dj_batch_launch(dj_batch* b, uint64_t stream) {
  clear_error();
  if (!b) return set_error(DJ_EINVAL, "NULL batch");
  return launch_batch(b, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int dj_batch_free(dj_batch* b) {
  clear_error();
  free_batch(b);
  return DJ_OK;
}

extern "C" int dj_batch_get_engine(const dj_batch* b, int32_t* engine) {
  clear_error();
  if (!b || !engine) return set_error(DJ_EINVAL, "NULL argument");
  *engine = b->lockstep ? DJ_BATCH_ENGINE_LOCKSTEP : DJ_BATCH_ENGINE_CLUSTER;
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
  auto time_it = [&](float* out_ms) {  // mean of two launches after a warm-up
    float sum = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, st);
      if (launch_batch(b, st) != DJ_OK) return false;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return false;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) sum += ms;
    }
    *out_ms = sum / 2.f;
    return true;
  };
  float best = 1e30f;
  int best_engine = DJ_BATCH_ENGINE_CLUSTER;
  ClusterLaunch best_cl = b->cl;
  const ClusterLaunch saved = b->cl;
  b->lockstep = false;
  for (int c : {2, 4, 8, 16}) {
    ClusterLaunch cl = saved;
    cl.cluster_size = c;
    if (!cluster_config_ok(b->max_pitch, cl)) continue;
    b->cl = cl;
    if (plan_cluster(b->max_pitch, b->cl, b->k, &b->plan) != DJ_OK) {
      clear_error();
      continue;
    }
    float ms = 0.f;
    if (!time_it(&ms)) {
      clear_error();
      cudaGetLastError();
      continue;
    }
    if (ms < best) {
      best = ms;
      best_cl = cl;
    }
  }
  if (b->ls_possible && prepare_lockstep(b) != DJ_OK) clear_error();
  if (b->ls_ok) {  // the lockstep engine as one more candidate
    b->lockstep = true;
    float ms = 0.f;
    if (time_it(&ms) && ms < best) {
      best = ms;
      best_engine = DJ_BATCH_ENGINE_LOCKSTEP;
    } else {
      clear_error();
      cudaGetLastError();
    }
    b->lockstep = false;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cl = best_cl;
  if (int rc = plan_cluster(b->max_pitch, b->cl, b->k, &b->plan)) return rc;
  b->lockstep = best_engine == DJ_BATCH_ENGINE_LOCKSTEP;
  b->tuned = true;
  if (b->graph) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_env_load_locked();
    tune_put_locked(tune_key(b->graph->n, b->graph->entries, ctx->num_sms),
                    TuneVal{best_engine, best_engine == DJ_BATCH_ENGINE_LOCKSTEP ? 0 : best_cl.cluster_size,
                            best_engine == DJ_BATCH_ENGINE_LOCKSTEP ? 512 : best_cl.threads, best});
    const char* f = std::getenv("DJ_TUNE_FILE");
    if (f && *f) tune_save_locked(f);
  }
  if (cluster_size) *cluster_size = best_engine == DJ_BATCH_ENGINE_LOCKSTEP ? 0 : best_cl.cluster_size;
  if (threads) *threads = best_engine == DJ_BATCH_ENGINE_LOCKSTEP ? 512 : best_cl.threads;
  if (best_ms) *best_ms = best;
  if (best >= 1e29f) return set_error(DJ_EUNSUPPORTED, "no batch configuration could run");
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
  dj_graph* g1 = shared_graph(graphs, k);
  TuneVal tv{};
  const bool have_tune = g1 && tune_find(tune_key(g1->n, g1->entries, ctx->num_sms), &tv);
  // solves of one graph whose tuned entry chose the lockstep engine
  LockstepPlan ls;
  if (g1 && have_tune && tv.engine == DJ_BATCH_ENGINE_LOCKSTEP && plan_lockstep(g1, k, &ls) == DJ_OK) {
    std::vector<LsSource> hs(static_cast<size_t>(k));
    for (int32_t i = 0; i < k; ++i) hs[i] = LsSource{dist[i], pred[i], sources[i], 0};
    const size_t tbytes = (hs.size() * sizeof(LsSource) + 255) & ~size_t(255);
    uint8_t* ws = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, tbytes + ls.ws_bytes, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(lockstep batch)");
    cudaMemcpyAsync(ws, hs.data(), hs.size() * sizeof(LsSource), cudaMemcpyHostToDevice, st);  // pageable: staged
    cudaMemsetAsync(ws + tbytes, 0, 256, st);
    const int32_t* tiled = nullptr;
    int rc = lockstep_tiles(g1, ls, st, &tiled);
    if (rc == DJ_OK)
      rc = run_lockstep(g1, ls, tiled, reinterpret_cast<LsSource*>(ws), ws + tbytes, ctx->words, 0, 1, st);
    cudaFreeAsync(ws, st);
    return rc;
  }
  clear_error();
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
  if (have_tune && tv.engine == DJ_BATCH_ENGINE_CLUSTER) cl.cluster_size = tv.cluster_size;
  int rc = launch_cluster(reinterpret_cast<SolveDesc*>(ws), k, max_n, max_pitch,
                          reinterpret_cast<uint32_t*>(ws + tbytes), cl, st);
  cudaFreeAsync(ws, st);
  return rc;
}
