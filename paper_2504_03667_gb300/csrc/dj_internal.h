// Host-side internals shared by the translation units of libdj.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dj.h"

struct dj_graph {
  int32_t n = 0;
  int32_t pitch = 0;  // row stride in int32 (n rounded up to 32)
  int32_t directed = 0;
  int32_t device = 0;
  int32_t wmin = DJ_INF;  // smallest finite off-diagonal weight
  int32_t wmax = 0;       // largest finite off-diagonal weight
  int32_t* W = nullptr;       // n x pitch, row-major
  int32_t* minout = nullptr;  // n row minima (then the n column minima, same allocation)
  int32_t* minin = nullptr;   // n column minima
  int32_t* tsrc = nullptr;    // n x tcap tie sources: the u != v with W[u][v] == minin[v]
  int32_t* tcnt = nullptr;    // n counts (above tcap: not listed)
  int32_t tcap = 0;
  // graphs that are not dense: the kInLists smallest finite in-weights of every column with their
  // rows, ascending by (weight, row), and a lower bound on every other in-weight (the dynamic IN
  // bound of the grid engine); nullptr otherwise
  uint2* inlist = nullptr;     // n x kInLists (weight, row); (INF, ~0) where a column has fewer
  uint32_t* inrest = nullptr;  // n: the kInLists-th weight if the column has more in-edges, else INF
  // the same for rows (out-edges, for the dynamic OUT bound): the in-lists themselves when the
  // matrix is symmetric (undirected graph)
  uint2* outlist = nullptr;
  uint32_t* outrest = nullptr;
  uint64_t bytes = 0;
  uint64_t entries = 0;       // finite off-diagonal matrix entries (directed edges)
  int32_t format = DJ_FORMAT_DENSE;  // DJ_FORMAT_CSR: no matrix, the arrays below
  int64_t nnz = 0;
  int64_t* row_ptr = nullptr;  // n + 1 edge offsets
  int32_t* col = nullptr;      // nnz targets, sorted within a row
  int32_t* wt = nullptr;       // nnz weights
  // set by dj_graph_upload: the next solve waits for the kernels before it on its stream
  // before it reads the matrix (solves otherwise read the graph while the previous kernel ends)
  int32_t upload_pending = 0;
  // lockstep batches: a column-tiled copy of the matrix for tiled_G slices (built on first use)
  int32_t* tiled = nullptr;
  int32_t tiled_G = 0;
  uint64_t tiled_bytes = 0;
};

namespace dj {

constexpr int kInLists = 4;  // in-edges listed per column for the dynamic IN bound

// Descriptor of one solve for the cluster engine (64 bytes).
struct SolveDesc {
  const int32_t* W;
  const int32_t* minout;
  int32_t* dist;
  int32_t* pred;
  int64_t pitch;
  int32_t n;
  int32_t source;
  uint32_t bits_u;
  uint32_t span;
  int32_t plain;
  int32_t use_in;  // settle by the IN bound too (every off-diagonal weight >= 1); minin = minout + n
};
static_assert(sizeof(SolveDesc) == 64, "descriptor layout");

// A workspace kept for one stream: solves enqueued on the same stream run one
// after another, so they can share it without any per-solve allocation.
struct StreamWs {
  cudaStream_t stream = nullptr;
  uint8_t* ptr = nullptr;
  size_t bytes = 0;
};

// A kernel's launch set-up on one device, done once: its dynamic shared-memory
// limit raised to all the device allows next to its static shared memory, the
// non-portable cluster size allowance, and its resident CTAs per SM at the
// shared memory and block size last queried.
struct FnSetup {
  const void* fn = nullptr;
  size_t smem = 0;  // the limit set (0: not yet)
  bool nonportable = false;
  size_t occ_smem = 0;
  int occ_threads = 0;
  int occ = -1;
};

struct DevCtx {
  int device = -1;
  int num_sms = 0;
  int max_smem_optin = 0;
  int coop = 0;
  int cluster_launch = 0;
  uint32_t* words = nullptr;  // device: [0] error bits, [1] phases of the last single solve
  std::vector<StreamWs> ws;   // per-stream workspaces of the grid engine (see stream_workspace)
  std::vector<FnSetup> fns;   // see prepare_function
};

// error reporting (thread-local message)
int set_error(int status, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);
void clear_error();

// per-device context of the current device (created on first use)
int get_ctx(DevCtx** out);

// Let `fn` launch with `smem` bytes of dynamic shared memory (and, with
// `nonportable`, clusters of more than 8 CTAs) on ctx's device.  The limit is
// set once, to the most the device allows, so the driver is asked only on a
// kernel's first launch (a small solve would otherwise pay those calls every
// time) and no later call lowers it.
int prepare_function(DevCtx* ctx, const void* fn, size_t smem, bool nonportable);
// The same limit for `fn` without a context (the allocation-free entry point).
int raise_smem_limit(const void* fn, int max_smem_optin);
// Resident CTAs per SM of `fn` at `threads` x `smem`, queried once per setting.
int function_occupancy(DevCtx* ctx, const void* fn, int threads, size_t smem, int* occ);

// A device buffer of at least `bytes` kept for stream `st` (its first
// `zero_bytes` zeroed on `st` when the buffer is created or grown), so that
// back-to-back solves on one stream allocate nothing.  Growing synchronises
// `st` once.  *out is nullptr when the stream is being captured or the table
// of streams is full: the caller then allocates per call, stream-ordered.
int stream_workspace(DevCtx* ctx, cudaStream_t st, size_t bytes, size_t zero_bytes, uint8_t** out);

inline uint32_t host_bits_for(uint32_t n) {
  uint32_t b = 1;
  while (b < 31 && (1u << b) < n) ++b;
  return b;
}
// Packing span of the tie word ((dist - m) << bits) | u: settled rows have
// dist - m < span.  One below the power of two, so no tie word is all ones
// (all ones marks "no stored tie" and "no candidate").
inline uint32_t host_span_for(uint32_t n) { return (1u << (32 - host_bits_for(n))) - 1u; }

SolveDesc make_desc(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, int plain);

// engines (dj_solve.cu)
int launch_grid(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, const dj_solve_opts& o,
                cudaStream_t st);
// compressed-row graphs (dj_csr.cu)
int launch_csr(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, const dj_solve_opts& o,
               cudaStream_t st);
// DJ_EUNSUPPORTED for a graph without a dense matrix (entry points that stream matrix rows)
int require_dense(const dj_graph* g);
struct ClusterLaunch {
  int cluster_size = 8;
  int threads = 256;
  int clusters = 0;  // 0 = as many as fit
  int copies = 0;    // DJ_COPIES_*: row-slice copy width of the rings (0 = auto)
};
// Launch the cluster engine over k descriptors already on the device.
// `queue` is a device word zeroed by this call before the launch.
int launch_cluster(const SolveDesc* descs_dev, int32_t k, int32_t max_n, int32_t max_pitch, uint32_t* queue,
                   const ClusterLaunch& cl, cudaStream_t st);
// A cluster-engine launch resolved ahead of time: running it is one memset
// and one kernel launch (both capturable in a CUDA graph).
struct ClusterPlan {
  void* fn = nullptr;
  int clusters = 0;
  int cluster_size = 0;
  int threads = 0;
  size_t smem = 0;
  int swcap = 0;
  int rgs_cap = 0;
  int depth = 0;
  int srows = 0;
  int rowcap = 0;
  int list_cap = 0;
  int amerge = 0;  // row groups merge through shared-memory atomicMin into one key per column
  uint32_t* words = nullptr;
};
// where a cluster launch takes its solves: a device table (batch), the serving
// ring, or one descriptor passed in the kernel's parameters
constexpr int kJobsBatch = 0;
constexpr int kJobsServe = 1;
constexpr int kJobsSingle = 2;
int plan_cluster(int32_t max_pitch, const ClusterLaunch& cl, int32_t k, ClusterPlan* plan, int kind = kJobsBatch);
// queue: two device words (next solve, exit count), zero when the launch starts; with
// zero_queue the launch zeroes them first, otherwise the previous launch left them zero
int run_cluster(const ClusterPlan& plan, const SolveDesc* descs_dev, int32_t k, uint32_t* queue, cudaStream_t st,
                bool zero_queue);
// one solve on one cluster, its descriptor in the kernel parameters (no device memory); rank 0
// writes the phase count to *phases_out, and the per-phase timeline to trace when given.
// Launched as a programmatic dependent of the previous kernel on the stream: it solves while
// that kernel ends and waits for it only before writing its outputs (and, unless `early`, before
// reading the graph).
int run_cluster_single(const ClusterPlan& plan, const SolveDesc& d, uint32_t* phases_out, uint64_t* trace,
                       int32_t trace_cap, bool early, cudaStream_t st);

// The serving request ring as the persistent kernel sees it (device-usable
// addresses of mapped pinned host memory, plus the device-side head).
struct ServeRing {
  const SolveDesc* ring;
  const uint32_t* tail;
  const uint32_t* stop;
  uint32_t* done;
  uint32_t* head;
  uint32_t cap_mask;
  int64_t idle_ns;
};
int run_serve_kernel(const ClusterPlan& plan, const ServeRing& r, cudaStream_t st);

// A cooperative launch (every CTA resident at once), as a programmatic dependent of the previous
// kernel on the stream when `pdl` (dj_solve.cu).
cudaError_t launch_cooperative(void* fn, int G, int threads, void** args, size_t smem, cudaStream_t st, bool pdl);

// Lockstep multi-source engine (dj_lockstep.cu): sources of one graph advance phase by phase
// together over every SM; one source's outputs.
struct LsSource {
  int32_t* dist;
  int32_t* pred;
  int32_t source;
  int32_t pad;
};
struct LockstepPlan {
  int G = 0, TPS = 0, swmax = 0, S_max = 0, S = 0, groups = 0, k = 0, nvec_total = 0, rstride = 0;
  size_t smem = 0, ws_bytes = 0, off_part = 0, off_dec = 0, off_tot = 0, off_reg = 0;
};
// Sizes and launch shape for k sources of g (groups of at most S_max sources, one launch each).
int plan_lockstep(const dj_graph* g, int32_t k, LockstepPlan* plan);
// The graph's column-tiled matrix copy for plan.G slices, built on `st` if missing.
int lockstep_tiles(dj_graph* g, const LockstepPlan& plan, cudaStream_t st, const int32_t** out);
// Launch every group.  ws: plan.ws_bytes of device memory whose first 256 bytes are zero (each
// launch leaves them zero again); src_dev: the k sources' descriptors on the device.
// allow_in = 0 keeps to the OUT bound (DJ_SETTLE_OUT).
int run_lockstep(const dj_graph* g, const LockstepPlan& plan, const int32_t* tiled, const LsSource* src_dev,
                 uint8_t* ws, uint32_t* words, int64_t timeout_ns, int allow_in, cudaStream_t st);
int cluster_max_clusters(int32_t max_pitch, const ClusterLaunch& cl, int* clusters);
bool cluster_config_ok(int32_t max_pitch, const ClusterLaunch& cl);

}  // namespace dj
