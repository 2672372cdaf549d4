/*
 * dj.h -- C ABI of the GB300 dense adjacency-matrix Dijkstra library.
 *
 * The operation is the paper's Algorithm 1 (Section III-A, "Serial Dijkstra's
 * Algorithm"): from a source s, n outer steps each take the unvisited node u
 * of smallest dist, mark it visited, and relax row u of the n x n weight
 * matrix G with  dist[v] = dist[u] + G[u][v], pred[v] = u  whenever that is a
 * strict improvement.  Inputs are edge lists turned into the matrix as in
 * Section III (Empirical methodology) and the -w flag of Section III-A.
 *
 * Results are defined as Algorithm 1's, read as follows where the paper is
 * silent: ties in the argmin go to the smallest index; pred starts at -1 (the
 * source and unreachable nodes keep -1); infinity is DJ_INF (INT32_MAX), also
 * the dist of unreachable nodes.  All arithmetic is int32; results are exact.
 *
 * Conventions for every call:
 *   - Return value: DJ_OK (0) or a negative DJ_E* status.  dj_last_error()
 *     returns a thread-local message for the last failing call on this thread.
 *   - `stream` is a cudaStream_t cast to uint64_t (0 = the legacy default
 *     stream).  Calls marked "asynchronous" only enqueue work on that stream;
 *     device-side failures (a bounded in-kernel wait that ran out) are
 *     reported by the next dj_sync() on the device.
 *   - "device pointer" means memory of the current CUDA device (for instance a
 *     torch tensor's data_ptr()); "host pointer" means ordinary host memory.
 *     Buffers stay owned by the caller unless stated otherwise.
 *   - The library keeps no global state other than a per-device context
 *     (error word, SM count) created on first use.
 */
#ifndef DJ_H
#define DJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define DJ_OK 0
#define DJ_EINVAL (-1)       /* bad argument: id out of range, negative or DJ_INF weight, n < 1 ... */
#define DJ_ENOMEM (-2)       /* device or pinned allocation failed, or over the serving HBM budget */
#define DJ_EOVERFLOW (-3)    /* (n-1) * max weight >= INT32_MAX: a path length could overflow int32 */
#define DJ_ECUDA (-4)        /* a CUDA runtime call failed (message in dj_last_error) */
#define DJ_ETIMEOUT (-5)     /* a bounded in-kernel wait ran out; the kernel returned early */
#define DJ_EBUSY (-6)        /* serving: no free slot or budget for the request right now */
#define DJ_EUNSUPPORTED (-7) /* configuration the device cannot run (e.g. cluster size) */

#define DJ_INF 2147483647

const char* dj_last_error(void);
const char* dj_status_string(int status);
int dj_version(void); /* major*10000 + minor*100 + patch */

/* ------------------------------------------------------------------ graphs */
typedef struct dj_graph dj_graph;

typedef struct dj_graph_info {
  int32_t n;             /* nodes */
  int32_t pitch;         /* row stride of the device matrix in int32 elements (n rounded up to 32) */
  int32_t directed;      /* 1 if built with the -w (directed) fill */
  int32_t min_weight;    /* smallest finite off-diagonal weight, DJ_INF if the graph has no edge */
  int32_t max_weight;    /* largest finite off-diagonal weight, 0 if none */
  int32_t device;        /* CUDA device holding the matrix */
  const int32_t* matrix; /* device pointer: n rows x pitch int32, row-major; columns >= n hold DJ_INF */
  const int32_t* minout; /* device pointer: n int32, min finite off-diagonal weight of row u (DJ_INF if none) */
  const int32_t* minin;  /* device pointer: n int32, min finite off-diagonal weight of column v (DJ_INF if none) */
  uint64_t bytes;        /* device bytes owned by the graph */
  uint64_t entries;      /* finite off-diagonal matrix entries (directed edges; twice the undirected ones) */
  int32_t format;        /* DJ_FORMAT_DENSE (matrix) or DJ_FORMAT_CSR (compressed rows, matrix NULL) */
  int32_t reserved;
} dj_graph_info;

#define DJ_FORMAT_DENSE 0
#define DJ_FORMAT_CSR 1

/* Build the n x n matrix on the current device from an edge list (Section
 * III: edge lists are written into the adjacency matrix; Section III-A
 * footnote: -w fills a directed graph, otherwise undirected).
 *   n          nodes, >= 1
 *   m          edges, >= 0
 *   src,dst,w  HOST pointers to m int32 each; read during the call only.
 *              Ids are 0-based in [0, n); 0 <= w < DJ_INF.
 *   directed   0: G[u][v] = G[v][u] = w;  1 (the paper's -w): G[u][v] = w only
 * The diagonal is 0, missing entries DJ_INF, a repeated pair keeps its minimum
 * weight, self-loops are ignored.  On success *out owns the device matrix until
 * dj_graph_free.  Synchronous with respect to the host (the edge arrays may be
 * reused on return); the device work is ordered on `stream`.
 * Errors: DJ_EINVAL (bad id/weight/n/m, NULL pointer), DJ_EOVERFLOW
 * ((n-1) * max weight >= INT32_MAX), DJ_ENOMEM, DJ_ECUDA. */
int dj_load_edges(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int32_t* w,
                  int directed, uint64_t stream, dj_graph** out);

/* The same graph kept in compressed-row form only: no n x n matrix (the paper
 * names that matrix's n^2 memory as the limit for sparse graphs, Section IV
 * and Conclusion).  Arguments, validation and fill rules as dj_load_edges
 * (repeats keep their smallest weight, self-loops are dropped, undirected
 * graphs store both directions); the edges are sorted on the host and the
 * device holds n + 1 64-bit row offsets, the targets and the weights
 * (8 bytes per directed edge) plus the row and column minima.  dj_sssp and
 * dj_sssp_ex solve it with the same phase logic and give the same dist and
 * pred as on the dense matrix; dj_graph_download / upload, dj_sssp_noalloc,
 * dj_sssp_lc, batches and serving need the matrix and return
 * DJ_EUNSUPPORTED.  Synchronous (uploads from host vectors). */
int dj_load_edges_csr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int32_t* w,
                      int directed, uint64_t stream, dj_graph** out);

/* Build a graph from an n x n row-major matrix W with row stride ld >= n
 * (same entry rules as above: diagonal must be 0, entries in [0, DJ_INF]).
 * `w_on_device` says whether W is a device (1) or host (0) pointer.  The
 * matrix is copied; the caller keeps W.  Errors as dj_load_edges (the entry
 * check runs on the device and reports DJ_EINVAL). Synchronous. */
int dj_load_dense(int32_t n, const int32_t* W, int64_t ld, int w_on_device, uint64_t stream,
                  dj_graph** out);

/* Overwrite an existing graph's matrix with a new n x n matrix of the same n
 * (host pointer W, row stride ld), then recompute its row and column minima and
 * tie sources.  This is the host-to-device matrix copy of the paper's CUDA
 * accounting (Section III-C, "Memory allocation and data transfer") without a
 * new allocation.  The copy is asynchronous on `stream` when W is pinned: a
 * kernel then reads W over the host link itself and takes the row minima (and,
 * for an undirected graph, the tie sources) on the way, so the matrix is not
 * read again for them (W must stay unchanged until the stream reaches it, as
 * for any asynchronous copy); pageable W goes through an ordinary copy first.
 * Entries are not re-validated (callers pass matrices that came from
 * dj_graph_download or a validated load, symmetric if the graph was loaded
 * undirected, whose column minima are taken from the row minima).  The next
 * solve of g waits for the kernels before it on its stream before it reads the
 * matrix. */
int dj_graph_upload(dj_graph* g, const int32_t* W, int64_t ld, uint64_t stream);

/* Copy the n x n matrix to HOST memory W (row stride ld >= n); synchronous. */
int dj_graph_download(const dj_graph* g, int32_t* W, int64_t ld, uint64_t stream);

int dj_graph_get_info(const dj_graph* g, dj_graph_info* info);

/* Release the device matrix.  The caller must have synchronised every stream
 * that still uses g.  NULL is accepted. */
int dj_graph_free(dj_graph* g);

/* ------------------------------------------------------------------ single solve */
#define DJ_MODE_AUTO 0  /* = DJ_MODE_PHASE */
#define DJ_MODE_PHASE 1 /* exact phase-batched: settles every node provably next in Algorithm 1's
                           visit order in one fused relaxation pass (same dist and pred) */
#define DJ_MODE_PLAIN 2 /* literal Algorithm 1: one argmin + one row relaxation per step */

#define DJ_ENGINE_AUTO 0     /* grid for n >= 4096, or n >= 2560 with at least n^2/4 finite entries */
#define DJ_ENGINE_GRID 1    /* one cooperative persistent kernel over every SM; column slices per CTA */
#define DJ_ENGINE_CLUSTER 2 /* one thread-block cluster; state in distributed shared memory */

typedef struct dj_solve_opts {
  int32_t mode;           /* DJ_MODE_* */
  int32_t engine;         /* DJ_ENGINE_* */
  int32_t cluster_size;   /* cluster engine: CTAs per cluster (1..16), 0 = auto */
  int32_t threads;        /* threads per CTA (256, 512 or 1024), 0 = auto */
  int32_t ctas_per_sm;    /* grid engine: resident CTAs per SM (1 or 2), 0 = auto */
  int32_t unroll;         /* rows in flight per warp (1, 2, 4 or 8), 0 = auto */
  int64_t timeout_ns;     /* limit of every in-kernel wait, 0 = 2 s */
  int32_t debug_skip_cta; /* testing only: this CTA leaves before the first grid barrier (-1 = none) */
  int32_t trace_cap;      /* profiling: entries of `trace` (0 = no trace) */
  uint64_t* trace;        /* DEVICE pointer to trace_cap uint64: per phase, CTA 0 (grid engine) or
                             rank 0 (cluster engine) records 8 words.  Grid engine: %globaltimer at
                             publish start, publish end, barrier arrival, barrier exit, decision
                             end, relaxation end, commit end, then the phase's candidate count
                             (low 32 bits) and CTA 0's live column groups (high 32 bits).  Cluster
                             engine: publish start, publish end, cluster barrier exit, decision
                             end, staging end, relaxation end (rank 0's warps), commit end, the
                             candidate count.  The last two entries get the kernel's (solve's)
                             entry and exit times (trace_cap >= 10); unused entries are left as is */
  int32_t settle;         /* phase mode's settle bounds: DJ_SETTLE_AUTO, DJ_SETTLE_OUT, DJ_SETTLE_OUT_IN */
  int32_t live;           /* grid engine column filter.  A settled row u offers column v at least
                             max(L, m + minin[v]), so a column whose stored dist is below that can
                             change neither dist nor pred in this phase.  0 = auto: a CTA with no
                             live column skips the phase's relaxation, one with few live columns
                             loads only those; > 0: load only the live columns when at most this
                             many 4-column groups of the CTA's slice are live; -1 = off (every
                             settled row's whole slice is streamed). */
  int32_t rowsplit;       /* grid engine: a phase with at least this many settled candidates streams
                             whole rows, each CTA a share of them, and merges the per-column bests
                             through global memory around one more grid barrier (reading a whole
                             row per CTA streams HBM faster than every CTA reading its slice of
                             every row).  0 = auto (n/8 clamped to 512..2048, on graphs with at
                             least n^2/32 finite entries; never on sparser ones), -1 = never. */
  int32_t rowpush;        /* grid engine, graphs with fewer than n^2/32 finite entries: a phase with at
                             least this many candidates (while a sixteenth of the nodes stays
                             unsettled) reads its settled rows whole, in 2048-column pieces spread over
                             every warp of the grid, and pushes each finite entry into per-column keys
                             that the owners commit from after one more grid barrier.  0 = auto (four
                             candidates per CTA), -1 = never; also forced (> 0) on dense graphs when
                             rowsplit is -1. */
  int32_t reserved[2];
} dj_solve_opts;

#define DJ_SETTLE_AUTO 0   /* OUT and IN bounds when every off-diagonal weight is >= 1, else OUT only;
                              the IN bound dynamic where the graph keeps in-lists (below) */
#define DJ_SETTLE_OUT 1    /* OUT bound only (nodes settled in Algorithm 1's visit order) */
#define DJ_SETTLE_OUT_IN 2 /* OUT and IN bounds, the IN bound from each column's smallest in-weight;
                              falls back to OUT when some weight is 0 */
#define DJ_SETTLE_OUT_DYN_IN 3 /* OUT and IN bounds, the IN bound (grid engine, graphs with fewer than
                              n^2/32 finite entries, which keep each column's 4 smallest in-weights
                              and their rows) from the smallest in-weight of the rows NOT yet settled:
                              a shorter path into v must enter it from an unsettled row.  Fewer phases
                              on sparse graphs (the directed n=32768, 8 out-edges per node graph:
                              about 90 instead of 140); same results. */
#define DJ_SETTLE_DYN 4    /* DJ_SETTLE_OUT_DYN_IN and the OUT bound dynamic too: each row's smallest
                              out-weight to columns not yet settled (rows' 4 smallest out-weights listed
                              at load).  A few phases fewer again (85 instead of 89 on that graph), but
                              measured slower there (1700 against 1663 us per solve: its row-push
                              phases take longer), so not the default. */

/* Fill opts with the defaults (AUTO everything, debug_skip_cta = -1). */
void dj_solve_opts_init(dj_solve_opts* opts);

/* One solve of Algorithm 1 from `source` on graph g.
 *   dist, pred  DEVICE pointers to n int32 each (caller-owned), written by the kernel.
 * Asynchronous on `stream`: one kernel launch.  The grid engine keeps a small
 * workspace per (device, stream) -- about 32 bytes per matrix column plus 16 *
 * pitch bytes with the row split, at least 1 MiB -- created on the first solve
 * on that stream (a cudaMalloc) and grown, after synchronising the stream,
 * when a larger graph comes; solves on one stream share it in stream order,
 * and it is held until the process exits.  While `stream` is being captured
 * into a CUDA graph the solve instead allocates and frees its workspace in
 * stream order (the graph owns it).  The cluster engine (small graphs) needs
 * no workspace: its solve descriptor travels in the launch's parameters.  The
 * first solve of a kernel configuration on a device sets that kernel's launch
 * attributes (its shared-memory limit) once; solve once before capturing a
 * stream under a capture mode that forbids such calls.  Replayed from a CUDA
 * graph, small solves run without the per-launch cost of a stream launch
 * (n=1024: 3.4 us per solve against about 11 us launched one by one).
 * Errors: DJ_EINVAL (source out of range, NULL), DJ_ECUDA (launch failed); a
 * device-side timeout shows at dj_sync(). */
int dj_sssp(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, uint64_t stream);
int dj_sssp_ex(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred,
               const dj_solve_opts* opts, uint64_t stream);

/* The same solve with HOST result buffers (n int32 each): launches, copies
 * dist and pred back, synchronises `stream` and returns the device status
 * (DJ_ETIMEOUT included).  Pinned buffers give the fastest copy. */
int dj_sssp_host(const dj_graph* g, int32_t source, int32_t* dist_host, int32_t* pred_host,
                 uint64_t stream);

/* Synchronise `stream`, then return and clear the device error word of the
 * current device: DJ_ETIMEOUT if a bounded wait ran out since the last
 * dj_sync, DJ_ECUDA on a CUDA error, DJ_OK otherwise. */
int dj_sync(uint64_t stream);

/* Phases (fused relaxation passes) taken by the last completed solve launched
 * by dj_sssp/dj_sssp_ex on this device (either engine); -1 if unknown.  Call
 * after dj_sync.  The count is one word per device written by every single
 * solve: with solves running concurrently on several streams it reports
 * whichever of them finished last. */
int dj_last_phases(void);

/* Allocation-free single solve.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory at solve
 * time -- for example code running while a stream is being captured under a
 * global capture mode (where cudaMalloc is forbidden), serving loops that
 * cannot afford the device-wide synchronisation or the failure of a late
 * allocation, or processes whose caching allocator already reserved nearly
 * all of HBM.  It runs the same grid-engine kernel and gives the same dist
 * and pred as dj_sssp, but its scratch (barrier and candidate counters,
 * per-CTA partials and two candidate lists of 16 bytes per column, about
 * 2 * 16 * pitch bytes) lives in one fixed 4 MiB array compiled into the
 * library: every GPU that loads the library holds those 4 MiB until the
 * process exits.  Graphs whose scratch does not fit are rejected with
 * DJ_EINVAL, whose message names this device's limit: n up to 130,720 on a
 * 152-SM GB300 (the bound moves by a few hundred with the SM count).
 *   g, source, dist, pred, stream: as dj_sssp (dist/pred DEVICE pointers).
 * The call allocates no device memory: it issues two small cudaMemsetAsync
 * calls (clearing the counters and setting dist[source] = -1) and one kernel
 * launch on `stream`.  DJ_EUNSUPPORTED if the slice layout cannot be resident
 * on every SM at once.  Asynchronous: once the stream has passed the kernel,
 * dist[source] == 0 means the solve completed; dist[source] == -1 means a
 * bounded in-kernel wait ran out and the outputs are not valid.
 * The first call on each device performs a one-time set-up (it looks up the
 * array's device address and the device's attributes); make that first call
 * before any stream capture.  Every call on a device shares the one array and
 * it keeps the previous call's contents, so calls whose kernels overlap on the
 * GPU (for instance on two streams) race: order them on one stream or
 * synchronise between them. */
int dj_sssp_noalloc(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, uint64_t stream);

/* Label-correcting solve: the paper's CUDA variant (Algorithms 3 and 4,
 * Section III-C), kept as a comparison point for Algorithm 1.  Sweeps relax
 * every row whose dist changed in the previous sweep until nothing changes
 * (a Bellman-Ford fixed point), all inside one cooperative kernel with no host
 * round trip between sweeps.
 *   g, source, dist, pred, stream: as dj_sssp (dist/pred DEVICE pointers).
 * dist equals Algorithm 1's exactly.  pred is a shortest-path tree
 * (dist[pred[v]] + G[pred[v]][v] == dist[v], -1 for the source and unreachable
 * nodes) but, where several shortest paths exist, not necessarily Algorithm 1's
 * choice; dj_last_phases() reports the number of sweeps.  Asynchronous; errors
 * as dj_sssp (DJ_EUNSUPPORTED for slices beyond 512 columns per SM). */
int dj_sssp_lc(const dj_graph* g, int32_t source, int32_t* dist, int32_t* pred, uint64_t stream);

/* ------------------------------------------------------------------ batched solves */
/* k solves (graph[i], sources[i]) in one persistent launch: one thread-block
 * cluster per solve at a time, solves pulled from a device queue (largest n
 * first), graphs of different n allowed, rows shared by concurrent solves of
 * one graph reused through L2; or, for solves of one graph whose shape the
 * autotuner found faster that way, the lockstep engine
 * (DJ_BATCH_ENGINE_LOCKSTEP).  Each solve's result equals dj_sssp's.
 *   graphs   HOST array of k graph handles (all on the current device)
 *   sources  HOST array of k int32
 *   dist, pred  HOST arrays of k DEVICE pointers, n_i int32 each
 * Asynchronous on `stream` (the descriptor table is copied before return). */
int dj_sssp_batch(const dj_graph* const* graphs, const int32_t* sources, int32_t k,
                  int32_t* const* dist, int32_t* const* pred, uint64_t stream);

typedef struct dj_batch_opts {
  int32_t mode;          /* DJ_MODE_* */
  int32_t cluster_size;  /* 0 = auto (autotuned table or heuristic) */
  int32_t threads;       /* 0 = auto */
  int32_t clusters;      /* clusters resident at once, 0 = as many as fit */
  int32_t settle;        /* DJ_SETTLE_* (defined below), 0 = auto */
  int32_t copies;        /* DJ_COPIES_*: how a CTA's ring copies its slice of a settled row */
  int32_t engine;        /* DJ_BATCH_ENGINE_*: which engine runs the batch */
  int32_t reserved[5];
} dj_batch_opts;

#define DJ_BATCH_ENGINE_AUTO 0     /* the tuned engine for this graph shape if there is one, else clusters */
#define DJ_BATCH_ENGINE_CLUSTER 1  /* one thread-block cluster per solve, solves pulled from a device queue */
#define DJ_BATCH_ENGINE_LOCKSTEP 2 /* every solve of ONE graph advances phase by phase together over every
                                      SM, so a row a phase needs is read once for all the sources that
                                      settle it (per-source results as Algorithm 1's).  The graph keeps
                                      a column-tiled copy of its matrix (about the matrix's size, counted
                                      in dj_graph_info.bytes) until it is freed.  Sources are taken in
                                      groups of at most 256 (fewer for n > 8192; DJ_EUNSUPPORTED where
                                      fewer than 32 fit, roughly n > 13000), one cooperative launch per
                                      group.  Fewer HBM bytes, but bound by instruction issue: slower
                                      than clusters on the shapes measured, so only chosen explicitly or
                                      by the autotuner. */

#define DJ_COPIES_AUTO 0   /* wide where the slice allows it */
#define DJ_COPIES_NARROW 1 /* every warp copies its own 512-byte part of each row */
#define DJ_COPIES_WIDE 2   /* a warp copies 2 KB (four 4-column groups per lane) of its rows; row groups
                              merge through shared-memory atomics.  Larger copies stream faster per SM. */

void dj_batch_opts_init(dj_batch_opts* opts);

/* A prepared batch: the descriptor table and the queue words live on the
 * device, so launching it is a single kernel launch (capturable in a CUDA
 * graph): the last cluster of each launch puts the queue back to zero for the
 * next one.  Launches of one batch must not overlap (one stream, or
 * synchronise between them).  The caller keeps the graphs and result buffers
 * alive while launched. */
typedef struct dj_batch dj_batch;
int dj_batch_create(const dj_graph* const* graphs, const int32_t* sources, int32_t k,
                    int32_t* const* dist, int32_t* const* pred, const dj_batch_opts* opts,
                    dj_batch** out);
int dj_batch_launch(dj_batch* b, uint64_t stream);
int dj_batch_free(dj_batch* b); /* caller synchronises first */

/* Autotuner: times every supported cluster size (2, 4, 8, 16) and, for
 * solves of one graph, the lockstep engine, on the device, and keeps the
 * fastest for the batch and in the process-wide table keyed by (n bucket =
 * floor(log2 n), density bucket = floor(log2(n^2 / finite entries)) capped at
 * 20, SM count), which later batches of one graph consult.  When the
 * environment variable DJ_TUNE_FILE names a file, the table is read from it on
 * first use and written back after every autotune, so another process picks up
 * the choice.  Synchronous; overwrites the batch's outputs.  Reports the choice
 * (cluster_size 0 for the lockstep engine) through the optional out-parameters. */
int dj_batch_autotune(dj_batch* b, uint64_t stream, int32_t* cluster_size, int32_t* threads,
                      float* best_ms);

/* The engine a prepared batch launches (DJ_BATCH_ENGINE_CLUSTER or _LOCKSTEP). */
int dj_batch_get_engine(const dj_batch* b, int32_t* engine);

/* The autotuner's table as JSON (host only, no GPU needed):
 *   {"version": 1, "entries": [{"n_bucket": 13, "density_bucket": 4, "sms": 152,
 *     "engine": "lockstep", "cluster_size": 0, "threads": 512, "ms": 3.1}, ...]}
 * dj_tune_load merges a file's entries into the table (DJ_EINVAL if it cannot
 * be read); dj_tune_save writes the table (atomically, through a temporary
 * file); dj_tune_lookup returns the entry for a graph of n nodes with
 * `entries` finite off-diagonal entries on a device of num_sms SMs (DJ_EINVAL
 * if none).  engine: DJ_BATCH_ENGINE_*. */
int dj_tune_load(const char* path);
int dj_tune_save(const char* path);
int dj_tune_lookup(int32_t n, uint64_t entries, int32_t num_sms, int32_t* engine, int32_t* cluster_size);

/* ------------------------------------------------------------------ serving */
typedef struct dj_server dj_server;

typedef struct dj_serve_opts {
  uint64_t hbm_budget;   /* bytes of device memory the server may hold (graphs + result pool) */
  int32_t max_slots;     /* requests in flight on the device at most (<= 4096) */
  int32_t cluster_size;  /* CTAs per solve cluster, 0 = auto */
  int32_t threads;       /* 0 = auto */
  int32_t clusters;      /* persistent solve clusters, 0 = as many as fit */
  int64_t idle_timeout_ns; /* the persistent kernel exits after this long without work, 0 = 200 ms */
  int32_t reserved[8];
} dj_serve_opts;

typedef struct dj_serve_stats {
  uint64_t submitted, completed, rejected;
  double p50_us, p90_us, p99_us, max_us, mean_us; /* submit-to-completion latency */
  double solves_per_s;                            /* completed / (last completion - first submit) */
  uint64_t resident_bytes;                        /* graphs + result pool held on the device */
  int32_t kernel_launches;                        /* persistent kernel (re)launches so far */
  int32_t reserved[7];
} dj_serve_stats;

void dj_serve_opts_init(dj_serve_opts* opts);

/* Create a server on the current device.  Allocates the pinned request ring
 * and completion words; device memory is admitted against hbm_budget. */
int dj_serve_create(const dj_serve_opts* opts, dj_server** out);

/* Make graph g resident for serving (counted against the budget); *graph_id
 * names it in requests.  DJ_ENOMEM if it does not fit the budget. */
int dj_serve_add_graph(dj_server* s, const dj_graph* g, int32_t* graph_id);

/* Submit one solve.  dist/pred are DEVICE or mapped-pinned HOST pointers of
 * n int32 each, or both NULL (the result then lands in a server-owned pool
 * buffer, counted against the budget, readable with dj_serve_result until the
 * next submit reuses it).  Returns DJ_EBUSY when every slot or the budget is
 * taken (the caller retries after a poll); the request then was not queued. */
int dj_serve_submit(dj_server* s, int32_t graph_id, int32_t source, int32_t* dist, int32_t* pred,
                    uint64_t* ticket);

/* *done = 1 once the ticket's result is in place (0 otherwise). */
int dj_serve_poll(dj_server* s, uint64_t ticket, int* done);

/* Block until the ticket completes or timeout_ns passes (DJ_ETIMEOUT). */
int dj_serve_wait(dj_server* s, uint64_t ticket, int64_t timeout_ns);

/* Copy a completed pool-buffered result to HOST memory (n int32 each). */
int dj_serve_result(dj_server* s, uint64_t ticket, int32_t* dist_host, int32_t* pred_host);

int dj_serve_stats_get(dj_server* s, dj_serve_stats* st);
int dj_serve_destroy(dj_server* s); /* waits for in-flight work */

/* Run a whole request trace on a fresh server: request r (graph req_graph[r],
 * source req_source[r]) is submitted no earlier than arrival_s[r] seconds
 * after the start (HOST arrays of R entries), admitted as slots and budget
 * free up, and completed by the persistent kernel while later requests keep
 * arriving (continuous batching).  out_dist/out_pred are optional HOST arrays
 * of R device pointers (entries may be NULL to drop that result).  Fills *st. */
int dj_serve(const dj_graph* const* graphs, int32_t num_graphs, int64_t R, const int32_t* req_graph,
             const int32_t* req_source, const double* arrival_s, int32_t* const* out_dist,
             int32_t* const* out_pred, const dj_serve_opts* opts, dj_serve_stats* st);

#ifdef __cplusplus
}
#endif

#endif /* DJ_H */
