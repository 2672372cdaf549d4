/*
 * CPU ORACLE -- test infrastructure only.
 *
 * A plain, serial, deliberately unoptimised restatement of the paper's
 * Algorithm 1 (Section III-A, "Serial Dijkstra's Algorithm") and of its
 * edge-list-to-adjacency-matrix input step (Section III, empirical
 * methodology, and the -w flag of Section III-A).  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline / reference legs may load it.
 * It shares no code, header or table with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Readings of the paper (where it is silent):
 *   - Infinity is INT32_MAX (the matrices of Section III-A print it as "inf").
 *   - The argmin of Algorithm 1 takes the smallest index among equal distances.
 *   - pred[] is never initialised by the paper: here it starts at -1, so the
 *     source and every unreachable node keep -1.
 *   - When the smallest unvisited distance is infinity, every remaining node is
 *     unreachable; the loop stops there instead of forming inf + G[u][v]
 *     (Algorithm 4 guards the same case with dist[tid] != INF).
 *   - Edge lists are (src, dst, w) triples with 0-based ids; a repeated pair
 *     keeps its smallest weight; a self-loop is ignored (the diagonal stays 0).
 *     Undirected input fills G[u][v] and G[v][u]; directed input (-w) fills
 *     G[u][v] only.
 *   - Sums dist[u] + G[u][v] are formed in 64-bit so that they are exact.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF INT32_MAX

/* Build the n x n matrix (row stride ld >= n) from an edge list.
 * Returns 0, or -1 for an id outside [0, n), a negative weight, or a weight
 * equal to the infinity sentinel. */
int orc_build_matrix(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                     const int32_t* w, int directed, int64_t ld, int32_t* G) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) G[i * ld + j] = (i == j) ? 0 : ORC_INF;
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e], x = w[e];
    if (u < 0 || u >= n || v < 0 || v >= n || x < 0 || x == ORC_INF) return -1;
    if (u == v) continue;
    if (x < G[(int64_t)u * ld + v]) G[(int64_t)u * ld + v] = x;
    if (!directed && x < G[(int64_t)v * ld + u]) G[(int64_t)v * ld + u] = x;
  }
  return 0;
}

/* Algorithm 1: Dijkstra(G, s).  dist[] and pred[] have n entries. */
void orc_dijkstra(int32_t n, const int32_t* G, int64_t ld, int32_t s, int32_t* dist,
                  int32_t* pred) {
  uint8_t* visited = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) {
    dist[i] = ORC_INF;
    visited[i] = 0;
    pred[i] = -1;
  }
  dist[s] = 0;
  for (int32_t i = 0; i < n; ++i) {
    /* u <- node with min dist[u] that is not visited (first index on ties) */
    int32_t u = -1;
    for (int32_t k = 0; k < n; ++k)
      if (!visited[k] && (u < 0 || dist[k] < dist[u])) u = k;
    if (u < 0 || dist[u] == ORC_INF) break;
    visited[u] = 1;
    /* for each neighbour v of u: relax with a strict improvement */
    const int32_t* row = G + (int64_t)u * ld;
    for (int32_t v = 0; v < n; ++v) {
      if (!visited[v] && row[v] != ORC_INF && (int64_t)dist[u] + row[v] < (int64_t)dist[v]) {
        dist[v] = (int32_t)((int64_t)dist[u] + row[v]);
        pred[v] = u;
      }
    }
  }
  free(visited);
}

/* The same solve for k sources of one matrix; outputs are k x n, row-major. */
void orc_dijkstra_many(int32_t n, const int32_t* G, int64_t ld, int32_t k, const int32_t* s,
                       int32_t* dist, int32_t* pred) {
  for (int32_t i = 0; i < k; ++i)
    orc_dijkstra(n, G, ld, s[i], dist + (int64_t)i * n, pred + (int64_t)i * n);
}

/* The same independent solves spread over `threads` host threads: thread t
 * runs orc_dijkstra for the sources t, t + threads, t + 2 threads, ...  Only
 * the scheduling differs from orc_dijkstra_many; every solve is the serial
 * Algorithm 1 above, and its outputs are written to the same places.
 * Returns the number of threads actually used (1 if threads could not be
 * started, in which case the solves run on the calling thread). */
typedef struct {
  int32_t n, k, t, threads;
  const int32_t* G;
  int64_t ld;
  const int32_t* s;
  int32_t* dist;
  int32_t* pred;
} orc_task;

static void* orc_worker(void* arg) {
  const orc_task* a = (const orc_task*)arg;
  for (int32_t i = a->t; i < a->k; i += a->threads)
    orc_dijkstra(a->n, a->G, a->ld, a->s[i], a->dist + (int64_t)i * a->n, a->pred + (int64_t)i * a->n);
  return NULL;
}

int orc_dijkstra_many_mt(int32_t n, const int32_t* G, int64_t ld, int32_t k, const int32_t* s,
                         int32_t* dist, int32_t* pred, int32_t threads) {
  if (threads > k) threads = k;
  if (threads < 2) {
    orc_dijkstra_many(n, G, ld, k, s, dist, pred);
    return 1;
  }
  pthread_t* tid = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
  orc_task* task = (orc_task*)malloc(sizeof(orc_task) * (size_t)threads);
  int32_t started = 0;
  for (int32_t t = 0; t < threads; ++t) {
    orc_task x = {n, k, t, threads, G, ld, s, dist, pred};
    task[t] = x;
    if (pthread_create(&tid[t], NULL, orc_worker, &task[t]) != 0) break;
    ++started;
  }
  for (int32_t t = 0; t < started; ++t) pthread_join(tid[t], NULL);
  /* sources whose thread never started run here */
  for (int32_t t = started; t < threads; ++t) orc_worker(&task[t]);
  free(tid);
  free(task);
  return started > 0 ? started : 1;
}
