/*
 * Seeded synthetic graph inputs, shared by the CPU oracle's tests and the GPU
 * path's tests and benchmark.  This file draws random numbers and lays them out
 * as edge lists; it holds none of the shortest-path arithmetic.
 *
 * Generator: a counter-based form of SplitMix64 (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014).  Draw number
 * `ctr` of stream `stream` under `seed` is the SplitMix64 output at position
 * ctr+1 of the sequence whose state starts at mix(seed + golden*(stream+1)).
 * Every draw is a pure function of (seed, stream, ctr), so rows can be
 * generated in any order or in parallel and give the same graph.
 *
 * Bounded integers use Lemire's multiply-and-reject method ("Fast random
 * integer generation in an interval", ACM TOMACS 2019); rejected draws retry
 * on a separate stream, so the result stays unbiased and reproducible.
 *
 * Graph shapes (the paper's workloads are dense and 1:3-sparse matrices of
 * int32 weights; its generator is unstated):
 *   - Bernoulli undirected: each unordered pair i<j is an edge with
 *     probability p, weight uniform in [wlo, whi].  Edges are listed once,
 *     as (i, j, w) with i < j, in row-major pair order.
 *   - Out-degree directed: each node u draws d targets uniform in [0, n);
 *     a draw equal to u is dropped; duplicates are kept in the list.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL

enum {
  GG_STREAM_EDGE = 1,
  GG_STREAM_WEIGHT = 2,
  GG_STREAM_TARGET = 3,
  GG_STREAM_SOURCE = 4,
  GG_STREAM_RETRY = 5,
  GG_STREAM_USER = 16
};

static inline uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t gg_draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  uint64_t key = gg_mix(seed + GG_GOLDEN * (stream + 1));
  return gg_mix(key + GG_GOLDEN * (ctr + 1));
}

/* Uniform integer in [0, range), range in [1, 2^32]. */
uint64_t gg_bounded(uint64_t seed, uint64_t stream, uint64_t ctr, uint64_t range) {
  uint64_t x = gg_draw(seed, stream, ctr) >> 32;
  uint64_t prod = x * range;
  uint64_t low = prod & 0xFFFFFFFFULL;
  if (low < range) {
    uint64_t thresh = ((1ULL << 32) - range) % range;
    uint64_t attempt = 0;
    while (low < thresh) {
      uint64_t r = gg_draw(seed ^ (stream * GG_GOLDEN), GG_STREAM_RETRY,
                           ctr * 64 + (attempt++ & 63));
      x = r >> 32;
      prod = x * range;
      low = prod & 0xFFFFFFFFULL;
    }
  }
  return prod >> 32;
}

/* Bulk draws for host-side workload shaping (arrival times, per-graph sizes). */
void gg_fill_u64(uint64_t seed, uint64_t stream, uint64_t ctr0, int64_t count, uint64_t* out) {
  for (int64_t i = 0; i < count; ++i) out[i] = gg_draw(seed, stream, ctr0 + (uint64_t)i);
}

void gg_fill_bounded(uint64_t seed, uint64_t stream, uint64_t ctr0, int64_t count,
                     uint64_t range, int64_t* out) {
  for (int64_t i = 0; i < count; ++i)
    out[i] = (int64_t)gg_bounded(seed, stream, ctr0 + (uint64_t)i, range);
}

static uint64_t gg_threshold(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return UINT64_MAX;
  return (uint64_t)ldexp(p, 64);
}

static inline int gg_pair_is_edge(uint64_t seed, int64_t n, int64_t i, int64_t j, uint64_t thr) {
  if (thr == UINT64_MAX) return 1;
  return gg_draw(seed, GG_STREAM_EDGE, (uint64_t)(i * n + j)) < thr;
}

/* Pass 1: per-row edge counts of the Bernoulli graph (pairs i<j). Returns m. */
int64_t gg_bernoulli_count(int32_t n, double p, uint64_t seed, int64_t* row_counts) {
  uint64_t thr = gg_threshold(p);
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int64_t j = i + 1; j < n; ++j) c += gg_pair_is_edge(seed, n, i, j, thr);
    row_counts[i] = c;
    total += c;
  }
  return total;
}

/* Pass 2: fill the edges; row_offsets[i] = exclusive prefix of row_counts. */
void gg_bernoulli_fill(int32_t n, double p, int32_t wlo, int32_t whi, uint64_t seed,
                       const int64_t* row_offsets, int32_t* src, int32_t* dst, int32_t* w) {
  uint64_t thr = gg_threshold(p);
  uint64_t range = (uint64_t)((int64_t)whi - (int64_t)wlo + 1);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    int64_t k = row_offsets[i];
    for (int64_t j = i + 1; j < n; ++j) {
      if (!gg_pair_is_edge(seed, n, i, j, thr)) continue;
      src[k] = (int32_t)i;
      dst[k] = (int32_t)j;
      w[k] = (int32_t)((int64_t)wlo +
                       (int64_t)gg_bounded(seed, GG_STREAM_WEIGHT, (uint64_t)(i * n + j), range));
      ++k;
    }
  }
}

/* Directed out-degree graph.  Arrays hold n*d entries; returns m (<= n*d). */
int64_t gg_outdeg_fill(int32_t n, int32_t d, int32_t wlo, int32_t whi, uint64_t seed,
                       int32_t* src, int32_t* dst, int32_t* w) {
  uint64_t range = (uint64_t)((int64_t)whi - (int64_t)wlo + 1);
  int64_t m = 0;
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t k = 0; k < d; ++k) {
      uint64_t ctr = (uint64_t)(u * d + k);
      int64_t t = (int64_t)gg_bounded(seed, GG_STREAM_TARGET, ctr, (uint64_t)n);
      if (t == u) continue;
      src[m] = (int32_t)u;
      dst[m] = (int32_t)t;
      w[m] = (int32_t)((int64_t)wlo + (int64_t)gg_bounded(seed, GG_STREAM_WEIGHT, ctr, range));
      ++m;
    }
  }
  return m;
}

/* k distinct nodes of [0, n) in draw order (k <= n). */
void gg_distinct_sources(int32_t n, int32_t k, uint64_t seed, int32_t* out, uint8_t* seen /* n */) {
  memset(seen, 0, (size_t)n);
  int32_t got = 0;
  for (uint64_t ctr = 0; got < k; ++ctr) {
    int32_t s = (int32_t)gg_bounded(seed, GG_STREAM_SOURCE, ctr, (uint64_t)n);
    if (seen[s]) continue;
    seen[s] = 1;
    out[got++] = s;
  }
}
