/*
 * parallel.c -- multi-threaded (OpenMP) CPU baseline for the three applications.
 *
 * MEASUREMENT INFRASTRUCTURE ONLY, like the serial oracle beside it: only the tests and the
 * CPU-baseline leg of the benchmark load it, and it shares nothing with the CUDA library.  It is
 * NOT the parity reference (the serial oracle is); it is a reasonable parallel CPU program for the
 * same step, timed next to the GPU, and the tests check it against the serial oracle.
 *
 *   par_bfs       hop distances from each of nsrc sources (Section 5.1's result).  With at least
 *                 as many sources as threads, the sources run in parallel, one serial FIFO search
 *                 per thread; otherwise each source runs a level-synchronous parallel search
 *                 (Algorithm 1's structure: the frontier is split over threads, a vertex joins the
 *                 next frontier through a compare-and-swap on its depth).
 *   par_pagerank  the fixed point of x = (1 - alpha) 1 + alpha P x (Section 5.2's result) by
 *                 parallel FP64 Jacobi sweeps in pull form, until the L1 change of a sweep is at
 *                 most tol_per_vertex * n.
 *   par_color     speculative greedy colouring in rounds (Algorithm 5's structure): every vertex
 *                 of the worklist takes the first colour that none of its neighbours holds, then
 *                 a vertex that shares its colour with a smaller neighbour goes to the next round.
 *
 * Counts returned for the throughput figures: neighbour entries read.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define UNREACHED INT32_MAX

static int64_t bfs_serial(const int32_t* rp, const int32_t* col, int32_t n, int32_t src, int32_t* depth,
                          int32_t* fifo) {
  for (int32_t v = 0; v < n; ++v) depth[v] = UNREACHED;
  int64_t head = 0, tail = 0, edges = 0;
  depth[src] = 0;
  fifo[tail++] = src;
  while (head < tail) {
    const int32_t u = fifo[head++];
    const int32_t nd = depth[u] + 1;
    edges += rp[u + 1] - rp[u];
    for (int32_t k = rp[u]; k < rp[u + 1]; ++k)
      if (depth[col[k]] == UNREACHED) {
        depth[col[k]] = nd;
        fifo[tail++] = col[k];
      }
  }
  return edges;
}

static int64_t bfs_levels(const int32_t* rp, const int32_t* col, int32_t n, int32_t src, int32_t* depth,
                          int32_t* front, int32_t* next) {
  int64_t edges = 0;
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < n; ++v) depth[v] = UNREACHED;
  depth[src] = 0;
  front[0] = src;
  int64_t fsize = 1;
  for (int32_t level = 0; fsize > 0; ++level) {
    int64_t nsize = 0;
#pragma omp parallel reduction(+ : edges)
    {
      int32_t buf[256];
      int nb = 0;
#pragma omp for schedule(dynamic, 64)
      for (int64_t i = 0; i < fsize; ++i) {
        const int32_t u = front[i];
        edges += rp[u + 1] - rp[u];
        for (int32_t k = rp[u]; k < rp[u + 1]; ++k) {
          const int32_t w = col[k];
          int32_t expect = UNREACHED;
          if (__atomic_load_n(depth + w, __ATOMIC_RELAXED) == UNREACHED &&
              __atomic_compare_exchange_n(depth + w, &expect, level + 1, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
            buf[nb++] = w;
            if (nb == 256) {
              const int64_t at = __atomic_fetch_add(&nsize, 256, __ATOMIC_RELAXED);
              memcpy(next + at, buf, sizeof(buf));
              nb = 0;
            }
          }
        }
      }
      if (nb) {
        const int64_t at = __atomic_fetch_add(&nsize, nb, __ATOMIC_RELAXED);
        memcpy(next + at, buf, sizeof(int32_t) * (size_t)nb);
      }
    }
    int32_t* t = front;
    front = next;
    next = t;
    fsize = nsize;
  }
  return edges;
}

/* depth: nsrc x n, row i for sources[i].  Returns the neighbour entries read, -1 on bad
 * arguments or allocation failure. */
int64_t par_bfs(const int32_t* rp, const int32_t* col, int32_t n, const int32_t* sources, int32_t nsrc,
                int32_t* depth, int32_t nthreads) {
  if (!rp || !sources || !depth || n < 1 || nsrc < 0) return -1;
  for (int32_t i = 0; i < nsrc; ++i)
    if (sources[i] < 0 || sources[i] >= n) return -1;
  if (nthreads < 1) nthreads = omp_get_max_threads();
  omp_set_num_threads(nthreads);
  int64_t edges = 0;
  int failed = 0;
  if (nsrc >= nthreads) {
#pragma omp parallel reduction(+ : edges)
    {
      int32_t* fifo = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      if (!fifo) __atomic_store_n(&failed, 1, __ATOMIC_RELAXED);
#pragma omp for schedule(dynamic, 1)
      for (int32_t i = 0; i < nsrc; ++i)
        if (fifo) edges += bfs_serial(rp, col, n, sources[i], depth + (size_t)i * n, fifo);
      free(fifo);
    }
  } else {
    int32_t* a = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* b = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (a && b)
      for (int32_t i = 0; i < nsrc; ++i) edges += bfs_levels(rp, col, n, sources[i], depth + (size_t)i * n, a, b);
    else
      failed = 1;
    free(a);
    free(b);
  }
  return failed ? -1 : edges;
}

/* x: n doubles, the unnormalised fixed point.  Returns the sweeps run (x after the last one), -1
 * on bad arguments, -2 without convergence in max_iter sweeps. */
int32_t par_pagerank(const int32_t* rp, const int32_t* col, int32_t n, double alpha, double tol_per_vertex,
                     int32_t max_iter, double* x, int32_t nthreads) {
  if (!rp || !x || n < 1 || max_iter < 1) return -1;
  if (nthreads < 1) nthreads = omp_get_max_threads();
  omp_set_num_threads(nthreads);
  double* share = (double*)malloc(sizeof(double) * (size_t)n);  /* x[u] / deg(u) */
  if (!share) return -1;
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < n; ++v) x[v] = 1.0 - alpha;
  int32_t it = 0;
  for (;;) {
#pragma omp parallel for schedule(static)
    for (int32_t u = 0; u < n; ++u) {
      const int32_t d = rp[u + 1] - rp[u];
      share[u] = d > 0 ? x[u] / d : 0.0;
    }
    double delta = 0.0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : delta)
    for (int32_t v = 0; v < n; ++v) {
      double s = 0.0;
      for (int32_t k = rp[v]; k < rp[v + 1]; ++k) s += share[col[k]];
      const double nv = (1.0 - alpha) + alpha * s;
      delta += nv > x[v] ? nv - x[v] : x[v] - nv;
      x[v] = nv;  /* v's own share for this sweep was taken above: a Jacobi sweep */
    }
    ++it;
    if (delta <= tol_per_vertex * n) break;
    if (it >= max_iter) {
      free(share);
      return -2;
    }
  }
  free(share);
  return it;
}

/* color: n int32.  Returns the number of colours, -1 on bad arguments or allocation failure.
 * *rounds and *edges (may be NULL) receive the rounds run and the neighbour entries read. */
int32_t par_color(const int32_t* rp, const int32_t* col, int32_t n, int32_t* color, int32_t nthreads,
                  int32_t* rounds, int64_t* edges) {
  if (!rp || !color || n < 1) return -1;
  if (nthreads < 1) nthreads = omp_get_max_threads();
  omp_set_num_threads(nthreads);
  int32_t maxd = 0;
  for (int32_t v = 0; v < n; ++v)
    if (rp[v + 1] - rp[v] > maxd) maxd = rp[v + 1] - rp[v];
  int32_t* work = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!work || !next) {
    free(work);
    free(next);
    return -1;
  }
#pragma omp parallel for schedule(static)
  for (int32_t v = 0; v < n; ++v) {
    color[v] = -1;
    work[v] = v;
  }
  int64_t wsize = n, ed = 0;
  int32_t r = 0, failed = 0;
  while (wsize > 0) {
    ++r;
#pragma omp parallel reduction(+ : ed)
    {
      /* mark[c] == v + 1: colour c is held by a neighbour of v (first fit needs at most deg + 1) */
      int32_t* mark = (int32_t*)calloc((size_t)maxd + 2, sizeof(int32_t));
      if (!mark) __atomic_store_n(&failed, 1, __ATOMIC_RELAXED);
#pragma omp for schedule(dynamic, 256)
      for (int64_t i = 0; i < wsize; ++i) {
        if (!mark) continue;
        const int32_t v = work[i];
        const int32_t d = rp[v + 1] - rp[v];
        for (int32_t k = rp[v]; k < rp[v + 1]; ++k) {
          const int32_t c = __atomic_load_n(color + col[k], __ATOMIC_RELAXED);
          if (c >= 0 && c <= d) mark[c] = v + 1;
        }
        int32_t c = 0;
        while (mark[c] == v + 1) ++c;
        __atomic_store_n(color + v, c, __ATOMIC_RELAXED);
        ed += d;
      }
      free(mark);
    }
    if (failed) break;
    int64_t nsize = 0;
#pragma omp parallel reduction(+ : ed)
    {
#pragma omp for schedule(dynamic, 256)
      for (int64_t i = 0; i < wsize; ++i) {
        const int32_t v = work[i];
        for (int32_t k = rp[v]; k < rp[v + 1]; ++k)
          if (col[k] < v && color[col[k]] == color[v]) {
            next[__atomic_fetch_add(&nsize, 1, __ATOMIC_RELAXED)] = v;
            break;
          }
        ed += rp[v + 1] - rp[v];
      }
    }
    int32_t* t = work;
    work = next;
    next = t;
    wsize = nsize;
  }
  free(work);
  free(next);
  if (failed) return -1;
  int32_t k = 0;
  for (int32_t v = 0; v < n; ++v)
    if (color[v] + 1 > k) k = color[v] + 1;
  if (rounds) *rounds = r;
  if (edges) *edges = ed;
  return k;
}
