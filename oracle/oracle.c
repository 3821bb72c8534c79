/*
 * oracle.c -- plain, serial, CPU reference for the three applications of the Atos paper.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this file: only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark use it.  It shares no code,
 * header, constant or helper with the CUDA library; the two meet only through the seeded input
 * graphs of the separate `graphgen` module.
 *
 * What it computes, and the passage each function follows:
 *
 *   oracle_bfs               Section 5.1 (Algorithms 1 and 2): the speculative BFS reaches the
 *                            exact hop distance from the source, i.e. what a textbook serial FIFO
 *                            breadth-first search computes.  That definition is written out here.
 *   oracle_bfs_certificate   the properties that characterise hop distances, checkable at any size.
 *   oracle_pagerank          Section 5.2 (Algorithms 3 and 4): push-residual PageRank converges to
 *                            the fixed point of x = (1 - alpha) 1 + alpha P x, P = A D^-1 on the
 *                            paper's unnormalised scale (initial rank 1 - alpha).  Solved here by
 *                            plain FP64 Jacobi power iteration.
 *   oracle_pr_residual       the FP64 residual (1 - alpha) 1 + alpha P x - x of any candidate x;
 *                            its L1 norm bounds the distance to the fixed point.
 *   oracle_pr_push_serial    the steps of Algorithm 3 run serially (initial residue, then push
 *                            exch / rank += / scatter while any residue exceeds epsilon), used for
 *                            workload statistics and to pin the reading of the initial residue.
 *   oracle_greedy_color      Section 5.3: serial greedy first-fit colouring in a given vertex order
 *                            (the sequential algorithm the speculative colouring parallelises).
 *   oracle_check_coloring    proper-colouring check and the first-fit range 0 <= c(v) <= deg(v).
 *
 * Readings of points where the paper is silent are fixed in the design notes; the ones that
 * matter here: unreached vertices get INT32_MAX; isolated vertices keep rank 1 - alpha and never
 * push; the initial residue of v is (1 - alpha) alpha sum_{u in N(v)} 1 / deg(u).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define UNREACHED INT32_MAX

/* ---------------------------------------------------------------- BFS */

/* Serial FIFO breadth-first search from src.  depth[v] = hop distance, UNREACHED if v is not in
 * src's component.  Returns the number of reached vertices, or -1 on bad arguments. */
int64_t oracle_bfs(const int32_t* row_ptr, const int32_t* col, int32_t n, int32_t src, int32_t* depth) {
  if (!row_ptr || !depth || n < 1 || src < 0 || src >= n) return -1;
  int32_t* fifo = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!fifo) return -1;
  for (int32_t v = 0; v < n; ++v) depth[v] = UNREACHED;
  int64_t head = 0, tail = 0;
  depth[src] = 0;
  fifo[tail++] = src;
  while (head < tail) {
    int32_t u = fifo[head++];
    int32_t du = depth[u];
    for (int32_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
      int32_t w = col[k];
      if (depth[w] == UNREACHED) {
        depth[w] = du + 1;
        fifo[tail++] = w;
      }
    }
  }
  free(fifo);
  return tail;
}

/* Certificate that depth[] holds the hop distances from src (valid for symmetric graphs):
 *   1. depth[src] == 0;
 *   2. every edge (u, w) has both ends reached or both unreached;
 *   3. every edge with both ends reached has |depth[u] - depth[w]| <= 1;
 *   4. every reached v != src has a neighbour at depth[v] - 1, and depth[v] > 0.
 * (1) and (4) give depth >= distance along a predecessor chain; (1) and (3) give depth <= distance
 * along a shortest path; (2) makes the reached set closed, hence exactly src's component.
 * Returns 0 if all hold, otherwise the failing property number, and stores the offending vertex. */
int oracle_bfs_certificate(const int32_t* row_ptr, const int32_t* col, int32_t n, int32_t src,
                           const int32_t* depth, int32_t* bad_vertex) {
  int32_t dummy;
  if (!bad_vertex) bad_vertex = &dummy;
  *bad_vertex = -1;
  if (!row_ptr || !depth || n < 1 || src < 0 || src >= n) return -1;
  if (depth[src] != 0) {
    *bad_vertex = src;
    return 1;
  }
  for (int32_t v = 0; v < n; ++v) {
    int32_t dv = depth[v];
    int has_parent = 0;
    if (dv != UNREACHED && dv < 0) {
      *bad_vertex = v;
      return 4;
    }
    for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
      int32_t w = col[k];
      int32_t dw = depth[w];
      if ((dv == UNREACHED) != (dw == UNREACHED)) {
        *bad_vertex = v;
        return 2;
      }
      if (dv == UNREACHED) continue;
      int64_t diff = (int64_t)dv - (int64_t)dw;
      if (diff > 1 || diff < -1) {
        *bad_vertex = v;
        return 3;
      }
      if ((int64_t)dw == (int64_t)dv - 1) has_parent = 1;
    }
    if (v != src && dv != UNREACHED && (!has_parent || dv <= 0)) {
      *bad_vertex = v;
      return 4;
    }
  }
  return 0;
}

/* ---------------------------------------------------------------- PageRank */

/* y = (1 - alpha) 1 + alpha P x with (P x)_v = sum_{u in N(v)} x_u / deg(u).  On a symmetric
 * graph the in-neighbours of v are its neighbours, so the product is a pull over v's row. */
static void pr_apply(const int32_t* row_ptr, const int32_t* col, int32_t n, double alpha, const double* x,
                     const double* inv_deg, double* y, double* scratch) {
  for (int32_t u = 0; u < n; ++u) scratch[u] = x[u] * inv_deg[u];
  for (int32_t v = 0; v < n; ++v) {
    double s = 0.0;
    for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) s += scratch[col[k]];
    y[v] = (1.0 - alpha) + alpha * s;
  }
}

static double* inverse_degrees(const int32_t* row_ptr, int32_t n) {
  double* inv = (double*)malloc(sizeof(double) * (size_t)n);
  if (!inv) return NULL;
  for (int32_t u = 0; u < n; ++u) {
    int32_t d = row_ptr[u + 1] - row_ptr[u];
    inv[u] = d > 0 ? 1.0 / (double)d : 0.0; /* isolated vertices push nothing */
  }
  return inv;
}

/* FP64 Jacobi power iteration x <- (1 - alpha) 1 + alpha P x from x = 1, until
 * ||x_new - x||_1 <= tol_per_vertex * n, or until the step has reached the FP64 rounding floor
 * (it is below 1e-9 per vertex and has not decreased for 3 sweeps; in exact arithmetic it shrinks
 * by at least alpha per sweep), or max_iter sweeps.  x_out is on the unnormalised scale (sum ~ n);
 * divide by its sum for the probability vector.  Returns 0, or 1 if max_iter was hit, or -1 on
 * bad arguments.  *iters and *last_delta report the sweeps and the final step size. */
int oracle_pagerank(const int32_t* row_ptr, const int32_t* col, int32_t n, double alpha, double tol_per_vertex,
                    int32_t max_iter, double* x_out, int32_t* iters, double* last_delta) {
  if (!row_ptr || !x_out || n < 1 || !(alpha >= 0.0 && alpha < 1.0) || max_iter < 1) return -1;
  double* inv = inverse_degrees(row_ptr, n);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* scratch = (double*)malloc(sizeof(double) * (size_t)n);
  if (!inv || !y || !scratch) {
    free(inv), free(y), free(scratch);
    return -1;
  }
  for (int32_t v = 0; v < n; ++v) x_out[v] = 1.0;
  int rc = 1;
  int32_t it = 0, flat = 0;
  double delta = INFINITY, prev = INFINITY;
  while (it < max_iter) {
    pr_apply(row_ptr, col, n, alpha, x_out, inv, y, scratch);
    delta = 0.0;
    for (int32_t v = 0; v < n; ++v) delta += fabs(y[v] - x_out[v]);
    memcpy(x_out, y, sizeof(double) * (size_t)n);
    it++;
    if (delta <= tol_per_vertex * (double)n) {
      rc = 0;
      break;
    }
    flat = (delta <= 1e-9 * (double)n && delta >= prev) ? flat + 1 : 0;
    if (flat >= 3) {
      rc = 0;
      break;
    }
    prev = delta;
  }
  if (iters) *iters = it;
  if (last_delta) *last_delta = delta;
  free(inv), free(y), free(scratch);
  return rc;
}

/* rho = (1 - alpha) 1 + alpha P x - x in FP64, for x given in FP64 on the unnormalised scale.
 * Writes rho (if rho_out) and returns ||rho||_1; since (I - alpha P) has an inverse of induced
 * L1 norm at most 1 / (1 - alpha), ||x - p||_1 <= ||rho||_1 / (1 - alpha) for the fixed point p. */
double oracle_pr_residual(const int32_t* row_ptr, const int32_t* col, int32_t n, double alpha, const double* x,
                          double* rho_out) {
  if (!row_ptr || !x || n < 1) return -1.0;
  double* inv = inverse_degrees(row_ptr, n);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* scratch = (double*)malloc(sizeof(double) * (size_t)n);
  if (!inv || !y || !scratch) {
    free(inv), free(y), free(scratch);
    return -1.0;
  }
  pr_apply(row_ptr, col, n, alpha, x, inv, y, scratch);
  double l1 = 0.0;
  for (int32_t v = 0; v < n; ++v) {
    double r = y[v] - x[v];
    if (rho_out) rho_out[v] = r;
    l1 += fabs(r);
  }
  free(inv), free(y), free(scratch);
  return l1;
}

/* Serial run of the push formulation (Algorithm 3's steps, one vertex at a time from a FIFO of
 * vertices whose residue exceeds epsilon; a vertex is in the FIFO at most once):
 *   init:  rank = 1 - alpha; residue[v] = (1 - alpha) alpha sum_{u in N(v)} 1/deg(u); all queued;
 *   pop v: r = residue[v]; residue[v] = 0; rank[v] += r; for n in N(v): residue[n] += alpha r/deg(v),
 *          queueing n when its residue exceeds epsilon.
 * FP64 throughout.  Returns the number of pushes (pops with deg > 0), or -1.  The invariant
 * p = rank + (I - alpha P)^-1 residue holds exactly in exact arithmetic. */
int64_t oracle_pr_push_serial(const int32_t* row_ptr, const int32_t* col, int32_t n, double alpha, double eps,
                              double* rank, double* residue, int64_t* edge_pushes) {
  if (!row_ptr || !rank || !residue || n < 1) return -1;
  int32_t* fifo = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  unsigned char* queued = (unsigned char*)calloc((size_t)n, 1);
  if (!fifo || !queued) {
    free(fifo), free(queued);
    return -1;
  }
  for (int32_t v = 0; v < n; ++v) {
    rank[v] = 1.0 - alpha;
    residue[v] = 0.0;
  }
  for (int32_t u = 0; u < n; ++u) {
    int32_t d = row_ptr[u + 1] - row_ptr[u];
    if (d == 0) continue;
    double share = (1.0 - alpha) * alpha / (double)d;
    for (int32_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) residue[col[k]] += share;
  }
  int64_t head = 0, count = 0; /* ring of capacity n: each vertex is queued at most once */
  for (int32_t v = 0; v < n; ++v) {
    fifo[v] = v;
    queued[v] = 1;
  }
  count = n;
  int64_t pushes = 0, epush = 0;
  while (count > 0) {
    int32_t v = fifo[head];
    head = (head + 1) % n;
    count--;
    queued[v] = 0;
    double r = residue[v];
    residue[v] = 0.0;
    rank[v] += r;
    int32_t d = row_ptr[v + 1] - row_ptr[v];
    if (d == 0 || r == 0.0) continue;
    double s = alpha * r / (double)d;
    pushes++;
    epush += d;
    for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
      int32_t w = col[k];
      residue[w] += s;
      if (residue[w] > eps && !queued[w]) {
        queued[w] = 1;
        fifo[(head + count) % n] = w;
        count++;
      }
    }
  }
  if (edge_pushes) *edge_pushes = epush;
  free(fifo), free(queued);
  return pushes;
}

/* ---------------------------------------------------------------- colouring */

/* Serial greedy first-fit: visit vertices in `order` (NULL = 0..n-1) and give each the smallest
 * colour not used by an already-coloured neighbour.  Returns the number of colours, or -1. */
int32_t oracle_greedy_color(const int32_t* row_ptr, const int32_t* col, int32_t n, const int32_t* order,
                            int32_t* color) {
  if (!row_ptr || !color || n < 1) return -1;
  int32_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] - row_ptr[v] > maxdeg) maxdeg = row_ptr[v + 1] - row_ptr[v];
  /* mark[c] == v + 1 means colour c is taken by a neighbour of v */
  int32_t* mark = (int32_t*)calloc((size_t)maxdeg + 2, sizeof(int32_t));
  if (!mark) return -1;
  for (int32_t v = 0; v < n; ++v) color[v] = -1;
  int32_t ncolors = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t v = order ? order[i] : i;
    if (v < 0 || v >= n) {
      free(mark);
      return -1;
    }
    for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
      int32_t c = color[col[k]];
      if (c >= 0 && c <= maxdeg) mark[c] = v + 1;
    }
    int32_t c = 0;
    while (mark[c] == v + 1) c++;
    color[v] = c;
    if (c + 1 > ncolors) ncolors = c + 1;
  }
  free(mark);
  return ncolors;
}

/* Returns 0 if color[] is a proper colouring with 0 <= color[v] <= deg(v) for every v;
 * 1 if an edge has equal colours, 2 if a colour is out of the first-fit range, 3 if a vertex is
 * uncoloured (negative).  *bad_vertex gets the offending vertex.  *num_colors (if given) gets
 * max colour + 1. */
int oracle_check_coloring(const int32_t* row_ptr, const int32_t* col, int32_t n, const int32_t* color,
                          int32_t* bad_vertex, int32_t* num_colors) {
  int32_t dummy;
  if (!bad_vertex) bad_vertex = &dummy;
  *bad_vertex = -1;
  if (!row_ptr || !color || n < 1) return -1;
  int32_t mx = -1;
  for (int32_t v = 0; v < n; ++v) {
    int32_t c = color[v];
    if (c < 0) {
      *bad_vertex = v;
      return 3;
    }
    if (c > row_ptr[v + 1] - row_ptr[v]) {
      *bad_vertex = v;
      return 2;
    }
    if (c > mx) mx = c;
    for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k)
      if (color[col[k]] == c && col[k] != v) {
        *bad_vertex = v;
        return 1;
      }
  }
  if (num_colors) *num_colors = mx + 1;
  return 0;
}
