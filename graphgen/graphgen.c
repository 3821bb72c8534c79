/*
 * graphgen.c -- seeded synthetic input graphs shared by the oracle and the CUDA path.
 *
 * This file holds no arithmetic of the scheduling method or of its three applications; it only
 * produces inputs:
 *   - RMAT graphs (recursive-matrix edge sampling with quadrant probabilities a, b, c, d),
 *   - 2-D 4-neighbour grids in row-major vertex order,
 *   - optional uniform deletion of a fraction of the undirected edges (seeded partial
 *     Fisher-Yates over the canonical edge list),
 *   - int32 CSR assembly: symmetrised, self-loops and duplicates removed, rows sorted,
 *   - a copy of a graph under a seeded uniform random relabelling of its vertices.
 *
 * Randomness is counter-based: value i of stream s under seed k is SplitMix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to a per-stream
 * base plus i times the golden-ratio increment.  Every value depends only on (k, s, i), so the
 * output is identical for any thread count and on any host architecture.
 *
 * The workload shapes stand in for the paper's SuiteSparse inputs (Section 6.2, Table 2): RMAT for
 * the scale-free graphs, the grid with deletions for the mesh-like road networks.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_OK 0
#define GG_ERR_ARG -1
#define GG_ERR_OOM -2
#define GG_ERR_TOO_BIG -3

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Base of stream s under seed k. */
static inline uint64_t stream_base(uint64_t seed, uint64_t stream) {
  return mix64(mix64(seed + GOLDEN) ^ (stream * 0xD1B54A32D192ED03ULL));
}

/* Value i of a stream: SplitMix64 output for counter i. */
static inline uint64_t stream_at(uint64_t base, uint64_t i) { return mix64(base + (i + 1) * GOLDEN); }

/* Uniform integer in [0, range) by the multiply-high method (Lemire 2019, without the rejection
 * step; the bias is below range / 2^64). */
static inline uint64_t below(uint64_t r, uint64_t range) {
  return (uint64_t)(((unsigned __int128)r * range) >> 64);
}

enum { STREAM_RMAT = 1, STREAM_DELETE = 2, STREAM_SOURCES = 3, STREAM_RELABEL = 4 };

/* ---------------------------------------------------------------- parallel for */

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct {
  range_fn fn;
  void* ctx;
  int64_t n, chunk;
  int64_t next;
  pthread_mutex_t mu;
} pfor_t;

static void* pfor_worker(void* p) {
  pfor_t* s = (pfor_t*)p;
  for (;;) {
    pthread_mutex_lock(&s->mu);
    int64_t lo = s->next;
    s->next += s->chunk;
    pthread_mutex_unlock(&s->mu);
    if (lo >= s->n) break;
    int64_t hi = lo + s->chunk < s->n ? lo + s->chunk : s->n;
    s->fn(s->ctx, lo, hi);
  }
  return NULL;
}

static void parallel_for(int nthreads, int64_t n, int64_t chunk, range_fn fn, void* ctx) {
  if (n <= 0) return;
  if (nthreads <= 1 || n <= chunk) {
    fn(ctx, 0, n);
    return;
  }
  if (nthreads > 64) nthreads = 64;
  pfor_t s;
  s.fn = fn;
  s.ctx = ctx;
  s.n = n;
  s.chunk = chunk;
  s.next = 0;
  pthread_mutex_init(&s.mu, NULL);
  pthread_t th[64];
  int started = 0;
  for (int t = 0; t < nthreads; ++t)
    if (pthread_create(&th[t], NULL, pfor_worker, &s) == 0) started++;
    else break;
  if (started == 0) pfor_worker(&s);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&s.mu);
}

/* ---------------------------------------------------------------- result handle */

typedef struct {
  int32_t n;
  int64_t nnz;
  int32_t* row_ptr; /* n + 1 */
  int32_t* col;     /* nnz */
} gg_graph;

void gg_destroy(gg_graph* g) {
  if (!g) return;
  free(g->row_ptr);
  free(g->col);
  free(g);
}

int32_t gg_num_vertices(const gg_graph* g) { return g ? g->n : -1; }
int64_t gg_num_entries(const gg_graph* g) { return g ? g->nnz : -1; }

/* Copies the CSR out into caller buffers of n + 1 and nnz int32 entries. */
int gg_copy_out(const gg_graph* g, int32_t* row_ptr, int32_t* col) {
  if (!g || !row_ptr || (g->nnz > 0 && !col)) return GG_ERR_ARG;
  memcpy(row_ptr, g->row_ptr, sizeof(int32_t) * ((size_t)g->n + 1));
  if (g->nnz) memcpy(col, g->col, sizeof(int32_t) * (size_t)g->nnz);
  return GG_OK;
}

/* ---------------------------------------------------------------- CSR assembly */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

typedef struct {
  const int32_t* rp;
  int32_t* col;
  int32_t* newdeg;
} sortdedup_ctx;

static void sortdedup_rows(void* p, int64_t lo, int64_t hi) {
  sortdedup_ctx* c = (sortdedup_ctx*)p;
  for (int64_t v = lo; v < hi; ++v) {
    int32_t* row = c->col + c->rp[v];
    int64_t len = (int64_t)c->rp[v + 1] - c->rp[v];
    if (len > 1) qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t w = 0;
    for (int64_t i = 0; i < len; ++i)
      if (w == 0 || row[i] != row[w - 1]) row[w++] = row[i];
    c->newdeg[v] = (int32_t)w;
  }
}

typedef struct {
  const int32_t* oldrp;
  const int32_t* oldcol;
  const int64_t* newrp;
  int32_t* newcol;
} compact_ctx;

static void compact_rows(void* p, int64_t lo, int64_t hi) {
  compact_ctx* c = (compact_ctx*)p;
  for (int64_t v = lo; v < hi; ++v) {
    int64_t len = c->newrp[v + 1] - c->newrp[v];
    if (len) memcpy(c->newcol + c->newrp[v], c->oldcol + c->oldrp[v], sizeof(int32_t) * (size_t)len);
  }
}

/* Builds a symmetric CSR from m undirected pairs (u[i], v[i]): both directions are inserted,
 * self-loops dropped, duplicate entries removed, rows sorted ascending. */
static int build_symmetric_csr(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, int nthreads,
                               gg_graph** out) {
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return GG_ERR_OOM;
  for (int64_t i = 0; i < m; ++i) {
    if (eu[i] == ev[i]) continue;
    cnt[eu[i] + 1]++;
    cnt[ev[i] + 1]++;
  }
  for (int32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
  int64_t total = cnt[n];
  if (total > INT32_MAX) {
    free(cnt);
    return GG_ERR_TOO_BIG;
  }
  int32_t* rp = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(total ? total : 1));
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!rp || !col || !pos) {
    free(cnt), free(rp), free(col), free(pos);
    return GG_ERR_OOM;
  }
  for (int32_t v = 0; v <= n; ++v) {
    rp[v] = (int32_t)cnt[v];
    pos[v] = cnt[v];
  }
  free(cnt);
  for (int64_t i = 0; i < m; ++i) {
    int32_t a = eu[i], b = ev[i];
    if (a == b) continue;
    col[pos[a]++] = b;
    col[pos[b]++] = a;
  }
  free(pos);
  int32_t* newdeg = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!newdeg) {
    free(rp), free(col);
    return GG_ERR_OOM;
  }
  sortdedup_ctx sc = {rp, col, newdeg};
  parallel_for(nthreads, n, 4096, sortdedup_rows, &sc);
  int64_t* nrp = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!nrp) {
    free(rp), free(col), free(newdeg);
    return GG_ERR_OOM;
  }
  nrp[0] = 0;
  for (int32_t v = 0; v < n; ++v) nrp[v + 1] = nrp[v] + newdeg[v];
  free(newdeg);
  int64_t nnz = nrp[n];
  int32_t* ncol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
  if (!ncol) {
    free(rp), free(col), free(nrp);
    return GG_ERR_OOM;
  }
  compact_ctx cc = {rp, col, nrp, ncol};
  parallel_for(nthreads, n, 4096, compact_rows, &cc);
  for (int32_t v = 0; v <= n; ++v) rp[v] = (int32_t)nrp[v];
  free(nrp);
  free(col);
  gg_graph* g = (gg_graph*)calloc(1, sizeof(gg_graph));
  if (!g) {
    free(rp), free(ncol);
    return GG_ERR_OOM;
  }
  g->n = n;
  g->nnz = nnz;
  g->row_ptr = rp;
  g->col = ncol;
  *out = g;
  return GG_OK;
}

/* Removes floor(frac * E) of the E undirected edges {u < v} of g, chosen by a seeded partial
 * Fisher-Yates shuffle of the edges in canonical (CSR, u ascending then v ascending) order, and
 * rebuilds the CSR. */
static int delete_fraction(gg_graph** gp, double frac, uint64_t seed, int nthreads) {
  gg_graph* g = *gp;
  if (frac <= 0.0) return GG_OK;
  int64_t E = 0;
  for (int32_t u = 0; u < g->n; ++u)
    for (int32_t k = g->row_ptr[u]; k < g->row_ptr[u + 1]; ++k)
      if (g->col[k] > u) E++;
  int64_t kdel = (int64_t)(frac * (double)E);
  if (kdel <= 0) return GG_OK;
  int32_t* eu = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E ? E : 1));
  int32_t* ev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E ? E : 1));
  int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(E ? E : 1));
  unsigned char* dead = (unsigned char*)calloc((size_t)(E ? E : 1), 1);
  if (!eu || !ev || !idx || !dead) {
    free(eu), free(ev), free(idx), free(dead);
    return GG_ERR_OOM;
  }
  int64_t e = 0;
  for (int32_t u = 0; u < g->n; ++u)
    for (int32_t k = g->row_ptr[u]; k < g->row_ptr[u + 1]; ++k)
      if (g->col[k] > u) {
        eu[e] = u;
        ev[e] = g->col[k];
        e++;
      }
  for (int64_t i = 0; i < E; ++i) idx[i] = i;
  uint64_t base = stream_base(seed, STREAM_DELETE);
  for (int64_t i = 0; i < kdel; ++i) {
    int64_t j = i + (int64_t)below(stream_at(base, (uint64_t)i), (uint64_t)(E - i));
    int64_t t = idx[i];
    idx[i] = idx[j];
    idx[j] = t;
    dead[idx[i]] = 1;
  }
  free(idx);
  int64_t w = 0;
  for (int64_t i = 0; i < E; ++i)
    if (!dead[i]) {
      eu[w] = eu[i];
      ev[w] = ev[i];
      w++;
    }
  free(dead);
  gg_graph* ng = NULL;
  int rc = build_symmetric_csr(g->n, w, eu, ev, nthreads, &ng);
  free(eu), free(ev);
  if (rc != GG_OK) return rc;
  gg_destroy(g);
  *gp = ng;
  return GG_OK;
}

/* ---------------------------------------------------------------- RMAT */

typedef struct {
  int scale;
  double a, ab, abc;
  uint64_t base;
  int32_t* eu;
  int32_t* ev;
} rmat_ctx;

static void rmat_edges(void* p, int64_t lo, int64_t hi) {
  rmat_ctx* c = (rmat_ctx*)p;
  const double inv53 = 1.0 / 9007199254740992.0;
  for (int64_t e = lo; e < hi; ++e) {
    uint32_t u = 0, v = 0;
    uint64_t ctr = (uint64_t)e * (uint64_t)c->scale;
    for (int l = 0; l < c->scale; ++l) {
      double r = (double)(stream_at(c->base, ctr + (uint64_t)l) >> 11) * inv53;
      uint32_t bu, bv;
      if (r < c->a) bu = 0, bv = 0;
      else if (r < c->ab) bu = 0, bv = 1;
      else if (r < c->abc) bu = 1, bv = 0;
      else bu = 1, bv = 1;
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    c->eu[e] = (int32_t)u;
    c->ev[e] = (int32_t)v;
  }
}

/* RMAT graph with 2^scale vertices and edge_factor * 2^scale sampled edges.  Quadrant
 * probabilities a, b, c and d = 1 - a - b - c are applied independently at every level (no noise,
 * no label permutation).  The samples are symmetrised, self-loops and duplicates are removed, and
 * then floor(delete_frac * E) of the E remaining undirected edges are deleted. */
int gg_rmat(int scale, int edge_factor, double a, double b, double c, uint64_t seed, double delete_frac,
            int nthreads, gg_graph** out) {
  if (!out || scale < 1 || scale > 30 || edge_factor < 1 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0 ||
      delete_frac < 0 || delete_frac >= 1)
    return GG_ERR_ARG;
  *out = NULL;
  int32_t n = (int32_t)1 << scale;
  int64_t m = (int64_t)edge_factor << scale;
  if (2 * m > INT32_MAX) return GG_ERR_TOO_BIG;
  int32_t* eu = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int32_t* ev = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  if (!eu || !ev) {
    free(eu), free(ev);
    return GG_ERR_OOM;
  }
  rmat_ctx rc = {scale, a, a + b, a + b + c, stream_base(seed, STREAM_RMAT), eu, ev};
  parallel_for(nthreads, m, 1 << 16, rmat_edges, &rc);
  gg_graph* g = NULL;
  int r = build_symmetric_csr(n, m, eu, ev, nthreads, &g);
  free(eu), free(ev);
  if (r != GG_OK) return r;
  r = delete_fraction(&g, delete_frac, seed, nthreads);
  if (r != GG_OK) {
    gg_destroy(g);
    return r;
  }
  *out = g;
  return GG_OK;
}

/* ---------------------------------------------------------------- grid */

/* width x height 4-neighbour grid; vertex (r, c) has id r * width + c.  Edge e enumerates the
 * horizontal edges row by row, then the vertical edges row by row; floor(delete_frac * E) of them
 * are deleted. */
int gg_grid(int32_t width, int32_t height, double delete_frac, uint64_t seed, int nthreads, gg_graph** out) {
  if (!out || width < 1 || height < 1 || delete_frac < 0 || delete_frac >= 1) return GG_ERR_ARG;
  *out = NULL;
  int64_t n64 = (int64_t)width * height;
  if (n64 > INT32_MAX / 4) return GG_ERR_TOO_BIG;
  int32_t n = (int32_t)n64;
  int64_t eh = (int64_t)height * (width - 1), evv = (int64_t)(height - 1) * width, E = eh + evv;
  int32_t* eu = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E ? E : 1));
  int32_t* ev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E ? E : 1));
  if (!eu || !ev) {
    free(eu), free(ev);
    return GG_ERR_OOM;
  }
  int64_t e = 0;
  for (int32_t r = 0; r < height; ++r)
    for (int32_t c = 0; c + 1 < width; ++c, ++e) {
      eu[e] = r * width + c;
      ev[e] = r * width + c + 1;
    }
  for (int32_t r = 0; r + 1 < height; ++r)
    for (int32_t c = 0; c < width; ++c, ++e) {
      eu[e] = r * width + c;
      ev[e] = (r + 1) * width + c;
    }
  gg_graph* g = NULL;
  int rc = build_symmetric_csr(n, E, eu, ev, nthreads, &g);
  free(eu), free(ev);
  if (rc != GG_OK) return rc;
  rc = delete_fraction(&g, delete_frac, seed, nthreads);
  if (rc != GG_OK) {
    gg_destroy(g);
    return rc;
  }
  *out = g;
  return GG_OK;
}

/* Builds a symmetric CSR from caller-given undirected pairs (used for small hand-made graphs). */
int gg_from_edges(int32_t n, int64_t m, const int32_t* eu, const int32_t* ev, gg_graph** out) {
  if (!out || n < 0 || m < 0 || (m > 0 && (!eu || !ev))) return GG_ERR_ARG;
  for (int64_t i = 0; i < m; ++i)
    if (eu[i] < 0 || eu[i] >= n || ev[i] < 0 || ev[i] >= n) return GG_ERR_ARG;
  return build_symmetric_csr(n, m, eu, ev, 1, out);
}

/* k distinct-not-required sources drawn uniformly from the vertices with nonzero degree. */
int gg_sources(const int32_t* row_ptr, int32_t n, int32_t k, uint64_t seed, int32_t* out) {
  if (!row_ptr || !out || n < 1 || k < 0) return GG_ERR_ARG;
  int64_t nz = 0;
  for (int32_t v = 0; v < n; ++v) nz += row_ptr[v + 1] > row_ptr[v];
  if (nz == 0) return GG_ERR_ARG;
  int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)nz);
  if (!cand) return GG_ERR_OOM;
  int64_t w = 0;
  for (int32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] > row_ptr[v]) cand[w++] = v;
  uint64_t base = stream_base(seed, STREAM_SOURCES);
  for (int32_t i = 0; i < k; ++i) out[i] = cand[below(stream_at(base, (uint64_t)i), (uint64_t)nz)];
  free(cand);
  return GG_OK;
}

/* Raw access to the counter-based stream, for inputs drawn on the Python side (graph sizes of a
 * batched mix, arrival times of a request stream). */
uint64_t gg_stream_u64(uint64_t seed, uint64_t stream, uint64_t i) { return stream_at(stream_base(seed, stream), i); }

/* ---------------------------------------------------------------- random relabelling */

typedef struct {
  const int32_t* rp;
  const int32_t* col;
  const int32_t* perm;
  const int32_t* newrp;
  int32_t* newcol;
} relabel_ctx;

static void relabel_rows(void* p, int64_t lo, int64_t hi) {
  relabel_ctx* c = (relabel_ctx*)p;
  for (int64_t v = lo; v < hi; ++v) {
    int32_t* dst = c->newcol + c->newrp[c->perm[v]];
    for (int64_t k = c->rp[v]; k < c->rp[v + 1]; ++k) *dst++ = c->perm[c->col[k]];
  }
}

/* Copy of the CSR (row_ptr, col) in which vertex v is renamed perm[v], perm a uniform random
 * permutation of 0..n-1 (Fisher-Yates driven by the counter-based stream), rows sorted again.
 * perm_out (n entries, may be NULL) receives the permutation. */
int gg_relabel(const int32_t* row_ptr, const int32_t* col, int32_t n, uint64_t seed, int nthreads, int32_t* perm_out,
               gg_graph** out) {
  if (!row_ptr || !out || n < 0 || row_ptr[0] != 0) return GG_ERR_ARG;
  const int64_t nnz = row_ptr[n];
  if (nnz > 0 && !col) return GG_ERR_ARG;
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  gg_graph* g = (gg_graph*)calloc(1, sizeof(gg_graph));
  if (g) {
    g->row_ptr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    g->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
  }
  if (!perm || !g || !g->row_ptr || !g->col) {
    free(perm);
    gg_destroy(g);
    return GG_ERR_OOM;
  }
  g->n = n;
  g->nnz = nnz;
  for (int32_t v = 0; v < n; ++v) perm[v] = v;
  const uint64_t base = stream_base(seed, STREAM_RELABEL);
  for (int64_t i = (int64_t)n - 1; i > 0; --i) {
    const int64_t j = (int64_t)below(stream_at(base, (uint64_t)i), (uint64_t)i + 1);
    const int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
  /* new row perm[v] has the length of old row v */
  for (int32_t v = 0; v < n; ++v) g->row_ptr[perm[v] + 1] = row_ptr[v + 1] - row_ptr[v];
  g->row_ptr[0] = 0;
  for (int32_t v = 0; v < n; ++v) g->row_ptr[v + 1] += g->row_ptr[v];
  relabel_ctx rc = {row_ptr, col, perm, g->row_ptr, g->col};
  parallel_for(nthreads, n, 4096, relabel_rows, &rc);
  int32_t* deg = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!deg) {
    free(perm);
    gg_destroy(g);
    return GG_ERR_OOM;
  }
  sortdedup_ctx sc = {g->row_ptr, g->col, deg};
  parallel_for(nthreads, n, 4096, sortdedup_rows, &sc);  /* no duplicates: only sorts */
  free(deg);
  if (perm_out) memcpy(perm_out, perm, sizeof(int32_t) * (size_t)n);
  free(perm);
  *out = g;
  return GG_OK;
}
