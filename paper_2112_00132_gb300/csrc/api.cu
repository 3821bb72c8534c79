// api.cu -- the C ABI (include/atos.h): argument checks, graph objects, scratch memory, and the
// host side of the persistent / discrete scheduling loops.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "atos.h"
#include "bsp.cuh"
#include "engine.cuh"
#include "launch.cuh"
#include "state.cuh"

namespace atos {
const void* pr_persistent_kernel(int worker);
const void* pr_discrete_kernel(int worker);
const void* gc_persistent_kernel(int worker);
const void* gc_discrete_kernel(int worker);
cudaError_t pr_verify_sweep(Instance* d_insts, int ninst, int max_n, DevCtl* d_ctl, cudaStream_t s);
cudaError_t pr_finish(Instance* d_insts, int ninst, int n, int64_t nnz, DevCtl* d_ctl, double* certificate_y,
                      double exact_sum, cudaStream_t s);
cudaError_t gc_finish(const Instance* h_inst, DevCtl* d_ctl, cudaStream_t s);
cudaError_t gc_split_build(const int32_t* row_ptr, const int32_t* col, int n, int32_t* mid, int32_t* scol,
                           int32_t* long_rows, int* long_count, cudaStream_t s);
cudaError_t gc_wait_init(const int32_t* mid, int n, int32_t* wait, cudaStream_t s);
int64_t gc_bitmap_scratch(int n);
cudaError_t gc_tail_segments(const int32_t* row_ptr, const int32_t* mid, int n, void* scratch, uint64_t* count,
                             cudaStream_t s);
uint64_t gc_tail_slack();
cudaError_t gc_bitmap_build(const int32_t* mid, int n, int2* fw, int32_t* scratch, uint32_t* total_words,
                            cudaStream_t s);
size_t spread_build_scratch_bytes(int32_t n);
cudaError_t spread_build(const int32_t* rp, const int32_t* col, int32_t n, int32_t* perm, int32_t* new_rp,
                         int32_t* new_col, int32_t* bsums, void* scratch, int32_t* h_hubs, HubMap* h_map,
                         cudaStream_t s);
cudaError_t unspread_f32(const float* src, float* dst, int32_t n, const int32_t* perm, cudaStream_t s);
cudaError_t unspread_i32(const int32_t* src, int32_t* dst, int32_t n, const int32_t* perm, cudaStream_t s);
unsigned long long launches_so_far();
}  // namespace atos

using namespace atos;

namespace {

constexpr int64_t kDefaultSpinNs = 4000000000LL;

uint32_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p > 0x80000000ULL ? 0 : (uint32_t)p;
}

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return ATOS_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? ATOS_ERR_OOM : ATOS_ERR_CUDA;
}

#define ATOS_TRY(expr)                          \
  do {                                          \
    int _rc = from_cuda(expr);                  \
    if (_rc != ATOS_OK) return _rc;             \
  } while (0)

template <class T>
cudaError_t dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return pool_malloc((void**)p, count * sizeof(T));
}

// Scratch owned by a graph: instance table, queue control blocks, rings, statistics and the
// device control block, grown on demand and reused by later calls.
struct Scratch {
  int ninst = 0;     // instances the arrays hold
  uint32_t cap = 0;  // ring slots per instance
  Instance* d_insts = nullptr;
  Instance* h_insts = nullptr;  // pinned
  QueueCtl* d_qctl = nullptr;
  unsigned long long* d_ring = nullptr;
  unsigned long long* d_stats = nullptr;
  unsigned long long* h_stats = nullptr;  // pinned
  DevCtl* d_ctl = nullptr;
  DevCtl* h_ctl = nullptr;  // pinned
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, upload_done = nullptr;
  bool upload_pending = false;

  void release() {
    pool_free(d_insts), pool_free_host(h_insts), pool_free(d_qctl), pool_free(d_ring);
    pool_free(d_stats), pool_free_host(h_stats), pool_free(d_ctl), pool_free_host(h_ctl);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (upload_done) cudaEventDestroy(upload_done);
    *this = Scratch();
  }
};

}  // namespace

struct atos_graph_s {
  int32_t n = 0;
  int64_t nnz = 0;
  int32_t max_degree = 0;
  int32_t n_isolated = 0;
  int32_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  bool owned = true;
  Scratch s;
  // application state that is not a caller output
  float* d_res = nullptr;
  uint32_t* d_qbits = nullptr;
  double* d_cert = nullptr;  // PageRank FP64 certificate scratch (n entries)
  void* d_bsp = nullptr;  // BSP comparator frontiers, scan space and control block
  size_t bsp_bytes = 0;
  void* h_bsp = nullptr;  // pinned: the BSP control block's upload image and read-back
  BspGraphs bsp_graphs;   // the device-loop graphs of the BSP comparator
  // the spread-id copy (ATOS_FLAG_SPREAD_IDS): CSR with vertex v renamed perm[v] (the
  // highest-degree vertices first, the rest spread over the id range), and an n-entry output
  // buffer in the copy's ids
  int32_t* sp_row_ptr = nullptr;
  int32_t* sp_col = nullptr;
  int32_t* sp_perm = nullptr;  // v -> the copy's id of v
  void* sp_out = nullptr;
  int32_t sp_hubs = 0;         // hubs of the copy (its highest-degree vertices)
  HubMap sp_hub = {0, 1, 1, 0};  // where they sit
  int32_t* d_expanded = nullptr;  // BFS: per source, the smallest depth each vertex was expanded at
  int4* d_segs = nullptr;         // BFS row splitting: per source, a segment table of seg_cap entries
  size_t seg_rows = 0;
  uint32_t seg_cap = 0;
  int32_t* d_gc_wait = nullptr;   // dependency-ordered colouring: per vertex, counts still to go
  // dependency-ordered colouring: per layout (input ids, spread-id copy), the rows with the
  // smaller-id neighbours first (gc_col) and how many they are (gc_mid); built on first use
  int32_t* gc_mid[2] = {nullptr, nullptr};
  int32_t* gc_col[2] = {nullptr, nullptr};
  int2* gc_fw[2] = {nullptr, nullptr};      // pushed colours: each vertex's bitmap (first word, words)
  uint32_t gc_fwords[2] = {0, 0};           // bitmap words of each layout
  unsigned* d_gc_forbid = nullptr;          // the bitmaps (gc_forbid_cap words)
  uint64_t gc_tails[2] = {0, 0};            // tail segments a run can create, per layout
  int4* d_gc_segs = nullptr;                // the tail-segment table (gc_segs_cap entries)
  uint64_t gc_segs_cap = 0;
  uint32_t gc_forbid_cap = 0;
  size_t expanded_rows = 0;
  unsigned long long* d_timeline = nullptr;  // throughput timeline (atos_timeline), 2 counters per bucket
  int64_t tl_bucket_ns = 0;
  int32_t tl_nbuckets = 0;
};

namespace {

// Builds the spread-id copy of g on `st` the first time it is needed (the build synchronises
// `st` once, to learn the size of the hub region).
int ensure_spread(atos_graph_s* g, cudaStream_t st) {
  if (g->sp_row_ptr) return ATOS_OK;
  const int32_t n = g->n;
  int32_t *bsums = nullptr, *rp = nullptr, *col = nullptr, *perm = nullptr;
  void *out = nullptr, *tmp = nullptr;
  int rc = from_cuda(dev_alloc(&rp, (size_t)n + 1));
  if (!rc) rc = from_cuda(dev_alloc(&perm, (size_t)n));
  if (!rc) rc = from_cuda(dev_alloc(&col, (size_t)std::max<int64_t>(g->nnz, 1)));
  if (!rc) rc = from_cuda(dev_alloc(&bsums, (size_t)n / 1024 + 2));
  if (!rc) rc = from_cuda(pool_malloc(&out, sizeof(int32_t) * std::max<size_t>((size_t)n, 1)));
  if (!rc) rc = from_cuda(pool_malloc(&tmp, spread_build_scratch_bytes(n)));
  int32_t hubs = 0;
  HubMap hm = {0, 1, 1, 0};
  if (!rc) rc = from_cuda(spread_build(g->row_ptr, g->col, n, perm, rp, col, bsums, tmp, &hubs, &hm, st));
  cudaStreamSynchronize(st);  // the build's scratch goes back now; nothing of a failed build may still run
  pool_free(tmp), pool_free(bsums);
  if (rc) {
    pool_free(rp), pool_free(col), pool_free(out), pool_free(perm);
    return rc;
  }
  g->sp_row_ptr = rp, g->sp_col = col, g->sp_out = out, g->sp_perm = perm, g->sp_hubs = hubs, g->sp_hub = hm;
  return ATOS_OK;
}

int ensure_scratch(atos_graph_s* g, int ninst, uint32_t cap) {
  Scratch& s = g->s;
  if (!s.ev0) {
    ATOS_TRY(cudaEventCreate(&s.ev0));
    ATOS_TRY(cudaEventCreate(&s.ev1));
    ATOS_TRY(cudaEventCreateWithFlags(&s.upload_done, cudaEventDisableTiming));
  }
  if (!s.d_ctl) {
    ATOS_TRY(dev_alloc(&s.d_ctl, 1));
    ATOS_TRY(pool_malloc_host((void**)&s.h_ctl, sizeof(DevCtl)));
    DevCtl init;
    memset(&init, 0, sizeof(init));
    init.dirty = 1;
    ATOS_TRY(cudaMemcpy(s.d_ctl, &init, sizeof(init), cudaMemcpyHostToDevice));
  }
  if (s.upload_pending) {
    cudaEventSynchronize(s.upload_done);
    s.upload_pending = false;
  }
  if (ninst <= s.ninst && cap == s.cap) return ATOS_OK;
  // (re)allocate; the device must be idle with respect to the old buffers
  cudaDeviceSynchronize();
  pool_free(s.d_insts), pool_free_host(s.h_insts), pool_free(s.d_qctl), pool_free(s.d_ring);
  pool_free(s.d_stats), pool_free_host(s.h_stats);
  s.d_insts = nullptr, s.h_insts = nullptr, s.d_qctl = nullptr, s.d_ring = nullptr;
  s.d_stats = nullptr, s.h_stats = nullptr;
  const int m = std::max(ninst, s.ninst);
  s.ninst = 0;
  s.cap = 0;
  ATOS_TRY(dev_alloc(&s.d_insts, m));
  ATOS_TRY(pool_malloc_host((void**)&s.h_insts, sizeof(Instance) * m));
  ATOS_TRY(dev_alloc(&s.d_qctl, m));
  ATOS_TRY(dev_alloc(&s.d_ring, (size_t)cap * m));
  ATOS_TRY(dev_alloc(&s.d_stats, (size_t)kNumStats * m));
  ATOS_TRY(pool_malloc_host((void**)&s.h_stats, sizeof(unsigned long long) * kNumStats * m));
  s.ninst = m;
  s.cap = cap;
  // fresh rings hold garbage: mark dirty so the next prepare fills them with EMPTY
  int one = 1;
  ATOS_TRY(cudaMemcpy(&s.d_ctl->dirty, &one, sizeof(int), cudaMemcpyHostToDevice));
  return ATOS_OK;
}

// Ring slots per instance.  Besides the tasks in flight the ring must cover the span between the
// oldest ticket a busy worker has not taken yet and the tail, so small graphs get a floor of 2^20
// slots (8 MiB); large ones 1.5 n plus the virtual prefix.
// BSP comparator scratch: frontiers, scan offsets, control block, grown on demand.
int ensure_bsp(atos_graph_s* g, size_t bytes) {
  if (!g->s.ev0) {
    int rc = ensure_scratch(g, 1, 1024);
    if (rc) return rc;
  }
  if (!g->h_bsp) ATOS_TRY(pool_malloc_host(&g->h_bsp, bsp_host_bytes()));
  if (g->bsp_bytes >= bytes) return ATOS_OK;
  cudaDeviceSynchronize();
  g->bsp_graphs.release();  // the graphs name the old control block
  pool_free(g->d_bsp);
  g->d_bsp = nullptr;
  g->bsp_bytes = 0;
  ATOS_TRY(pool_malloc(&g->d_bsp, bytes));
  g->bsp_bytes = bytes;
  return ATOS_OK;
}

// One BSP run on g's comparator scratch; accumulates into *acc.
int run_bsp(atos_graph_s* g, const BspRun& r, cudaStream_t st, BspResult* acc) {
  int rc = ensure_bsp(g, bsp_scratch_bytes(r.app, r.n, r.nnz, r.nsrc));
  if (rc) return rc;
  BspResult one = {};
  rc = bsp_run(r, g->d_bsp, g->bsp_bytes, g->h_bsp, &g->bsp_graphs, st, acc ? &one : nullptr);
  if (rc) return rc;
  if (acc) {
    acc->iters += one.iters, acc->edges += one.edges, acc->tasks += one.tasks;
    if (!acc->status) acc->status = one.status;
  }
  return ATOS_OK;
}

uint32_t ring_capacity(const atos_config& cfg, int32_t n, uint32_t prefix) {
  if (cfg.queue_capacity > 0) return next_pow2(std::max<uint64_t>((uint64_t)cfg.queue_capacity, 1024));
  const uint64_t want = (uint64_t)n + (uint64_t)n / 2 + prefix + 1024;
  return next_pow2(std::max<uint64_t>(want, 1u << 20));
}

// ATOS_FLAG_USE_TUNED: the configuration cached by the autotuner for g's class, if any.
void apply_tuned(atos_graph_t g, int32_t app, atos_config* cfg) {
  if (!(cfg->flags & ATOS_FLAG_USE_TUNED)) return;
  atos_config t;
  if (atos_tuned_config(g, app, &t) == ATOS_OK) *cfg = t;
  cfg->flags &= ~ATOS_FLAG_USE_TUNED;
}

int check_config(const atos_config& c) {
  if (!worker_supported(c.worker_size)) return ATOS_ERR_UNSUPPORTED;
  if (c.fetch_size < 1 || c.fetch_size > 1024) return ATOS_ERR_INVALID_ARG;
  if (c.fetch_size > (warp_hosted(c.worker_size) ? 32 : c.worker_size)) return ATOS_ERR_INVALID_ARG;
  if (c.strategy < ATOS_PERSISTENT || c.strategy > ATOS_BSP) return ATOS_ERR_INVALID_ARG;
  if (c.fetch_policy < ATOS_FETCH_FIXED || c.fetch_policy > ATOS_FETCH_SPREAD) return ATOS_ERR_INVALID_ARG;
  if (c.num_blocks < 0 || c.check_size < 0 || c.window < 0 || c.queue_capacity < 0 || c.spin_limit_ns < 0)
    return ATOS_ERR_INVALID_ARG;
  if (c.flags & ~(ATOS_FLAG_PHANTOM_TASK | ATOS_FLAG_PR_CROSSING | ATOS_FLAG_SPREAD_IDS | ATOS_FLAG_USE_TUNED |
                  ATOS_FLAG_GC_ORDERED | ATOS_FLAG_BFS_EXPAND_ONCE | ATOS_FLAG_BSP_DEVICE_LOOP |
                  ATOS_FLAG_BSP_PER_SOURCE | ATOS_FLAG_GC_DEPENDENCY | ATOS_FLAG_BFS_SPLIT_ROWS))
    return ATOS_ERR_INVALID_ARG;
  return ATOS_OK;
}

void default_config(atos_config* c) {
  memset(c, 0, sizeof(*c));
  c->worker_size = 256;
  c->fetch_size = 256;
  c->strategy = ATOS_PERSISTENT;
  c->fetch_policy = ATOS_FETCH_SPREAD;
  c->num_blocks = 0;
  c->check_size = 32;
  c->window = 0;
  c->queue_capacity = 0;
  c->spin_limit_ns = 0;
}

// Uploads the instance table (from pinned memory, so the copy is asynchronous; the next call
// waits for it before rewriting the table).
int upload_instances(Scratch& s, int ninst, cudaStream_t st) {
  ATOS_TRY(cudaMemcpyAsync(s.d_insts, s.h_insts, sizeof(Instance) * ninst, cudaMemcpyHostToDevice, st));
  ATOS_TRY(cudaEventRecord(s.upload_done, st));
  s.upload_pending = true;
  return ATOS_OK;
}

// The BSP strategy records no timeline: clear it, so a read after such a call shows nothing.
int clear_timeline(atos_graph_s* g, cudaStream_t st) {
  if (g->d_timeline && g->tl_nbuckets > 0)
    ATOS_TRY(cudaMemsetAsync(g->d_timeline, 0, sizeof(unsigned long long) * 2 * g->tl_nbuckets, st));
  return ATOS_OK;
}

// Runs the scheduling loop over the instances in s.h_insts[0, ninst).  The caller has filled the
// table; `kp` / `kd` are the body's persistent / discrete kernels.
int run_instances(atos_graph_s* g, int ninst, int max_n, const atos_config& cfg, const void* (*kp)(int),
                  const void* (*kd)(int), int app, cudaStream_t st, int64_t* iterations) {
  Scratch& s = g->s;
  const int worker = cfg.worker_size;
  const int threads = block_threads(worker);
  int window = cfg.window > 0 ? std::min(cfg.window, ninst) : ninst;
  Launch L;
  memset(&L, 0, sizeof(L));
  L.insts = s.d_insts;
  L.ninst = ninst;
  L.window = window;
  L.fetch = cfg.fetch_size;
  L.policy = cfg.fetch_policy;
  L.flags = cfg.flags;
  L.status = &s.d_ctl->status;
  L.next_inst = &s.d_ctl->next_inst;
  L.spin_limit_ns = cfg.spin_limit_ns > 0 ? cfg.spin_limit_ns : kDefaultSpinNs;
  L.lifetime_ns = L.spin_limit_ns * 16;
  L.fail_site = &s.d_ctl->fail_site;
  int rc = upload_instances(s, ninst, st);
  if (rc) return rc;
  if (g->d_timeline && g->tl_nbuckets > 0) {
    ATOS_TRY(cudaMemsetAsync(g->d_timeline, 0, sizeof(unsigned long long) * 2 * g->tl_nbuckets, st));
    L.timeline = g->d_timeline;
    L.t_origin = &s.d_ctl->t_origin;
    L.bucket_ns = g->tl_bucket_ns;
    L.nbuckets = g->tl_nbuckets;
  }
  ATOS_TRY(launch_prepare(s.d_insts, ninst, max_n, s.d_ctl, cfg.flags, (unsigned)window, st));
  if (app == kAppPr) ATOS_TRY(launch_pr_init(s.d_insts, ninst, g->nnz, st));
  int64_t iters = 0;
  if (cfg.strategy == ATOS_PERSISTENT) {
    const void* fn = kp(worker);
    if (!fn) return ATOS_ERR_UNSUPPORTED;
    int nb = cfg.num_blocks > 0 ? cfg.num_blocks : resident_blocks(fn, threads);
    if (nb <= 0) return ATOS_ERR_CUDA;
    const int workers_per_block = warp_hosted(worker) ? kWarpBlock / 32 : 1;
    L.nworkers = std::max(1, nb * workers_per_block / window);
    ATOS_TRY(launch_kernel(fn, dim3(nb), threads, L, st));
    iters = 1;
  } else {
    const void* fn = kd(worker);
    if (!fn) return ATOS_ERR_UNSUPPORTED;
    const int per_block = warp_hosted(worker) ? std::min(cfg.fetch_size, 32) * (kWarpBlock / 32) : cfg.fetch_size;
    unsigned gen = 0;
    for (int i = 0; i < ninst; ++i) gen = std::max(gen, s.h_insts[i].prefix_len);
    ATOS_TRY(discrete_loop(fn, threads, per_block, L, s.d_insts, ninst, max_n, gen, app == kAppPr, s.d_ctl, s.h_ctl,
                           st, &iters));
    if (iters > (1 << 24)) return ATOS_ERR_TIMEOUT;
  }
  ATOS_TRY(launch_finalize(s.d_insts, ninst, s.d_ctl, st));
  if (iterations) *iterations = iters;
  return ATOS_OK;
}

// Synchronises and reads back the statistics of a launch over `ninst` instances.
int collect_stats(atos_graph_s* g, int ninst, cudaStream_t st, atos_stats* out) {
  Scratch& s = g->s;
  ATOS_TRY(cudaMemcpyAsync(s.h_stats, s.d_stats, sizeof(unsigned long long) * kNumStats * ninst,
                           cudaMemcpyDeviceToHost, st));
  ATOS_TRY(cudaMemcpyAsync(s.h_ctl, s.d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
  ATOS_TRY(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, s.ev0, s.ev1);
  out->ms = ms;
  out->tasks = out->edges = out->pushes = out->batches = out->idle_polls = 0;
  for (int i = 0; i < ninst; ++i) {
    out->tasks += (int64_t)s.h_stats[i * kNumStats + kStatTasks];
    out->edges += (int64_t)s.h_stats[i * kNumStats + kStatEdges];
    out->pushes += (int64_t)s.h_stats[i * kNumStats + kStatPushes];
    out->batches += (int64_t)s.h_stats[i * kNumStats + kStatBatches];
    out->idle_polls += (int64_t)s.h_stats[i * kNumStats + kStatIdle];
  }
  out->status = s.h_ctl->status;
  return ATOS_OK;
}

Instance base_instance(atos_graph_s* g, int i, int app, uint32_t cap, uint32_t prefix_len, int32_t prefix_item) {
  Scratch& s = g->s;
  Instance I;
  memset(&I, 0, sizeof(I));
  I.row_ptr = g->row_ptr;
  I.col = g->col;
  I.n = g->n;
  I.app = app;
  I.ring = s.d_ring + (size_t)cap * i;
  I.cap = cap;
  I.prefix_len = prefix_len;
  I.prefix_item = prefix_item;
  I.ctl = s.d_qctl + i;
  I.stats = s.d_stats + (size_t)kNumStats * i;
  return I;
}

}  // namespace

namespace atos {
// Device CSR of a graph, for the batch API.
int graph_spread_csr(atos_graph_t g, const int32_t** row_ptr, const int32_t** col, cudaStream_t st,
                     const int32_t** perm, int32_t* hubs, HubMap* hub) {
  if (!g) return ATOS_ERR_INVALID_ARG;
  const int rc = ensure_spread(g, st);
  if (rc) return rc;
  *row_ptr = g->sp_row_ptr;
  *col = g->sp_col;
  if (perm) *perm = g->sp_perm;
  if (hubs) *hubs = g->sp_hubs;
  if (hub) *hub = g->sp_hub;
  return ATOS_OK;
}

int graph_device_csr(atos_graph_t g, const int32_t** row_ptr, const int32_t** col, int32_t* n_isolated) {
  if (!g) return ATOS_ERR_INVALID_ARG;
  *row_ptr = g->row_ptr;
  *col = g->col;
  *n_isolated = g->n_isolated;
  return ATOS_OK;
}
}  // namespace atos

// ============================================================================ C ABI

namespace {
// Device CSR validation: sets *bad when a column index lies outside [0, n).  Reads col only.
__global__ void csr_col_range_kernel(const int32_t* __restrict__ col, int64_t nnz, int32_t n, int* bad) {
  bool out = false;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = col[k];
    out |= c < 0 || c >= n;
  }
  if (__syncthreads_or(out) && threadIdx.x == 0) atomicExch(bad, 1);
}

// Validates a CSR held in device memory: row_ptr (already copied to the host, `hrp`) on the host,
// the column range by a kernel, and symmetry (ATOS_CHECK_SYMMETRIC) on a host copy of col.
int validate_device_csr(const int32_t* hrp, const int32_t* col, int32_t n, int64_t nnz, uint32_t flags,
                        cudaStream_t st) {
  if (hrp[0] != 0 || hrp[n] != nnz) return ATOS_ERR_BAD_CSR;
  for (int32_t v = 0; v < n; ++v)
    if (hrp[v + 1] < hrp[v]) return ATOS_ERR_BAD_CSR;
  if (nnz == 0) return ATOS_OK;
  if (flags & ATOS_CHECK_SYMMETRIC) {
    std::vector<int32_t> hcol((size_t)nnz);
    ATOS_TRY(cudaMemcpyAsync(hcol.data(), col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st));
    ATOS_TRY(cudaStreamSynchronize(st));
    return atos_csr_validate(hrp, hcol.data(), n, nnz, flags);
  }
  int* d_bad = nullptr;
  ATOS_TRY(dev_alloc(&d_bad, 1));
  int h_bad = 0;
  cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = std::min<int64_t>((int64_t)sms * 8, (nnz + 255) / 256);
    count_launches(1);
    csr_col_range_kernel<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, st>>>(col, nnz, n, d_bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  pool_free(d_bad);
  if (e != cudaSuccess) return from_cuda(e);
  return h_bad ? ATOS_ERR_BAD_CSR : ATOS_OK;
}
}  // namespace

extern "C" {

const char* atos_status_string(int status) {
  switch (status) {
    case ATOS_OK: return "ok";
    case ATOS_ERR_INVALID_ARG: return "invalid argument";
    case ATOS_ERR_BAD_CSR: return "malformed CSR graph";
    case ATOS_ERR_OOM: return "device out of memory";
    case ATOS_ERR_QUEUE_OVERFLOW: return "worklist ring overflow";
    case ATOS_ERR_TIMEOUT: return "device wait exceeded its time budget";
    case ATOS_ERR_CUDA: return "CUDA runtime error";
    case ATOS_ERR_UNSUPPORTED: return "unsupported configuration";
    case ATOS_ERR_BUSY: return "no free slot or arena memory for the request now";
    case ATOS_ERR_BOUNDS: return "an index outside its array was caught (bounds-checked build)";
  }
  return "unknown status";
}

const char* atos_version(void) { return "atos-gb300 0.1 (sm_103a)"; }

int atos_queue_config(atos_config* cfg, const char* preset) {
  if (!cfg) return ATOS_ERR_INVALID_ARG;
  default_config(cfg);
  if (!preset || !strcmp(preset, "default") || !strcmp(preset, "persist-cta")) return ATOS_OK;
  if (!strcmp(preset, "persist-warp")) {
    cfg->worker_size = 32;
    cfg->fetch_size = 1;
    cfg->fetch_policy = ATOS_FETCH_FIXED;
    return ATOS_OK;
  }
  if (!strcmp(preset, "discrete-cta")) {
    cfg->strategy = ATOS_DISCRETE;
    return ATOS_OK;
  }
  if (!strcmp(preset, "discrete-warp")) {
    cfg->worker_size = 32;
    cfg->fetch_size = 1;
    cfg->strategy = ATOS_DISCRETE;
    return ATOS_OK;
  }
  if (!strcmp(preset, "bsp")) {
    cfg->strategy = ATOS_BSP;
    return ATOS_OK;
  }
  if (!strcmp(preset, "autotune")) {
    cfg->flags |= ATOS_FLAG_USE_TUNED;
    return ATOS_OK;
  }
  return ATOS_ERR_INVALID_ARG;
}

int atos_csr_validate(const int32_t* row_ptr, const int32_t* col, int32_t n, int64_t nnz, uint32_t flags) {
  if (n < 0 || nnz < 0 || nnz > INT32_MAX || !row_ptr || (nnz > 0 && !col)) return ATOS_ERR_INVALID_ARG;
  if (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz) return ATOS_ERR_BAD_CSR;
  for (int32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return ATOS_ERR_BAD_CSR;
  for (int64_t k = 0; k < nnz; ++k)
    if (col[k] < 0 || col[k] >= n) return ATOS_ERR_BAD_CSR;
  if (flags & ATOS_CHECK_SYMMETRIC) {
    // every (v, w) needs (w, v): count mirrored entries row by row with a per-row cursor
    std::vector<int32_t> cur(row_ptr, row_ptr + n);
    for (int32_t v = 0; v < n; ++v)
      for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
        const int32_t w = col[k];
        bool found = false;
        for (int32_t j = row_ptr[w]; j < row_ptr[w + 1]; ++j)
          if (col[j] == v) {
            found = true;
            break;
          }
        if (!found) return ATOS_ERR_BAD_CSR;
      }
  }
  return ATOS_OK;
}

int atos_graph_create(const int32_t* row_ptr, const int32_t* col, int32_t n, int64_t nnz, uint32_t flags,
                      void* stream, atos_graph_t* out) {
  if (!out) return ATOS_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 0 || nnz < 0 || nnz > INT32_MAX || !row_ptr || (nnz > 0 && !col)) return ATOS_ERR_INVALID_ARG;
  if ((flags & ATOS_BORROW) && !(flags & ATOS_DEVICE_PTRS)) return ATOS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> hrp;
  const int32_t* rp_host = nullptr;
  if (!(flags & ATOS_DEVICE_PTRS)) {
    if (!(flags & ATOS_SKIP_VALIDATION)) {
      int rc = atos_csr_validate(row_ptr, col, n, nnz, flags);
      if (rc) return rc;
    } else if (row_ptr[0] != 0 || row_ptr[n] != nnz) {
      return ATOS_ERR_BAD_CSR;
    }
    rp_host = row_ptr;
  } else {
    hrp.resize((size_t)n + 1);
    ATOS_TRY(cudaMemcpyAsync(hrp.data(), row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    ATOS_TRY(cudaStreamSynchronize(st));
    rp_host = hrp.data();
    if (flags & ATOS_SKIP_VALIDATION) {
      if (rp_host[0] != 0 || rp_host[n] != nnz) return ATOS_ERR_BAD_CSR;
    } else {
      const int rc = validate_device_csr(rp_host, col, n, nnz, flags, st);
      if (rc) return rc;
    }
  }
  atos_graph_s* g = new (std::nothrow) atos_graph_s();
  if (!g) return ATOS_ERR_OOM;
  g->n = n;
  g->nnz = nnz;
  for (int32_t v = 0; v < n; ++v) {
    const int32_t d = rp_host[v + 1] - rp_host[v];
    g->max_degree = std::max(g->max_degree, d);
    g->n_isolated += d == 0;
  }
  int rc = ATOS_OK;
  if (flags & ATOS_BORROW) {
    g->row_ptr = const_cast<int32_t*>(row_ptr);
    g->col = const_cast<int32_t*>(col);
    g->owned = false;
  } else {
    const cudaMemcpyKind kind = (flags & ATOS_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    rc = from_cuda(dev_alloc(&g->row_ptr, (size_t)n + 1));
    if (!rc) rc = from_cuda(dev_alloc(&g->col, (size_t)nnz));
    if (!rc) rc = from_cuda(cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(int32_t) * (n + 1), kind, st));
    if (!rc && nnz) rc = from_cuda(cudaMemcpyAsync(g->col, col, sizeof(int32_t) * nnz, kind, st));
    if (!rc) rc = from_cuda(cudaStreamSynchronize(st));
  }
  if (rc) {
    atos_graph_destroy(g);
    return rc;
  }
  *out = g;
  return ATOS_OK;
}

int atos_graph_destroy(atos_graph_t g) {
  if (!g) return ATOS_OK;
  cudaDeviceSynchronize();
  if (g->owned) pool_free(g->row_ptr), pool_free(g->col);
  g->bsp_graphs.release();
  pool_free(g->d_res), pool_free(g->d_qbits), pool_free(g->d_bsp), pool_free(g->d_cert);
  pool_free_host(g->h_bsp);
  pool_free(g->sp_row_ptr), pool_free(g->sp_col), pool_free(g->sp_out), pool_free(g->sp_perm);
  pool_free(g->d_expanded);
  pool_free(g->d_segs);
  pool_free(g->d_gc_wait);
  for (int k = 0; k < 2; ++k) pool_free(g->gc_mid[k]), pool_free(g->gc_col[k]), pool_free(g->gc_fw[k]);
  pool_free(g->d_gc_forbid);
  pool_free(g->d_gc_segs);
  pool_free(g->d_timeline);
  g->s.release();
  delete g;
  return ATOS_OK;
}

int atos_graph_info(atos_graph_t g, int32_t* n, int64_t* nnz, int32_t* max_degree) {
  if (!g) return ATOS_ERR_INVALID_ARG;
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (max_degree) *max_degree = g->max_degree;
  return ATOS_OK;
}

int atos_bfs(atos_graph_t g, const int32_t* sources, int32_t nsrc, int32_t* depths, const atos_config* cfg_in,
             void* stream, atos_stats* stats) {
  if (!g || !sources || !depths || nsrc < 1 || nsrc > 65535) return ATOS_ERR_INVALID_ARG;
  for (int32_t i = 0; i < nsrc; ++i)
    if (sources[i] < 0 || sources[i] >= g->n) return ATOS_ERR_INVALID_ARG;
  atos_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else default_config(&cfg);
  apply_tuned(g, ATOS_APP_BFS, &cfg);
  int rc = check_config(cfg);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = g->n;
  if (cfg.strategy == ATOS_BSP) {
    // Algorithm 1: the frontiers of a group of sources advance in the same launches, one level at
    // a time (one source after another with ATOS_FLAG_BSP_PER_SOURCE)
    rc = clear_timeline(g, st);
    if (rc) return rc;
    // sources advance together in groups of cfg.window (0: as many as keep their depth arrays
    // within about half of L2, as for the persistent strategy)
    int32_t group = nsrc;
    if (cfg.flags & ATOS_FLAG_BSP_PER_SOURCE) group = 1;
    else if (cfg.window > 0) group = std::min(cfg.window, nsrc);
    else group = (int32_t)std::max<int64_t>(1, std::min<int64_t>(nsrc, (64LL << 20) / (4 * n + 1)));
    BspRun r = {};
    r.app = kAppBfs;
    r.row_ptr = g->row_ptr, r.col = g->col, r.n = g->n, r.nnz = g->nnz;
    r.device_loop = (cfg.flags & ATOS_FLAG_BSP_DEVICE_LOOP) != 0;
    rc = ensure_bsp(g, bsp_scratch_bytes(kAppBfs, g->n, g->nnz, group));
    if (rc) return rc;
    ATOS_TRY(cudaEventRecord(g->s.ev0, st));
    BspResult acc = {};
    for (int32_t i = 0; i < nsrc; i += group) {
      r.sources = sources + i;
      r.nsrc = std::min(group, nsrc - i);
      r.depth = depths + (size_t)i * n;
      rc = run_bsp(g, r, st, stats ? &acc : nullptr);
      if (rc) return rc;
    }
    ATOS_TRY(cudaEventRecord(g->s.ev1, st));
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      ATOS_TRY(cudaStreamSynchronize(st));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, g->s.ev0, g->s.ev1);
      stats->ms = ms;
      stats->iterations = acc.iters;
      stats->edges = acc.edges;
      stats->tasks = acc.tasks;
      stats->pushes = acc.tasks;
      stats->status = acc.status;
      return acc.status;
    }
    return ATOS_OK;
  }
  const uint32_t cap = ring_capacity(cfg, g->n, 1);
  if (!cap) return ATOS_ERR_INVALID_ARG;
  rc = ensure_scratch(g, nsrc, cap);
  if (rc) return rc;
  const bool marks = (cfg.flags & ATOS_FLAG_BFS_EXPAND_ONCE) != 0;
  if (marks && (size_t)nsrc > g->expanded_rows) {  // expansion markers, one row of n per source
    cudaDeviceSynchronize();               // the old rows may still be in use
    pool_free(g->d_expanded);
    g->d_expanded = nullptr;
    g->expanded_rows = 0;
    ATOS_TRY(dev_alloc(&g->d_expanded, (size_t)nsrc * (size_t)n));
    g->expanded_rows = (size_t)nsrc;
  }
  // row splitting needs a CTA worker (the warp and thread workers expand a row themselves)
  const bool split = (cfg.flags & ATOS_FLAG_BFS_SPLIT_ROWS) != 0 && cfg.worker_size > 32;
  if (split && (size_t)nsrc > g->seg_rows) {
    // per source, room for every row longer than the split threshold split twice over (a row
    // split again after an improvement of its vertex); a full table expands rows whole
    cudaDeviceSynchronize();
    pool_free(g->d_segs);
    g->d_segs = nullptr;
    g->seg_rows = 0;
    const uint64_t cap_segs = std::max<uint64_t>(1024, 2 * (uint64_t)g->nnz / 4096 + 64);
    g->seg_cap = (uint32_t)std::min<uint64_t>(cap_segs, 1u << 30);
    ATOS_TRY(dev_alloc(&g->d_segs, (size_t)nsrc * g->seg_cap));
    g->seg_rows = (size_t)nsrc;
  }
  for (int32_t i = 0; i < nsrc; ++i) {
    Instance I = base_instance(g, i, kAppBfs, cap, 1, sources[i]);
    I.depth = depths + (size_t)i * n;
    I.expanded = marks ? g->d_expanded + (size_t)i * n : nullptr;
    if (split) I.segs = g->d_segs + (size_t)i * g->seg_cap, I.seg_cap = g->seg_cap;
    g->s.h_insts[i] = I;
  }
  if (cfg.window == 0) {
    // keep the depth arrays of the active searches within about half of L2 (129 MB)
    const int64_t per = 4 * n + 1;
    cfg.window = (int)std::max<int64_t>(1, std::min<int64_t>(nsrc, (64LL << 20) / per));
  }
  ATOS_TRY(cudaEventRecord(g->s.ev0, st));
  int64_t iters = 0;
  rc = run_instances(g, nsrc, g->n, cfg, bfs_persistent_kernel, bfs_discrete_kernel, kAppBfs, st, &iters);
  if (rc) return rc;
  ATOS_TRY(cudaEventRecord(g->s.ev1, st));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    rc = collect_stats(g, nsrc, st, stats);
    if (rc) return rc;
    stats->iterations = iters;
    return stats->status;
  }
  return ATOS_OK;
}

int atos_pagerank(atos_graph_t g, float alpha, float eps, float* rank, const atos_config* cfg_in, void* stream,
                  atos_stats* stats) {
  if (!g || !rank || !(alpha > 0.0f && alpha < 1.0f) || !(eps > 0.0f)) return ATOS_ERR_INVALID_ARG;
  atos_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else default_config(&cfg);
  apply_tuned(g, ATOS_APP_PAGERANK, &cfg);
  int rc = check_config(cfg);
  if (rc) return rc;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (g->n == 0) return ATOS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  const bool bsp = cfg.strategy == ATOS_BSP;
  if (bsp) {
    cfg.strategy = ATOS_PERSISTENT;  // the prepare step below is shared; the loop is not run
    rc = ensure_bsp(g, bsp_scratch_bytes(kAppPr, n, g->nnz, 1));
    if (rc) return rc;
  }
  const uint32_t cap = ring_capacity(cfg, n, (uint32_t)n);
  if (!cap) return ATOS_ERR_INVALID_ARG;
  rc = ensure_scratch(g, 1, cap);
  if (rc) return rc;
  if (!g->d_res) ATOS_TRY(dev_alloc(&g->d_res, (size_t)n));
  if (!g->d_qbits) ATOS_TRY(dev_alloc(&g->d_qbits, (size_t)(n + 31) / 32));
  const bool spread = (cfg.flags & ATOS_FLAG_SPREAD_IDS) != 0;
  if (spread) {
    rc = ensure_spread(g, st);
    if (rc) return rc;
  }
  Instance I = base_instance(g, 0, kAppPr, cap, (uint32_t)n, -1);
  I.rank = spread ? (float*)g->sp_out : rank;
  if (spread) I.row_ptr = g->sp_row_ptr, I.col = g->sp_col, I.hubs = g->sp_hubs, I.hub = g->sp_hub;
  I.res = g->d_res;
  I.qbits = g->d_qbits;
  I.alpha = alpha;
  I.eps = eps;
  I.check_size = cfg.check_size > 0 ? (uint32_t)cfg.check_size : 32u;
  I.pr_crossing = (cfg.flags & ATOS_FLAG_PR_CROSSING) ? 1 : 0;
  g->s.h_insts[0] = I;
  cfg.window = 1;
  const double exact_sum = (double)n - (double)alpha * (double)g->n_isolated;
  ATOS_TRY(cudaEventRecord(g->s.ev0, st));
  int64_t iters = 0;
  BspResult bsp_acc = {};
  if (bsp) {
    // Algorithm 3: same initial state (prepare + initial residue), then level-synchronous sweeps
    rc = clear_timeline(g, st);
    if (rc) return rc;
    rc = upload_instances(g->s, 1, st);
    if (rc) return rc;
    ATOS_TRY(launch_prepare(g->s.d_insts, 1, n, g->s.d_ctl, 0u, 1u, st));
    ATOS_TRY(launch_pr_init(g->s.d_insts, 1, g->nnz, st));
    BspRun r = {};
    r.app = kAppPr;
    r.row_ptr = I.row_ptr, r.col = I.col, r.n = n, r.nnz = g->nnz;
    r.rank = I.rank, r.res = g->d_res, r.alpha = alpha, r.eps = eps;
    r.device_loop = (cfg.flags & ATOS_FLAG_BSP_DEVICE_LOOP) != 0;
    rc = run_bsp(g, r, st, stats ? &bsp_acc : nullptr);
    if (rc) return rc;
    iters = bsp_acc.iters;
  } else {
    rc = run_instances(g, 1, n, cfg, pr_persistent_kernel, pr_discrete_kernel, kAppPr, st, &iters);
    if (rc) return rc;
  }
  if (stats && !g->d_cert) ATOS_TRY(dev_alloc(&g->d_cert, (size_t)n));
  ATOS_TRY(pr_finish(g->s.d_insts, 1, n, g->nnz, g->s.d_ctl, stats ? g->d_cert : nullptr, exact_sum, st));
  if (spread) ATOS_TRY(unspread_f32((const float*)g->sp_out, rank, n, g->sp_perm, st));
  ATOS_TRY(cudaEventRecord(g->s.ev1, st));
  if (stats) {
    rc = collect_stats(g, 1, st, stats);
    if (rc) return rc;
    stats->iterations = iters;
    if (bsp) {
      stats->tasks = bsp_acc.tasks;
      stats->edges = bsp_acc.edges;
      stats->pushes = bsp_acc.tasks;
      if (!stats->status) stats->status = bsp_acc.status;
    }
    stats->residual_l1 = g->s.h_ctl->sum_res;
    const double denom = (1.0 - (double)alpha) * exact_sum;
    stats->error_bound = g->s.h_ctl->cert_l1 / denom + 5.96e-8;  // + FP32 rounding of the output
    return stats->status;
  }
  return ATOS_OK;
}

int atos_color(atos_graph_t g, int32_t* colors, int32_t* num_colors, const atos_config* cfg_in, void* stream,
               atos_stats* stats) {
  if (!g || !colors) return ATOS_ERR_INVALID_ARG;
  atos_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else default_config(&cfg);
  apply_tuned(g, ATOS_APP_COLOR, &cfg);
  int rc = check_config(cfg);
  if (rc) return rc;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (num_colors) *num_colors = 0;
  if (g->n == 0) return ATOS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = g->n;
  if (cfg.strategy == ATOS_BSP) {
    rc = ensure_bsp(g, bsp_scratch_bytes(kAppGc, n, g->nnz, 1));
    if (rc) return rc;
    const bool spread_bsp = (cfg.flags & ATOS_FLAG_SPREAD_IDS) != 0;
    if (spread_bsp) {
      rc = ensure_spread(g, st);
      if (rc) return rc;
    }
    int32_t* out = spread_bsp ? (int32_t*)g->sp_out : colors;
    rc = clear_timeline(g, st);
    if (rc) return rc;
    ATOS_TRY(cudaEventRecord(g->s.ev0, st));
    BspRun r = {};
    r.app = kAppGc;
    r.row_ptr = spread_bsp ? g->sp_row_ptr : g->row_ptr, r.col = spread_bsp ? g->sp_col : g->col, r.n = n;
    r.nnz = g->nnz;
    r.color = out;
    r.device_loop = (cfg.flags & ATOS_FLAG_BSP_DEVICE_LOOP) != 0;
    BspResult acc = {};
    rc = run_bsp(g, r, st, (stats || num_colors) ? &acc : nullptr);
    if (rc) return rc;
    Instance I;
    memset(&I, 0, sizeof(I));
    I.n = n;
    I.color = out;
    ATOS_TRY(gc_finish(&I, g->s.d_ctl, st));
    if (spread_bsp) ATOS_TRY(unspread_i32(out, colors, n, g->sp_perm, st));
    ATOS_TRY(cudaEventRecord(g->s.ev1, st));
    if (stats || num_colors) {
      ATOS_TRY(cudaMemcpyAsync(g->s.h_ctl, g->s.d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
      ATOS_TRY(cudaStreamSynchronize(st));
      if (num_colors) *num_colors = g->s.h_ctl->num_colors;
      if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->s.ev0, g->s.ev1);
        stats->ms = ms;
        stats->iterations = acc.iters;
        stats->edges = acc.edges;
        stats->tasks = acc.tasks;
        stats->pushes = acc.tasks;
        stats->num_colors = g->s.h_ctl->num_colors;
        stats->status = acc.status;
      }
    }
    return ATOS_OK;
  }
  const uint32_t cap = ring_capacity(cfg, n, (uint32_t)n);
  if (!cap) return ATOS_ERR_INVALID_ARG;
  rc = ensure_scratch(g, 1, cap);
  if (rc) return rc;
  if (!g->d_qbits) ATOS_TRY(dev_alloc(&g->d_qbits, (size_t)(n + 31) / 32));
  const bool spread = (cfg.flags & ATOS_FLAG_SPREAD_IDS) != 0;
  if (spread) {
    rc = ensure_spread(g, st);
    if (rc) return rc;
  }
  Instance I = base_instance(g, 0, kAppGc, cap, (uint32_t)n, -1);
  I.color = spread ? (int32_t*)g->sp_out : colors;
  I.gc_ordered = (cfg.flags & ATOS_FLAG_GC_ORDERED) ? 1 : 0;
  if (spread) I.row_ptr = g->sp_row_ptr, I.col = g->sp_col;
  I.qbits = g->d_qbits;
  const bool dependency = (cfg.flags & ATOS_FLAG_GC_DEPENDENCY) != 0;
  if (dependency) {
    if (!g->d_gc_wait) ATOS_TRY(dev_alloc(&g->d_gc_wait, (size_t)n));
    const int lay = spread ? 1 : 0;
    if (!g->gc_mid[lay]) {  // the split rows of this layout, built once per graph
      int32_t *mid = nullptr, *scol = nullptr, *tmp = nullptr;
      int rc2 = from_cuda(dev_alloc(&mid, (size_t)n));
      if (!rc2) rc2 = from_cuda(dev_alloc(&scol, (size_t)std::max<int64_t>(g->nnz, 1)));
      if (!rc2) rc2 = from_cuda(dev_alloc(&tmp, (size_t)n + 1));  // long rows and their count
      if (!rc2) rc2 = from_cuda(gc_split_build(I.row_ptr, I.col, n, mid, scol, tmp + 1, (int*)tmp, st));
      cudaStreamSynchronize(st);  // the list's scratch goes back now
      pool_free(tmp);
      if (rc2) {
        pool_free(mid), pool_free(scol);
        return rc2;
      }
      g->gc_mid[lay] = mid, g->gc_col[lay] = scol;
    }
    if (!g->gc_fw[lay]) {  // pushed colours: the bitmaps' places, built once per layout
      int2* fw = nullptr;
      int32_t* tmp = nullptr;
      uint32_t words = 0;
      int rc2 = from_cuda(dev_alloc(&fw, (size_t)n));
      if (!rc2) rc2 = from_cuda(dev_alloc(&tmp, (size_t)gc_bitmap_scratch(n)));
      if (!rc2) rc2 = from_cuda(gc_bitmap_build(g->gc_mid[lay], n, fw, tmp, &words, st));  // synchronises
      uint64_t tails = 0;
      if (!rc2) rc2 = from_cuda(gc_tail_segments(I.row_ptr, g->gc_mid[lay], n, tmp, &tails, st));  // synchronises
      pool_free(tmp);
      if (rc2) {
        pool_free(fw);
        return rc2;
      }
      g->gc_fw[lay] = fw, g->gc_fwords[lay] = words, g->gc_tails[lay] = tails ? tails + gc_tail_slack() : 0;
    }
    // tail segments (CTA workers): room for every one the run can create, plus the chunks CTAs
    // may leave partly used; item -(n + 1 + entry) must stay within int32
    const uint64_t tails = g->gc_tails[lay];
    const bool use_tails = cfg.worker_size > 32 && tails > 0 && (uint64_t)n + 1 + tails < (1ull << 31);
    if (use_tails && g->gc_segs_cap < tails) {
      cudaDeviceSynchronize();  // a previous call may still use the old table
      pool_free(g->d_gc_segs);
      g->d_gc_segs = nullptr;
      g->gc_segs_cap = 0;
      ATOS_TRY(dev_alloc(&g->d_gc_segs, (size_t)tails));
      g->gc_segs_cap = tails;
    }
    if (use_tails) I.segs = g->d_gc_segs, I.seg_cap = (uint32_t)tails;
    if (g->gc_forbid_cap < g->gc_fwords[lay]) {
      cudaDeviceSynchronize();  // a previous call may still use the old bitmaps
      pool_free(g->d_gc_forbid);
      g->d_gc_forbid = nullptr;
      g->gc_forbid_cap = 0;
      ATOS_TRY(dev_alloc(&g->d_gc_forbid, (size_t)std::max<uint32_t>(g->gc_fwords[lay], 1)));
      g->gc_forbid_cap = g->gc_fwords[lay];
    }
    I.gc_wait = g->d_gc_wait;
    I.gc_mid = g->gc_mid[lay];
    I.col = g->gc_col[lay];
    I.gc_fw = g->gc_fw[lay];
    I.gc_forbid = g->d_gc_forbid;
    I.gc_forbid_words = g->gc_fwords[lay];
  }
  g->s.h_insts[0] = I;
  cfg.window = 1;
  ATOS_TRY(cudaEventRecord(g->s.ev0, st));
  if (dependency) {
    ATOS_TRY(gc_wait_init(I.gc_mid, n, I.gc_wait, st));
    if (I.gc_forbid) ATOS_TRY(cudaMemsetAsync(I.gc_forbid, 0, sizeof(unsigned) * I.gc_forbid_words, st));
  }
  int64_t iters = 0;
  rc = run_instances(g, 1, n, cfg, gc_persistent_kernel, gc_discrete_kernel, kAppGc, st, &iters);
  if (rc) return rc;
  ATOS_TRY(gc_finish(&I, g->s.d_ctl, st));
  if (spread) ATOS_TRY(unspread_i32((const int32_t*)g->sp_out, colors, n, g->sp_perm, st));
  ATOS_TRY(cudaEventRecord(g->s.ev1, st));
  if (stats || num_colors) {
    atos_stats local;
    atos_stats* out = stats ? stats : &local;
    memset(out, 0, sizeof(*out));
    rc = collect_stats(g, 1, st, out);
    if (rc) return rc;
    out->iterations = iters;
    out->num_colors = g->s.h_ctl->num_colors;
    if (num_colors) *num_colors = g->s.h_ctl->num_colors;
    return out->status;
  }
  return ATOS_OK;
}

int atos_timeline(atos_graph_t g, int64_t bucket_ns, int32_t nbuckets) {
  if (!g || nbuckets < 0 || nbuckets > (1 << 20) || (nbuckets > 0 && bucket_ns < 1)) return ATOS_ERR_INVALID_ARG;
  cudaDeviceSynchronize();  // a running call may still count into the old buffer
  pool_free(g->d_timeline);
  g->d_timeline = nullptr;
  g->tl_nbuckets = 0;
  if (nbuckets == 0) return ATOS_OK;
  ATOS_TRY(dev_alloc(&g->d_timeline, (size_t)2 * nbuckets));
  ATOS_TRY(cudaMemset(g->d_timeline, 0, sizeof(unsigned long long) * 2 * nbuckets));
  g->tl_bucket_ns = bucket_ns;
  g->tl_nbuckets = nbuckets;
  return ATOS_OK;
}

int atos_timeline_read(atos_graph_t g, int64_t* tasks, int64_t* edges, int32_t nbuckets) {
  if (!g || nbuckets != g->tl_nbuckets || nbuckets < 1) return ATOS_ERR_INVALID_ARG;
  std::vector<unsigned long long> h((size_t)2 * nbuckets);
  ATOS_TRY(cudaDeviceSynchronize());
  ATOS_TRY(cudaMemcpy(h.data(), g->d_timeline, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost));
  for (int32_t b = 0; b < nbuckets; ++b) {
    if (tasks) tasks[b] = (int64_t)h[2 * b];
    if (edges) edges[b] = (int64_t)h[2 * b + 1];
  }
  return ATOS_OK;
}

int atos_debug_queue_state(atos_graph_t g, int32_t ninst, uint64_t* words, uint32_t* heads, int32_t* fail_site) {
  if (!g || ninst < 0 || ninst > g->s.ninst) return ATOS_ERR_INVALID_ARG;
  ATOS_TRY(cudaDeviceSynchronize());
  for (int32_t i = 0; i < ninst; ++i) {
    QueueCtl c;
    ATOS_TRY(cudaMemcpy(&c, g->s.d_qctl + i, sizeof(c), cudaMemcpyDeviceToHost));
    if (words) words[i] = c.word;
    if (heads) heads[i] = c.head;
  }
  if (fail_site && g->s.d_ctl) {
    DevCtl d;
    ATOS_TRY(cudaMemcpy(&d, g->s.d_ctl, sizeof(d), cudaMemcpyDeviceToHost));
    *fail_site = d.fail_site;
  }
  return ATOS_OK;
}

uint64_t atos_kernel_launches(void) { return (uint64_t)launches_so_far(); }

int atos_debug_spread_layout(atos_graph_t g, int32_t* perm, int32_t* hubs, void* stream) {
  if (!g) return ATOS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (g->n == 0) {
    if (hubs) *hubs = 0;
    return ATOS_OK;
  }
  const int rc = ensure_spread(g, st);
  if (rc) return rc;
  if (perm) {
    ATOS_TRY(cudaMemcpyAsync(perm, g->sp_perm, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, st));
    ATOS_TRY(cudaStreamSynchronize(st));
  }
  if (hubs) *hubs = g->sp_hubs;
  return ATOS_OK;
}

int atos_debug_scratch_check(atos_graph_t g, uint64_t* set_bits, uint64_t* busy_slots) {
  if (!g) return ATOS_ERR_INVALID_ARG;
  ATOS_TRY(cudaDeviceSynchronize());
  if (set_bits) {
    *set_bits = 0;
    if (g->d_qbits && g->n) {
      std::vector<uint32_t> b((g->n + 31) / 32);
      ATOS_TRY(cudaMemcpy(b.data(), g->d_qbits, b.size() * 4, cudaMemcpyDeviceToHost));
      for (uint32_t w : b) *set_bits += (uint64_t)__builtin_popcount(w);
    }
  }
  if (busy_slots) {
    *busy_slots = 0;
    if (g->s.d_ring && g->s.cap) {
      std::vector<unsigned long long> r((size_t)g->s.cap * g->s.ninst);
      ATOS_TRY(cudaMemcpy(r.data(), g->s.d_ring, r.size() * 8, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < r.size(); ++i)
        if (r[i] != ~0ull) {
          if (*busy_slots < 4)
            fprintf(stderr, "atos: busy slot %zu holds ticket %u item %d\n", i, (unsigned)(r[i] >> 32), (int)(unsigned)r[i]);
          *busy_slots += 1;
        }
    }
  }
  return ATOS_OK;
}

}  // extern "C"
