// batch.cu -- many instances (BFS sources, PageRanks, colourings, over several graphs) in one
// persistent launch, each with its own worklist, and the same launch replayed as a CUDA graph.
//
// The instance table, rings, control blocks and application scratch are allocated once when the
// batch is created; a run is then a fixed sequence of stream-ordered kernel launches and memsets
// (prepare, initial PageRank residues, one persistent launch of the mixed body, bookkeeping and
// per-instance result reductions), so it can be captured into a CUDA graph and replayed with one
// launch per batch.  Workers pick instances through the windowed hand-over of the engine: at most
// `window` instances are active at once, and the workers of a finished instance move on to the
// next one.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "atos.h"
#include "bfs.cuh"
#include "color.cuh"
#include "engine.cuh"
#include "launch.cuh"
#include "pagerank.cuh"
#include "state.cuh"

namespace atos {

// Per-CTA shared state of the mixed body: a CTA runs one application's batch at a time, so the
// colouring bitmaps and the PageRank hub accumulators share their space.
template <int B>
struct MixedExtra {
  union {
    unsigned bits[2 * B];
    float hub[HubSlots<B>::value];
  };
};

// Dispatches to the body of the instance's application (uniform across a CTA / warp).
struct MixedBody {
  template <int B>
  using Extra = MixedExtra<B>;
  static constexpr int kResidentThreads = 1536;
  template <int B>
  static constexpr int kLbsR = LbsRun<B>::R;

  template <int BLOCK, class S>
  __device__ static void cta_batch(S& sm, int cnt, const Launch& L, unsigned long long* st) {
    switch (sm.I.app) {
      case kAppBfs: BfsBody::template cta_batch<BLOCK>(sm, cnt, L, st); break;
      case kAppPr: PrBody::template cta_batch<BLOCK>(sm, cnt, L, st); break;
      default: GcBody::template cta_batch<BLOCK>(sm, cnt, L, st); break;
    }
  }
  template <int BLOCK, class S>
  __device__ static int cta_idle(S& sm, const Launch& L, unsigned long long* st) {
    switch (sm.I.app) {
      case kAppBfs: return BfsBody::template cta_idle<BLOCK>(sm, L, st);
      case kAppPr: return PrBody::template cta_idle<BLOCK>(sm, L, st);
      default: return GcBody::template cta_idle<BLOCK>(sm, L, st);
    }
  }
  __device__ static void warp_item(WarpSmem& ws, const Instance& I, int item, const Launch& L,
                                   unsigned long long* st) {
    switch (I.app) {
      case kAppBfs: BfsBody::warp_item(ws, I, item, L, st); break;
      case kAppPr: PrBody::warp_item(ws, I, item, L, st); break;
      default: GcBody::warp_item(ws, I, item, L, st); break;
    }
  }
  __device__ static void lane_items(WarpSmem& ws, const Instance& I, int item, const Launch& L,
                                    unsigned long long* st) {
    switch (I.app) {
      case kAppBfs: BfsBody::lane_items(ws, I, item, L, st); break;
      case kAppPr: PrBody::lane_items(ws, I, item, L, st); break;
      default: GcBody::lane_items(ws, I, item, L, st); break;
    }
  }
  __device__ static int warp_idle(WarpSmem& ws, const Instance& I, const Launch& L, unsigned long long* st) {
    switch (I.app) {
      case kAppBfs: return BfsBody::warp_idle(ws, I, L, st);
      case kAppPr: return PrBody::warp_idle(ws, I, L, st);
      default: return GcBody::warp_idle(ws, I, L, st);
    }
  }
};

// Per-instance results of a batch.
struct InstResult {
  double sum_rank;  // PageRank: FP64 sum of the ranks before normalisation
  double sum_res;   // PageRank: FP64 sum of the residues left
  int num_colors;   // colouring
  int pad;
};

// only_finished: skip instances whose worklist has not terminated (serving epochs).
__global__ void batch_reduce_kernel(const Instance* insts, InstResult* out, int only_finished) {
  const Instance I = insts[blockIdx.y];
  if (I.app == kAppBfs) return;
  if (only_finished && !ld_relaxed(&I.ctl->finished)) return;
  double a = 0.0, b = 0.0;
  int m = -1;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < I.n; v += gridDim.x * blockDim.x) {
    if (I.app == kAppPr) {
      a += (double)I.rank[v];
      b += (double)I.res[v];
    } else {
      m = max(m, I.color[v]);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) {
    InstResult* r = out + blockIdx.y;
    if (I.app == kAppPr) {
      atomicAdd(&r->sum_rank, a);
      atomicAdd(&r->sum_res, b);
    } else {
      atomicMax(&r->num_colors, m + 1);
    }
  }
}

__global__ void batch_normalise_kernel(const Instance* insts, const InstResult* res, int only_finished) {
  const Instance I = insts[blockIdx.y];
  if (I.app != kAppPr) return;
  if (only_finished && !ld_relaxed(&I.ctl->finished)) return;
  const double inv = 1.0 / res[blockIdx.y].sum_rank;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < I.n; v += gridDim.x * blockDim.x)
    I.rank[v] = (float)((double)I.rank[v] * inv);
}

const void* mixed_persistent_kernel(int worker) {
  return worker == 1 ? (const void*)warp_persistent_kernel<MixedBody, true> : persistent_kernel_ptr<MixedBody>(worker);
}
const void* mixed_discrete_kernel(int worker) {
  return worker == 1 ? (const void*)warp_discrete_kernel<MixedBody, true> : discrete_kernel_ptr<MixedBody>(worker);
}

// Finishes the terminated instances among d_insts[0, ninst) (PageRank normalisation, colour
// count) into d_results[k] (InstResult each); instances still running are left alone.
cudaError_t batch_finish_terminated(const Instance* d_insts, int ninst, int max_n, void* d_results, cudaStream_t s) {
  cudaMemsetAsync(d_results, 0, sizeof(InstResult) * ninst, s);
  int gx = (max_n + 255) / 256;
  gx = gx < 1 ? 1 : (gx > 256 ? 256 : gx);
  count_launches(2);
  batch_reduce_kernel<<<dim3(gx, ninst), 256, 0, s>>>(d_insts, (InstResult*)d_results, 1);
  batch_normalise_kernel<<<dim3(gx, ninst), 256, 0, s>>>(d_insts, (const InstResult*)d_results, 1);
  return cudaGetLastError();
}

size_t batch_result_bytes() { return sizeof(InstResult); }

void batch_result_read(const void* h_result, double* sum_rank, double* sum_res, int* num_colors) {
  const InstResult* r = (const InstResult*)h_result;
  *sum_rank = r->sum_rank;
  *sum_res = r->sum_res;
  *num_colors = r->num_colors;
}

}  // namespace atos

using namespace atos;

namespace {

uint32_t pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p > 0x80000000ULL ? 0 : (uint32_t)p;
}

}  // namespace

struct atos_batch_s {
  int ninst = 0;
  int window = 1;
  int nb = 0;
  int threads = 0;
  atos_config cfg;
  const void* fn = nullptr;
  int max_n = 0;
  int64_t max_nnz = 0;
  bool has_pr = false;
  std::vector<Instance> h_insts;
  std::vector<double> exact_sum;  // PageRank instances: n - alpha * isolated
  std::vector<float> alpha;
  Instance* d_insts = nullptr;
  QueueCtl* d_qctl = nullptr;
  unsigned long long* d_ring = nullptr;
  unsigned long long* d_stats = nullptr;
  unsigned long long* h_stats = nullptr;
  DevCtl* d_ctl = nullptr;
  DevCtl* h_ctl = nullptr;
  float* d_res = nullptr;
  uint32_t* d_qbits = nullptr;
  InstResult* d_results = nullptr;
  InstResult* h_results = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned graph_kernels = 0;  // library kernels one replay of the captured graph launches
  // PageRank output certificates: instance indices, FP64 scratch, results (device / pinned host)
  int n_pr = 0, max_n_pr = 0;
  int64_t max_nnz_pr = 0;
  int* d_pr_idx = nullptr;
  double* d_cert_y = nullptr;
  double* d_cert = nullptr;
  double* h_cert = nullptr;
  // ATOS_FLAG_SPREAD_IDS: PageRank / colouring instances run on their graph's spread-id copy,
  // write into d_sp_out and are mapped back to the caller's outputs at the end of a run
  char* d_sp_out = nullptr;
  SpreadJob* d_jobs = nullptr;
  int njobs = 0, max_n_jobs = 0;
  const void* fn_discrete = nullptr;
  unsigned first_gen = 0;      // discrete strategy: the largest virtual prefix (first generation)

  ~atos_batch_s() {
    cudaDeviceSynchronize();
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    pool_free(d_insts), pool_free(d_qctl), pool_free(d_ring), pool_free(d_stats), pool_free_host(h_stats);
    pool_free(d_ctl), pool_free_host(h_ctl), pool_free(d_res), pool_free(d_qbits), pool_free(d_results);
    pool_free(d_pr_idx), pool_free(d_cert_y), pool_free(d_cert), pool_free_host(h_cert);
    pool_free(d_sp_out), pool_free(d_jobs);
    pool_free_host(h_results);
  }
};

namespace {

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return ATOS_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? ATOS_ERR_OOM : ATOS_ERR_CUDA;
}
#define BATCH_TRY(expr)                \
  do {                                 \
    int _rc = cuda_rc(expr);           \
    if (_rc != ATOS_OK) return _rc;    \
  } while (0)

// The stream-ordered sequence of one batch run: no allocation, and no host synchronisation with
// the persistent strategy (the discrete one reads each generation's size back).
int enqueue_run(atos_batch_s* b, cudaStream_t st) {
  Launch L;
  memset(&L, 0, sizeof(L));
  L.insts = b->d_insts;
  L.ninst = b->ninst;
  L.window = b->window;
  L.fetch = b->cfg.fetch_size;
  L.policy = b->cfg.fetch_policy;
  L.flags = b->cfg.flags;
  L.status = &b->d_ctl->status;
  L.next_inst = &b->d_ctl->next_inst;
  L.fail_site = &b->d_ctl->fail_site;
  L.spin_limit_ns = b->cfg.spin_limit_ns > 0 ? b->cfg.spin_limit_ns : 4000000000LL;
  L.lifetime_ns = L.spin_limit_ns * 16;
  const int workers_per_block = warp_hosted(b->cfg.worker_size) ? kWarpBlock / 32 : 1;
  L.nworkers = std::max(1, b->nb * workers_per_block / b->window);
  const bool discrete = b->cfg.strategy == ATOS_DISCRETE;
  BATCH_TRY(launch_prepare(b->d_insts, b->ninst, b->max_n, b->d_ctl, b->cfg.flags,
                           discrete ? (unsigned)b->ninst : (unsigned)b->window, st));
  if (b->has_pr) BATCH_TRY(launch_pr_init(b->d_insts, b->ninst, b->max_nnz, st));
  if (discrete) {
    // one launch per generation over every instance, the generation size read back each time
    L.window = b->ninst;
    const int per_block = warp_hosted(b->cfg.worker_size) ? std::min(b->cfg.fetch_size, 32) * (kWarpBlock / 32)
                                                   : b->cfg.fetch_size;
    BATCH_TRY(discrete_loop(b->fn_discrete, b->threads, per_block, L, b->d_insts, b->ninst, b->max_n, b->first_gen,
                            b->has_pr, b->d_ctl, b->h_ctl, st, nullptr));
  } else {
    BATCH_TRY(launch_kernel(b->fn, dim3(b->nb), b->threads, L, st));
  }
  BATCH_TRY(launch_finalize(b->d_insts, b->ninst, b->d_ctl, st));
  BATCH_TRY(cudaMemsetAsync(b->d_results, 0, sizeof(InstResult) * b->ninst, st));
  int gx = (b->max_n + 255) / 256;
  gx = std::max(1, std::min(gx, 256));
  count_launches(2);
  batch_reduce_kernel<<<dim3(gx, b->ninst), 256, 0, st>>>(b->d_insts, b->d_results, 0);
  batch_normalise_kernel<<<dim3(gx, b->ninst), 256, 0, st>>>(b->d_insts, b->d_results, 0);
  BATCH_TRY(cudaGetLastError());
  // FP64 certificate of every PageRank output (it certifies the FP32 vector returned)
  BATCH_TRY(pr_certify_outputs(b->d_insts, b->d_pr_idx, b->n_pr, b->max_n_pr, b->max_nnz_pr, b->d_cert, st));
  BATCH_TRY(unspread_jobs(b->d_jobs, b->njobs, b->max_n_jobs, st));  // spread-id results to caller ids
  return ATOS_OK;
}

}  // namespace

// the graph accessors of api.cu
extern "C" int atos_graph_info(atos_graph_t g, int32_t* n, int64_t* nnz, int32_t* max_degree);
namespace atos {
int graph_device_csr(atos_graph_t g, const int32_t** row_ptr, const int32_t** col, int32_t* n_isolated);
int graph_spread_csr(atos_graph_t g, const int32_t** row_ptr, const int32_t** col, cudaStream_t st,
                     const int32_t** perm, int32_t* hubs, HubMap* hub);
}

extern "C" {

int atos_batch_create(const atos_graph_t* graphs, int32_t ngraphs, const atos_instance* inst, int32_t ninst,
                      const atos_config* cfg_in, atos_batch_t* out) {
  if (!out) return ATOS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!graphs || ngraphs < 1 || !inst || ninst < 1 || ninst > 65535) return ATOS_ERR_INVALID_ARG;
  atos_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else atos_queue_config(&cfg, nullptr);
  if (!worker_supported(cfg.worker_size)) return ATOS_ERR_UNSUPPORTED;
  if (cfg.strategy != ATOS_PERSISTENT && cfg.strategy != ATOS_DISCRETE) return ATOS_ERR_UNSUPPORTED;
  if (cfg.flags & ATOS_FLAG_GC_DEPENDENCY) return ATOS_ERR_UNSUPPORTED;  // atos_color only
  if (cfg.fetch_size < 1 || cfg.fetch_size > (warp_hosted(cfg.worker_size) ? 32 : cfg.worker_size))
    return ATOS_ERR_INVALID_ARG;
  // validate every instance before allocating anything
  std::vector<int32_t> gn(ngraphs);
  std::vector<int64_t> gnnz(ngraphs);
  for (int32_t i = 0; i < ngraphs; ++i) {
    if (!graphs[i]) return ATOS_ERR_INVALID_ARG;
    atos_graph_info(graphs[i], &gn[i], &gnnz[i], nullptr);
  }
  for (int32_t i = 0; i < ninst; ++i) {
    const atos_instance& q = inst[i];
    if (q.graph < 0 || q.graph >= ngraphs || !q.out || gn[q.graph] < 1) return ATOS_ERR_INVALID_ARG;
    if (q.app == ATOS_APP_BFS && (q.source < 0 || q.source >= gn[q.graph])) return ATOS_ERR_INVALID_ARG;
    if (q.app == ATOS_APP_PAGERANK && !(q.alpha > 0.0f && q.alpha < 1.0f && q.eps > 0.0f)) return ATOS_ERR_INVALID_ARG;
    if (q.app != ATOS_APP_BFS && q.app != ATOS_APP_PAGERANK && q.app != ATOS_APP_COLOR) return ATOS_ERR_INVALID_ARG;
  }
  atos_batch_s* b = new (std::nothrow) atos_batch_s();
  if (!b) return ATOS_ERR_OOM;
  b->cfg = cfg;
  b->ninst = ninst;
  b->threads = block_threads(cfg.worker_size);
  b->fn = mixed_persistent_kernel(cfg.worker_size);
  b->fn_discrete = mixed_discrete_kernel(cfg.worker_size);
  int rc = ATOS_OK;
  // sizes: one ring per instance, PageRank residues and queued bits, colouring bits
  std::vector<uint64_t> ring_off(ninst), res_off(ninst), bits_off(ninst);
  std::vector<uint32_t> caps(ninst);
  uint64_t ring_total = 0, res_total = 0, bits_total = 0;
  double footprint = 0.0;
  for (int32_t i = 0; i < ninst; ++i) {
    const int32_t n = gn[inst[i].graph];
    const uint32_t prefix = inst[i].app == ATOS_APP_BFS ? 1u : (uint32_t)n;
    uint32_t cap = cfg.queue_capacity > 0 ? pow2_at_least((uint64_t)cfg.queue_capacity)
                                         : pow2_at_least(std::max<uint64_t>((uint64_t)n + n / 2 + prefix + 1024, 1u << 20));
    if (!cap) {
      delete b;
      return ATOS_ERR_INVALID_ARG;
    }
    caps[i] = cap;
    ring_off[i] = ring_total;
    ring_total += cap;
    res_off[i] = res_total;
    if (inst[i].app == ATOS_APP_PAGERANK) res_total += ((uint64_t)n + 63) & ~(uint64_t)63;  // 256-byte aligned rows
    bits_off[i] = bits_total;
    if (inst[i].app != ATOS_APP_BFS) bits_total += (uint64_t)(n + 31) / 32;
    b->max_n = std::max(b->max_n, n);
    b->max_nnz = std::max(b->max_nnz, gnnz[inst[i].graph]);
    b->has_pr |= inst[i].app == ATOS_APP_PAGERANK;
    if (inst[i].app == ATOS_APP_PAGERANK) {
      b->n_pr++;
      b->max_n_pr = std::max(b->max_n_pr, n);
      b->max_nnz_pr = std::max(b->max_nnz_pr, gnnz[inst[i].graph]);
    }
    footprint += (inst[i].app == ATOS_APP_PAGERANK ? 8.0 : 4.0) * n;
  }
  if (!rc) rc = cuda_rc(pool_malloc((void**)&b->d_insts, sizeof(Instance) * ninst));
  if (!rc) rc = cuda_rc(pool_malloc((void**)&b->d_qctl, sizeof(QueueCtl) * ninst));
  if (!rc) rc = cuda_rc(pool_malloc((void**)&b->d_ring, sizeof(unsigned long long) * ring_total));
  if (!rc) rc = cuda_rc(pool_malloc((void**)&b->d_stats, sizeof(unsigned long long) * kNumStats * ninst));
  if (!rc) rc = cuda_rc(pool_malloc_host((void**)&b->h_stats, sizeof(unsigned long long) * kNumStats * ninst));
  if (!rc) rc = cuda_rc(pool_malloc((void**)&b->d_ctl, sizeof(DevCtl)));
  if (!rc) rc = cuda_rc(pool_malloc_host((void**)&b->h_ctl, sizeof(DevCtl)));
  if (!rc && res_total) rc = cuda_rc(pool_malloc((void**)&b->d_res, sizeof(float) * res_total));
  if (!rc && bits_total) rc = cuda_rc(pool_malloc((void**)&b->d_qbits, sizeof(uint32_t) * bits_total));
  const bool spread = (cfg.flags & ATOS_FLAG_SPREAD_IDS) != 0;
  std::vector<uint64_t> sp_off(ninst, 0);
  uint64_t sp_total = 0;
  if (spread)
    for (int32_t i = 0; i < ninst; ++i)
      if (inst[i].app != ATOS_APP_BFS) {
        sp_off[i] = sp_total;
        sp_total += ((uint64_t)gn[inst[i].graph] + 63) & ~(uint64_t)63;
        b->njobs++;
        b->max_n_jobs = std::max(b->max_n_jobs, gn[inst[i].graph]);
      }
  if (!rc && sp_total) rc = cuda_rc(pool_malloc((void**)&b->d_sp_out, sizeof(int32_t) * sp_total));
  if (!rc && b->njobs) rc = cuda_rc(pool_malloc((void**)&b->d_jobs, sizeof(SpreadJob) * b->njobs));
  if (!rc && b->n_pr) {
    rc = cuda_rc(pool_malloc((void**)&b->d_cert_y, sizeof(double) * res_total));  // same row offsets as res
    if (!rc) rc = cuda_rc(pool_malloc((void**)&b->d_pr_idx, sizeof(int) * b->n_pr));
    if (!rc) rc = cuda_rc(pool_malloc((void**)&b->d_cert, sizeof(double) * b->n_pr));
    if (!rc) rc = cuda_rc(pool_malloc_host((void**)&b->h_cert, sizeof(double) * b->n_pr));
  }
  if (!rc) rc = cuda_rc(pool_malloc((void**)&b->d_results, sizeof(InstResult) * ninst));
  if (!rc) rc = cuda_rc(pool_malloc_host((void**)&b->h_results, sizeof(InstResult) * ninst));
  if (!rc) rc = cuda_rc(cudaEventCreate(&b->ev0));
  if (!rc) rc = cuda_rc(cudaEventCreate(&b->ev1));
  if (rc) {
    delete b;
    return rc;
  }
  b->h_insts.resize(ninst);
  b->exact_sum.assign(ninst, 0.0);
  b->alpha.assign(ninst, 0.0f);
  std::vector<int> pr_idx;
  std::vector<SpreadJob> jobs;
  for (int32_t i = 0; i < ninst; ++i) {
    const atos_instance& q = inst[i];
    const int32_t* rp = nullptr;
    const int32_t* col = nullptr;
    int32_t iso = 0;
    graph_device_csr(graphs[q.graph], &rp, &col, &iso);
    SpreadJob job;
    memset(&job, 0, sizeof(job));
    int32_t hubs = 0;
    HubMap hub = {0, 1, 1, 0};
    if (spread && q.app != ATOS_APP_BFS) {
      // the spread-id copy of the graph (built on the legacy stream the first time; create is synchronous)
      const int rc2 = graph_spread_csr(graphs[q.graph], &rp, &col, 0, &job.perm, &hubs, &hub);
      if (rc2) {
        delete b;
        return rc2;
      }
      job.src = b->d_sp_out + sizeof(int32_t) * sp_off[i];
      job.dst = q.out;
      job.n = gn[q.graph];
    }
    Instance I;
    memset(&I, 0, sizeof(I));
    I.row_ptr = rp;
    I.col = col;
    I.n = gn[q.graph];
    I.ring = b->d_ring + ring_off[i];
    I.cap = caps[i];
    I.ctl = b->d_qctl + i;
    I.stats = b->d_stats + (size_t)kNumStats * i;
    if (q.app == ATOS_APP_BFS) {
      I.app = kAppBfs;
      I.prefix_len = 1;
      I.prefix_item = q.source;
      I.depth = (int32_t*)q.out;
    } else if (q.app == ATOS_APP_PAGERANK) {
      I.app = kAppPr;
      I.prefix_len = (uint32_t)I.n;
      I.prefix_item = -1;
      I.rank = job.src ? (float*)job.src : (float*)q.out;
      I.hubs = hubs;
      I.hub = hub;
      I.res = b->d_res + res_off[i];
      I.qbits = b->d_qbits + bits_off[i];
      I.alpha = q.alpha;
      I.eps = q.eps;
      I.check_size = cfg.check_size > 0 ? (uint32_t)cfg.check_size : 32u;
      I.pr_crossing = (cfg.flags & ATOS_FLAG_PR_CROSSING) ? 1 : 0;
      b->exact_sum[i] = (double)I.n - (double)q.alpha * iso;
      b->alpha[i] = q.alpha;
      I.cert_y = b->d_cert_y + res_off[i];
      I.exact_sum = b->exact_sum[i];
      pr_idx.push_back(i);
    } else {
      I.app = kAppGc;
      I.prefix_len = (uint32_t)I.n;
      I.prefix_item = -1;
      I.color = job.src ? (int32_t*)job.src : (int32_t*)q.out;
      I.gc_ordered = (cfg.flags & ATOS_FLAG_GC_ORDERED) ? 1 : 0;
      I.qbits = b->d_qbits + bits_off[i];
    }
    b->h_insts[i] = I;
    b->first_gen = std::max(b->first_gen, I.prefix_len);
    if (job.src) jobs.push_back(job);
  }
  rc = cuda_rc(cudaMemcpy(b->d_insts, b->h_insts.data(), sizeof(Instance) * ninst, cudaMemcpyHostToDevice));
  if (!rc && b->n_pr)
    rc = cuda_rc(cudaMemcpy(b->d_pr_idx, pr_idx.data(), sizeof(int) * b->n_pr, cudaMemcpyHostToDevice));
  if (!rc && b->njobs)
    rc = cuda_rc(cudaMemcpy(b->d_jobs, jobs.data(), sizeof(SpreadJob) * b->njobs, cudaMemcpyHostToDevice));
  DevCtl init;
  memset(&init, 0, sizeof(init));
  init.dirty = 1;  // fresh rings: the first prepare fills them
  if (!rc) rc = cuda_rc(cudaMemcpy(b->d_ctl, &init, sizeof(init), cudaMemcpyHostToDevice));
  if (!rc) {
    b->nb = cfg.num_blocks > 0 ? cfg.num_blocks : resident_blocks(b->fn, b->threads);
    if (b->nb <= 0) rc = ATOS_ERR_CUDA;
  }
  if (rc) {
    delete b;
    return rc;
  }
  if (cfg.window > 0) {
    b->window = std::min(cfg.window, ninst);
  } else {
    // keep the state of the active instances within about half of L2, with at least one CTA each
    const double per = footprint / ninst;
    int w = (int)std::max(1.0, (64.0 * (1 << 20)) / std::max(per, 1.0));
    b->window = std::max(1, std::min(std::min(w, ninst), b->nb));
  }
  *out = b;
  return ATOS_OK;
}

int atos_batch_run(atos_batch_t b, void* stream) {
  if (!b) return ATOS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  BATCH_TRY(cudaEventRecord(b->ev0, st));
  int rc = enqueue_run(b, st);
  if (rc) return rc;
  BATCH_TRY(cudaEventRecord(b->ev1, st));
  return ATOS_OK;
}

int atos_batch_run_graph(atos_batch_t b, void* stream) {
  if (!b) return ATOS_ERR_INVALID_ARG;
  if (b->cfg.strategy != ATOS_PERSISTENT) return ATOS_ERR_UNSUPPORTED;  // host-driven generations
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->exec) {
    // capture the run once on a private stream (the legacy default stream cannot be captured)
    BATCH_TRY(cudaStreamSynchronize(st));
    if (!b->cap_stream) BATCH_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    BATCH_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    const unsigned long long before = launches_so_far();
    int rc = enqueue_run(b, b->cap_stream);
    b->graph_kernels = (unsigned)(launches_so_far() - before);
    uncount_launches(b->graph_kernels);  // captured, not run: each replay counts them
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    BATCH_TRY(e);
    b->graph = graph;
    BATCH_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  BATCH_TRY(cudaEventRecord(b->ev0, st));
  BATCH_TRY(cudaGraphLaunch(b->exec, st));
  count_launches(b->graph_kernels);
  BATCH_TRY(cudaEventRecord(b->ev1, st));
  return ATOS_OK;
}

int atos_batch_stats(atos_batch_t b, atos_stats* total, atos_stats* per_instance, void* stream) {
  if (!b) return ATOS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  BATCH_TRY(cudaMemcpyAsync(b->h_stats, b->d_stats, sizeof(unsigned long long) * kNumStats * b->ninst,
                            cudaMemcpyDeviceToHost, st));
  BATCH_TRY(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
  BATCH_TRY(cudaMemcpyAsync(b->h_results, b->d_results, sizeof(InstResult) * b->ninst, cudaMemcpyDeviceToHost, st));
  if (b->n_pr) BATCH_TRY(cudaMemcpyAsync(b->h_cert, b->d_cert, sizeof(double) * b->n_pr, cudaMemcpyDeviceToHost, st));
  BATCH_TRY(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  atos_stats sum;
  memset(&sum, 0, sizeof(sum));
  sum.ms = ms;
  sum.iterations = 1;
  sum.status = b->h_ctl->status;
  int kpr = 0;
  for (int i = 0; i < b->ninst; ++i) {
    atos_stats one;
    memset(&one, 0, sizeof(one));
    one.ms = ms;
    one.iterations = 1;
    one.status = b->h_ctl->status;
    one.tasks = (int64_t)b->h_stats[i * kNumStats + kStatTasks];
    one.edges = (int64_t)b->h_stats[i * kNumStats + kStatEdges];
    one.pushes = (int64_t)b->h_stats[i * kNumStats + kStatPushes];
    const Instance& I = b->h_insts[i];
    if (I.app == kAppPr) {
      one.residual_l1 = b->h_results[i].sum_res;
      // FP64 certificate of the returned vector q: ||q - p / sum p||_1 <= ||rho||_1 / ((1 - alpha) S)
      one.error_bound = b->h_cert[kpr++] / ((1.0 - (double)b->alpha[i]) * b->exact_sum[i]);
    } else if (I.app == kAppGc) {
      one.num_colors = b->h_results[i].num_colors;
    }
    if (per_instance) per_instance[i] = one;
    sum.tasks += one.tasks;
    sum.edges += one.edges;
    sum.pushes += one.pushes;
    sum.residual_l1 += one.residual_l1;
    sum.error_bound = std::max(sum.error_bound, one.error_bound);
    sum.num_colors = std::max(sum.num_colors, one.num_colors);
  }
  if (total) *total = sum;
  return sum.status;
}

int atos_batch_info(atos_batch_t b, int32_t* ninst, int32_t* window, int32_t* grid) {
  if (!b) return ATOS_ERR_INVALID_ARG;
  if (ninst) *ninst = b->ninst;
  if (window) *window = b->window;
  if (grid) *grid = b->nb;
  return ATOS_OK;
}

int atos_batch_destroy(atos_batch_t b) {
  delete b;
  return ATOS_OK;
}

}  // extern "C"
