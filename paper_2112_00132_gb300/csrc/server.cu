// server.cu -- serving: resident graphs, requests admitted by HBM footprint, continuous batching.
//
// A server holds a set of resident graphs, a fixed number of request slots and an arena of
// device memory of a fixed budget.  A request (BFS from a source, PageRank, colouring, on one of
// the graphs) is admitted when a slot is free and its scratch -- worklist ring, the tickets a
// paused epoch may leave pending, PageRank residues, queued bitmap -- fits in the arena (first
// fit); its state is initialised at once on the server's stream.  Work runs in epochs: one
// persistent launch over every active request, bounded by a time slice, after which each worker
// pauses at a safe point and records the pop tickets it still holds; the next epoch takes those
// over.  Queue state therefore stays on the device across epochs, requests admitted while others
// are in flight join at the next epoch, and the work of all of them overlaps on the GPU.  When a
// request's instance has terminated, its result is finished (PageRank normalised, colours
// counted), a completion record is queued for the host, and its slot and memory are released.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "atos.h"
#include "engine.cuh"
#include "launch.cuh"
#include "state.cuh"

namespace atos {
const void* mixed_persistent_kernel(int worker);
int graph_device_csr(atos_graph_t g, const int32_t** row_ptr, const int32_t** col, int32_t* n_isolated);
int graph_spread_csr(atos_graph_t g, const int32_t** row_ptr, const int32_t** col, cudaStream_t st,
                     const int32_t** perm, int32_t* hubs, HubMap* hub);
cudaError_t batch_finish_terminated(const Instance* d_insts, int ninst, int max_n, void* d_results, cudaStream_t s);
size_t batch_result_bytes();
void batch_result_read(const void* h_result, double* sum_rank, double* sum_res, int* num_colors);

// Start of epoch e for each active instance (one block per instance).  Epoch e hands out the
// tickets the pauses of epoch e-1 recorded (buffer e & 1).  Tickets of epoch e-1's own read
// buffer that were not handed out before its slice ended are appended to them, so no pending
// ticket is ever dropped; then epoch e's pauses get an empty buffer ((e + 1) & 1).
__global__ void server_epoch_begin(Instance* active, unsigned epoch, int* status) {
  const Instance I = active[blockIdx.x];
  QueueCtl* c = I.ctl;
  const unsigned r = epoch & 1, prev = (epoch + 1) & 1;
  const unsigned head = c->orphan_head, prev_cnt = c->orphan_count[prev], cnt = c->orphan_count[r];
  const unsigned left = prev_cnt > head ? prev_cnt - head : 0;
  if (cnt + left > I.orphan_cap) {
    if (threadIdx.x == 0) atomicCAS(status, 0, ATOS_ERR_QUEUE_OVERFLOW);
    return;
  }
  for (unsigned k = threadIdx.x; k < left; k += blockDim.x) I.orphans[r][cnt + k] = I.orphans[prev][head + k];
  __syncthreads();
  if (threadIdx.x == 0) {
    c->orphan_count[r] = cnt + left;
    c->orphan_count[prev] = 0;
    c->orphan_head = 0;
    c->succ = -2;
  }
}

__global__ void server_gather_finished(const Instance* active, int nactive, int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nactive; i += gridDim.x * blockDim.x)
    out[i] = active[i].ctl->finished;
}

}  // namespace atos

using namespace atos;

namespace {

// First-fit arena over one device allocation (host-side bookkeeping; offsets aligned to 256 B).
struct Arena {
  char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  size_t used = 0;

  void init(char* b, size_t n) {
    base = b;
    size = n;
    free_.clear();
    free_[0] = n;
    used = 0;
  }
  // returns offset or SIZE_MAX
  size_t alloc(size_t n) {
    n = (n + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[off + n] = len - n;
        used += n;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) & ~(size_t)255;
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
};

enum SlotState { kFree = 0, kActive = 1 };

struct Slot {
  int state = kFree;
  int64_t id = -1;
  int app = 0;
  int graph = 0;
  size_t off = 0, bytes = 0;
  float alpha = 0.85f;
  double exact_sum = 0.0;
  Instance inst;
  SpreadJob job;  // spread-id requests: the result's way back to the caller's ids (src == nullptr: none)
};

uint32_t pow2_ceil(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p > 0x80000000ULL ? 0 : (uint32_t)p;
}

int rc_of(cudaError_t e) {
  if (e == cudaSuccess) return ATOS_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? ATOS_ERR_OOM : ATOS_ERR_CUDA;
}
#define SRV_TRY(expr)              \
  do {                             \
    int _rc = rc_of(expr);         \
    if (_rc != ATOS_OK) return _rc; \
  } while (0)

}  // namespace

struct atos_server_s {
  std::vector<atos_graph_t> graphs;
  std::vector<int32_t> gn, giso;
  std::vector<int64_t> gnnz;
  atos_config cfg;
  int max_slots = 0;
  int nb = 0, threads = 0;
  const void* fn = nullptr;
  uint32_t orphan_cap = 0;
  cudaStream_t stream = nullptr;
  unsigned epoch = 0;
  int64_t next_id = 0;
  Arena arena;
  char* d_arena = nullptr;
  std::vector<Slot> slots;
  Instance* d_slots = nullptr;   // descriptor of every slot
  Instance* h_slots = nullptr;   // pinned staging of the descriptors (submit copies from it)
  Instance* d_active = nullptr;  // the active slots of the current epoch, compacted
  Instance* h_active = nullptr;  // pinned
  std::vector<int> active_idx;
  QueueCtl* d_qctl = nullptr;
  unsigned long long* d_stats = nullptr;
  unsigned long long* h_stats = nullptr;  // pinned
  DevCtl* d_ctl = nullptr;
  DevCtl* h_ctl = nullptr;  // pinned
  int* d_fin = nullptr;
  int* h_fin = nullptr;  // pinned
  char* d_results = nullptr;
  char* h_results = nullptr;  // pinned
  int* d_cert_idx = nullptr;  // PageRank certificates of the requests an epoch finished
  int* h_cert_idx = nullptr;  // pinned
  double* d_cert = nullptr;
  double* h_cert = nullptr;   // pinned
  SpreadJob* d_jobs = nullptr;
  SpreadJob* h_jobs = nullptr;  // pinned
  std::deque<atos_completion> done;
  int64_t epochs = 0;

  ~atos_server_s() {
    cudaDeviceSynchronize();
    pool_free(d_arena), pool_free(d_slots), pool_free_host(h_slots), pool_free(d_active), pool_free_host(h_active);
    pool_free(d_qctl);
    pool_free(d_stats), pool_free_host(h_stats), pool_free(d_ctl), pool_free_host(h_ctl), pool_free(d_fin);
    pool_free_host(h_fin), pool_free(d_results), pool_free_host(h_results);
    pool_free(d_cert_idx), pool_free_host(h_cert_idx), pool_free(d_cert), pool_free_host(h_cert);
    pool_free(d_jobs), pool_free_host(h_jobs);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

// Device bytes a request needs from the arena.
size_t request_bytes(const atos_server_s* s, int app, int32_t n, uint32_t* cap_out) {
  const uint32_t prefix = app == ATOS_APP_BFS ? 1u : (uint32_t)n;
  // a full lap of the ring must take longer than one epoch slice: a push that wraps onto a slot
  // whose item waits for the next epoch (its ticket's worker paused) would otherwise wait for it
  const uint32_t cap = pow2_ceil(std::max<uint64_t>((uint64_t)n + n / 2 + prefix + 1024, 1u << 20));
  if (cap_out) *cap_out = cap;
  size_t b = (size_t)cap * 8 + 256;                 // ring
  b += 2 * ((size_t)s->orphan_cap * 4 + 256);       // pending tickets of a pause, two epochs
  if (app == ATOS_APP_PAGERANK) b += (size_t)n * 4 + 256 + (size_t)n * 8 + 256;  // residues, certificate
  if (app != ATOS_APP_BFS) b += (size_t)(n + 31) / 32 * 4 + 256;  // queued bits
  if (app != ATOS_APP_BFS && (s->cfg.flags & ATOS_FLAG_SPREAD_IDS)) b += (size_t)n * 4 + 256;  // spread-id output
  return b;
}

void release_slot(atos_server_s* s, int i) {
  Slot& sl = s->slots[i];
  s->arena.release(sl.off, sl.bytes);
  sl.state = kFree;
  sl.id = -1;
}

}  // namespace

extern "C" {

int atos_server_create(const atos_graph_t* graphs, int32_t ngraphs, int32_t max_slots, int64_t budget_bytes,
                       const atos_config* cfg_in, atos_server_t* out) {
  if (!out) return ATOS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!graphs || ngraphs < 1 || max_slots < 1 || max_slots > 4096 || budget_bytes < (1 << 20))
    return ATOS_ERR_INVALID_ARG;
  atos_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else atos_queue_config(&cfg, nullptr);
  if (cfg.strategy != ATOS_PERSISTENT || warp_hosted(cfg.worker_size) || !worker_supported(cfg.worker_size))
    return ATOS_ERR_UNSUPPORTED;  // serving pauses CTA workers only
  if (cfg.flags & ATOS_FLAG_GC_DEPENDENCY) return ATOS_ERR_UNSUPPORTED;  // atos_color only
  if (cfg.fetch_size < 1 || cfg.fetch_size > cfg.worker_size) return ATOS_ERR_INVALID_ARG;
  atos_server_s* s = new (std::nothrow) atos_server_s();
  if (!s) return ATOS_ERR_OOM;
  s->cfg = cfg;
  s->max_slots = max_slots;
  for (int32_t i = 0; i < ngraphs; ++i) {
    if (!graphs[i]) {
      delete s;
      return ATOS_ERR_INVALID_ARG;
    }
    int32_t n = 0;
    int64_t nnz = 0;
    atos_graph_info(graphs[i], &n, &nnz, nullptr);
    const int32_t *rp, *col;
    int32_t iso = 0;
    graph_device_csr(graphs[i], &rp, &col, &iso);
    s->graphs.push_back(graphs[i]);
    s->gn.push_back(n);
    s->gnnz.push_back(nnz);
    s->giso.push_back(iso);
  }
  s->threads = cfg.worker_size;
  s->fn = mixed_persistent_kernel(cfg.worker_size);
  s->nb = cfg.num_blocks > 0 ? cfg.num_blocks : resident_blocks(s->fn, s->threads);
  // tickets one pause can leave is at most one reservation per CTA; twice that covers a pause
  // recorded next to the undrained remainder of the previous one
  s->orphan_cap = (uint32_t)(2 * s->nb * cfg.worker_size);
  int rc = s->nb > 0 ? ATOS_OK : ATOS_ERR_CUDA;
  if (!rc) rc = rc_of(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_arena, (size_t)budget_bytes));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_slots, sizeof(Instance) * max_slots));
  if (!rc) rc = rc_of(pool_malloc_host((void**)&s->h_slots, sizeof(Instance) * max_slots));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_active, sizeof(Instance) * max_slots));
  if (!rc) rc = rc_of(pool_malloc_host((void**)&s->h_active, sizeof(Instance) * max_slots));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_qctl, sizeof(QueueCtl) * max_slots));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_stats, sizeof(unsigned long long) * kNumStats * max_slots));
  if (!rc) rc = rc_of(pool_malloc_host((void**)&s->h_stats, sizeof(unsigned long long) * kNumStats * max_slots));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_ctl, sizeof(DevCtl)));
  if (!rc) rc = rc_of(pool_malloc_host((void**)&s->h_ctl, sizeof(DevCtl)));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_fin, sizeof(int) * max_slots));
  if (!rc) rc = rc_of(pool_malloc_host((void**)&s->h_fin, sizeof(int) * max_slots));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_results, batch_result_bytes() * max_slots));  // by active index
  if (!rc) rc = rc_of(pool_malloc_host((void**)&s->h_results, batch_result_bytes() * max_slots));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_cert_idx, sizeof(int) * max_slots));
  if (!rc) rc = rc_of(pool_malloc_host((void**)&s->h_cert_idx, sizeof(int) * max_slots));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_cert, sizeof(double) * max_slots));
  if (!rc) rc = rc_of(pool_malloc_host((void**)&s->h_cert, sizeof(double) * max_slots));
  if (!rc) rc = rc_of(pool_malloc((void**)&s->d_jobs, sizeof(SpreadJob) * max_slots));
  if (!rc) rc = rc_of(pool_malloc_host((void**)&s->h_jobs, sizeof(SpreadJob) * max_slots));
  if (!rc) rc = rc_of(cudaMemsetAsync(s->d_ctl, 0, sizeof(DevCtl), s->stream));
  if (rc) {
    delete s;
    return rc;
  }
  s->arena.init(s->d_arena, (size_t)budget_bytes);
  s->slots.resize(max_slots);
  *out = s;
  return ATOS_OK;
}

int atos_server_submit(atos_server_t s, const atos_instance* q, int64_t* id) {
  if (!s || !q || !id) return ATOS_ERR_INVALID_ARG;
  if (q->graph < 0 || q->graph >= (int)s->graphs.size() || !q->out) return ATOS_ERR_INVALID_ARG;
  const int32_t n = s->gn[q->graph];
  if (n < 1) return ATOS_ERR_INVALID_ARG;
  if (q->app == ATOS_APP_BFS && (q->source < 0 || q->source >= n)) return ATOS_ERR_INVALID_ARG;
  if (q->app == ATOS_APP_PAGERANK && !(q->alpha > 0.0f && q->alpha < 1.0f && q->eps > 0.0f)) return ATOS_ERR_INVALID_ARG;
  if (q->app != ATOS_APP_BFS && q->app != ATOS_APP_PAGERANK && q->app != ATOS_APP_COLOR) return ATOS_ERR_INVALID_ARG;
  int slot = -1;
  for (int i = 0; i < s->max_slots; ++i)
    if (s->slots[i].state == kFree) {
      slot = i;
      break;
    }
  if (slot < 0) return ATOS_ERR_BUSY;
  uint32_t cap = 0;
  const size_t bytes = request_bytes(s, q->app, n, &cap);
  const size_t off = s->arena.alloc(bytes);
  if (off == SIZE_MAX) return ATOS_ERR_BUSY;  // not admitted: the footprint does not fit now
  // carve the scratch
  char* p = s->d_arena + off;
  auto take = [&](size_t nb) {
    char* r = p;
    p += (nb + 255) & ~(size_t)255;
    return r;
  };
  const int32_t *rp, *col;
  int32_t iso = 0;
  graph_device_csr(s->graphs[q->graph], &rp, &col, &iso);
  SpreadJob job;
  memset(&job, 0, sizeof(job));
  int32_t hubs = 0;
  HubMap hub = {0, 1, 1, 0};
  if (q->app != ATOS_APP_BFS && (s->cfg.flags & ATOS_FLAG_SPREAD_IDS)) {
    // the graph's spread-id copy (built the first time, synchronising the server stream)
    const int rc2 = graph_spread_csr(s->graphs[q->graph], &rp, &col, s->stream, &job.perm, &hubs, &hub);
    if (rc2) {
      s->arena.release(off, bytes);
      return rc2;
    }
    job.src = take((size_t)n * 4);
    job.dst = q->out;
    job.n = n;
  }
  Instance I;
  memset(&I, 0, sizeof(I));
  I.row_ptr = rp;
  I.col = col;
  I.n = n;
  I.ring = (unsigned long long*)take((size_t)cap * 8);
  I.cap = cap;
  I.orphans[0] = (unsigned*)take((size_t)s->orphan_cap * 4);
  I.orphans[1] = (unsigned*)take((size_t)s->orphan_cap * 4);
  I.orphan_cap = s->orphan_cap;
  I.ctl = s->d_qctl + slot;
  I.stats = s->d_stats + (size_t)kNumStats * slot;
  Slot& sl = s->slots[slot];
  sl.alpha = 0.85f;
  sl.exact_sum = 0.0;
  if (q->app == ATOS_APP_BFS) {
    I.app = kAppBfs;
    I.prefix_len = 1;
    I.prefix_item = q->source;
    I.depth = (int32_t*)q->out;
  } else if (q->app == ATOS_APP_PAGERANK) {
    I.app = kAppPr;
    I.prefix_len = (uint32_t)n;
    I.prefix_item = -1;
    I.rank = job.src ? (float*)job.src : (float*)q->out;
    I.hubs = hubs;
    I.hub = hub;
    I.res = (float*)take((size_t)n * 4);
    I.cert_y = (double*)take((size_t)n * 8);
    I.exact_sum = (double)n - (double)q->alpha * iso;
    I.qbits = (uint32_t*)take((size_t)(n + 31) / 32 * 4);
    I.alpha = q->alpha;
    I.eps = q->eps;
    I.check_size = s->cfg.check_size > 0 ? (uint32_t)s->cfg.check_size : 32u;
    I.pr_crossing = (s->cfg.flags & ATOS_FLAG_PR_CROSSING) ? 1 : 0;
    sl.alpha = q->alpha;
    sl.exact_sum = (double)n - (double)q->alpha * iso;
  } else {
    I.app = kAppGc;
    I.prefix_len = (uint32_t)n;
    I.prefix_item = -1;
    I.color = job.src ? (int32_t*)job.src : (int32_t*)q->out;
    I.gc_ordered = (s->cfg.flags & ATOS_FLAG_GC_ORDERED) ? 1 : 0;
    I.qbits = (uint32_t*)take((size_t)(n + 31) / 32 * 4);
  }
  sl.state = kActive;
  sl.id = s->next_id++;
  sl.app = q->app;
  sl.graph = q->graph;
  sl.off = off;
  sl.bytes = bytes;
  sl.inst = I;
  sl.job = job;
  // initialise on the server stream: descriptor, free ring, state (prepare), PageRank residues.
  // Nothing waits here: the descriptor is copied from pinned staging that this slot alone uses
  // (the slot is not reused before a later step has synchronised the stream), and the next
  // epoch is ordered after these operations on the same stream.
  s->h_slots[slot] = I;
  int rc = rc_of(cudaMemcpyAsync(s->d_slots + slot, s->h_slots + slot, sizeof(Instance), cudaMemcpyHostToDevice,
                                 s->stream));
  if (!rc) rc = rc_of(cudaMemsetAsync(I.ring, 0xff, (size_t)cap * 8, s->stream));
  if (!rc) rc = rc_of(launch_prepare(s->d_slots + slot, 1, n, s->d_ctl, 0u, 1u, s->stream));
  if (!rc && I.app == kAppPr) rc = rc_of(launch_pr_init(s->d_slots + slot, 1, s->gnnz[q->graph], s->stream));
  if (rc) {
    release_slot(s, slot);
    return rc;
  }
  *id = sl.id;
  return ATOS_OK;
}

int atos_server_step(atos_server_t s, int64_t slice_ns, int32_t* active_left) {
  if (!s || slice_ns < 0) return ATOS_ERR_INVALID_ARG;
  s->active_idx.clear();
  for (int i = 0; i < s->max_slots; ++i)
    if (s->slots[i].state == kActive) {
      s->h_active[s->active_idx.size()] = s->slots[i].inst;
      s->active_idx.push_back(i);
    }
  const int na = (int)s->active_idx.size();
  if (na == 0) {
    if (active_left) *active_left = 0;
    return ATOS_OK;
  }
  cudaStream_t st = s->stream;
  SRV_TRY(cudaMemcpyAsync(s->d_active, s->h_active, sizeof(Instance) * na, cudaMemcpyHostToDevice, st));
  memset(s->h_ctl, 0, sizeof(DevCtl));  // pinned: the copy may run after this call returns
  s->h_ctl->next_inst = (unsigned)na;
  SRV_TRY(cudaMemcpyAsync(s->d_ctl, s->h_ctl, sizeof(DevCtl), cudaMemcpyHostToDevice, st));
  count_launches(1);
  server_epoch_begin<<<na, 256, 0, st>>>(s->d_active, s->epoch, &s->d_ctl->status);
  Launch L;
  memset(&L, 0, sizeof(L));
  L.insts = s->d_active;
  L.ninst = na;
  L.window = na;
  L.fetch = s->cfg.fetch_size;
  L.policy = s->cfg.fetch_policy;
  L.nworkers = std::max(1, s->nb / na);
  L.status = &s->d_ctl->status;
  L.next_inst = &s->d_ctl->next_inst;
  L.fail_site = &s->d_ctl->fail_site;
  L.spin_limit_ns = s->cfg.spin_limit_ns > 0 ? s->cfg.spin_limit_ns : 4000000000LL;
  L.lifetime_ns = L.spin_limit_ns * 16;
  L.slice_ns = slice_ns > 0 ? slice_ns : 1000000;
  L.epoch = s->epoch;
  SRV_TRY(launch_kernel(s->fn, dim3(s->nb), s->threads, L, st));
  // finish the requests that terminated in this epoch on the device (PageRank normalised, colours
  // counted), then read flags, statistics and results back: one synchronisation per epoch
  count_launches(1);
  server_gather_finished<<<(na + 255) / 256, 256, 0, st>>>(s->d_active, na, s->d_fin);
  int max_n = 1;
  for (int k = 0; k < na; ++k) max_n = std::max(max_n, (int)s->h_active[k].n);
  SRV_TRY(batch_finish_terminated(s->d_active, na, max_n, s->d_results, st));
  const size_t rb = batch_result_bytes();
  SRV_TRY(cudaMemcpyAsync(s->h_fin, s->d_fin, sizeof(int) * na, cudaMemcpyDeviceToHost, st));
  SRV_TRY(cudaMemcpyAsync(s->h_ctl, s->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
  SRV_TRY(cudaMemcpyAsync(s->h_stats, s->d_stats, sizeof(unsigned long long) * kNumStats * s->max_slots,
                          cudaMemcpyDeviceToHost, st));
  SRV_TRY(cudaMemcpyAsync(s->h_results, s->d_results, rb * na, cudaMemcpyDeviceToHost, st));
  SRV_TRY(cudaStreamSynchronize(st));
  s->epoch++;
  s->epochs++;
  const int status = s->h_ctl->status;
  // complete the terminated requests (or fail every active one if the epoch failed)
  std::vector<int> finished, finished_k;
  for (int k = 0; k < na; ++k)
    if (status != 0 || s->h_fin[k]) finished.push_back(s->active_idx[k]), finished_k.push_back(k);
  // FP64 certificates of the finished PageRank outputs (a second synchronisation, only in epochs
  // that finished one)
  int ncert = 0, cert_n = 1;
  int64_t cert_nnz = 1;
  std::vector<int> cert_of(finished.size(), -1);
  if (status == 0)
    for (size_t f = 0; f < finished.size(); ++f) {
      const Slot& sl = s->slots[finished[f]];
      if (sl.app != ATOS_APP_PAGERANK) continue;
      cert_of[f] = ncert;
      s->h_cert_idx[ncert++] = finished_k[f];
      cert_n = std::max(cert_n, (int)sl.inst.n);
      cert_nnz = std::max(cert_nnz, s->gnnz[sl.graph]);
    }
  // spread-id results back to the callers' ids
  int njobs = 0, jobs_n = 1;
  if (status == 0)
    for (size_t f = 0; f < finished.size(); ++f) {
      const Slot& sl = s->slots[finished[f]];
      if (!sl.job.src) continue;
      s->h_jobs[njobs++] = sl.job;
      jobs_n = std::max(jobs_n, (int)sl.job.n);
    }
  if (njobs) {
    SRV_TRY(cudaMemcpyAsync(s->d_jobs, s->h_jobs, sizeof(SpreadJob) * njobs, cudaMemcpyHostToDevice, st));
    SRV_TRY(unspread_jobs(s->d_jobs, njobs, jobs_n, st));
  }
  if (ncert) {
    SRV_TRY(cudaMemcpyAsync(s->d_cert_idx, s->h_cert_idx, sizeof(int) * ncert, cudaMemcpyHostToDevice, st));
    SRV_TRY(pr_certify_outputs(s->d_active, s->d_cert_idx, ncert, cert_n, cert_nnz, s->d_cert, st));
    SRV_TRY(cudaMemcpyAsync(s->h_cert, s->d_cert, sizeof(double) * ncert, cudaMemcpyDeviceToHost, st));
  }
  if (ncert || njobs) SRV_TRY(cudaStreamSynchronize(st));
  for (size_t f = 0; f < finished.size(); ++f) {
    const int i = finished[f];
    Slot& sl = s->slots[i];
    atos_completion c;
    memset(&c, 0, sizeof(c));
    c.id = sl.id;
    c.status = status;
    c.app = sl.app;
    c.graph = sl.graph;
    c.tasks = (int64_t)s->h_stats[i * kNumStats + kStatTasks];
    c.edges = (int64_t)s->h_stats[i * kNumStats + kStatEdges];
    c.epochs = s->epochs;
    double sum_rank = 0, sum_res = 0;
    int ncol = 0;
    batch_result_read(s->h_results + rb * finished_k[f], &sum_rank, &sum_res, &ncol);
    if (sl.app == ATOS_APP_PAGERANK && cert_of[f] >= 0)
      c.error_bound = s->h_cert[cert_of[f]] / ((1.0 - (double)sl.alpha) * std::max(sl.exact_sum, 1e-300));
    if (sl.app == ATOS_APP_COLOR) c.num_colors = ncol;
    s->done.push_back(c);
    release_slot(s, i);
  }

  if (active_left) *active_left = na - (int)finished.size();
  return ATOS_OK;
}

int atos_server_poll(atos_server_t s, atos_completion* out, int32_t max, int32_t* count) {
  if (!s || !count || max < 0 || (max > 0 && !out)) return ATOS_ERR_INVALID_ARG;
  int32_t k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *count = k;
  return ATOS_OK;
}

int atos_server_info(atos_server_t s, int32_t* active, int64_t* arena_used, int64_t* arena_size, int64_t* epochs) {
  if (!s) return ATOS_ERR_INVALID_ARG;
  if (active) {
    int a = 0;
    for (const Slot& sl : s->slots) a += sl.state == kActive;
    *active = a;
  }
  if (arena_used) *arena_used = (int64_t)s->arena.used;
  if (arena_size) *arena_size = (int64_t)s->arena.size;
  if (epochs) *epochs = s->epochs;
  return ATOS_OK;
}

int atos_server_destroy(atos_server_t s) {
  delete s;
  return ATOS_OK;
}

}  // extern "C"
