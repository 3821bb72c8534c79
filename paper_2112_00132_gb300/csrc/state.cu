// state.cu -- per-launch preparation and bookkeeping kernels shared by all applications.
//
//   prepare_kernel      resets every instance's queue control block and statistics, refills the
//                       rings with EMPTY when the previous launch on this scratch failed (after a
//                       clean run every slot is already EMPTY), and writes the initial state of
//                       the application: BFS depth (INT32_MAX, source 0), PageRank rank = 1 -
//                       alpha and the initial residue (one push of the initial rank, i.e.
//                       (1 - alpha) alpha sum_{u in N(v)} 1/deg(u)), colouring colour = -1.
//   next_generation     discrete strategy: the tasks pushed during the last launch become the
//                       next generation; reports the largest generation over instances.
//   finalize_kernel     remembers whether the launch failed (so the next prepare refills rings).
#include <atomic>

#include "engine.cuh"
#include "launch.cuh"
#include "state.cuh"

namespace atos {

static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(unsigned n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

__global__ void prepare_kernel(Instance* insts, DevCtl* ctl, uint32_t flags, unsigned window) {
  const Instance I = insts[blockIdx.y];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (ctl->dirty)
    for (uint32_t k = tid; k < I.cap; k += stride) I.ring[k] = kFreeSlot;
  if (tid == 0 && blockIdx.y == 0) ctl->t_origin = globaltimer();
  if (tid == 0) {
    QueueCtl* c = I.ctl;
    const unsigned phantom = (flags & ATOS_FLAG_PHANTOM_TASK) ? 1u : 0u;
    c->word = (unsigned long long)(I.prefix_len + phantom) << 32;
    c->head = 0;
    c->check = 0;
    c->vword = 0;
    c->vdone = 0;
    c->finished = 0;
    c->succ = -2;
    c->gen_begin = 0;
    c->gen_end = I.prefix_len;
    c->orphan_count[0] = c->orphan_count[1] = 0;
    c->orphan_head = 0;
    c->seg_next = 0;
    for (int k = 0; k < kNumStats; ++k) I.stats[k] = 0;
    if (blockIdx.y == 0) {
      ctl->status = 0;
      ctl->fail_site = 0;
      ctl->next_inst = window;
      ctl->maxgen = 0;
    }
  }
  const int n = I.n;
  switch (I.app) {
    case kAppBfs:
      for (int v = tid; v < n; v += stride) I.depth[v] = v == I.prefix_item ? 0 : kUnreached;
      if (I.expanded)
        for (int v = tid; v < n; v += stride) I.expanded[v] = kUnreached;
      break;
    case kAppPr: {
      const float a = I.alpha, base = (1.0f - I.alpha) * I.alpha;
      for (int v = tid; v < n; v += stride) I.rank[v] = 1.0f - a;
      const int words = (n + 31) >> 5;
      for (int w = tid; w < words; w += stride) {
        const int rem = n - (w << 5);
        I.qbits[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
      }
      // the initial residue is accumulated by pr_init_residue_kernel (edge-balanced)
      for (int v = tid; v < n; v += stride) I.res[v] = 0.0f;
      (void)base;
      break;
    }
    case kAppGc: {
      for (int v = tid; v < n; v += stride) I.color[v] = -1;
      const int words = (n + 31) >> 5;  // every vertex starts with its assign task queued
      for (int w = tid; w < words; w += stride) {
        const int rem = n - (w << 5);
        I.qbits[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
      }
      break;
    }
  }
}

// Largest i in [lo, hi) with row_ptr[i] <= k (the row holding CSR entry k).
__device__ __forceinline__ int row_of(const int32_t* row_ptr, int lo, int hi, int k) {
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(row_ptr + mid) <= k) lo = mid;
    else hi = mid;
  }
  return lo;
}

// residue[v] = (1 - alpha) alpha sum_{u in N(v)} 1/deg(u), edge-balanced: each thread takes
// kRun consecutive CSR entries (so a hub row is spread over many threads), finds the row of its
// first entry by binary search, and adds one partial sum per row it touches.
constexpr int kInitRun = 8;

__global__ void pr_init_residue_kernel(Instance* insts) {
  const Instance I = insts[blockIdx.y];
  if (I.app != kAppPr) return;
  const int64_t nnz = __ldg(I.row_ptr + I.n);
  const float base = (1.0f - I.alpha) * I.alpha;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kInitRun;
  for (int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kInitRun; k0 < nnz; k0 += stride) {
    const int k1 = (int)(k0 + kInitRun < nnz ? k0 + kInitRun : nnz);
    int r = row_of(I.row_ptr, 0, I.n, (int)k0);
    int next = __ldg(I.row_ptr + r + 1);
    float acc = 0.0f;
    for (int k = (int)k0; k < k1; ++k) {
      while (k >= next) {  // entry k starts a later row: flush the finished one
        if (acc != 0.0f) atomicAdd(I.res + r, base * acc);
        acc = 0.0f;
        ++r;
        next = __ldg(I.row_ptr + r + 1);
      }
      const int u = __ldg(I.col + k);
      acc += 1.0f / (float)(__ldg(I.row_ptr + u + 1) - __ldg(I.row_ptr + u));
    }
    if (acc != 0.0f) atomicAdd(I.res + r, base * acc);
  }
}

cudaError_t launch_pr_init(Instance* d_insts, int ninst, int64_t max_nnz, cudaStream_t s) {
  int64_t per = (max_nnz + 256 * kInitRun - 1) / (256 * kInitRun);
  int gx = (int)(per < 1 ? 1 : (per > 4096 ? 4096 : per));
  count_launches(1);
  pr_init_residue_kernel<<<dim3(gx, ninst), 256, 0, s>>>(d_insts);
  return cudaGetLastError();
}

__global__ void next_generation_kernel(Instance* insts, int ninst, DevCtl* ctl) {
  __shared__ unsigned red[32];
  unsigned mx = 0;
  for (int i = threadIdx.x; i < ninst; i += blockDim.x) {
    QueueCtl* c = insts[i].ctl;
    const unsigned tail = (unsigned)(c->word >> 32);
    const unsigned b = c->gen_end;
    c->gen_begin = b;
    c->gen_end = tail;
    c->head = b;  // tickets below b are consumed: the overflow check may reuse their slots
    mx = max(mx, tail - b);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) ctl->maxgen = mx;
  }
}

// The rings are clean after a run only if it succeeded and every instance ended with as many
// tasks completed as pushed (then every written slot was taken and freed).
__global__ void finalize_kernel(const Instance* insts, int ninst, DevCtl* ctl) {
  __shared__ int unbalanced;
  if (threadIdx.x == 0) unbalanced = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < ninst; i += blockDim.x) {
    const unsigned long long w = insts[i].ctl->word;
    if ((unsigned)(w >> 32) != (unsigned)w) unbalanced = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) ctl->dirty = (ctl->status != 0 || unbalanced) ? 1 : 0;
}

cudaError_t launch_prepare(Instance* d_insts, int ninst, int max_n, DevCtl* d_ctl, uint32_t flags, unsigned window,
                           cudaStream_t s) {
  int per = (max_n + 255) / 256;
  int gx = per < 1 ? 1 : (per > 1024 ? 1024 : per);
  if (ninst > 65535) return cudaErrorInvalidValue;
  count_launches(1);
  prepare_kernel<<<dim3(gx, ninst), 256, 0, s>>>(d_insts, d_ctl, flags, window);
  return cudaGetLastError();
}

cudaError_t launch_next_generation(Instance* d_insts, int ninst, DevCtl* d_ctl, cudaStream_t s) {
  count_launches(1);
  next_generation_kernel<<<1, 1024, 0, s>>>(d_insts, ninst, d_ctl);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Instance* d_insts, int ninst, DevCtl* d_ctl, cudaStream_t s) {
  count_launches(1);
  finalize_kernel<<<1, 256, 0, s>>>(d_insts, ninst, d_ctl);
  return cudaGetLastError();
}

cudaError_t pr_verify_sweep(Instance* d_insts, int ninst, int max_n, DevCtl* d_ctl, cudaStream_t s);

cudaError_t discrete_loop(const void* fn, int threads, int per_block, Launch L, Instance* d_insts, int ninst,
                          int max_n, unsigned first_gen, bool has_pr, DevCtl* d_ctl, DevCtl* h_ctl, cudaStream_t st,
                          int64_t* iterations) {
#define DL_TRY(expr)                     \
  do {                                   \
    cudaError_t _e = (expr);             \
    if (_e != cudaSuccess) return _e;    \
  } while (0)
  int64_t iters = 0;
  unsigned gen = first_gen;
  for (;;) {
    if (iters > (1 << 24)) break;  // the caller sees the unbalanced queues as a failed run
    if (gen == 0) {
      if (!has_pr) break;
      // PageRank: the queues drained; sweep every residue once (Algorithm 4's scan over all ids)
      // and stop only if nothing exceeds epsilon
      DL_TRY(pr_verify_sweep(d_insts, ninst, max_n, d_ctl, st));
      DL_TRY(launch_next_generation(d_insts, ninst, d_ctl, st));
      DL_TRY(cudaMemcpyAsync(h_ctl, d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
      DL_TRY(cudaStreamSynchronize(st));
      if (h_ctl->status) break;
      gen = h_ctl->maxgen;
      if (gen == 0) break;
    }
    const unsigned gx = (gen + per_block - 1) / per_block;
    L.nworkers = (int)gx;
    Launch copy = L;
    void* args[] = {&copy};
    count_launches(1);
    DL_TRY(cudaLaunchKernel(fn, dim3(gx, ninst), dim3(threads), args, 0, st));
    DL_TRY(launch_next_generation(d_insts, ninst, d_ctl, st));
    DL_TRY(cudaMemcpyAsync(h_ctl, d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
    DL_TRY(cudaStreamSynchronize(st));
    iters++;
    if (h_ctl->status) break;
    gen = h_ctl->maxgen;
  }
#undef DL_TRY
  if (iterations) *iterations = iters;
  return cudaSuccess;
}

}  // namespace atos
