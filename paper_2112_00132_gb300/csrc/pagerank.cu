// pagerank.cu -- PageRank kernels: the persistent / discrete instantiations of the task body in
// pagerank.cuh, the discrete final sweep, and the FP64 result reductions and certificate.
//
// Task body summary (Section 5.2, Algorithm 4):
//
// A task is a vertex v.  The worker takes v's residue with an atomic exchange, adds it to
// rank[v], and scatters alpha * residue / deg(v) to every neighbour (red.global.add.f32, no
// return).  It then reserves Check_Size consecutive vertex ids from a round-robin cursor and
// enqueues those whose residue exceeds epsilon.  All arithmetic on ranks and residues is FP32.
//
// Two points the paper leaves open are fixed here:
//   * a vertex is in the queue at most once: a bitmap bit is set by whoever enqueues it and
//     cleared by the worker that pops it (before it takes the residue), so the ring never needs
//     more than n slots and duplicate pops disappear;
//   * termination: the queue draining is not enough, because Algorithm 4 enqueues only through
//     the Check_Size scan.  Workers whose pops come back empty run the scan as their idle
//     function (f2 of the launch API), and once the instance is quiescent (tasks pushed ==
//     tasks completed, value T) they split one full sweep of all n residues into chunks; the
//     instance ends when a sweep that started at quiescence T has covered all n vertices without
//     enqueueing anything and the queue word still reads (T, T).  Nothing can change a residue
//     during such a sweep, so every residue is then at most epsilon.
#include "engine.cuh"
#include "launch.cuh"
#include "pagerank.cuh"
#include "state.cuh"

namespace atos {

// worker 1: thread workers (each lane of a warp runs its own task, PrBody::lane_items)
const void* pr_persistent_kernel(int worker) {
  return worker == 1 ? (const void*)warp_persistent_kernel<PrBody, true> : persistent_kernel_ptr<PrBody>(worker);
}
const void* pr_discrete_kernel(int worker) {
  return worker == 1 ? (const void*)warp_discrete_kernel<PrBody, true> : discrete_kernel_ptr<PrBody>(worker);
}

// Discrete strategy: after a generation comes back empty, one full sweep enqueues every vertex
// whose residue still exceeds epsilon (they form the next generation).
__global__ void pr_sweep_kernel(Instance* insts, int* status) {
  const Instance I = insts[blockIdx.y];
  if (I.app != kAppPr) return;  // batches mix applications
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x; r < I.n; r += stride) {
    const int u = r + threadIdx.x;
    const bool want = u < I.n && pr_try_enqueue(I, u);
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) continue;
    unsigned base = 0;
    if (lane == 0) {
      const unsigned long long old = atomicAdd(&I.ctl->word, (unsigned long long)__popc(m) << 32);
      base = (unsigned)(old >> 32);
      const long long last = (long long)base + __popc(m) - 1;
      const long long prev = last - (long long)I.cap;
      if (prev >= (long long)I.prefix_len && (long long)I.ctl->head <= prev) {
        atomicCAS(status, 0, ATOS_ERR_QUEUE_OVERFLOW);
        base = 0xffffffffu;
      }
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (want && base != 0xffffffffu) {
      const unsigned idx = base + __popc(m & lanemask_lt());
      I.ring[idx & (I.cap - 1)] = ((unsigned long long)idx << 32) | (unsigned)u;
    }
  }
}

cudaError_t pr_verify_sweep(Instance* d_insts, int ninst, int max_n, DevCtl* d_ctl, cudaStream_t s) {
  int gx = (max_n + 255) / 256;
  gx = gx < 1 ? 1 : (gx > 2048 ? 2048 : gx);
  count_launches(1);
  pr_sweep_kernel<<<dim3(gx, ninst), 256, 0, s>>>(d_insts, &d_ctl->status);
  return cudaGetLastError();
}

// FP64 reductions of the result: sum of ranks and of the residues left.
__global__ void pr_sums_kernel(const Instance* inst, DevCtl* ctl) {
  const Instance I = *inst;
  double a = 0.0, b = 0.0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < I.n; v += gridDim.x * blockDim.x) {
    a += (double)I.rank[v];
    b += (double)I.res[v];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&ctl->sum_rank, a);
    atomicAdd(&ctl->sum_res, b);
  }
}

// A posteriori certificate in FP64: with x = rank * (S / sum_rank), where S = n - alpha * (isolated
// vertices) is the exact sum of the fixed point, ||(1 - alpha) 1 + alpha P x - x||_1.  First
// y[v] = sum_{u in N(v)} rank[u] / deg(u) is accumulated edge-balanced (kCertRun consecutive CSR
// entries per thread, FP64 atomics per row touched), then a vertex pass sums |rho_v|.
constexpr int kCertRun = 8;

__device__ __forceinline__ int cert_row_of(const int32_t* row_ptr, int lo, int hi, int k) {
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(row_ptr + mid) <= k) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void pr_cert_pull_kernel(const Instance* inst, double* y) {
  const Instance I = *inst;
  const int64_t nnz = __ldg(I.row_ptr + I.n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kCertRun;
  for (int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kCertRun; k0 < nnz; k0 += stride) {
    const int k1 = (int)(k0 + kCertRun < nnz ? k0 + kCertRun : nnz);
    int r = cert_row_of(I.row_ptr, 0, I.n, (int)k0);
    int next = __ldg(I.row_ptr + r + 1);
    double acc = 0.0;
    for (int k = (int)k0; k < k1; ++k) {
      while (k >= next) {
        if (acc != 0.0) atomicAdd(y + r, acc);
        acc = 0.0;
        ++r;
        next = __ldg(I.row_ptr + r + 1);
      }
      const int u = __ldg(I.col + k);
      acc += (double)I.rank[u] / (double)(__ldg(I.row_ptr + u + 1) - __ldg(I.row_ptr + u));
    }
    if (acc != 0.0) atomicAdd(y + r, acc);
  }
}

__global__ void pr_cert_sum_kernel(const Instance* inst, const double* y, DevCtl* ctl, double S) {
  const Instance I = *inst;
  const double scale = S / ctl->sum_rank;
  const double a = (double)I.alpha;
  double acc = 0.0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < I.n; v += gridDim.x * blockDim.x)
    acc += fabs((1.0 - a) + a * y[v] * scale - (double)I.rank[v] * scale);
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&ctl->cert_l1, acc);
}

__global__ void pr_normalise_kernel(const Instance* inst, const DevCtl* ctl) {
  const Instance I = *inst;
  const double inv = 1.0 / ctl->sum_rank;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < I.n; v += gridDim.x * blockDim.x)
    I.rank[v] = (float)((double)I.rank[v] * inv);
}

// Output certificates of several instances (see state.cuh): blockIdx.y selects d_idx[y].
__global__ void pr_out_cert_zero_kernel(const Instance* insts, const int* idx) {
  const Instance I = insts[idx[blockIdx.y]];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < I.n; v += gridDim.x * blockDim.x) I.cert_y[v] = 0.0;
}

__global__ void pr_out_cert_pull_kernel(const Instance* insts, const int* idx) {
  const Instance I = insts[idx[blockIdx.y]];
  const int64_t nnz = __ldg(I.row_ptr + I.n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kCertRun;
  for (int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kCertRun; k0 < nnz; k0 += stride) {
    const int k1 = (int)(k0 + kCertRun < nnz ? k0 + kCertRun : nnz);
    int r = cert_row_of(I.row_ptr, 0, I.n, (int)k0);
    int next = __ldg(I.row_ptr + r + 1);
    double acc = 0.0;
    for (int k = (int)k0; k < k1; ++k) {
      while (k >= next) {
        if (acc != 0.0) atomicAdd(I.cert_y + r, acc);
        acc = 0.0;
        ++r;
        next = __ldg(I.row_ptr + r + 1);
      }
      const int u = __ldg(I.col + k);
      acc += (double)I.rank[u] / (double)(__ldg(I.row_ptr + u + 1) - __ldg(I.row_ptr + u));
    }
    if (acc != 0.0) atomicAdd(I.cert_y + r, acc);
  }
}

__global__ void pr_out_cert_sum_kernel(const Instance* insts, const int* idx, double* out) {
  const Instance I = insts[idx[blockIdx.y]];
  const double S = I.exact_sum, a = (double)I.alpha;
  double acc = 0.0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < I.n; v += gridDim.x * blockDim.x)
    acc += fabs((1.0 - a) + a * S * I.cert_y[v] - S * (double)I.rank[v]);
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out + blockIdx.y, acc);
}

cudaError_t pr_certify_outputs(const Instance* d_insts, const int* d_idx, int count, int max_n, int64_t max_nnz,
                               double* d_out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (count > 65535) return cudaErrorInvalidValue;
  cudaMemsetAsync(d_out, 0, sizeof(double) * (size_t)count, s);
  int gx = (max_n + 255) / 256;
  gx = gx < 1 ? 1 : (gx > 1024 ? 1024 : gx);
  int64_t per = (max_nnz + 256 * kCertRun - 1) / (256 * kCertRun);
  const int gy = (int)(per < 1 ? 1 : (per > 2048 ? 2048 : per));
  count_launches(3);
  pr_out_cert_zero_kernel<<<dim3(gx, count), 256, 0, s>>>(d_insts, d_idx);
  pr_out_cert_pull_kernel<<<dim3(gy, count), 256, 0, s>>>(d_insts, d_idx);
  pr_out_cert_sum_kernel<<<dim3(gx, count), 256, 0, s>>>(d_insts, d_idx, d_out);
  return cudaGetLastError();
}

// certificate_y: FP64 scratch of n entries (needed only when `certificate`).
cudaError_t pr_finish(Instance* d_insts, int ninst, int n, int64_t nnz, DevCtl* d_ctl, double* certificate_y,
                      double exact_sum, cudaStream_t s) {
  (void)ninst;
  cudaMemsetAsync(&d_ctl->sum_rank, 0, 3 * sizeof(double), s);
  int gx = (n + 255) / 256;
  gx = gx < 1 ? 1 : (gx > 2048 ? 2048 : gx);
  count_launches(2);
  pr_sums_kernel<<<gx, 256, 0, s>>>(d_insts, d_ctl);
  if (certificate_y) {
    cudaMemsetAsync(certificate_y, 0, sizeof(double) * (size_t)n, s);
    int64_t per = (nnz + 256 * kCertRun - 1) / (256 * kCertRun);
    const int gy = (int)(per < 1 ? 1 : (per > 4096 ? 4096 : per));
    count_launches(2);
    pr_cert_pull_kernel<<<gy, 256, 0, s>>>(d_insts, certificate_y);
    pr_cert_sum_kernel<<<gx, 256, 0, s>>>(d_insts, certificate_y, d_ctl, exact_sum);
  }
  pr_normalise_kernel<<<gx, 256, 0, s>>>(d_insts, d_ctl);
  return cudaGetLastError();
}

}  // namespace atos
