// relabel.cu -- an internal copy of a graph with its vertex ids spread over the id range.
//
// RMAT-like graphs put their hubs at the smallest ids, and CSR rows are sorted, so every row
// starts with the same few hubs.  A warp of a task body then updates (PageRank's residue
// scatter) or reads (colouring) 32 entries of a state array that lie in a few cache lines, all in
// the same few L2 slices, and those slices become the bottleneck.  The copy renames vertex v to
// pi(v) = (a v + c) mod n with a ~ 0.618 n coprime to n: a bijection that sends neighbouring ids
// far apart, so the same row touches lines spread over all slices.  Row pi(v) of the copy lists
// pi(u) for the neighbours u of v, in v's order.  Results computed on the copy are mapped back
// with one gather (out[v] = copy_out[pi(v)]).
#include <cuda_runtime.h>
#include <stdint.h>

#include <numeric>

#include "launch.cuh"
#include "state.cuh"

namespace atos {
namespace bsp {
cudaError_t scan_inplace(int32_t* a, int32_t F, int32_t* bsums, cudaStream_t s);
}

namespace {

__device__ __forceinline__ int32_t spread_id(uint32_t v, uint64_t a, uint64_t c, uint32_t n) {
  return (int32_t)((a * v + c) % n);
}

// perm[v] = pi(v) for every v (the one place the 64-bit product and remainder are computed), and
// the degrees of the copy's rows.
__global__ void spread_perm_kernel(const int32_t* __restrict__ rp, int32_t n, uint64_t a, uint64_t c,
                                   int32_t* __restrict__ perm, int32_t* __restrict__ new_rp) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t p = spread_id((uint32_t)v, a, c, (uint32_t)n);
    perm[v] = p;
    new_rp[p] = __ldg(rp + v + 1) - __ldg(rp + v);
  }
}

// One warp per row of the original graph; lanes stride the row and rename through perm.
__global__ void spread_cols_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n,
                                   const int32_t* __restrict__ perm, const int32_t* __restrict__ new_rp,
                                   int32_t* __restrict__ new_col) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int s = __ldg(rp + v), e = __ldg(rp + v + 1);
    const int d = __ldg(new_rp + __ldg(perm + v));
    for (int k = s + lane; k < e; k += 32) new_col[d + (k - s)] = __ldg(perm + __ldg(col + k));
  }
}

template <class T>
__global__ void unspread_kernel(const T* __restrict__ src, T* __restrict__ dst, int32_t n, uint64_t a, uint64_t c) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    dst[v] = src[spread_id((uint32_t)v, a, c, (uint32_t)n)];
}

int grid_for(int64_t work, int threads, int cap) {
  const int64_t g = (work + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

// The multiplier of the spreading permutation: the integer nearest 0.618 n that is coprime to n.
uint64_t spread_multiplier(int32_t n) {
  if (n <= 2) return 1;
  uint64_t a = (uint64_t)((double)n * 0.6180339887498949);
  if (a < 1) a = 1;
  while (std::gcd(a, (uint64_t)n) != 1) ++a;
  return a % (uint64_t)n;
}

// Builds the spread copy: perm (n entries, v -> pi(v)), new_rp (n + 1 entries) and new_col (nnz
// entries); bsums needs n / 1024 + 2 entries of scratch.
cudaError_t spread_build(const int32_t* rp, const int32_t* col, int32_t n, uint64_t a, uint64_t c, int32_t* perm,
                         int32_t* new_rp, int32_t* new_col, int32_t* bsums, cudaStream_t s) {
  count_launches(2);
  spread_perm_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(rp, n, a, c, perm, new_rp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = bsp::scan_inplace(new_rp, n, bsums, s);  // exclusive scan; new_rp[n] = nnz
  if (e != cudaSuccess) return e;
  spread_cols_kernel<<<grid_for((int64_t)n * 32, 256, 8192), 256, 0, s>>>(rp, col, n, perm, new_rp, new_col);
  return cudaGetLastError();
}

__global__ void unspread_jobs_kernel(const SpreadJob* jobs) {
  const SpreadJob J = jobs[blockIdx.y];
  const int32_t* src = (const int32_t*)J.src;  // 4-byte elements (float ranks or int32 colours)
  int32_t* dst = (int32_t*)J.dst;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < J.n; v += gridDim.x * blockDim.x)
    dst[v] = src[spread_id((uint32_t)v, J.a, J.c, (uint32_t)J.n)];
}

cudaError_t unspread_jobs(const SpreadJob* d_jobs, int njobs, int max_n, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  count_launches(1);
  unspread_jobs_kernel<<<dim3(grid_for(max_n, 256, 1024), njobs), 256, 0, s>>>(d_jobs);
  return cudaGetLastError();
}

cudaError_t unspread_f32(const float* src, float* dst, int32_t n, uint64_t a, uint64_t c, cudaStream_t s) {
  count_launches(1);
  unspread_kernel<float><<<grid_for(n, 256, 4096), 256, 0, s>>>(src, dst, n, a, c);
  return cudaGetLastError();
}

cudaError_t unspread_i32(const int32_t* src, int32_t* dst, int32_t n, uint64_t a, uint64_t c, cudaStream_t s) {
  count_launches(1);
  unspread_kernel<int32_t><<<grid_for(n, 256, 4096), 256, 0, s>>>(src, dst, n, a, c);
  return cudaGetLastError();
}

}  // namespace atos
