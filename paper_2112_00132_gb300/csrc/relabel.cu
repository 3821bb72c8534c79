// relabel.cu -- an internal copy of a graph with its vertex ids rearranged for the task bodies.
//
// RMAT-like graphs put their hubs at the smallest ids, and CSR rows are sorted, so every row
// starts with the same few hubs.  A warp of a task body then updates (PageRank's residue
// scatter) or reads (colouring) 32 entries of a state array that lie in a few cache lines, all in
// the same few L2 slices, and those slices become the bottleneck.  The copy renames the vertices
// so that neighbouring ids are far apart and no line of the state arrays holds two hubs:
//
//   * the hubs: the (at most kHubRegion, and at most 2^k = the largest power of two <= n / 32)
//     vertices of highest degree, taken as whole degree classes (four classes per power of two)
//     while they fit, ranked by decreasing class and increasing id within a class.  The hub of
//     rank i gets the id 32 ((mul i + add) mod 2^k): the first entry of a 128-byte line of every
//     4-byte state array, the lines of consecutive ranks far apart (mul ~ 0.618 2^k, odd).  A
//     PageRank CTA adds the residue updates its batch sends to the first hubs in shared memory
//     (the rank of the hub at id u is one multiplication away, see HubMap) and sends each touched
//     hub one update per batch;
//   * every other vertex, of rank r among the non-hubs in id order, takes the r'-th id that no hub
//     holds, r' = (a r + c) mod m, m = n - H, a ~ 0.618 m coprime to m: a bijection that sends
//     neighbouring ids far apart, so a row's updates land on lines spread over all L2 slices.
//
// perm[v] is the copy's id of v.  Row perm[v] of the copy lists perm[u] for the neighbours u of v,
// in v's order.  Results computed on the copy are mapped back with one gather
// (out[v] = copy_out[perm[v]]).  The plan (H, the hub map, a, c) is made on the device from a
// histogram of the degree classes; the host reads it back once the build is done.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.cuh"
#include "state.cuh"

namespace atos {
namespace bsp {
cudaError_t scan_inplace(int32_t* a, int32_t F, int32_t* bsums, cudaStream_t s);
}

namespace {

constexpr int kDegBuckets = 128;

// Degree class: 0 for isolated vertices, else 1 + 4 floor(log2 d) + the two bits below d's
// leading one (four classes per power of two, non-decreasing in d).
__device__ __forceinline__ int degree_bucket(int d) {
  if (d <= 0) return 0;
  const int lg = 31 - __clz(d);
  const int sub = lg >= 2 ? (d >> (lg - 2)) & 3 : (d << (2 - lg)) & 3;
  return 1 + 4 * lg + sub;
}

struct HubPlan {
  int32_t hubs;        // H
  int32_t bmin;        // lowest degree class of the hubs (kDegBuckets: none)
  int32_t m;           // n - H
  int32_t long_count;  // rows longer than kLongRow, listed for the renaming of their entries
  uint64_t a, c;       // spreading map of the non-hubs
  HubMap map;          // where the hubs sit
  int32_t hist[kDegBuckets];
};

__device__ __forceinline__ int32_t spread_id(uint32_t r, uint64_t a, uint64_t c, uint32_t m) {
  return (int32_t)((a * r + c) % m);
}

__global__ void hub_hist_kernel(const int32_t* __restrict__ rp, int32_t n, HubPlan* plan) {
  __shared__ int h[kDegBuckets];
  for (int b = threadIdx.x; b < kDegBuckets; b += blockDim.x) h[b] = 0;
  __syncthreads();
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    atomicAdd(&h[degree_bucket(__ldg(rp + v + 1) - __ldg(rp + v))], 1);
  __syncthreads();
  for (int b = threadIdx.x; b < kDegBuckets; b += blockDim.x)
    if (h[b]) atomicAdd(&plan->hist[b], h[b]);
}

__device__ uint64_t gcd_u64(uint64_t x, uint64_t y) {
  while (y) {
    const uint64_t t = x % y;
    x = y;
    y = t;
  }
  return x;
}

// One thread: take whole degree classes from the top while they fit (at most kHubRegion hubs and
// one per line of the first 2^k lines), the hub map, then the spreading map of the rest.
__global__ void hub_plan_kernel(HubPlan* plan, int32_t n, int32_t region) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t lines = 0;  // 2^k, the largest power of two <= n / 32 (0: no hubs)
  if (n >= 32) {
    lines = 1;
    while (lines * 2 <= (uint32_t)(n / 32)) lines *= 2;
  }
  if ((uint32_t)region > lines) region = (int32_t)lines;
  int cum = 0, bmin = kDegBuckets;
  for (int b = kDegBuckets - 1; b >= 1; --b) {
    const int c = plan->hist[b];
    if (cum + c > region) break;
    cum += c;
    bmin = b;
  }
  HubMap hm;
  hm.mask = lines ? lines - 1 : 0;
  hm.mul = ((uint32_t)((double)lines * 0.6180339887498949) | 1u) & hm.mask;
  if (hm.mask == 0) hm.mul = 1;
  hm.mul |= 1u;
  uint32_t x = hm.mul;  // Newton's iteration for mul^-1 mod 2^32 (odd mul: 3 bits, doubling each step)
  for (int it = 0; it < 5; ++it) x *= 2u - hm.mul * x;
  hm.inv = x;
  hm.add = lines / 2;
  const int32_t m = n - cum;
  uint64_t a = 1;
  if (m > 2) {
    a = (uint64_t)((double)m * 0.6180339887498949);
    if (a < 1) a = 1;
    while (gcd_u64(a, (uint64_t)m) != 1) ++a;
    a %= (uint64_t)m;
  }
  plan->hubs = cum;
  plan->bmin = bmin;
  plan->m = m;
  plan->a = a;
  plan->c = (uint64_t)(m / 2);
  plan->map = hm;
}

__device__ __forceinline__ bool is_hub(const int32_t* rp, int v, int bmin) {
  const int b = degree_bucket(__ldg(rp + v + 1) - __ldg(rp + v));
  return b >= 1 && b >= bmin;
}

__global__ void hub_flag_kernel(const int32_t* __restrict__ rp, int32_t n, const HubPlan* plan, int32_t* flags) {
  const int bmin = plan->bmin;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    flags[v] = is_hub(rp, v, bmin) ? 1 : 0;
}

// After the scan, before[v] = hubs with a smaller id than v.  Hubs are listed in id order.
__global__ void hub_list_kernel(const int32_t* __restrict__ rp, int32_t n, const HubPlan* plan,
                                const int32_t* __restrict__ before, int32_t* list) {
  const int bmin = plan->bmin;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (is_hub(rp, v, bmin)) list[before[v]] = v;
}

// One CTA of 1024 threads: bitonic sort of the hub list by (degree class descending, id), keys
// in dynamic shared memory (kHubRegion 64-bit keys); then perm[hub of rank i] = map.id_of(i), and
// occ marks the ids the hubs hold (occ zeroed before).
constexpr int kSortThreads = 1024;

__global__ void __launch_bounds__(kSortThreads) hub_sort_kernel(const int32_t* __restrict__ rp, const HubPlan* plan,
                                                               const int32_t* __restrict__ list, int32_t* perm,
                                                               int32_t* occ) {
  extern __shared__ unsigned long long key[];
  const int H = plan->hubs;
  if (H == 0) return;
  int P = 1;
  while (P < H) P <<= 1;
  for (int i = threadIdx.x; i < P; i += kSortThreads) {
    if (i < H) {
      const int v = list[i];
      const int b = degree_bucket(__ldg(rp + v + 1) - __ldg(rp + v));
      key[i] = ((unsigned long long)(kDegBuckets - 1 - b) << 32) | (unsigned)v;
    } else {
      key[i] = ~0ull;
    }
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += kSortThreads) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long x = key[i], y = key[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) key[i] = y, key[l] = x;
        }
      }
      __syncthreads();
    }
  }
  const HubMap hm = plan->map;
  for (int i = threadIdx.x; i < H; i += kSortThreads) {
    const int32_t id = hm.id_of((uint32_t)i);
    perm[(int)(unsigned)key[i]] = id;
    occ[id] = 1;
  }
}

// After the scan of occ (occ[u] = hub ids below u), list the free ids in order.
__global__ void free_ids_kernel(int32_t n, const int32_t* __restrict__ occ_before, int32_t* free_list) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
    if (occ_before[u + 1] == occ_before[u]) free_list[u - occ_before[u]] = u;
}

// perm[v] for the non-hubs, and the degrees of every row of the copy.
__global__ void spread_perm_kernel(const int32_t* __restrict__ rp, int32_t n, const HubPlan* plan,
                                   const int32_t* __restrict__ before, const int32_t* __restrict__ free_list,
                                   int32_t* __restrict__ perm, int32_t* __restrict__ new_rp) {
  const int bmin = plan->bmin;
  const uint64_t a = plan->a, c = plan->c;
  const uint32_t m = (uint32_t)plan->m;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int p;
    if (is_hub(rp, v, bmin)) {
      p = perm[v];  // placed by the sort
    } else {
      p = free_list[spread_id((uint32_t)(v - before[v]), a, c, m)];
      perm[v] = p;
    }
    new_rp[p] = __ldg(rp + v + 1) - __ldg(rp + v);
  }
}

// One warp per row of the original graph of at most kLongRow entries; lanes stride the row and
// rename through perm.  Longer rows are listed for spread_cols_long_kernel, so that a hub row
// does not hold one warp for its whole length.
constexpr int kLongRow = 2048;

__global__ void spread_cols_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n,
                                   const int32_t* __restrict__ perm, const int32_t* __restrict__ new_rp,
                                   int32_t* __restrict__ new_col, int32_t* long_rows, int* long_count) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int s = __ldg(rp + v), e = __ldg(rp + v + 1);
    if (e - s > kLongRow) {
      if (lane == 0) long_rows[atomicAdd(long_count, 1)] = v;
      continue;
    }
    const int d = __ldg(new_rp + __ldg(perm + v));
    for (int k = s + lane; k < e; k += 32) new_col[d + (k - s)] = __ldg(perm + __ldg(col + k));
  }
}

// The listed long rows, one CTA per row at a time.
__global__ void spread_cols_long_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                        const int32_t* __restrict__ perm, const int32_t* __restrict__ new_rp,
                                        int32_t* __restrict__ new_col, const int32_t* long_rows, const int* long_count) {
  for (int i = blockIdx.x; i < *long_count; i += gridDim.x) {
    const int v = long_rows[i];
    const int s = __ldg(rp + v), e = __ldg(rp + v + 1);
    const int d = __ldg(new_rp + __ldg(perm + v));
    for (int k = s + threadIdx.x; k < e; k += blockDim.x) new_col[d + (k - s)] = __ldg(perm + __ldg(col + k));
  }
}

template <class T>
__global__ void unspread_kernel(const T* __restrict__ src, T* __restrict__ dst, int32_t n,
                                const int32_t* __restrict__ perm) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) dst[v] = src[perm[v]];
}

int grid_for(int64_t work, int threads, int cap) {
  const int64_t g = (work + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

size_t spread_build_scratch_bytes(int32_t n) {
  return sizeof(HubPlan) + sizeof(int32_t) * (3 * ((size_t)n + 1) + kHubRegion);
}

// Builds the copy: perm (n entries, v -> copy id), new_rp (n + 1 entries) and new_col (nnz
// entries).  bsums needs n / 1024 + 2 entries; `scratch` spread_build_scratch_bytes(n) bytes,
// free again once the stream has passed the build.  *h_hubs and *h_map (host) receive the hub
// count and map after a synchronisation of `s`.
cudaError_t spread_build(const int32_t* rp, const int32_t* col, int32_t n, int32_t* perm, int32_t* new_rp,
                         int32_t* new_col, int32_t* bsums, void* scratch, int32_t* h_hubs, HubMap* h_map,
                         cudaStream_t s) {
  HubPlan* plan = (HubPlan*)scratch;
  int32_t* before = (int32_t*)(plan + 1);  // n + 1: hubs of smaller vertex id
  int32_t* occ = before + n + 1;           // n + 1: hub ids below each id
  int32_t* free_list = occ + n + 1;        // n: the ids no hub holds, in order
  int32_t* list = free_list + n + 1;       // kHubRegion
  *h_hubs = 0;
  *h_map = HubMap{0, 1, 1, 0};
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(hub_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(unsigned long long) * kHubRegion));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(plan, 0, sizeof(HubPlan), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(occ, 0, sizeof(int32_t) * ((size_t)n + 1), s);
  if (e != cudaSuccess) return e;
  count_launches(3);
  hub_hist_kernel<<<grid_for(n, 256, 1024), 256, 0, s>>>(rp, n, plan);
  hub_plan_kernel<<<1, 32, 0, s>>>(plan, n, kHubRegion);
  hub_flag_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(rp, n, plan, before);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = bsp::scan_inplace(before, n, bsums, s);  // exclusive: before[v] = hubs below v
  if (e != cudaSuccess) return e;
  count_launches(2);
  hub_list_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(rp, n, plan, before, list);
  hub_sort_kernel<<<1, kSortThreads, sizeof(unsigned long long) * kHubRegion, s>>>(rp, plan, list, perm, occ);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = bsp::scan_inplace(occ, n, bsums, s);  // exclusive: occ[u] = hub ids below u
  if (e != cudaSuccess) return e;
  count_launches(2);
  free_ids_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(n, occ, free_list);
  spread_perm_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(rp, n, plan, before, free_list, perm, new_rp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = bsp::scan_inplace(new_rp, n, bsums, s);  // exclusive scan; new_rp[n] = nnz
  if (e != cudaSuccess) return e;
  count_launches(2);
  // `before` is free again: it lists the long rows
  spread_cols_kernel<<<grid_for((int64_t)n * 32, 256, 8192), 256, 0, s>>>(rp, col, n, perm, new_rp, new_col, before,
                                                                          &plan->long_count);
  spread_cols_long_kernel<<<512, 1024, 0, s>>>(rp, col, perm, new_rp, new_col, before, &plan->long_count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  HubPlan h;
  e = cudaMemcpyAsync(&h, plan, sizeof(HubPlan), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  *h_hubs = h.hubs;
  *h_map = h.map;
  return cudaSuccess;
}

__global__ void unspread_jobs_kernel(const SpreadJob* jobs) {
  const SpreadJob J = jobs[blockIdx.y];
  const int32_t* src = (const int32_t*)J.src;  // 4-byte elements (float ranks or int32 colours)
  int32_t* dst = (int32_t*)J.dst;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < J.n; v += gridDim.x * blockDim.x) dst[v] = src[J.perm[v]];
}

cudaError_t unspread_jobs(const SpreadJob* d_jobs, int njobs, int max_n, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  count_launches(1);
  unspread_jobs_kernel<<<dim3(grid_for(max_n, 256, 1024), njobs), 256, 0, s>>>(d_jobs);
  return cudaGetLastError();
}

cudaError_t unspread_f32(const float* src, float* dst, int32_t n, const int32_t* perm, cudaStream_t s) {
  count_launches(1);
  unspread_kernel<float><<<grid_for(n, 256, 4096), 256, 0, s>>>(src, dst, n, perm);
  return cudaGetLastError();
}

cudaError_t unspread_i32(const int32_t* src, int32_t* dst, int32_t n, const int32_t* perm, cudaStream_t s) {
  count_launches(1);
  unspread_kernel<int32_t><<<grid_for(n, 256, 4096), 256, 0, s>>>(src, dst, n, perm);
  return cudaGetLastError();
}

}  // namespace atos
