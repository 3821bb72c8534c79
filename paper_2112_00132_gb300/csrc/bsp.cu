// bsp.cu -- level-synchronous BFS comparator (Algorithm 1): one level per iteration, a
// device-wide scan of the frontier degrees, a load-balanced advance in which each CTA relaxes a
// fixed chunk of edges (atomicMin(depth, level + 1), appending improved vertices to the next
// frontier), and a host read of the next frontier's size.
#include <algorithm>

#include "bsp.cuh"
#include "launch.cuh"

namespace atos {
namespace bsp {

__global__ void __launch_bounds__(kBlock) degree_chunk_sums(const int32_t* __restrict__ frontier, int32_t F,
                                                            const int32_t* __restrict__ row_ptr,
                                                            int32_t* __restrict__ offs, int32_t* __restrict__ bsums) {
  __shared__ int tmp[33];
  const int base = blockIdx.x * kChunk;
  int local = 0;
  int d[kPerThread];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int i = base + threadIdx.x * kPerThread + k;
    d[k] = 0;
    if (i < F) {
      const int v = __ldg(frontier + i);
      d[k] = __ldg(row_ptr + v + 1) - __ldg(row_ptr + v);
    }
    local += d[k];
  }
  int total;
  int pre = block_exclusive_scan<kBlock>(local, tmp, total);
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int i = base + threadIdx.x * kPerThread + k;
    if (i < F) offs[i] = pre;
    pre += d[k];
  }
  if (threadIdx.x == 0) bsums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_chunk_sums(int32_t* bsums, int nb, int32_t* offs, int32_t F) {
  __shared__ int tmp[33];
  // one block: each thread owns a contiguous run of chunk sums
  const int per = (nb + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  int local = 0;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) local += bsums[b0 + k];
  int total;
  int pre = block_exclusive_scan<1024>(local, tmp, total);
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) {
      const int x = bsums[b0 + k];
      bsums[b0 + k] = pre;
      pre += x;
    }
  if (threadIdx.x == 0) offs[F] = total;
}

__global__ void __launch_bounds__(kBlock) add_chunk_offsets(int32_t* offs, int32_t F, const int32_t* bsums) {
  const int base = blockIdx.x * kChunk;
  const int add = bsums[blockIdx.x];
  for (int k = threadIdx.x; k < kChunk; k += kBlock) {
    const int i = base + k;
    if (i < F) offs[i] += add;
  }
}

cudaError_t scan_degrees(const int32_t* frontier, int32_t F, const int32_t* row_ptr, int32_t* offs, int32_t* bsums,
                         cudaStream_t s) {
  const int nb = (F + kChunk - 1) / kChunk;
  count_launches(3);
  degree_chunk_sums<<<nb, kBlock, 0, s>>>(frontier, F, row_ptr, offs, bsums);
  scan_chunk_sums<<<1, 1024, 0, s>>>(bsums, nb, offs, F);
  add_chunk_offsets<<<nb, kBlock, 0, s>>>(offs, F, bsums);
  return cudaGetLastError();
}

// Relaxes edge chunks [c * kChunk, (c + 1) * kChunk) of the scanned frontier (grid-stride over
// chunks; the total is read on the device so the host does not wait for it).
__global__ void __launch_bounds__(kBlock) bfs_advance(const int32_t* __restrict__ frontier, int32_t F,
                                                      const int32_t* __restrict__ offs,
                                                      const int32_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col, int32_t* depth, int32_t nd,
                                                      int32_t* __restrict__ out, int32_t* out_count) {
  __shared__ int s_off[kChunk + 1];
  __shared__ int s_start[kChunk + 1];
  __shared__ int s_lo, s_cnt;
  const int total = offs[F];
  const int nchunks = (total + kChunk - 1) / kChunk;
  const int lane = threadIdx.x & 31;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int e0 = c * kChunk, e1 = min(total, e0 + kChunk);
    if (threadIdx.x == 0) {
      const int lo = upper_bound_global(offs, F, e0);
      const int hi = upper_bound_global(offs, F, e1 - 1);
      s_lo = lo;
      s_cnt = hi - lo + 1;
    }
    __syncthreads();
    const int lo = s_lo, cnt = s_cnt;
    // Frontier items of degree 0 can make the owning range longer than the chunk; such a
    // chunk searches the global offsets instead of a staged copy.
    const bool staged = cnt <= kChunk + 1;
    if (staged)
      for (int k = threadIdx.x; k < cnt; k += kBlock) {
        s_off[k] = offs[lo + k];
        s_start[k] = __ldg(row_ptr + __ldg(frontier + lo + k));
      }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) {
      const int e = e0 + r * kBlock + threadIdx.x;
      bool want = false;
      int nb = 0;
      if (e < e1) {
        int i, first, o;
        if (staged) {
          i = owner_of(s_off, cnt, e);
          first = s_start[i];
          o = s_off[i];
        } else {
          i = lo + upper_bound_global(offs + lo, cnt, e);
          first = __ldg(row_ptr + __ldg(frontier + i));
          o = offs[i];
        }
        nb = __ldg(col + first + (e - o));
        if (nd < __ldcg(depth + nb)) want = nd < atomicMin(depth + nb, nd);
      }
      const unsigned m = __ballot_sync(0xffffffffu, want);
      if (m) {
        const int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(out_count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (want) out[base + __popc(m & lanemask_lt())] = nb;
      }
    }
    __syncthreads();
  }
}

__global__ void bfs_init(int32_t* depth, int32_t n, int32_t src, int32_t* frontier, int32_t* count) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) depth[v] = v == src ? 0 : kUnreached;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    frontier[0] = src;
    *count = 0;
  }
}


// In-place exclusive scan of a[0, F) into a[0, F]; a[F] receives the total.
__global__ void __launch_bounds__(kBlock) chunk_sums_inplace(int32_t* a, int32_t F, int32_t* bsums) {
  __shared__ int tmp[33];
  const int base = blockIdx.x * kChunk;
  int local = 0;
  int d[kPerThread];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int i = base + threadIdx.x * kPerThread + k;
    d[k] = i < F ? a[i] : 0;
    local += d[k];
  }
  int total;
  int pre = block_exclusive_scan<kBlock>(local, tmp, total);
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int i = base + threadIdx.x * kPerThread + k;
    if (i < F) a[i] = pre;
    pre += d[k];
  }
  if (threadIdx.x == 0) bsums[blockIdx.x] = total;
}

cudaError_t scan_inplace(int32_t* a, int32_t F, int32_t* bsums, cudaStream_t s) {
  const int nb = (F + kChunk - 1) / kChunk;
  count_launches(3);
  chunk_sums_inplace<<<nb, kBlock, 0, s>>>(a, F, bsums);
  scan_chunk_sums<<<1, 1024, 0, s>>>(bsums, nb, a, F);
  add_chunk_offsets<<<nb, kBlock, 0, s>>>(a, F, bsums);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ PageRank (Algorithm 3)

// Kernel 1a: per frontier vertex, take the residue, add it to the rank, and record the share
// alpha * r / deg(v) to scatter; cnt[i] = deg(v) if there is anything to scatter.
__global__ void pr_bsp_take(const int32_t* __restrict__ frontier, int32_t F, const int32_t* __restrict__ row_ptr,
                            float* rank, float* res, float alpha, float* share, int32_t* cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F; i += gridDim.x * blockDim.x) {
    const int v = frontier[i];
    const float r = atomicExch(res + v, 0.0f);
    const int d = __ldg(row_ptr + v + 1) - __ldg(row_ptr + v);
    rank[v] += r;
    const bool go = r != 0.0f && d > 0;
    share[i] = go ? alpha * r / (float)d : 0.0f;
    cnt[i] = go ? d : 0;
  }
}

// Kernel 1b: load-balanced scatter over the frontier's edges (offsets from the scan of cnt).
__global__ void __launch_bounds__(kBlock) pr_bsp_scatter(const int32_t* __restrict__ frontier, int32_t F,
                                                         const int32_t* __restrict__ offs,
                                                         const int32_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col,
                                                         const float* __restrict__ share, float* res) {
  const int total = offs[F];
  const int nchunks = (total + kChunk - 1) / kChunk;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int e0 = c * kChunk, e1 = min(total, e0 + kChunk);
    // each thread: kPerThread consecutive edges, one owner search
    const int ea = e0 + threadIdx.x * kPerThread;
    if (ea >= e1) continue;
    int i = upper_bound_global(offs, F, ea);
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      const int e = ea + k;
      if (e >= e1) break;
      while (i + 1 < F && __ldg(offs + i + 1) <= e) ++i;
      const int v = __ldg(frontier + i);
      const int nb = __ldg(col + __ldg(row_ptr + v) + (e - __ldg(offs + i)));
      red_add_f32(res + nb, __ldg(share + i));
    }
  }
}

// Kernel 2: the next frontier is every vertex whose residue exceeds eps.
__global__ void pr_bsp_filter(const float* __restrict__ res, int32_t n, float eps, int32_t* out, int32_t* count) {
  const int lane = threadIdx.x & 31;
  for (int r = blockIdx.x * blockDim.x; r < n; r += gridDim.x * blockDim.x) {
    const int v = r + threadIdx.x;
    const bool want = v < n && res[v] > eps;
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) continue;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) out[base + __popc(m & lanemask_lt())] = v;
  }
}

__global__ void iota_kernel(int32_t* f, int32_t n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) f[v] = v;
}

// ------------------------------------------------------------------ colouring (Algorithm 5)

// Kernel 1: every frontier vertex takes the smallest colour none of its neighbours holds (one
// warp per vertex, colour windows of 64 combined by an OR reduction over the lanes).
__global__ void gc_bsp_assign(const int32_t* __restrict__ frontier, int32_t F, const int32_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ col, int32_t* color, int64_t* edges) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  long long ed = 0;
  for (int i = gw; i < F; i += nw) {
    const int v = frontier[i];
    const int s = __ldg(row_ptr + v), e = __ldg(row_ptr + v + 1);
    int colour = -1;
    for (int base = 0; colour < 0; base += 64) {
      unsigned lo = 0, hi = 0;
      for (int k = s + lane; k < e; k += 32) {
        const int rel = __ldcg(color + __ldg(col + k)) - base;
        if (rel >= 0 && rel < 32) lo |= 1u << rel;
        else if (rel >= 32 && rel < 64) hi |= 1u << (rel - 32);
      }
      ed += e - s;
      lo = __reduce_or_sync(0xffffffffu, lo);
      hi = __reduce_or_sync(0xffffffffu, hi);
      const unsigned long long used = ((unsigned long long)hi << 32) | lo;
      if (~used) colour = base + __ffsll((long long)~used) - 1;
    }
    if (lane == 0) color[v] = colour;
  }
  if (lane == 0 && ed) atomicAdd((unsigned long long*)edges, (unsigned long long)ed);
}

// Kernel 2: a frontier vertex whose colour a smaller neighbour also holds goes to the next
// frontier (of a conflicting pair the larger id recolours).
__global__ void gc_bsp_conflicts(const int32_t* __restrict__ frontier, int32_t F, const int32_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col, const int32_t* __restrict__ color, int32_t* out,
                                 int32_t* count) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = gw; i < F; i += nw) {
    const int v = frontier[i];
    const int s = __ldg(row_ptr + v), e = __ldg(row_ptr + v + 1);
    const int cv = color[v];
    bool conflict = false;
    for (int k = s + lane; k < e; k += 32) {
      const int u = __ldg(col + k);
      conflict |= u < v && color[u] == cv;
    }
    if (__any_sync(0xffffffffu, conflict) && lane == 0) out[atomicAdd(count, 1)] = v;
  }
}

__global__ void fill_kernel(int32_t* a, int32_t n, int32_t value) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) a[v] = value;
}

}  // namespace bsp

// Level-synchronous BFS from src.  scratch holds two frontiers of n entries, the scan offsets,
// the chunk sums and a counter; `hcount` is pinned host memory receiving the next frontier size.
int bsp_bfs(const int32_t* row_ptr, const int32_t* col, int32_t n, int32_t src, int32_t* depth, void* scratch,
            size_t scratch_bytes, int32_t* hcount, cudaStream_t s, int64_t* iterations, int64_t* edges) {
  using namespace bsp;
  int32_t* fa = (int32_t*)scratch;
  int32_t* fb = fa + n;
  int32_t* offs = fb + n;  // n + 1
  int32_t* bsums = offs + n + 1;
  int32_t* count = bsums + (n / kChunk + 2);
  if ((size_t)((char*)(count + 1) - (char*)scratch) > scratch_bytes) return ATOS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  count_launches(1);
  bfs_init<<<std::max(1, std::min(1024, (n + 255) / 256)), 256, 0, s>>>(depth, n, src, fa, count);
  int32_t F = 1, level = 0;
  int64_t iters = 0, ed = 0;
  int rc = ATOS_OK;
  while (F > 0) {
    if (scan_degrees(fa, F, row_ptr, offs, bsums, s) != cudaSuccess) {
      rc = ATOS_ERR_CUDA;
      break;
    }
    cudaMemsetAsync(count, 0, sizeof(int32_t), s);
    count_launches(1);
    bfs_advance<<<sms * 8, kBlock, 0, s>>>(fa, F, offs, row_ptr, col, depth, level + 1, fb, count);
    int32_t tot = 0;
    cudaMemcpyAsync(hcount, count, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&tot, offs + F, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      rc = ATOS_ERR_CUDA;
      break;
    }
    ed += tot;
    F = *hcount;
    int32_t* t = fa;
    fa = fb;
    fb = t;
    level++;
    iters++;
  }
  if (iterations) *iterations = iters;
  if (edges) *edges = ed;
  return rc;
}


// Level-synchronous PageRank (Algorithm 3): rank and residue are initialised by the caller (the
// same prepare step as the asynchronous form); frontier 0 is every vertex.  Each iteration takes
// the residues of the frontier, scatters them over its edges, then collects every vertex whose
// residue exceeds eps.  Scratch: two frontiers (n), scan offsets (n + 1), shares (n floats),
// chunk sums; `hcount` is pinned host memory.
int bsp_pagerank(const int32_t* row_ptr, const int32_t* col, int32_t n, float alpha, float eps, float* rank,
                 float* res, void* scratch, size_t scratch_bytes, int32_t* hcount, cudaStream_t s,
                 int64_t* iterations, int64_t* edges, int64_t* tasks) {
  using namespace bsp;
  int32_t* fa = (int32_t*)scratch;
  int32_t* fb = fa + n;
  int32_t* offs = fb + n;
  float* share = (float*)(offs + n + 1);
  int32_t* bsums = (int32_t*)(share + n);
  int32_t* count = bsums + (n / kChunk + 2);
  if ((size_t)((char*)(count + 1) - (char*)scratch) > scratch_bytes) return ATOS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int gv = std::max(1, std::min(sms * 8, (n + 255) / 256));
  count_launches(1);
  iota_kernel<<<gv, 256, 0, s>>>(fa, n);
  int32_t F = n;
  int64_t iters = 0, ed = 0, tk = 0;
  while (F > 0) {
    count_launches(1);
    pr_bsp_take<<<std::max(1, std::min(sms * 8, (F + 255) / 256)), 256, 0, s>>>(fa, F, row_ptr, rank, res, alpha,
                                                                                 share, offs);
    if (scan_inplace(offs, F, bsums, s) != cudaSuccess) return ATOS_ERR_CUDA;
    count_launches(2);
    pr_bsp_scatter<<<sms * 8, kBlock, 0, s>>>(fa, F, offs, row_ptr, col, share, res);
    cudaMemsetAsync(count, 0, sizeof(int32_t), s);
    pr_bsp_filter<<<gv, 256, 0, s>>>(res, n, eps, fb, count);
    int32_t tot = 0;
    cudaMemcpyAsync(hcount, count, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&tot, offs + F, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return ATOS_ERR_CUDA;
    ed += tot;
    tk += F;
    F = *hcount;
    int32_t* t = fa;
    fa = fb;
    fb = t;
    if (++iters > (1 << 22)) return ATOS_ERR_TIMEOUT;
  }
  if (iterations) *iterations = iters;
  if (edges) *edges = ed;
  if (tasks) *tasks = tk;
  return ATOS_OK;
}

// Level-synchronous speculative colouring (Algorithm 5): frontier 0 is every vertex, colours
// start at -1; each iteration assigns first-fit colours to the frontier, then keeps the frontier
// vertices that conflict with a smaller neighbour.
int bsp_color(const int32_t* row_ptr, const int32_t* col, int32_t n, int32_t* color, void* scratch,
              size_t scratch_bytes, int32_t* hcount, cudaStream_t s, int64_t* iterations, int64_t* edges,
              int64_t* tasks) {
  using namespace bsp;
  int32_t* fa = (int32_t*)scratch;
  int32_t* fb = fa + n;
  int64_t* d_edges = (int64_t*)(((uintptr_t)(fb + n) + 15) & ~(uintptr_t)15);
  int32_t* count = (int32_t*)(d_edges + 1);
  if ((size_t)((char*)(count + 1) - (char*)scratch) > scratch_bytes) return ATOS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int gv = std::max(1, std::min(sms * 8, (n + 255) / 256));
  count_launches(2);
  iota_kernel<<<gv, 256, 0, s>>>(fa, n);
  fill_kernel<<<gv, 256, 0, s>>>(color, n, -1);
  cudaMemsetAsync(d_edges, 0, sizeof(int64_t), s);
  int32_t F = n;
  int64_t iters = 0, tk = 0;
  while (F > 0) {
    const int gw = std::max(1, std::min(sms * 16, (F + 7) / 8));
    count_launches(2);
    gc_bsp_assign<<<gw, 256, 0, s>>>(fa, F, row_ptr, col, color, d_edges);
    cudaMemsetAsync(count, 0, sizeof(int32_t), s);
    gc_bsp_conflicts<<<gw, 256, 0, s>>>(fa, F, row_ptr, col, color, fb, count);
    cudaMemcpyAsync(hcount, count, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return ATOS_ERR_CUDA;
    tk += F;
    F = *hcount;
    int32_t* t = fa;
    fa = fb;
    fb = t;
    if (++iters > (1 << 22)) return ATOS_ERR_TIMEOUT;
  }
  int64_t ed = 0;
  cudaMemcpy(&ed, d_edges, sizeof(int64_t), cudaMemcpyDeviceToHost);
  if (iterations) *iterations = iters;
  if (edges) *edges = ed;
  if (tasks) *tasks = tk;
  return ATOS_OK;
}

}  // namespace atos
