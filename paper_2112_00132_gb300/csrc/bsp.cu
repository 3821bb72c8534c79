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

}  // namespace atos
