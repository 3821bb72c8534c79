// color.cu -- colouring kernels: persistent / discrete instantiations of the task body in
// color.cuh and the colour-count reduction.
#include "bsp.cuh"
#include "color.cuh"
#include "engine.cuh"
#include "launch.cuh"
#include "state.cuh"

namespace atos {

// worker 1: thread workers (each lane of a warp runs its own task, GcBody::lane_items)
const void* gc_persistent_kernel(int worker) {
  return worker == 1 ? (const void*)warp_persistent_kernel<GcBody, true> : persistent_kernel_ptr<GcBody>(worker);
}
const void* gc_discrete_kernel(int worker) {
  return worker == 1 ? (const void*)warp_discrete_kernel<GcBody, true> : discrete_kernel_ptr<GcBody>(worker);
}

__global__ void gc_max_kernel(const int32_t* color, int n, int* out) {
  int m = -1;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) m = max(m, color[v]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m + 1);
}

// Dependency-ordered colouring uses a copy of the CSR columns whose rows list the smaller-id
// neighbours first and then the larger ones, each part in the row's order (mid[v]: how many are
// smaller).  One warp per row of at most kLongRow entries (a ballot per 32 entries gives each
// entry its place); longer rows are listed and split by a whole CTA each, so a hub row does not
// hold one warp for its whole length.
constexpr int kLongRow = 2048;

__global__ void gc_split_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int n,
                                int32_t* __restrict__ mid, int32_t* __restrict__ scol, int32_t* long_rows,
                                int* long_count) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int s = __ldg(row_ptr + v), e = __ldg(row_ptr + v + 1);
    if (e - s > kLongRow) {
      if (lane == 0) long_rows[atomicAdd(long_count, 1)] = v;
      continue;
    }
    int lower = 0;
    for (int k = s + lane; k < e; k += 32) lower += __ldg(col + k) < v;
    lower = __reduce_add_sync(0xffffffffu, lower);
    int lo = s, hi = s + lower;  // next slot of the lower and of the upper part
    for (int k0 = s; k0 < e; k0 += 32) {
      const int k = k0 + lane;
      const int u = k < e ? __ldg(col + k) : 0;
      const bool below = k < e && u < v;
      const unsigned mb = __ballot_sync(0xffffffffu, below);
      const unsigned ma = __ballot_sync(0xffffffffu, k < e && !below);
      const unsigned lt = (1u << lane) - 1u;
      if (below) scol[lo + __popc(mb & lt)] = u;
      else if (k < e) scol[hi + __popc(ma & lt)] = u;
      lo += __popc(mb);
      hi += __popc(ma);
    }
    if (lane == 0) mid[v] = lower;
  }
}

// The listed long rows, one CTA of kSplitBlock threads per row at a time: count the smaller
// neighbours, then place each chunk of kSplitBlock entries with one block scan.
constexpr int kSplitBlock = 1024;

__global__ void __launch_bounds__(kSplitBlock) gc_split_long_kernel(const int32_t* __restrict__ row_ptr,
                                                                   const int32_t* __restrict__ col,
                                                                   int32_t* __restrict__ mid,
                                                                   int32_t* __restrict__ scol,
                                                                   const int32_t* long_rows, const int* long_count) {
  __shared__ int tmp[33];
  const int t = threadIdx.x;
  for (int i = blockIdx.x; i < *long_count; i += gridDim.x) {
    const int v = long_rows[i];
    const int s = __ldg(row_ptr + v), e = __ldg(row_ptr + v + 1);
    int c = 0;
    for (int k = s + t; k < e; k += kSplitBlock) c += __ldg(col + k) < v;
    int lower;
    block_exclusive_scan<kSplitBlock>(c, tmp, lower);
    int lo = 0, hi = 0;  // entries of each part placed so far
    for (int k0 = s; k0 < e; k0 += kSplitBlock) {
      const int k = k0 + t;
      const int u = k < e ? __ldg(col + k) : 0;
      const bool below = k < e && u < v;
      int below_total;
      const int pre = block_exclusive_scan<kSplitBlock>(below ? 1 : 0, tmp, below_total);
      if (below) scol[s + lo + pre] = u;
      else if (k < e) scol[s + lower + hi + (t - pre)] = u;
      lo += below_total;
      hi += min(kSplitBlock, e - k0) - below_total;
    }
    if (t == 0) mid[v] = lower;
    __syncthreads();
  }
}

__global__ void gc_wait_init_kernel(const int32_t* __restrict__ mid, int n, int32_t* wait) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) wait[v] = 1 + mid[v];
}

// scratch: long_rows of up to n entries and one counter, device memory the caller provides
cudaError_t gc_split_build(const int32_t* row_ptr, const int32_t* col, int n, int32_t* mid, int32_t* scol,
                           int32_t* long_rows, int* long_count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(long_count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  int64_t blocks = ((int64_t)n * 32 + 255) / 256;
  blocks = blocks < 1 ? 1 : (blocks > 8192 ? 8192 : blocks);
  count_launches(2);
  gc_split_kernel<<<(int)blocks, 256, 0, s>>>(row_ptr, col, n, mid, scol, long_rows, long_count);
  gc_split_long_kernel<<<256, kSplitBlock, 0, s>>>(row_ptr, col, mid, scol, long_rows, long_count);
  return cudaGetLastError();
}

// Pushed colours: vertex v's bitmap has (mid[v] + 32) / 32 words (room for colours 0..mid[v],
// which holds its first-fit colour): its own word in [0, n), then the rest (overflow) at
// fw[v] = (first word, words), laid out in id order after the n first words.
__global__ void gc_words_kernel(const int32_t* __restrict__ mid, int n, int32_t* __restrict__ words) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    words[v] = ((mid[v] + 32) >> 5) - 1;
}

__global__ void gc_fw_kernel(const int32_t* __restrict__ first, int n, int2* __restrict__ fw) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    fw[v] = make_int2(n + first[v], first[v + 1] - first[v]);
}

int64_t gc_bitmap_scratch(int n) { return (int64_t)n + 1 + n / 1024 + 2; }

// Tail segments the dependency-ordered colouring can create: a ready vertex's larger neighbours
// after its first kGcHead, in segments of up to kGcSegment entries (each vertex is ready once).
__global__ void gc_tail_count_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ mid, int n,
                                     unsigned long long* out) {
  unsigned long long c = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int upper = row_ptr[v + 1] - row_ptr[v] - mid[v];
    if (upper > kGcHead) c += (unsigned long long)((upper - kGcHead + kGcSegment - 1) / kGcSegment);
  }
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Table entries a run may leave unused: every CTA (at most 32 per SM) may hold a partly used chunk.
uint64_t gc_tail_slack() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 160;
  return (uint64_t)kGcSegChunk * 32u * (uint64_t)sms;
}

// scratch: 8 bytes of device memory; synchronises s
cudaError_t gc_tail_segments(const int32_t* row_ptr, const int32_t* mid, int n, void* scratch, uint64_t* count,
                             cudaStream_t s) {
  *count = 0;
  if (n <= 0) return cudaSuccess;
  unsigned long long* d = (unsigned long long*)scratch;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(*d), s);
  if (e != cudaSuccess) return e;
  int blocks = (n + 255) / 256;
  blocks = blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks);
  count_launches(1);
  gc_tail_count_kernel<<<blocks, 256, 0, s>>>(row_ptr, mid, n, d);
  unsigned long long h = 0;
  e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) *count = h;
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t gc_bitmap_build(const int32_t* mid, int n, int2* fw, int32_t* scratch, uint32_t* total_words,
                            cudaStream_t s) {
  *total_words = 0;
  if (n <= 0) return cudaSuccess;
  int blocks = (n + 255) / 256;
  blocks = blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks);
  count_launches(2);
  gc_words_kernel<<<blocks, 256, 0, s>>>(mid, n, scratch);
  cudaError_t e = bsp::scan_inplace(scratch, n, scratch + n + 1, s);
  if (e != cudaSuccess) return e;
  gc_fw_kernel<<<blocks, 256, 0, s>>>(scratch, n, fw);
  int32_t words = 0;
  e = cudaMemcpyAsync(&words, scratch + n, sizeof(words), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) *total_words = (uint32_t)n + (uint32_t)words;
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t gc_wait_init(const int32_t* mid, int n, int32_t* wait, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (n + 255) / 256;
  blocks = blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks);
  count_launches(1);
  gc_wait_init_kernel<<<blocks, 256, 0, s>>>(mid, n, wait);
  return cudaGetLastError();
}

cudaError_t gc_finish(const Instance* h_inst, DevCtl* d_ctl, cudaStream_t s) {
  cudaMemsetAsync(&d_ctl->num_colors, 0, sizeof(int), s);
  int gx = (h_inst->n + 255) / 256;
  gx = gx < 1 ? 1 : (gx > 2048 ? 2048 : gx);
  count_launches(1);
  gc_max_kernel<<<gx, 256, 0, s>>>(h_inst->color, h_inst->n, &d_ctl->num_colors);
  return cudaGetLastError();
}

}  // namespace atos
