// ceiling.cu -- the memory-system ceilings of the task bodies' inner loops, measured on the
// caller's graph with no scheduler around them.
//
// A task body's edge loop gathers col[e] for a run of consecutive CSR entries and then either
// scatters to the neighbour (PageRank: red.add.f32 into res[col[e]]) or reads the neighbour's
// state (BFS and colouring: a load of depth[col[e]] / color[col[e]]).  The kernels here do exactly
// that over every entry of the CSR once, in CSR order, with a grid-stride loop, coalesced col reads
// and nothing else.  On a scale-free graph the scatter is limited by same-address atomics at the
// hubs (they serialise in their L2 slice), not by DRAM bandwidth; the measured rate is the
// roofline the persistent PageRank kernel is compared with.
#include <cuda_runtime.h>
#include <stdint.h>

#include "atos.h"
#include "launch.cuh"

namespace atos {
int graph_device_csr(atos_graph_t g, const int32_t** row_ptr, const int32_t** col, int32_t* n_isolated);
int graph_spread_csr(atos_graph_t g, const int32_t** row_ptr, const int32_t** col, cudaStream_t st,
                     const int32_t** perm, int32_t* hubs, HubMap* hub);

namespace {

__global__ void ideal_scatter_kernel(const int32_t* __restrict__ col, int64_t nnz, float* state) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
    red_add_f32(state + __ldg(col + e), 1.0e-9f);
}

__global__ void ideal_gather_kernel(const int32_t* __restrict__ col, int64_t nnz, const float* state, float* sink) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float acc = 0.0f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
    acc += __ldcg(state + __ldg(col + e));
  if (acc == -1.0f) sink[0] = acc;  // never true (state holds non-negative values): keeps the loads
}

}  // namespace
}  // namespace atos

using namespace atos;

extern "C" int atos_edge_ceiling(atos_graph_t g, int32_t kind, int32_t repeats, double* ms_per_pass, void* stream) {
  const int base_kind = kind & ~ATOS_CEILING_SPREAD_IDS;
  if (!g || !ms_per_pass || repeats < 1 || (base_kind != ATOS_CEILING_SCATTER && base_kind != ATOS_CEILING_GATHER) ||
      (kind & ~(ATOS_CEILING_SPREAD_IDS | 1)))
    return ATOS_ERR_INVALID_ARG;
  int32_t n = 0;
  int64_t nnz = 0;
  atos_graph_info(g, &n, &nnz, nullptr);
  *ms_per_pass = 0.0;
  if (n < 1 || nnz < 1) return ATOS_OK;
  const int32_t *rp = nullptr, *col = nullptr;
  int32_t iso = 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (kind & ATOS_CEILING_SPREAD_IDS) {
    const int rc0 = graph_spread_csr(g, &rp, &col, st, nullptr, nullptr, nullptr);
    if (rc0) return rc0;
  } else {
    graph_device_csr(g, &rp, &col, &iso);
  }
  float* state = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = ATOS_OK;
  if (cudaMalloc((void**)&state, sizeof(float) * ((size_t)n + 1)) != cudaSuccess) rc = ATOS_ERR_OOM;
  if (!rc && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)) rc = ATOS_ERR_CUDA;
  if (!rc && cudaMemsetAsync(state, 0, sizeof(float) * ((size_t)n + 1), st) != cudaSuccess) rc = ATOS_ERR_CUDA;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  for (int r = 0; !rc && r <= repeats; ++r) {  // pass 0 warms up
    if (r == 1) cudaEventRecord(a, st);
    count_launches(1);
    if (base_kind == ATOS_CEILING_SCATTER) ideal_scatter_kernel<<<blocks, threads, 0, st>>>(col, nnz, state);
    else ideal_gather_kernel<<<blocks, threads, 0, st>>>(col, nnz, state, state + n);
    if (cudaGetLastError() != cudaSuccess) rc = ATOS_ERR_CUDA;
  }
  if (!rc) {
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) rc = ATOS_ERR_CUDA;
    float ms = 0.0f;
    if (!rc) cudaEventElapsedTime(&ms, a, b);
    *ms_per_pass = (double)ms / repeats;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (state) cudaFree(state);
  return rc;
}
