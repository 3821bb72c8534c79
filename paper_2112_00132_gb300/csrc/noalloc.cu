// noalloc.cu -- single-source BFS that allocates no memory at all.
//
// Some callers cannot call cudaMalloc: code that runs inside a host application whose own memory
// manager has reserved the whole device (a fixed pool handed out by that manager, where a foreign
// cudaMalloc would fail or fragment it), plug-ins that are forbidden from allocating by their
// host, and latency-critical loops that cannot afford the implicit device-wide synchronisation a
// cudaMalloc / cudaFree may cause.  For them atos_bfs_noalloc takes the caller's device CSR and
// output buffer and keeps every piece of scratch it needs (worklist ring, queue control block,
// instance descriptor, status block, counters, the CSR check flag) in one fixed-size array of
// device memory that is part of the library image itself: every GPU that loads the library holds
// it until the process exits.
//
// In host code the array's name only stands for the symbol, not for a device address.  Every call
// asks for the device address with cudaGetSymbolAddress, with the calling device current (a cheap
// host call), so a module that cudaDeviceReset reloaded at another address is picked up.  The
// set-up of the array itself happens on the device: it carries a marker word that the first
// kernel of every call checks, so a zero-filled array (the first call on a device, or a module
// reloaded by cudaDeviceReset) is recognised and its ring made valid before use.  Device code
// could name the array directly, but the kernels used here take pointers.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "atos.h"
#include "engine.cuh"
#include "launch.cuh"
#include "state.cuh"

namespace atos {

namespace {

constexpr uint32_t kNoAllocRingSlots = 1u << 20;  // 8 MiB of 64-bit ring slots, as atos_bfs's floor
constexpr unsigned kScratchMarker = 0x41544f53u;  // "ATOS": the array has been set up on this device

struct NoAllocScratch {
  unsigned long long ring[kNoAllocRingSlots];
  QueueCtl qctl;
  DevCtl dctl;
  Instance inst;
  unsigned long long stats[kNumStats];  // reset by the prepare step of every call
  int csr_bad;                           // set by the CSR check of the current call
  unsigned marker;                       // kScratchMarker once the ring has been made valid
};

static_assert((uint64_t)ATOS_NOALLOC_MAX_VERTICES + ATOS_NOALLOC_MAX_VERTICES / 2 + 1024 <= kNoAllocRingSlots,
              "the fixed ring must cover 1.5 n plus slack for the largest accepted graph");

// The scratch: file scope, fixed size, 256-byte aligned, shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Writes the call's instance descriptor.  A zero-filled array (first use on this device, or a
// module reloaded by cudaDeviceReset) has no marker: its ring is all zeros, not free slots, so
// the control block is marked dirty and the prepare step that follows refills the ring.
__global__ void noalloc_write_instance(NoAllocScratch* s, Instance I) {
  if (s->marker != kScratchMarker) {
    s->dctl.dirty = 1;
    s->marker = kScratchMarker;
  }
  s->inst = I;
}

// The caller's CSR, checked before any kernel reads it as a graph: row_ptr[0] == 0,
// row_ptr[n] == nnz, rows non-decreasing, every column index in [0, n).  Reads row_ptr[0, n] and
// col[0, nnz) only; any violation sets *bad.
__global__ void noalloc_check_csr(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n,
                                  int64_t nnz, int* bad) {
  bool wrong = false;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (t == 0) wrong |= rp[0] != 0 || (int64_t)rp[n] != nnz;
  for (int64_t v = t; v < n; v += stride) wrong |= rp[v + 1] < rp[v];
  for (int64_t k = t; k < nnz; k += stride) {
    const int32_t c = col[k];
    wrong |= c < 0 || c >= n;
  }
  if (__syncthreads_or(wrong) && threadIdx.x == 0) atomicExch(bad, 1);
}

// Device address of the scratch on the current device.
int scratch_for_current_device(NoAllocScratch** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return ATOS_ERR_CUDA;
  }
  *out = (NoAllocScratch*)p;
  return ATOS_OK;
}

}  // namespace

}  // namespace atos

using namespace atos;

extern "C" int atos_bfs_noalloc(const int32_t* row_ptr, const int32_t* col, int32_t n, int64_t nnz, int32_t source,
                                int32_t* depth, void* stream) {
  if (!row_ptr || !depth || (nnz > 0 && !col) || n < 1 || nnz < 0 || nnz > INT32_MAX || source < 0 ||
      source >= n)
    return ATOS_ERR_INVALID_ARG;
  if (n > ATOS_NOALLOC_MAX_VERTICES) return ATOS_ERR_INVALID_ARG;  // beyond the fixed scratch
  cudaStream_t st = (cudaStream_t)stream;
  NoAllocScratch* s = nullptr;
  int rc = scratch_for_current_device(&s);
  if (rc) return rc;

  // check the CSR before any kernel reads it as a graph (one round trip to the host)
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t work = std::max<int64_t>((int64_t)n + 1, nnz);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 4, (work + 255) / 256));
  int bad = 0;
  if (cudaMemsetAsync(&s->csr_bad, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return ATOS_ERR_CUDA;
  }
  count_launches(1);
  noalloc_check_csr<<<blocks, 256, 0, st>>>(row_ptr, col, n, nnz, &s->csr_bad);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&bad, &s->csr_bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return ATOS_ERR_CUDA;
  }
  if (bad) return ATOS_ERR_BAD_CSR;

  Instance I;
  memset(&I, 0, sizeof(I));
  I.row_ptr = row_ptr;
  I.col = col;
  I.n = n;
  I.app = kAppBfs;
  I.ring = s->ring;
  I.cap = kNoAllocRingSlots;
  I.prefix_len = 1;
  I.prefix_item = source;
  I.ctl = &s->qctl;
  I.depth = depth;
  I.stats = s->stats;
  count_launches(1);
  noalloc_write_instance<<<1, 1, 0, st>>>(s, I);
  if (cudaGetLastError() != cudaSuccess) return ATOS_ERR_CUDA;

  if (launch_prepare(&s->inst, 1, n, &s->dctl, 0u, 1u, st) != cudaSuccess) return ATOS_ERR_CUDA;
  const int worker = 256;
  const void* fn = bfs_persistent_kernel(worker);
  const int nb = resident_blocks(fn, worker);
  if (!fn || nb <= 0) return ATOS_ERR_CUDA;
  Launch L;
  memset(&L, 0, sizeof(L));
  L.insts = &s->inst;
  L.ninst = 1;
  L.window = 1;
  L.fetch = 256;
  L.policy = ATOS_FETCH_SPREAD;
  L.nworkers = nb;
  L.status = &s->dctl.status;
  L.next_inst = &s->dctl.next_inst;
  L.spin_limit_ns = 4000000000LL;
  L.lifetime_ns = 16 * L.spin_limit_ns;
  L.fail_site = &s->dctl.fail_site;
  if (launch_kernel(fn, dim3(nb), worker, L, st) != cudaSuccess) return ATOS_ERR_CUDA;
  if (launch_finalize(&s->inst, 1, &s->dctl, st) != cudaSuccess) return ATOS_ERR_CUDA;

  // report the device status: a plain copy into a host stack variable, then wait for the stream
  int status = 0;
  if (cudaMemcpyAsync(&status, &s->dctl.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return ATOS_ERR_CUDA;
  }
  return status;
}
