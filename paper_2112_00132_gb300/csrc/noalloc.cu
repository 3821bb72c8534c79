// noalloc.cu -- single-source BFS that allocates no memory at all.
//
// Some callers cannot call cudaMalloc: code that runs inside a host application whose own memory
// manager has reserved the whole device (a fixed pool handed out by that manager, where a foreign
// cudaMalloc would fail or fragment it), plug-ins that are forbidden from allocating by their
// host, and latency-critical loops that cannot afford the implicit device-wide synchronisation a
// cudaMalloc / cudaFree may cause.  For them atos_bfs_noalloc takes the caller's device CSR and
// output buffer and keeps every piece of scratch it needs (worklist ring, queue control block,
// instance descriptor, status block, counters) in one fixed-size array of device memory that is
// part of the library image itself: every GPU that loads the library holds it until the process
// exits.
//
// In host code the array's name only stands for the symbol, not for a device address; its device
// address is obtained once per device with cudaGetSymbolAddress (with that device current) and
// cached.  Device code could name the array directly, but the kernels used here take pointers.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "atos.h"
#include "engine.cuh"
#include "launch.cuh"
#include "state.cuh"

namespace atos {

namespace {

constexpr uint32_t kNoAllocRingSlots = 1u << 19;  // 4 MiB of 64-bit ring slots

struct NoAllocScratch {
  unsigned long long ring[kNoAllocRingSlots];
  QueueCtl qctl;
  DevCtl dctl;
  Instance inst;
  unsigned long long stats[kNumStats];
};

static_assert((uint64_t)ATOS_NOALLOC_MAX_VERTICES + ATOS_NOALLOC_MAX_VERTICES / 2 + 1024 <= kNoAllocRingSlots,
              "the fixed ring must cover 1.5 n plus slack for the largest accepted graph");

// The scratch: file scope, fixed size, 256-byte aligned, shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};

__global__ void noalloc_first_use(NoAllocScratch* s) {
  // the library image zero-fills the array; the ring must start with every slot free (all ones),
  // which the next prepare step does when the block is marked dirty
  s->dctl.dirty = 1;
}

__global__ void noalloc_write_instance(NoAllocScratch* s, Instance I) { s->inst = I; }

// Device address of the scratch on the current device (set-up on the first call per device).
int scratch_for_current_device(NoAllocScratch** out, cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ATOS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return ATOS_ERR_CUDA;
    }
    count_launches(1);
    noalloc_first_use<<<1, 1, 0, stream>>>((NoAllocScratch*)p);
    if (cudaGetLastError() != cudaSuccess) return ATOS_ERR_CUDA;
    g_scratch_ptr[dev] = (NoAllocScratch*)p;
  }
  *out = g_scratch_ptr[dev];
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
  int rc = scratch_for_current_device(&s, st);
  if (rc) return rc;

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
