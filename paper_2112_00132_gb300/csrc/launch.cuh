// launch.cuh -- host-side launch helpers for the worker engines (one instantiation per body).
#pragma once

#include <cuda_runtime.h>

#include "engine.cuh"

namespace atos {

// Worker shapes that are compiled: thread workers (1), the warp worker (32) and CTA
// workers of 64 .. 1024 threads.
inline bool worker_supported(int w) {
  return w == 1 || w == 32 || w == 64 || w == 128 || w == 256 || w == 512 || w == 1024;
}
// Workers that a warp hosts (thread and warp workers are scheduled per warp).
inline bool warp_hosted(int w) { return w == 1 || w == 32; }

template <class Body>
const void* persistent_kernel_ptr(int worker) {
  switch (worker) {
    case 32: return (const void*)warp_persistent_kernel<Body>;
    case 64: return (const void*)cta_persistent_kernel<Body, 64>;
    case 128: return (const void*)cta_persistent_kernel<Body, 128>;
    case 256: return (const void*)cta_persistent_kernel<Body, 256>;
    case 512: return (const void*)cta_persistent_kernel<Body, 512>;
    case 1024: return (const void*)cta_persistent_kernel<Body, 1024>;
  }
  return nullptr;
}

template <class Body>
const void* discrete_kernel_ptr(int worker) {
  switch (worker) {
    case 32: return (const void*)warp_discrete_kernel<Body>;
    case 64: return (const void*)cta_discrete_kernel<Body, 64>;
    case 128: return (const void*)cta_discrete_kernel<Body, 128>;
    case 256: return (const void*)cta_discrete_kernel<Body, 256>;
    case 512: return (const void*)cta_discrete_kernel<Body, 512>;
    case 1024: return (const void*)cta_discrete_kernel<Body, 1024>;
  }
  return nullptr;
}

inline int block_threads(int worker) { return warp_hosted(worker) ? kWarpBlock : worker; }

// CTAs of this kernel that fit on the whole GPU at once (the persistent grid of Section 3.4).
inline int resident_blocks(const void* fn, int threads) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess) return 0;
  return per_sm * sms;
}

// The library's caching allocator (pool.cu): blocks are reused by later requests of the same size
// class instead of going back to the driver.  Free only blocks the device no longer uses.
cudaError_t pool_malloc(void** p, size_t bytes);
cudaError_t pool_malloc_host(void** p, size_t bytes);
void pool_free(void* p);
void pool_free_host(void* p);

// Kernels this library has launched (all launch sites add to it; read by atos_kernel_launches).
void count_launches(unsigned n);
void uncount_launches(unsigned n);  // launches recorded into a CUDA graph, not run
unsigned long long launches_so_far();

inline cudaError_t launch_kernel(const void* fn, dim3 grid, int threads, const Launch& L, cudaStream_t s) {
  Launch copy = L;
  void* args[] = {&copy};
  count_launches(1);
  return cudaLaunchKernel(fn, grid, dim3(threads), args, 0, s);
}

// Entry points each application translation unit defines.
struct AppKernels {
  const void* (*persistent)(int worker);
  const void* (*discrete)(int worker);
};

}  // namespace atos
