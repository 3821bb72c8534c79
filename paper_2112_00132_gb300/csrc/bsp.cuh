// bsp.cuh -- building blocks of the level-synchronous (BSP) comparator (Algorithms 1, 3, 5).
//
// The comparator is a "GPU-wide worker" (Section 3.2): every level is one or more kernels over
// the whole frontier, with a device-wide exclusive scan of the frontier's degrees so that each
// CTA advances exactly `kChunk` edges (load-balanced advance), and the host reads the size of the
// next frontier between levels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.cuh"

namespace atos {
namespace bsp {

constexpr int kBlock = 256;
constexpr int kPerThread = 4;
constexpr int kChunk = kBlock * kPerThread;  // edges per CTA per advance step

// Device-wide exclusive scan of the degrees of frontier[0, F) into offs[0, F], offs[F] = total.
// Scratch `bsums` needs ceil(F / kChunk) + 1 entries.
cudaError_t scan_degrees(const int32_t* frontier, int32_t F, const int32_t* row_ptr, int32_t* offs, int32_t* bsums,
                         cudaStream_t s);

// The frontier item owning edge e in a CTA chunk: stage offs[lo..hi] and search in shared memory.
struct ChunkMap {
  int lo, cnt;  // frontier items [lo, lo + cnt) intersect the chunk
};

__device__ __forceinline__ int upper_bound_global(const int32_t* offs, int count, int e) {
  // largest i in [0, count) with offs[i] <= e
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(offs + mid) <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace bsp
}  // namespace atos
