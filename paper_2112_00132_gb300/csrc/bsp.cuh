// bsp.cuh -- the level-synchronous (BSP) comparator (Algorithms 1, 3, 5): host interface.
//
// The comparator is a "GPU-wide worker" (Section 3.2): every level is a fixed sequence of kernels
// over the whole frontier.  All of a run's level state (frontier sizes, which frontier buffer is
// current, the level number, counters) lives in one device-side control block, and every level
// kernel reads the sizes it needs from there and covers them with a fixed grid (grid-stride
// loops).  The same level sequence can therefore be driven two ways:
//   * from the host: after each level one small read-back of the control block decides whether
//     to launch the next level (one host round trip per level, as a BSP framework does);
//   * on the device: the level sequence is the body of a CUDA graph whose conditional WHILE node
//     repeats it while the last kernel of the level (cudaGraphSetConditional) finds a non-empty
//     next frontier; a run is one graph launch, with no host synchronisation per level.
// BFS advances the frontiers of all its sources together: a frontier item is (source, vertex) and
// one launch per level relaxes the edges of every source's frontier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.cuh"

namespace atos {

// One BSP run (host-side description).
struct BspRun {
  int app;                  // kAppBfs, kAppPr or kAppGc
  const int32_t* row_ptr;   // device CSR of the graph the run works on
  const int32_t* col;
  int32_t n;
  int64_t nnz;
  const int32_t* sources;   // BFS: HOST array of nsrc source vertices
  int32_t nsrc;
  int32_t* depth;           // BFS: DEVICE nsrc x n depths
  float* rank;              // PageRank: DEVICE rank and residue, already initialised
  float* res;
  float alpha, eps;
  int32_t* color;           // colouring: DEVICE colours
  bool device_loop;         // drive the levels from a CUDA graph's conditional WHILE node
};

struct BspResult {
  int64_t iters;   // levels run
  int64_t edges;   // neighbour entries read (BFS, colouring) or scattered to (PageRank)
  int64_t tasks;   // frontier items processed, summed over the levels
  int32_t status;  // ATOS_OK or ATOS_ERR_TIMEOUT (level budget exhausted)
};

// Device-side CUDA graphs of the device-loop form, one per application, built on first use for a
// scratch area and reused while it stays the same.
struct BspGraphs {
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  const void* scratch = nullptr;  // the scratch area the graphs were built for
  cudaStream_t capture = nullptr;
  void release();
};

// Bytes of device scratch a run of `app` needs (frontiers, scan offsets, control block).
size_t bsp_scratch_bytes(int app, int32_t n, int64_t nnz, int32_t nsrc);

// Runs r on `s`.  scratch: bsp_scratch_bytes(...) bytes of device memory; host_buf: pinned host
// memory of at least bsp_host_bytes() bytes.  With `result` non-NULL (or in the host-driven form)
// the call synchronises `s` and fills it.  Returns ATOS_OK, ATOS_ERR_CUDA or ATOS_ERR_INVALID_ARG.
size_t bsp_host_bytes();
int bsp_run(const BspRun& r, void* scratch, size_t scratch_bytes, void* host_buf, BspGraphs* graphs, cudaStream_t s,
            BspResult* result);

namespace bsp {
// In-place exclusive scan of a[0, F) into a[0, F]; a[F] receives the total.  bsums needs
// F / 1024 + 2 entries.
cudaError_t scan_inplace(int32_t* a, int32_t F, int32_t* bsums, cudaStream_t s);
}  // namespace bsp

}  // namespace atos
