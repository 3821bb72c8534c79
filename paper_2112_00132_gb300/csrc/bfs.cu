// bfs.cu -- speculative BFS task body (Section 5.1, Algorithm 2) on the worker engines.
//
// A task is a vertex v.  The worker re-reads depth[v] when it pops v (the depth may have improved
// since v was pushed), and relaxes every neighbour n with atomicMin(depth[n], depth[v] + 1),
// pushing n whenever the minimum actually decreased.  Depths only decrease, so a neighbour whose
// current depth is already <= depth[v] + 1 is skipped with a plain L2 load and no atomic.  Since
// every improvement is pushed and re-relaxed, the fixed point is the exact hop distance whatever
// the order of pops; the discrete strategy processes the queue one generation at a time, which
// makes each generation one BFS level.
#include "bfs.cuh"
#include "launch.cuh"

namespace atos {

// worker 1: thread workers (each lane of a warp expands its own vertex, BfsBody::lane_items)
const void* bfs_persistent_kernel(int worker) {
  return worker == 1 ? (const void*)warp_persistent_kernel<BfsBody, true> : persistent_kernel_ptr<BfsBody>(worker);
}
const void* bfs_discrete_kernel(int worker) {
  return worker == 1 ? (const void*)warp_discrete_kernel<BfsBody, true> : discrete_kernel_ptr<BfsBody>(worker);
}

}  // namespace atos
