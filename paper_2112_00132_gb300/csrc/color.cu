// color.cu -- colouring kernels: persistent / discrete instantiations of the task body in
// color.cuh and the colour-count reduction.
#include "color.cuh"
#include "engine.cuh"
#include "launch.cuh"
#include "state.cuh"

namespace atos {

const void* gc_persistent_kernel(int worker) { return persistent_kernel_ptr<GcBody>(worker); }
const void* gc_discrete_kernel(int worker) { return discrete_kernel_ptr<GcBody>(worker); }

__global__ void gc_max_kernel(const int32_t* color, int n, int* out) {
  int m = -1;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) m = max(m, color[v]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m + 1);
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
