// pool.cu -- the library's caching allocator for device memory and pinned host memory.
//
// Graph objects, batches and servers allocate their scratch (rings, control blocks, residues,
// the spread-id copy, certificate buffers) when they are created or first used, and free it when
// they are destroyed.  A program that creates a graph, runs it and destroys it in a loop (a
// request pipeline, or the end-to-end benchmark) would otherwise pay cudaMalloc / cudaFree and
// cudaMallocHost / cudaFreeHost for several GB on every iteration.  Freed blocks are kept in
// per-device free lists keyed by a size class and handed out again to requests of the same
// class; atos_pool_trim returns them to the driver, and a failed cudaMalloc trims and retries.
//
// Blocks are only freed by the library after the device is idle with respect to them (object
// destruction and scratch reallocation synchronise first), so a reused block is never still in
// use by a kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <tuple>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

#include "atos.h"

namespace atos {

namespace {

std::mutex g_mu;
// key: (device, host?, size class) -> cached blocks
std::map<std::tuple<int, int, size_t>, std::vector<void*>> g_free;
std::unordered_map<void*, std::tuple<int, int, size_t>> g_live;  // block -> its key
size_t g_cached_bytes = 0;

size_t size_class(size_t bytes) {
  if (bytes <= (1u << 20)) {
    size_t c = 256;
    while (c < bytes) c <<= 1;
    return c;
  }
  const size_t g = (size_t)2 << 20;
  return (bytes + g - 1) / g * g;
}

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

void trim_locked() {
  for (auto& kv : g_free) {
    const bool host = std::get<1>(kv.first) != 0;
    for (void* p : kv.second) {
      if (host) cudaFreeHost(p);
      else cudaFree(p);
    }
  }
  g_free.clear();
  g_cached_bytes = 0;
}

cudaError_t pool_get(void** p, size_t bytes, int host) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  const size_t cls = size_class(bytes);
  const auto key = std::make_tuple(host ? -1 : current_device(), host, cls);
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_free.find(key);
  if (it != g_free.end() && !it->second.empty()) {
    *p = it->second.back();
    it->second.pop_back();
    g_cached_bytes -= cls;
    g_live[*p] = key;
    return cudaSuccess;
  }
  cudaError_t e = host ? cudaMallocHost(p, cls) : cudaMalloc(p, cls);
  if (e != cudaSuccess && g_cached_bytes) {  // give the cached blocks back and try once more
    cudaGetLastError();
    trim_locked();
    e = host ? cudaMallocHost(p, cls) : cudaMalloc(p, cls);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  g_live[*p] = key;
  return cudaSuccess;
}

void pool_put(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_live.find(p);
  if (it == g_live.end()) return;  // not ours
  g_free[it->second].push_back(p);
  g_cached_bytes += std::get<2>(it->second);
  g_live.erase(it);
}

}  // namespace

cudaError_t pool_malloc(void** p, size_t bytes) { return pool_get(p, bytes, 0); }
cudaError_t pool_malloc_host(void** p, size_t bytes) { return pool_get(p, bytes, 1); }
void pool_free(void* p) { pool_put(p); }
void pool_free_host(void* p) { pool_put(p); }

}  // namespace atos

extern "C" int atos_pool_trim(int64_t* cached_bytes_before) {
  std::lock_guard<std::mutex> lock(atos::g_mu);
  if (cached_bytes_before) *cached_bytes_before = (int64_t)atos::g_cached_bytes;
  atos::trim_locked();
  return ATOS_OK;
}
