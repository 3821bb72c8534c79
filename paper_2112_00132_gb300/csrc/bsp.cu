// bsp.cu -- the level-synchronous comparator (Algorithms 1, 3, 5), driven level by level from the
// host or by a conditional WHILE node of a CUDA graph (see bsp.cuh).
//
// Level sequences (every kernel reads the sizes it covers from the control block):
//   BFS (Algorithm 1)        degrees -> scan -> advance (relax with atomicMin, append the
//                            improved (source, vertex) pairs to the next frontier) -> end
//   PageRank (Algorithm 3)   take (residue into rank, share per item) -> scan -> scatter (red.add
//                            of the shares over the frontier's edges) -> filter (every vertex
//                            whose residue exceeds eps forms the next frontier) -> end
//   colouring (Algorithm 5)  assign (first fit over the neighbours' colours) -> conflicts (of two
//                            adjacent vertices with one colour the larger id goes to the next
//                            frontier) -> end
// The scan is a device-wide exclusive scan of the frontier items' degrees (64-bit: a level of a
// multi-source BFS can hold more than 2^31 edges), so that each CTA of the advance and scatter
// kernels takes exactly kChunk consecutive edges (load-balanced advance).
#include <algorithm>

#include "bsp.cuh"
#include "launch.cuh"

namespace atos {
namespace bsp {

constexpr int kBlock = 256;
constexpr int kPerThread = 4;
constexpr int kChunk = kBlock * kPerThread;  // items per scan chunk, edges per CTA per advance step
constexpr int kPerLevel[3] = {7, 8, 3};      // kernels in a level of BFS, PageRank, colouring

// The control block: level state first (what the host reads back), then the run's parameters.
struct Ctl {
  long long F[2];    // frontier sizes; F[cur] is the current frontier, F[cur ^ 1] the next one
  long long total;   // edges of the current (scanned) frontier
  long long edges, tasks, iters;
  long long max_iters;
  int cur, level, status, app;
  int fail_site;     // checked builds: the first bounds violation's site
  int pad;
  long long cap_items;   // frontier buffer capacity (items)
  long long cap_chunks;  // chunk_lo capacity
  long long nnz;
  // parameters
  const int32_t* row_ptr;
  const int32_t* col;
  int32_t n, nsrc;
  int32_t* depth;
  float* rank;
  float* res;
  float alpha, eps;
  int32_t* color;
  void* fr[2];       // BFS: uint64 (source << 32 | vertex); PageRank, colouring: int32 vertex
  long long* offs;   // scan of the current frontier's degrees (F + 1 entries)
  long long* bsums;  // per-chunk sums of the scan
  int32_t* chunk_lo; // per edge chunk of kChunk edges: the frontier item owning its first edge
  float* share;      // PageRank: alpha * residue / degree per frontier item
  int32_t* sources;  // BFS: the nsrc sources
};

struct Header {  // the leading fields of Ctl, as read back by the host
  long long F[2];
  long long total, edges, tasks, iters, max_iters;
  int cur, level, status, app;
};
static_assert(sizeof(Header) <= sizeof(Ctl), "header");

// Where checked builds record a violation (the control block's status and site words).
struct CtlErr {
  int* status;
  int* fail_site;
  __device__ explicit CtlErr(Ctl* c) : status(&c->status), fail_site(&c->fail_site) {}
};

// col[k] with the entry index and the neighbour id checked in checked builds.
__device__ __forceinline__ int col_at(const int32_t* __restrict__ col, long long k, const Ctl* c, const CtlErr& ce) {
#ifdef ATOS_CHECKED
  return ATOS_IX(__ldg(col + ATOS_IX(k, c->nnz, ce, kSiteEntry)), c->n, ce, kSiteNeighbour);
#else
  (void)c, (void)ce;
  return __ldg(col + k);
#endif
}

__device__ __forceinline__ long long warp_incl_scan64(long long x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive prefix sum of 64-bit values over a block of BLOCK threads (tmp: 33 entries).
template <int BLOCK>
__device__ long long block_excl_scan64(long long x, long long* tmp, long long& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long inc = warp_incl_scan64(x);
  if (lane == 31) tmp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const long long s = lane < BLOCK / 32 ? tmp[lane] : 0;
    const long long si = warp_incl_scan64(s);
    if (lane < BLOCK / 32) tmp[lane] = si - s;
    if (lane == 31) tmp[32] = si;
  }
  __syncthreads();
  total = tmp[32];
  const long long r = tmp[wid] + inc - x;
  __syncthreads();
  return r;
}

// Largest i in [0, cnt) with off[i] <= e (off non-decreasing, off[0] <= e).
__device__ __forceinline__ long long owner64(const long long* off, long long cnt, long long e) {
  long long lo = 0, hi = cnt - 1;
  while (lo < hi) {
    const long long mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Appends `item` (when `want`) to the next frontier with one atomic per warp.
template <class T>
__device__ __forceinline__ void append_next(Ctl* c, int nxt, bool want, T item) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd((unsigned long long*)&c->F[nxt], (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  const CtlErr ce(c);
  if (want) ((T*)c->fr[nxt])[ATOS_IX((long long)(base + __popc(m & lanemask_lt())), c->cap_items, ce, kSiteFrontier)] = item;
}

// ------------------------------------------------------------------------------------ scan

// Chunk-local exclusive scan of offs[0, F) (the items' degrees) and the chunk sums.
__global__ void __launch_bounds__(kBlock) scan_chunks_kernel(Ctl* c) {
  __shared__ long long tmp[33];
  const long long F = c->F[c->cur];
  const long long nchunks = (F + kChunk - 1) / kChunk;
  long long* __restrict__ offs = c->offs;
  long long* __restrict__ bsums = c->bsums;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long base = ch * kChunk + (long long)threadIdx.x * kPerThread;
    long long d[kPerThread], local = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      d[k] = base + k < F ? offs[base + k] : 0;
      local += d[k];
    }
    long long total;
    long long pre = block_excl_scan64<kBlock>(local, tmp, total);
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      if (base + k < F) offs[base + k] = pre;
      pre += d[k];
    }
    if (threadIdx.x == 0) bsums[ch] = total;
  }
}

// One block: exclusive scan of the chunk sums; offs[F] and c->total receive the frontier's edges.
__global__ void __launch_bounds__(1024) scan_top_kernel(Ctl* c) {
  __shared__ long long tmp[33];
  const long long F = c->F[c->cur];
  const long long nchunks = (F + kChunk - 1) / kChunk;
  const long long per = (nchunks + 1023) / 1024;
  const long long b0 = (long long)threadIdx.x * per;
  long long* __restrict__ bsums = c->bsums;
  long long local = 0;
  for (long long k = 0; k < per; ++k)
    if (b0 + k < nchunks) local += bsums[b0 + k];
  long long total;
  long long pre = block_excl_scan64<1024>(local, tmp, total);
  for (long long k = 0; k < per; ++k)
    if (b0 + k < nchunks) {
      const long long x = bsums[b0 + k];
      bsums[b0 + k] = pre;
      pre += x;
    }
  if (threadIdx.x == 0) {
    c->offs[F] = total;
    c->total = total;
  }
}

__global__ void scan_add_kernel(Ctl* c) {
  const long long F = c->F[c->cur];
  long long* __restrict__ offs = c->offs;
  const long long* __restrict__ bsums = c->bsums;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < F; i += (long long)gridDim.x * blockDim.x)
    offs[i] += bsums[i / kChunk];
}

// Owner of each edge chunk's first edge: item i writes itself for every chunk that starts in its
// edge range [offs[i], offs[i + 1]) (a parallel scatter instead of a binary search per chunk).
__global__ void mark_chunks_kernel(Ctl* c) {
  const long long F = c->F[c->cur];
  const long long* __restrict__ offs = c->offs;
  int32_t* __restrict__ lo = c->chunk_lo;
  const CtlErr ce(c);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < F; i += (long long)gridDim.x * blockDim.x) {
    const long long a = offs[i], b = offs[i + 1];
    for (long long ch = (a + kChunk - 1) / kChunk; ch * kChunk < b; ++ch) lo[ATOS_IX(ch, c->cap_chunks, ce, kSiteChunk)] = (int32_t)i;
  }
}

// Stages the frontier items that own the edges of chunk `ch` (shared: their scan offsets, item
// words and row starts); returns the first item and the count through *lo / *cnt, or cnt > kChunk
// + 1 when the range (degree-0 items included) does not fit, then nothing is staged.
template <class Item, class RowOf>
__device__ __forceinline__ void stage_chunk(const Ctl* c, long long ch, long long nchunks, long long F,
                                            const Item* __restrict__ fr, long long* s_off, Item* s_item,
                                            int* s_start, long long* s_lo, long long* s_cnt, RowOf row_of) {
  if (threadIdx.x == 0) {
    const long long lo = c->chunk_lo[ch];
    const long long hi = ch + 1 < nchunks ? c->chunk_lo[ch + 1] : F - 1;
    *s_lo = lo;
    *s_cnt = hi - lo + 1;
  }
  __syncthreads();
  const long long lo = *s_lo, cnt = *s_cnt;
  if (cnt <= kChunk + 1)
    for (int k = threadIdx.x; k < cnt; k += kBlock) {
      s_off[k] = c->offs[lo + k];
      s_item[k] = fr[lo + k];
      s_start[k] = __ldg(c->row_ptr + row_of(s_item[k]));
    }
  __syncthreads();
}

// ---------------------------------------------------------------------------- level end

// One thread: account the level, make the next frontier current, decide whether to go on.
__global__ void level_end_kernel(Ctl* c, cudaGraphConditionalHandle handle, int use_handle) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int cur = c->cur;
  c->edges += c->total;
  c->tasks += c->F[cur];
  c->iters += 1;
  c->total = 0;
  c->cur = cur ^ 1;
  c->F[cur] = 0;  // the old frontier's buffer receives the next level's items
  c->level += 1;
  bool more = c->F[cur ^ 1] > 0;
  if (more && c->iters >= c->max_iters) {
    c->status = ATOS_ERR_TIMEOUT;
    more = false;
  }
  if (use_handle) cudaGraphSetConditional(handle, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------------- BFS

__global__ void bfs_fill_kernel(Ctl* c) {
  const long long total = (long long)c->nsrc * c->n;
  int32_t* __restrict__ depth = c->depth;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    depth[i] = kUnreached;
}

__global__ void bfs_seed_kernel(Ctl* c) {
  unsigned long long* fr = (unsigned long long*)c->fr[c->cur];
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < c->nsrc; s += gridDim.x * blockDim.x) {
    const int v = c->sources[s];
    c->depth[(long long)s * c->n + v] = 0;
    fr[s] = ((unsigned long long)s << 32) | (unsigned)v;
  }
}

__global__ void bfs_degrees_kernel(Ctl* c) {
  const long long F = c->F[c->cur];
  const unsigned long long* __restrict__ fr = (const unsigned long long*)c->fr[c->cur];
  const int32_t* __restrict__ row_ptr = c->row_ptr;
  long long* __restrict__ offs = c->offs;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < F; i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(unsigned)fr[i];
    offs[i] = __ldg(row_ptr + v + 1) - __ldg(row_ptr + v);
  }
}

// Relaxes edge chunks [k kChunk, (k + 1) kChunk) of the scanned frontier, grid-stride over chunks.
__global__ void __launch_bounds__(kBlock) bfs_advance_kernel(Ctl* c) {
  __shared__ long long s_off[kChunk + 1];
  __shared__ unsigned long long s_item[kChunk + 1];
  __shared__ int s_start[kChunk + 1];
  __shared__ long long s_lo, s_cnt;
  const int cur = c->cur, nxt = cur ^ 1;
  const long long F = c->F[cur];
  const long long total = c->total;
  const int nd = c->level + 1;
  const long long n = c->n;
  const unsigned long long* fr = (const unsigned long long*)c->fr[cur];
  const long long* offs = c->offs;
  const int32_t* __restrict__ row_ptr = c->row_ptr;
  const int32_t* __restrict__ col = c->col;
  int32_t* depth = c->depth;
  const CtlErr ce(c);
  const long long nchunks = (total + kChunk - 1) / kChunk;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long e0 = ch * kChunk, e1 = min(total, e0 + kChunk);
    stage_chunk(c, ch, nchunks, F, fr, s_off, s_item, s_start, &s_lo, &s_cnt,
                [](unsigned long long it) { return (int)(unsigned)it; });
    const long long lo = s_lo, cnt = s_cnt;
    // items of degree 0 can make the owning range longer than the chunk; such a chunk searches
    // the global offsets of its range instead of a staged copy
    const bool staged = cnt <= kChunk + 1;
    // each thread: kPerThread consecutive edges, one owner search
    const long long ea = e0 + (long long)threadIdx.x * kPerThread;
    long long i = 0;
    if (ea < e1) i = staged ? owner64(s_off, cnt, ea) : owner64(offs + lo, cnt, ea);
    int nbs[kPerThread], cur_d[kPerThread];
    unsigned srcs[kPerThread];
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) {
      const long long e = ea + r;
      nbs[r] = -1;
      srcs[r] = 0;
      if (e < e1) {
        if (staged) {
          while (i + 1 < cnt && s_off[i + 1] <= e) ++i;
          srcs[r] = (unsigned)(s_item[i] >> 32);
          nbs[r] = col_at(col, s_start[i] + (e - s_off[i]), c, ce);
        } else {
          while (i + 1 < cnt && offs[lo + i + 1] <= e) ++i;
          const unsigned long long it = fr[lo + i];
          srcs[r] = (unsigned)(it >> 32);
          nbs[r] = col_at(col, __ldg(row_ptr + (int)(unsigned)it) + (e - offs[lo + i]), c, ce);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) cur_d[r] = nbs[r] >= 0 ? __ldcg(depth + (long long)srcs[r] * n + nbs[r]) : 0;
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) {
      bool want = false;
      if (nbs[r] >= 0 && nd < cur_d[r]) want = nd < atomicMin(depth + (long long)srcs[r] * n + nbs[r], nd);
      append_next(c, nxt, want, ((unsigned long long)srcs[r] << 32) | (unsigned)(nbs[r] < 0 ? 0 : nbs[r]));
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- PageRank

__global__ void iota_kernel(Ctl* c) {
  int32_t* fr = (int32_t*)c->fr[c->cur];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < c->n; v += gridDim.x * blockDim.x) fr[v] = v;
}

// Per frontier vertex: take the residue, add it to the rank, record the share to scatter and its
// degree (0 when there is nothing to scatter) for the scan.
__global__ void pr_take_kernel(Ctl* c) {
  const long long F = c->F[c->cur];
  const int32_t* __restrict__ fr = (const int32_t*)c->fr[c->cur];
  const int32_t* __restrict__ row_ptr = c->row_ptr;
  float* __restrict__ res = c->res;
  float* __restrict__ rank = c->rank;
  float* __restrict__ share = c->share;
  long long* __restrict__ offs = c->offs;
  const float alpha = c->alpha;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < F; i += (long long)gridDim.x * blockDim.x) {
    const int v = fr[i];
    const float r = atomicExch(res + v, 0.0f);
    const int d = __ldg(row_ptr + v + 1) - __ldg(row_ptr + v);
    rank[v] += r;
    const bool go = r != 0.0f && d > 0;
    share[i] = go ? alpha * r / (float)d : 0.0f;
    offs[i] = go ? d : 0;
  }
}

// Load-balanced scatter over the frontier's edges: each thread kPerThread consecutive edges, one
// owner search.
__global__ void __launch_bounds__(kBlock) pr_scatter_kernel(Ctl* c) {
  __shared__ long long s_off[kChunk + 1];
  __shared__ int32_t s_item[kChunk + 1];
  __shared__ int s_start[kChunk + 1];
  __shared__ long long s_lo, s_cnt;
  const long long F = c->F[c->cur];
  const long long total = c->total;
  const int32_t* __restrict__ fr = (const int32_t*)c->fr[c->cur];
  const long long* __restrict__ offs = c->offs;
  const int32_t* __restrict__ row_ptr = c->row_ptr;
  const int32_t* __restrict__ col = c->col;
  const float* __restrict__ share = c->share;
  float* res = c->res;
  const CtlErr ce(c);
  const long long nchunks = (total + kChunk - 1) / kChunk;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long e0 = ch * kChunk, e1 = min(total, e0 + kChunk);
    stage_chunk(c, ch, nchunks, F, fr, s_off, s_item, s_start, &s_lo, &s_cnt, [](int32_t v) { return v; });
    const long long lo = s_lo, cnt = s_cnt;
    const bool staged = cnt <= kChunk + 1;
    // each thread: kPerThread consecutive edges, one owner search
    const long long ea = e0 + (long long)threadIdx.x * kPerThread;
    if (ea < e1) {
      long long i = staged ? owner64(s_off, cnt, ea) : owner64(offs + lo, cnt, ea);
#pragma unroll
      for (int k = 0; k < kPerThread; ++k) {
        const long long e = ea + k;
        if (e >= e1) break;
        int nb;
        if (staged) {
          while (i + 1 < cnt && s_off[i + 1] <= e) ++i;
          nb = col_at(col, s_start[i] + (e - s_off[i]), c, ce);
        } else {
          while (i + 1 < cnt && offs[lo + i + 1] <= e) ++i;
          nb = col_at(col, __ldg(row_ptr + fr[lo + i]) + (e - offs[lo + i]), c, ce);
        }
        red_add_f32(res + nb, share[lo + i]);
      }
    }
    __syncthreads();
  }
}

// The next frontier: every vertex whose residue exceeds eps.
__global__ void pr_filter_kernel(Ctl* c) {
  const int nxt = c->cur ^ 1;
  const float eps = c->eps;
  const int n = c->n;
  const float* __restrict__ res = c->res;
  unsigned long long* count = (unsigned long long*)&c->F[nxt];
  int32_t* out = (int32_t*)c->fr[nxt];
  const long long cap = c->cap_items;
  const CtlErr ce(c);
  (void)cap, (void)ce;
  const int lane = threadIdx.x & 31;
  for (int r = blockIdx.x * blockDim.x; r < n; r += gridDim.x * blockDim.x) {
    const int v = r + threadIdx.x;
    const bool want = v < n && __ldcg(res + v) > eps;
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) continue;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) out[ATOS_IX((long long)(base + __popc(m & lanemask_lt())), cap, ce, kSiteFrontier)] = v;
  }
}

// ---------------------------------------------------------------------------- colouring

__global__ void gc_init_kernel(Ctl* c) {
  int32_t* fr = (int32_t*)c->fr[c->cur];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < c->n; v += gridDim.x * blockDim.x) {
    fr[v] = v;
    c->color[v] = -1;
  }
}

// Every frontier vertex takes the smallest colour none of its neighbours holds (one warp per
// vertex, colour windows of 64 combined by an OR reduction over the lanes).
__global__ void gc_assign_kernel(Ctl* c) {
  const long long F = c->F[c->cur];
  const int32_t* __restrict__ fr = (const int32_t*)c->fr[c->cur];
  const int32_t* __restrict__ row_ptr = c->row_ptr;
  const int32_t* __restrict__ col = c->col;
  int32_t* color = c->color;
  const CtlErr ce(c);
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  long long ed = 0;
  for (long long i = gw; i < F; i += nw) {
    const int v = fr[i];
    const int s = __ldg(row_ptr + v), e = __ldg(row_ptr + v + 1);
    int colour = -1;
    for (int base = 0; colour < 0; base += 64) {
      unsigned lo = 0, hi = 0;
      for (int k = s + lane; k < e; k += 32) {
        const int rel = __ldcg(color + col_at(col, k, c, ce)) - base;
        if (rel >= 0 && rel < 32) lo |= 1u << rel;
        else if (rel >= 32 && rel < 64) hi |= 1u << (rel - 32);
      }
      ed += e - s;
      lo = __reduce_or_sync(0xffffffffu, lo);
      hi = __reduce_or_sync(0xffffffffu, hi);
      const unsigned long long used = ((unsigned long long)hi << 32) | lo;
      if (~used) colour = base + __ffsll((long long)~used) - 1;
    }
    if (lane == 0) color[v] = colour;
  }
  if (lane == 0 && ed) atomicAdd((unsigned long long*)&c->edges, (unsigned long long)ed);
}

// A frontier vertex whose colour a smaller neighbour also holds goes to the next frontier (of a
// conflicting pair the larger id recolours).
__global__ void gc_conflicts_kernel(Ctl* c) {
  const int cur = c->cur, nxt = cur ^ 1;
  const long long F = c->F[cur];
  const int32_t* __restrict__ fr = (const int32_t*)c->fr[cur];
  const int32_t* __restrict__ row_ptr = c->row_ptr;
  const int32_t* __restrict__ col = c->col;
  const int32_t* __restrict__ color = c->color;
  unsigned long long* count = (unsigned long long*)&c->F[nxt];
  int32_t* out = (int32_t*)c->fr[nxt];
  const CtlErr ce(c);
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = gw; i < F; i += nw) {
    const int v = fr[i];
    const int s = __ldg(row_ptr + v), e = __ldg(row_ptr + v + 1);
    const int cv = color[v];
    bool conflict = false;
    for (int k = s + lane; k < e; k += 32) {
      const int u = col_at(col, k, c, ce);
      conflict |= u < v && color[u] == cv;
    }
    if (__any_sync(0xffffffffu, conflict) && lane == 0)
      out[ATOS_IX((long long)atomicAdd(count, 1ull), c->cap_items, ce, kSiteFrontier)] = v;
  }
}

// ---------------------------------------------------------------------------- int32 scan

__global__ void __launch_bounds__(kBlock) chunk_sums_inplace(int32_t* a, int32_t F, int32_t* bsums) {
  __shared__ int tmp[33];
  const int base = blockIdx.x * kChunk;
  int local = 0;
  int d[kPerThread];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int i = base + threadIdx.x * kPerThread + k;
    d[k] = i < F ? a[i] : 0;
    local += d[k];
  }
  int total;
  int pre = block_exclusive_scan<kBlock>(local, tmp, total);
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int i = base + threadIdx.x * kPerThread + k;
    if (i < F) a[i] = pre;
    pre += d[k];
  }
  if (threadIdx.x == 0) bsums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_chunk_sums(int32_t* bsums, int nb, int32_t* offs, int32_t F) {
  __shared__ int tmp[33];
  const int per = (nb + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  int local = 0;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) local += bsums[b0 + k];
  int total;
  int pre = block_exclusive_scan<1024>(local, tmp, total);
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) {
      const int x = bsums[b0 + k];
      bsums[b0 + k] = pre;
      pre += x;
    }
  if (threadIdx.x == 0) offs[F] = total;
}

__global__ void __launch_bounds__(kBlock) add_chunk_offsets(int32_t* offs, int32_t F, const int32_t* bsums) {
  const int base = blockIdx.x * kChunk;
  const int add = bsums[blockIdx.x];
  for (int k = threadIdx.x; k < kChunk; k += kBlock) {
    const int i = base + k;
    if (i < F) offs[i] += add;
  }
}

cudaError_t scan_inplace(int32_t* a, int32_t F, int32_t* bsums, cudaStream_t s) {
  if (F <= 0) return cudaMemsetAsync(a, 0, sizeof(int32_t), s);
  const int nb = (F + kChunk - 1) / kChunk;
  count_launches(3);
  chunk_sums_inplace<<<nb, kBlock, 0, s>>>(a, F, bsums);
  scan_chunk_sums<<<1, 1024, 0, s>>>(bsums, nb, a, F);
  add_chunk_offsets<<<nb, kBlock, 0, s>>>(a, F, bsums);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------- driver

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t ctl, fr0, fr1, offs, bsums, chunk_lo, share, sources, total;
  size_t items, chunks;  // frontier capacity (items) and chunk_lo capacity (entries)
};

Layout layout_for(int app, int32_t n, int64_t nnz, int32_t nsrc) {
  const size_t items = app == kAppBfs ? (size_t)n * (size_t)std::max(nsrc, 1) : (size_t)n;
  // a level scans at most every source's whole CSR: nsrc * nnz edges
  const size_t edges = app == kAppBfs ? (size_t)nnz * (size_t)std::max(nsrc, 1) : (size_t)nnz;
  const size_t isz = app == kAppBfs ? 8 : 4;
  Layout L;
  size_t p = 0;
  L.ctl = p, p += align256(sizeof(Ctl));
  L.fr0 = p, p += align256(isz * std::max<size_t>(items, 1));
  L.fr1 = p, p += align256(isz * std::max<size_t>(items, 1));
  L.offs = p, p += app == kAppGc ? 0 : align256(8 * (items + 1));
  L.bsums = p, p += app == kAppGc ? 0 : align256(8 * (items / kChunk + 2));
  L.chunk_lo = p, p += app == kAppGc ? 0 : align256(4 * (edges / kChunk + 2));
  L.share = p, p += app == kAppPr ? align256(4 * std::max<size_t>(items, 1)) : 0;
  L.sources = p, p += app == kAppBfs ? align256(4 * (size_t)std::max(nsrc, 1)) : 0;
  L.total = p;
  L.items = std::max<size_t>(items, 1);
  L.chunks = app == kAppGc ? 0 : edges / kChunk + 2;
  return L;
}

struct Grids {
  int items, edges, warps;
};

Grids grids() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return Grids{sms * 8, sms * 8, sms * 16};
}

// The kernels of one level (launched on `s`; captured into a graph when `s` is capturing).
cudaError_t launch_level(int app, Ctl* c, const Grids& g, cudaGraphConditionalHandle h, int use_handle,
                         cudaStream_t s) {
  if (app == kAppBfs) {
    bfs_degrees_kernel<<<g.items, kBlock, 0, s>>>(c);
    scan_chunks_kernel<<<g.items, kBlock, 0, s>>>(c);
    scan_top_kernel<<<1, 1024, 0, s>>>(c);
    scan_add_kernel<<<g.items, kBlock, 0, s>>>(c);
    mark_chunks_kernel<<<g.items, kBlock, 0, s>>>(c);
    bfs_advance_kernel<<<g.edges, kBlock, 0, s>>>(c);
  } else if (app == kAppPr) {
    pr_take_kernel<<<g.items, kBlock, 0, s>>>(c);
    scan_chunks_kernel<<<g.items, kBlock, 0, s>>>(c);
    scan_top_kernel<<<1, 1024, 0, s>>>(c);
    scan_add_kernel<<<g.items, kBlock, 0, s>>>(c);
    mark_chunks_kernel<<<g.items, kBlock, 0, s>>>(c);
    pr_scatter_kernel<<<g.edges, kBlock, 0, s>>>(c);
    pr_filter_kernel<<<g.items, kBlock, 0, s>>>(c);
  } else {
    gc_assign_kernel<<<g.warps, kBlock, 0, s>>>(c);
    gc_conflicts_kernel<<<g.warps, kBlock, 0, s>>>(c);
  }
  level_end_kernel<<<1, 32, 0, s>>>(c, h, use_handle);
  return cudaGetLastError();
}

int app_index(int app) { return app == kAppBfs ? 0 : (app == kAppPr ? 1 : 2); }

// The device-loop graph of `app` for the control block at c: one conditional WHILE node whose
// body is one level (the level's last kernel sets the condition).
cudaError_t build_graph(int app, Ctl* c, const Grids& g, BspGraphs* graphs) {
  cudaError_t e = cudaSuccess;
  if (!graphs->capture) e = cudaStreamCreateWithFlags(&graphs->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaGraph_t graph = nullptr;
  e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle handle;
  e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams params = {};
  params.type = cudaGraphNodeTypeConditional;
  params.conditional.handle = handle;
  params.conditional.type = cudaGraphCondTypeWhile;
  params.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &params);
  if (e == cudaSuccess) {
    cudaGraph_t body = params.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(graphs->capture, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e1 = launch_level(app, c, g, handle, 1, graphs->capture);
      const cudaError_t e2 = cudaStreamEndCapture(graphs->capture, &body);
      e = e1 != cudaSuccess ? e1 : e2;
    }
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e == cudaSuccess) graphs->exec[app_index(app)] = exec;
  return e;
}

}  // namespace bsp

void BspGraphs::release() {
  for (auto& e : exec)
    if (e) cudaGraphExecDestroy(e), e = nullptr;
  if (capture) cudaStreamDestroy(capture), capture = nullptr;
  scratch = nullptr;
}

size_t bsp_scratch_bytes(int app, int32_t n, int64_t nnz, int32_t nsrc) {
  return bsp::layout_for(app, n, nnz, nsrc).total;
}

size_t bsp_host_bytes() { return 2 * bsp::align256(sizeof(bsp::Ctl)); }

int bsp_run(const BspRun& r, void* scratch, size_t scratch_bytes, void* host_buf, BspGraphs* graphs, cudaStream_t s,
            BspResult* result) {
  using namespace bsp;
  const int nsrc = r.app == kAppBfs ? r.nsrc : 1;
  const Layout Lo = layout_for(r.app, r.n, r.nnz, nsrc);
  if (!scratch || scratch_bytes < Lo.total || !host_buf || r.n < 1 || nsrc < 1) return ATOS_ERR_INVALID_ARG;
  char* base = (char*)scratch;
  Ctl* d_ctl = (Ctl*)(base + Lo.ctl);
  Ctl* h_img = (Ctl*)host_buf;                                  // the parameters uploaded
  Header* h_back = (Header*)((char*)host_buf + align256(sizeof(Ctl)));  // the level state read back
  Ctl c;
  memset(&c, 0, sizeof(c));
  c.F[0] = r.app == kAppBfs ? nsrc : r.n;
  c.max_iters = r.app == kAppBfs ? (long long)r.n + 2 : (1LL << 22);
  c.app = r.app;
  c.row_ptr = r.row_ptr, c.col = r.col, c.n = r.n, c.nsrc = nsrc;
  c.depth = r.depth, c.rank = r.rank, c.res = r.res, c.alpha = r.alpha, c.eps = r.eps, c.color = r.color;
  c.fr[0] = base + Lo.fr0, c.fr[1] = base + Lo.fr1;
  c.offs = (long long*)(base + Lo.offs);
  c.bsums = (long long*)(base + Lo.bsums);
  c.chunk_lo = (int32_t*)(base + Lo.chunk_lo);
  c.cap_items = (long long)Lo.items;
  c.cap_chunks = (long long)Lo.chunks;
  c.nnz = r.nnz;
  c.share = (float*)(base + Lo.share);
  c.sources = (int32_t*)(base + Lo.sources);
  // the pinned image may still be in flight from the previous run on this scratch
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ATOS_ERR_CUDA;
  *h_img = c;
  e = cudaMemcpyAsync(d_ctl, h_img, sizeof(Ctl), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && r.app == kAppBfs)
    e = cudaMemcpyAsync(c.sources, r.sources, sizeof(int32_t) * nsrc, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return ATOS_ERR_CUDA;
  const Grids g = grids();
  count_launches(2);
  if (r.app == kAppBfs) {
    bfs_fill_kernel<<<g.items, kBlock, 0, s>>>(d_ctl);
    bfs_seed_kernel<<<std::max(1, std::min(g.items, (nsrc + kBlock - 1) / kBlock)), kBlock, 0, s>>>(d_ctl);
  } else if (r.app == kAppPr) {
    iota_kernel<<<g.items, kBlock, 0, s>>>(d_ctl);
    uncount_launches(1);
  } else {
    gc_init_kernel<<<g.items, kBlock, 0, s>>>(d_ctl);
    uncount_launches(1);
  }
  if (cudaGetLastError() != cudaSuccess) return ATOS_ERR_CUDA;
  const int per_level = kPerLevel[app_index(r.app)];
  if (r.device_loop) {
    if (graphs->scratch != scratch) {
      graphs->release();
      graphs->scratch = scratch;
    }
    cudaGraphExec_t& exec = graphs->exec[app_index(r.app)];
    if (!exec && build_graph(r.app, d_ctl, g, graphs) != cudaSuccess) {
      cudaGetLastError();
      return ATOS_ERR_CUDA;
    }
    count_launches(1);
    if (cudaGraphLaunch(exec, s) != cudaSuccess) return ATOS_ERR_CUDA;
    if (result) {
      if (cudaMemcpyAsync(h_back, d_ctl, sizeof(Header), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return ATOS_ERR_CUDA;
      count_launches((unsigned)(h_back->iters * per_level));  // the kernels the graph ran
    }
  } else {
    for (;;) {
      count_launches(per_level);
      if (launch_level(r.app, d_ctl, g, 0, 0, s) != cudaSuccess) return ATOS_ERR_CUDA;
      if (cudaMemcpyAsync(h_back, d_ctl, sizeof(Header), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return ATOS_ERR_CUDA;
      if (h_back->status || h_back->F[h_back->cur] == 0) break;
    }
  }
  if (result) {
    result->iters = h_back->iters;
    result->edges = h_back->edges;
    result->tasks = h_back->tasks;
    result->status = h_back->status;
  }
  return ATOS_OK;
}

}  // namespace atos
