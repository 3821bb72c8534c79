// bfs.cuh -- the speculative BFS task body (Section 5.1, Algorithm 2).
#pragma once

#include "engine.cuh"

namespace atos {

constexpr int kMarkMinDegree = 16;  // ATOS_FLAG_BFS_EXPAND_ONCE: rows this long or longer are marked
constexpr int kSplitDegree = 8192;  // ATOS_FLAG_BFS_SPLIT_ROWS: longer rows become segment tasks
constexpr int kSegment = 4096;      // entries per segment task

struct BfsBody {
  template <int B>
  using Extra = NoExtra;
  static constexpr int kResidentThreads = 1536;
  // edges per thread of a load-balancing round (RMAT 22 x64: 2 beats 4 at 256 threads)
  template <int B>
  static constexpr int kLbsR = B <= 512 ? 2 : 1;

  // Reads the neighbours' depths of one load-balancing round, relaxes them (atomicMin) and
  // pushes the neighbours it improved.
  template <int BLOCK, class S>
  __device__ static void relax_round(S& sm, int32_t* __restrict__ depth, const int (&item)[S::kR],
                                     const int (&nb)[S::kR]) {
    constexpr int R = S::kR;
    int cur[R];
#pragma unroll
    for (int j = 0; j < R; ++j) cur[j] = item[j] >= 0 ? __ldcg(depth + nb[j]) : 0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      bool want = false;
      if (item[j] >= 0) {
        const int nd = sm.aux[item[j]];
        if (nd < cur[j]) want = nd < atomicMin(depth + nb[j], nd);
      }
      cta_push(sm, want, nb[j]);
    }
  }

  // Row splitting: the rows of `parts` > 0 become segment tasks of kSegment entries, table entry
  // (vertex, first entry, depth the row was popped at) and item -(entry + 1); returns false
  // (nothing split) when the table is full.  Whole block.
  template <int BLOCK, class S>
  __device__ static bool split_rows(S& sm, int parts, int v, int s, int d, const Launch& L, unsigned long long* st) {
    const Instance& I = sm.I;
    int total;
    const int off = block_exclusive_scan<BLOCK>(parts, sm.tmp, total);  // ends with a barrier
    if (threadIdx.x == 0) sm.base = atomicAdd(&I.ctl->seg_next, (unsigned)total);
    __syncthreads();
    const unsigned j0 = sm.base;
    if (j0 + (unsigned)total > I.seg_cap || j0 + (unsigned)total < j0) return false;  // uniform
    for (int k = 0; k < parts; ++k) I.segs[j0 + off + k] = make_int4(v, s + k * kSegment, d, 0);
    for (int w = 0; w < total; w += S::kPushCap) {  // push the segment items, a buffer at a time
      const int need = min(S::kPushCap, total - w);
      if (sm.npush + need > S::kPushCap) cta_flush<BLOCK>(sm, I, 0, L, st);
      const int at = sm.npush - w;
      for (int k = 0; k < parts; ++k) {
        const int idx = off + k;
        if (idx >= w && idx < w + need) sm.push[ATOS_IX(at + idx, S::kPushCap, sm, kSitePushBuffer)] = -(int)(j0 + idx + 1);
      }
      __syncthreads();
      if (threadIdx.x == 0) sm.npush += need;
      __syncthreads();
    }
    return true;
  }

  // CTA worker: stage (row start, depth + 1) of the popped vertices, scan their degrees and map
  // the flattened neighbour range onto the threads (load-balancing search inside the worker).
  // With a segment table (ATOS_FLAG_BFS_SPLIT_ROWS) a popped vertex whose row exceeds
  // kSplitDegree entries is pushed back as segment tasks, which any worker expands (re-reading the
  // vertex's depth then), so one long row is spread over the grid instead of holding one CTA.
  template <int BLOCK, class S>
  __device__ static void cta_batch(S& sm, int cnt, const Launch& L, unsigned long long* st) {
    const Instance& I = sm.I;
    int deg = 0, parts = 0, v = 0, s = 0, d = 0;
    if ((int)threadIdx.x < cnt) {
      const int item = sm.items[threadIdx.x];
      int e;
      if (item >= 0) {
        v = item;
        s = ldg(I.row_ptr + v), e = ldg(I.row_ptr + v + 1);
        d = ld_relaxed(I.depth + v);
      } else {  // a segment of a split row (entries are written once per run: read past L1)
        const int4 sg = __ldcg(I.segs + ATOS_IX(-(item + 1), I.seg_cap, sm, kSiteItem));
        v = sg.x, s = sg.y;
        e = min(ldg(I.row_ptr + v + 1), s + kSegment);
        d = ld_relaxed(I.depth + v);
        // the vertex improved since the row was split: the copy pushed by that improvement
        // expands the whole row at the better depth
        if (d < sg.z) e = s;
      }
      sm.start[threadIdx.x] = s;
      sm.aux[threadIdx.x] = d + 1;
      deg = d == kUnreached ? 0 : e - s;  // a queued vertex always has a depth; never relax from INT32_MAX
      // a vertex queued twice is expanded once per depth: a task finding it already expanded at
      // this depth or a better one (by a copy popped after the improvement) skips the expansion;
      // rows shorter than kMarkMinDegree are cheaper to re-expand than to mark
      if (item >= 0 && deg >= kMarkMinDegree && I.expanded && atomicMin(I.expanded + v, d) <= d) deg = 0;
      if (item >= 0 && deg > kSplitDegree && I.segs) parts = (deg + kSegment - 1) / kSegment;
    }
    if (I.segs && __syncthreads_or(parts > 0) && split_rows<BLOCK>(sm, parts, v, s, d, L, st) && parts > 0) deg = 0;
    int total;
    const int off = block_exclusive_scan<BLOCK>(deg, sm.tmp, total);
    if ((int)threadIdx.x < cnt) sm.off[threadIdx.x] = off;
    __syncthreads();
    int32_t* __restrict__ depth = I.depth;
    constexpr int R = S::kR;
    int rounds = 0;
    if (BLOCK >= 512) {
      // software-pipelined: the next round's col gathers are in flight while this round's
      // neighbour depths are read and relaxed (smaller CTAs run under a 40-register cap, where
      // the extra live registers spill)
      int item[R], nb[R];
      lbs_round<BLOCK>(sm, I.col, cnt, total, 0, item, nb);
      for (int base = 0; base < total; base += BLOCK * R) {
        int item2[R], nb2[R];
        lbs_round<BLOCK>(sm, I.col, cnt, total, base + BLOCK * R, item2, nb2);
        relax_round<BLOCK>(sm, depth, item, nb);
#pragma unroll
        for (int j = 0; j < R; ++j) item[j] = item2[j], nb[j] = nb2[j];
        if (base + BLOCK * R < total && flush_round<S>(rounds)) cta_maybe_flush<BLOCK>(sm, I, L, st);
      }
    } else {
      for (int base = 0; base < total; base += BLOCK * R) {
        int item[R], nb[R];
        lbs_round<BLOCK>(sm, I.col, cnt, total, base, item, nb);
        relax_round<BLOCK>(sm, depth, item, nb);
        if (base + BLOCK * R < total && flush_round<S>(rounds)) cta_maybe_flush<BLOCK>(sm, I, L, st);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      st[kStatTasks] += cnt;
      st[kStatEdges] += total;
    }
    cta_flush<BLOCK>(sm, I, cnt, L, st);
  }

  template <int BLOCK, class S>
  __device__ static int cta_idle(S& sm, const Launch&, unsigned long long*) {
    return threadIdx.x == 0 ? (instance_quiescent(sm.I) ? 1 : 0) : 0;
  }

  // Warp worker: the 32 lanes stride the neighbour list of one vertex.
  __device__ static void warp_item(WarpSmem& ws, const Instance& I, int v, const Launch& L, unsigned long long* st) {
    const int lane = threadIdx.x & 31;
    int d = 0, skip = 0;
    if (lane == 0) {
      d = ld_relaxed(I.depth + v);
      skip = d == kUnreached;
      if (!skip && I.expanded && ldg(I.row_ptr + v + 1) - ldg(I.row_ptr + v) >= kMarkMinDegree)
        skip = atomicMin(I.expanded + v, d) <= d;  // see cta_batch
    }
    d = __shfl_sync(0xffffffffu, d, 0);  // one read, so every lane relaxes with the same depth
    skip = __shfl_sync(0xffffffffu, skip, 0);
    const int nd = d + 1;
    const int s = ldg(I.row_ptr + v), e = skip ? s : ldg(I.row_ptr + v + 1);
    for (int k = s; k < e; k += 32) {
      const int j = k + lane;
      bool want = false;
      int nb = 0;
      if (j < e) {
        nb = nbr_at(I, j, L);
        if (nd < __ldcg(I.depth + nb)) want = nd < atomicMin(I.depth + nb, nd);
      }
      warp_push(ws, want, nb);
      warp_maybe_flush(ws, I, L, st);
    }
    if (lane == 0) st[kStatEdges] += e - s;
  }

  // Thread worker (worker_size 1, Section 3.2's smallest worker): each lane expands its own
  // vertex v (kEmpty: none), walking its row one entry per step; the warp steps together until
  // every lane's row is done, and pushes through the warp's buffer.  A row longer than
  // kLaneRowMax would hold the whole warp for its length, so those vertices are expanded after
  // the short rows by the warp worker's path, 32 entries per step (the thread/warp split of
  // load-balanced graph frameworks).
  static constexpr int kLaneRowMax = 32;
  __device__ static void lane_items(WarpSmem& ws, const Instance& I, int v, const Launch& L, unsigned long long* st) {
    int k = 0, e = 0, nd = 0;
    bool longrow = false;
    if (v != kEmpty) {
      const int d = ld_relaxed(I.depth + v);
      if (d != kUnreached) {
        k = ldg(I.row_ptr + v);
        e = ldg(I.row_ptr + v + 1);
        nd = d + 1;
        if (e - k > kLaneRowMax) {
          longrow = true;
          e = k;
        } else if (I.expanded && e - k >= kMarkMinDegree && atomicMin(I.expanded + v, d) <= d) {
          e = k;  // see cta_batch
        }
      }
    }
    unsigned long long edges = (unsigned long long)(e - k);
    while (__any_sync(0xffffffffu, k < e)) {
      bool want = false;
      int nb = 0;
      if (k < e) {
        nb = nbr_at(I, k, L);
        if (nd < __ldcg(I.depth + nb)) want = nd < atomicMin(I.depth + nb, nd);
        ++k;
      }
      warp_push(ws, want, nb);
      warp_maybe_flush(ws, I, L, st);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) edges += __shfl_xor_sync(0xffffffffu, edges, o);
    if ((threadIdx.x & 31) == 0) st[kStatEdges] += edges;
    for (unsigned big = __ballot_sync(0xffffffffu, longrow); big; big &= big - 1)
      warp_item(ws, I, __shfl_sync(0xffffffffu, v, __ffs(big) - 1), L, st);
  }

  __device__ static int warp_idle(WarpSmem&, const Instance& I, const Launch&, unsigned long long*) {
    return (threadIdx.x & 31) == 0 ? (instance_quiescent(I) ? 1 : 0) : 0;
  }
};

}  // namespace atos
