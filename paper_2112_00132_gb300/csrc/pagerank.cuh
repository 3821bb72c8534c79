// pagerank.cuh -- asynchronous push-residual PageRank task body (Section 5.2, Algorithm 4).
//
// A task is a vertex v.  The worker takes v's residue with an atomic exchange, adds it to
// rank[v], and scatters alpha * residue / deg(v) to every neighbour (red.global.add.f32, no
// return).  It then reserves Check_Size consecutive vertex ids from a round-robin cursor and
// enqueues those whose residue exceeds epsilon.  All arithmetic on ranks and residues is FP32.
//
// Two points the paper leaves open are fixed here:
//   * a vertex is in the queue at most once: a bitmap bit is set by whoever enqueues it and
//     cleared by the worker that pops it (before it takes the residue), so the ring never needs
//     more than n slots and duplicate pops disappear;
//   * termination: the queue draining is not enough, because Algorithm 4 enqueues only through
//     the Check_Size scan.  Workers whose pops come back empty run the scan as their idle
//     function (f2 of the launch API), and once the instance is quiescent (tasks pushed ==
//     tasks completed, value T) they split one full sweep of all n residues into chunks; the
//     instance ends when a sweep that started at quiescence T has covered all n vertices without
//     enqueueing anything and the queue word still reads (T, T).  Nothing can change a residue
//     during such a sweep, so every residue is then at most epsilon.
//
// Hub combining: on the spread-id copy the highest-degree vertices sit at the first entry of
// distinct 128-byte lines of the residue array (I.hub gives the id of the hub of each rank and the
// rank of the hub at an id; rank 0 has the largest degree).  A CTA worker keeps FP32 accumulators
// for the first hubs in shared memory, slot i for the hub of rank i; its batch adds every
// residue share bound for such a hub there (a shared-memory atomic) and, once the batch's
// scatter is done, sends each accumulator that is not zero to the residue array with one
// red.add.  The batch's updates are all in global memory before it reports its tasks complete,
// as without combining, so the termination rule above is unchanged.  On scale-free graphs a few
// thousand hubs receive a large share of all updates; each CTA then sends each of them one update
// per batch instead of one per edge.
//
// Variant (ATOS_FLAG_PR_CROSSING): instead of the Check_Size scan, the scatter uses an atomic add
// that returns the old residue, and the push that lifts a neighbour from <= epsilon to above it
// enqueues that neighbour (through the same queued bit).  Every residue above epsilon is then
// queued or being processed without any scan; the verification sweep above still decides
// termination (it also catches the rare residue stranded by a pop that clears the bit after a
// concurrent crossing set it).
#pragma once

#include "engine.cuh"

namespace atos {

__device__ __forceinline__ bool pr_try_enqueue(const Instance& I, int u) {
  if (!(__ldcg(I.res + u) > I.eps)) return false;
  const unsigned bit = 1u << (u & 31);
  return !(atomicOr(I.qbits + (u >> 5), bit) & bit);
}

// Final-sweep check of u: returns 1 if u must be pushed (residue above eps, bit claimed), and
// sets *dirty whenever the residue is above eps at all.  A set bit does not make a vertex clean:
// another worker may have set it and not yet reserved the ticket, so the control word can still
// read quiescent while that push is pending.
__device__ __forceinline__ bool pr_sweep_vertex(const Instance& I, int u, bool* dirty) {
  if (!(__ldcg(I.res + u) > I.eps)) return false;
  *dirty = true;
  const unsigned bit = 1u << (u & 31);
  return !(atomicOr(I.qbits + (u >> 5), bit) & bit);
}

// Verification sweep protocol (see the file comment).  Returns the claimed chunk (>= 0), -1 when
// the epoch has no chunk left, -2 when the instance is not quiescent or the epoch is stale.
__device__ __forceinline__ int pr_claim_chunk(const Instance& I, int chunk, unsigned& T) {
  const unsigned long long w = ld_relaxed_u64(&I.ctl->word);
  T = (unsigned)(w >> 32);
  if (T != (unsigned)w) return -2;
  const unsigned nchunks = ((unsigned)I.n + chunk - 1) / chunk;
  for (int tries = 0; tries < 64; ++tries) {
    const unsigned long long vw = ld_relaxed_u64(&I.ctl->vword);
    const unsigned e = (unsigned)(vw >> 32);
    if (e != T) {
      if ((int)(e - T) > 0) return -2;  // a newer epoch exists: our view is stale
      atomicCAS(&I.ctl->vword, vw, (unsigned long long)T << 32);
      continue;
    }
    const unsigned k = (unsigned)vw;
    if (k >= nchunks) return -1;
    if (atomicCAS(&I.ctl->vword, vw, vw + 1) == vw) return (int)k;
  }
  return -1;
}

// Records `len` clean vertices for epoch T; returns true if that completes a clean sweep while
// the instance is still quiescent at T (then the instance is finished).
__device__ __forceinline__ bool pr_record_clean(const Instance& I, unsigned T, unsigned len) {
  for (int tries = 0; tries < 1 << 20; ++tries) {
    const unsigned long long vd = ld_relaxed_u64(&I.ctl->vdone);
    const unsigned e = (unsigned)(vd >> 32);
    unsigned long long nv;
    if (e == T) nv = vd + len;
    else if ((int)(e - T) < 0) nv = ((unsigned long long)T << 32) | len;
    else return false;
    if (atomicCAS(&I.ctl->vdone, vd, nv) == vd) {
      if ((unsigned)nv < (unsigned)I.n) return false;
      const unsigned long long w = ld_relaxed_u64(&I.ctl->word);
      if (w == (((unsigned long long)T << 32) | T)) {
        atomicExch(&I.ctl->finished, 1);
        return true;
      }
      return false;
    }
  }
  return false;
}

// The Check_Size scan reads residues in groups of 4 consecutive vertices (group g = vertices
// 4g .. 4g+3): one 16-byte load per group (res rows are 16-byte aligned), and the queued bits of
// a group sit in one bitmap word, so one atomicOr claims all of its vertices at once.
__device__ __forceinline__ float4 pr_load_group(const Instance& I, unsigned g) {
  const int v = (int)(g << 2);
  if (v + 3 < I.n) return __ldcg(reinterpret_cast<const float4*>(I.res) + g);
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (v < I.n) r.x = __ldcg(I.res + v);
  if (v + 1 < I.n) r.y = __ldcg(I.res + v + 1);
  if (v + 2 < I.n) r.z = __ldcg(I.res + v + 2);
  return r;
}

// Claims the group's vertices whose residue is above eps and whose queued bit was clear; returns
// them as a 4-bit mask (bit b = vertex 4g + b).
__device__ __forceinline__ unsigned pr_claim_group(const Instance& I, unsigned g, float4 r) {
  const float e = I.eps;
  const unsigned m = (r.x > e ? 1u : 0u) | (r.y > e ? 2u : 0u) | (r.z > e ? 4u : 0u) | (r.w > e ? 8u : 0u);
  if (!m) return 0u;
  const unsigned sh = (g & 7u) * 4u;
  const unsigned old = atomicOr(I.qbits + (g >> 3), m << sh);
  return m & ~(old >> sh) & 0xfu;
}

// Appends to the CTA push buffer the vertices of each thread's claimed groups: bit 4j + b of
// `claimed` is vertex 4 grp[j] + b.  One block scan places every thread's items; the buffer is
// flushed first when they do not fit (several times if they exceed it).  Whole block.
template <int BLOCK, int G, class S>
__device__ __forceinline__ void cta_push_claimed(S& sm, unsigned claimed, const unsigned (&grp)[G], const Launch& L,
                                                 unsigned long long* st) {
  int total;
  const int off = block_exclusive_scan<BLOCK>(__popc(claimed), sm.tmp, total);  // ends with a barrier
  for (int w = 0; w < total; w += S::kPushCap) {
    const int need = min(S::kPushCap, total - w);
    if (sm.npush + need > S::kPushCap) cta_flush<BLOCK>(sm, sm.I, 0, L, st);
    const int at = sm.npush - w;
    int idx = off;
#pragma unroll
    for (int j = 0; j < G; ++j) {  // static indices: grp stays in registers
      unsigned c = (claimed >> (4 * j)) & 0xfu;
      while (c) {
        const int b = __ffs(c) - 1;
        c &= c - 1;
        if (idx >= w && idx < w + need) sm.push[at + idx] = (int)(grp[j] << 2) + b;
        ++idx;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) sm.npush += need;
    __syncthreads();
  }
}

// Threshold-crossing scatter: adds s to u's residue; true if this add lifted it from <= eps to
// above eps and claimed u's queued bit (the caller then enqueues u).
__device__ __forceinline__ bool pr_add_crossing(const Instance& I, int u, float s) {
  const float old = atomicAdd(I.res + u, s);
  if (!(old <= I.eps && old + s > I.eps)) return false;
  const unsigned bit = 1u << (u & 31);
  return !(atomicOr(I.qbits + (u >> 5), bit) & bit);
}

// Shared-memory hub accumulators of a B-thread CTA worker.  Only a hub that receives several of
// a batch's updates gains (the others cost a shared atomic and a flush instead of one red.add),
// so the slots cover the top hubs only: measured on RMAT 22, 1024 slots were best for 512-thread
// workers (9% faster than none, against 3% for 8192 slots) and 2048 for 256-thread ones.
template <int B>
struct HubSlots {
  static constexpr int value = B >= 512 ? 1024 : 8 * B;
};

template <int B>
struct PrExtra {
  float hub[HubSlots<B>::value];
};

struct PrBody {
  template <int B>
  using Extra = PrExtra<B>;
  // 1536 threads per SM (the 40-register cap spills a little below 1024-thread CTAs); 1024 at
  // 64 registers measured faster on RMAT at 256 and 512 threads but slower on the grid, and the
  // tuned RMAT configuration (1024 threads, one CTA per SM) is the same either way
  static constexpr int kResidentThreads = 1536;
  // edges per thread of a load-balancing round (RMAT 22: 4 at up to 512 threads, 2 at 1024)
  template <int B>
  static constexpr int kLbsR = B <= 512 ? 4 : 2;

  // Algorithm 4's Check_Size scan of `nchk` vertex ids (rounded up to whole groups of 4) from
  // the round-robin cursor, which counts groups.  Each thread issues its G group loads, then its
  // G claims, before using any result: two round trips per round instead of one per id.
  template <int BLOCK, class S>
  __device__ static void check_scan(S& sm, int nchk, const Launch& L, unsigned long long* st) {
    const Instance& I = sm.I;
    constexpr int G = BLOCK >= 1024 ? 4 : 2;  // smaller CTAs run under a 40-register cap
    const unsigned ngroups = ((unsigned)I.n + 3u) >> 2;
    const int ng = (nchk + 3) >> 2;
    if (threadIdx.x == 0) sm.base = atomicAdd(&I.ctl->check, (unsigned)ng);
    __syncthreads();
    const unsigned gbase = sm.base;
    for (int r = 0; r < ng; r += BLOCK * G) {
      unsigned grp[G];
      float4 v[G];
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const int k = r + j * BLOCK + (int)threadIdx.x;
        grp[j] = (gbase + (unsigned)k) % ngroups;
        v[j] = k < ng ? pr_load_group(I, grp[j]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      unsigned claimed = 0;
#pragma unroll
      for (int j = 0; j < G; ++j) claimed |= pr_claim_group(I, grp[j], v[j]) << (4 * j);
      cta_push_claimed<BLOCK, G>(sm, claimed, grp, L, st);
    }
  }

  template <int BLOCK, class S>
  __device__ static void cta_batch(S& sm, int cnt, const Launch& L, unsigned long long* st) {
    const Instance& I = sm.I;
    // hub accumulators of this batch: slot i for the hub of rank i < nhub (the space may hold
    // another body's state in a mixed launch, so it is cleared here; the scan below orders it
    // before the scatter)
    const int nhub = I.pr_crossing ? 0 : min(HubSlots<BLOCK>::value, I.hubs);
    for (int k = threadIdx.x; k < nhub; k += BLOCK) sm.x.hub[k] = 0.0f;
    int deg = 0;
    if ((int)threadIdx.x < cnt) {
      const int v = sm.items[threadIdx.x];
      atomicAnd(I.qbits + (v >> 5), ~(1u << (v & 31)));
      const float r = atomicExch(I.res + v, 0.0f);
      const int s = ldg(I.row_ptr + v), e = ldg(I.row_ptr + v + 1);
      float share = 0.0f;
      if (r != 0.0f) {
        red_add_f32(I.rank + v, r);
        if (e > s) {
          share = I.alpha * r / (float)(e - s);
          deg = e - s;
        }
      }
      sm.start[threadIdx.x] = s;
      sm.aux[threadIdx.x] = __float_as_int(share);
    }
    int total;
    const int off = block_exclusive_scan<BLOCK>(deg, sm.tmp, total);
    if ((int)threadIdx.x < cnt) sm.off[threadIdx.x] = off;
    __syncthreads();
    float* __restrict__ res = I.res;
    constexpr int R = S::kR;
    if (I.pr_crossing) {
      int rounds = 0;
      for (int base = 0; base < total; base += BLOCK * R) {
        int item[R], nb[R];
        lbs_round<BLOCK>(sm, I.col, cnt, total, base, item, nb);
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const bool want = item[j] >= 0 && pr_add_crossing(I, nb[j], __int_as_float(sm.aux[item[j]]));
          cta_push(sm, want, nb[j]);
        }
        if (base + BLOCK * R < total && flush_round<S>(rounds)) cta_maybe_flush<BLOCK>(sm, I, L, st);
      }
    } else {
      for (int base = 0; base < total; base += BLOCK * R) {
        int item[R], nb[R];
        lbs_round<BLOCK>(sm, I.col, cnt, total, base, item, nb);
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (item[j] >= 0) {
            const float share = __int_as_float(sm.aux[item[j]]);
            const uint32_t slot = I.hub.rank_of(nb[j]);
            if (slot < (uint32_t)nhub) atomicAdd(&sm.x.hub[ATOS_IX(slot, HubSlots<BLOCK>::value, sm, kSiteShared)], share);
            else red_add_f32(res + nb[j], share);
          }
      }
      if (nhub > 0) {  // one update per touched hub
        __syncthreads();
        for (int k = threadIdx.x; k < nhub; k += BLOCK) {
          const float a = sm.x.hub[k];
          if (a != 0.0f) red_add_f32(res + I.hub.id_of((uint32_t)k), a);
        }
      }
    }
    if (threadIdx.x == 0) {
      st[kStatTasks] += cnt;
      st[kStatEdges] += total;
    }
    if (!I.pr_crossing) check_scan<BLOCK>(sm, cnt * (int)I.check_size, L, st);
    __syncthreads();
    cta_flush<BLOCK>(sm, I, cnt, L, st);
  }

  template <int BLOCK, class S>
  __device__ static int cta_idle(S& sm, const Launch& L, unsigned long long* st) {
    const Instance& I = sm.I;
    constexpr int kChunk = BLOCK * 2;  // at most one push per vertex: fits the push buffer
    if (threadIdx.x == 0) {
      unsigned T = 0;
      int k = -3;
      if (ld_relaxed(&I.ctl->finished)) k = -4;
      else k = pr_claim_chunk(I, kChunk, T);
      sm.cnt = k;
      sm.base = T;
    }
    __syncthreads();
    const int k = sm.cnt;
    const unsigned T = sm.base;
    __syncthreads();
    if (k == -4) return 1;
    if (k == -1) return 0;  // the rest of the sweep is in other workers' hands
    if (k == -2) {
      if (I.pr_crossing) return 0;  // crossings enqueue everything: wait for work or quiescence
      // not quiescent: Algorithm 4's scan as the idle function
      check_scan<BLOCK>(sm, BLOCK, L, st);
      __syncthreads();
      cta_flush<BLOCK>(sm, I, 0, L, st);
      return 0;
    }
    const int v0 = k * kChunk;
    const int v1 = min(I.n, v0 + kChunk);
    bool dirty = false;
    for (int r = v0; r < v1; r += BLOCK) {
      const int u = r + threadIdx.x;
      const bool want = u < v1 && pr_sweep_vertex(I, u, &dirty);
      cta_push(sm, want, u);
    }
    const int any_dirty = __syncthreads_or(dirty);
    cta_flush<BLOCK>(sm, I, 0, L, st);
    if (any_dirty) return 0;
    if (threadIdx.x == 0) sm.cnt = pr_record_clean(I, T, (unsigned)(v1 - v0)) ? 1 : 0;
    __syncthreads();
    return sm.cnt;
  }

  // Warp worker.
  __device__ static void warp_item(WarpSmem& ws, const Instance& I, int v, const Launch& L, unsigned long long* st) {
    const int lane = threadIdx.x & 31;
    float share = 0.0f;
    int s = 0, e = 0;
    if (lane == 0) {
      atomicAnd(I.qbits + (v >> 5), ~(1u << (v & 31)));
      const float r = atomicExch(I.res + v, 0.0f);
      s = ldg(I.row_ptr + v);
      e = ldg(I.row_ptr + v + 1);
      if (r != 0.0f) {
        red_add_f32(I.rank + v, r);
        if (e > s) share = I.alpha * r / (float)(e - s);
      }
      if (share == 0.0f) e = s;
    }
    share = __shfl_sync(0xffffffffu, share, 0);
    s = __shfl_sync(0xffffffffu, s, 0);
    e = __shfl_sync(0xffffffffu, e, 0);
    if (lane == 0) st[kStatEdges] += e - s;
    if (I.pr_crossing) {
      for (int k0 = s; k0 < e; k0 += 32) {
        const int k = k0 + lane;
        int u = 0;
        bool want = false;
        if (k < e) {
          u = nbr_at(I, k, L);
          want = pr_add_crossing(I, u, share);
        }
        warp_push(ws, want, u);
        warp_maybe_flush(ws, I, L, st);
      }
      return;
    }
    for (int k = s + lane; k < e; k += 32) red_add_f32(I.res + nbr_at(I, k, L), share);
    warp_check_scan(ws, I, I.check_size, L, st);
  }

  // Thread worker (worker_size 1, Section 3.2's smallest worker): each lane runs its own task v
  // (kEmpty: none) -- takes the residue, and walks its row one entry per step, the warp stepping
  // together until every lane's row is done -- then the warp runs one Check_Size scan for all of
  // them.  A row longer than kLaneRowMax would hold the whole warp for its length, so such a task
  // is run afterwards by the warp worker's path, 32 entries per step.
  static constexpr int kLaneRowMax = 32;
  __device__ static void lane_items(WarpSmem& ws, const Instance& I, int v, const Launch& L, unsigned long long* st) {
    int k = 0, e = 0;
    float share = 0.0f;
    bool longrow = false;
    if (v != kEmpty) {
      const int s = ldg(I.row_ptr + v), end = ldg(I.row_ptr + v + 1);
      if (end - s > kLaneRowMax) {
        longrow = true;  // the whole task goes to the warp path below
      } else {
        atomicAnd(I.qbits + (v >> 5), ~(1u << (v & 31)));
        const float r = atomicExch(I.res + v, 0.0f);
        if (r != 0.0f) {
          red_add_f32(I.rank + v, r);
          if (end > s) share = I.alpha * r / (float)(end - s), k = s, e = end;
        }
      }
    }
    unsigned long long edges = (unsigned long long)(e - k);
    while (__any_sync(0xffffffffu, k < e)) {
      bool want = false;
      int u = 0;
      if (k < e) {
        u = nbr_at(I, k, L);
        if (I.pr_crossing) want = pr_add_crossing(I, u, share);
        else red_add_f32(I.res + u, share);
        ++k;
      }
      if (I.pr_crossing) {
        warp_push(ws, want, u);
        warp_maybe_flush(ws, I, L, st);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) edges += __shfl_xor_sync(0xffffffffu, edges, o);
    if ((threadIdx.x & 31) == 0) st[kStatEdges] += edges;
    const unsigned shortm = __ballot_sync(0xffffffffu, v != kEmpty && !longrow);
    if (!I.pr_crossing && shortm) warp_check_scan(ws, I, (unsigned)__popc(shortm) * I.check_size, L, st);
    for (unsigned big = __ballot_sync(0xffffffffu, longrow); big; big &= big - 1)
      warp_item(ws, I, __shfl_sync(0xffffffffu, v, __ffs(big) - 1), L, st);
  }

  // The Check_Size scan for a warp: lane k takes group k of the range (see check_scan).
  __device__ static void warp_check_scan(WarpSmem& ws, const Instance& I, unsigned nchk, const Launch& L,
                                         unsigned long long* st) {
    const int lane = threadIdx.x & 31;
    const unsigned ngroups = ((unsigned)I.n + 3u) >> 2;
    const unsigned ng = (nchk + 3u) >> 2;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&I.ctl->check, ng);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (unsigned r = 0; r < ng; r += 32) {
      const unsigned k = r + lane;
      const unsigned g = (base + k) % ngroups;
      const unsigned claimed = k < ng ? pr_claim_group(I, g, pr_load_group(I, g)) : 0u;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        warp_push(ws, (claimed >> b) & 1u, (int)(g << 2) + b);
        warp_maybe_flush(ws, I, L, st);
      }
    }
  }

  __device__ static int warp_idle(WarpSmem& ws, const Instance& I, const Launch& L, unsigned long long* st) {
    const int lane = threadIdx.x & 31;
    constexpr int kChunk = kWarpPushCap;  // at most one push per vertex: fits the push buffer
    int k = 0;
    unsigned T = 0;
    if (lane == 0) k = ld_relaxed(&I.ctl->finished) ? -4 : pr_claim_chunk(I, kChunk, T);
    k = __shfl_sync(0xffffffffu, k, 0);
    T = __shfl_sync(0xffffffffu, T, 0);
    if (k == -4) return 1;
    if (k == -1) return 0;
    if (k == -2) {
      if (I.pr_crossing) return 0;
      warp_check_scan(ws, I, 128u, L, st);
      warp_flush(ws, I, 0, L, st);
      return 0;
    }
    const int v0 = k * kChunk, v1 = min(I.n, v0 + kChunk);
    bool dirty = false;
    for (int r = v0; r < v1; r += 32) {
      const int u = r + lane;
      warp_push(ws, u < v1 && pr_sweep_vertex(I, u, &dirty), u);
    }
    const bool any_dirty = __any_sync(0xffffffffu, dirty);
    warp_flush(ws, I, 0, L, st);
    if (any_dirty) return 0;
    int done = 0;
    if (lane == 0) done = pr_record_clean(I, T, (unsigned)(v1 - v0)) ? 1 : 0;
    return __shfl_sync(0xffffffffu, done, 0);
  }
};

}  // namespace atos
