// color.cuh -- asynchronous speculative greedy colouring task body (Section 5.3, Algorithm 6).
//
// One uberkernel handles two kinds of task, told apart by the sign of the item:
//   * item v >= 0 (assign): read the colours of v's neighbours, give v the smallest colour none
//     of them holds (first fit; the colour is at most deg(v)), then push the check task ~v;
//   * item ~v < 0 (check): for every neighbour u holding v's colour, the larger of u and v must
//     recolour: push v itself (once) if some u < v, and push u for each such u > v.
// Only the larger id of a conflicting pair recolours, so the smallest id of any conflict keeps its
// colour.  A vertex has at most one assign task queued: a bitmap bit is set by whoever queues the
// assign and cleared when it is popped, before the neighbours' colours are read (a request that
// finds the bit set is covered by the pending assign, which will read the newer colours).  Pushing the larger endpoint from the smaller one's check closes the race in which the
// smaller vertex's assign read a stale colour and wrote its own after the larger vertex's last
// check.  The check task is encoded as ~v = -v - 1 so that vertex 0 has a distinct check task.
//
// Memory ordering: an assign writes its colour and then executes a sequentially consistent
// device fence; a check executes the same fence before it reads any colour.  For two adjacent
// vertices x and y this is the store-buffering pattern W(x); fence; R(y) against W(y); fence;
// R(x), so at least one of the two checks that follow their final writes sees the other's colour,
// and the conflict is found.  Colours are read from L2 (ld.global.cg).
//
// Dependency-ordered mode (ATOS_FLAG_GC_DEPENDENCY, I.gc_wait set): a vertex is coloured once,
// after all of its smaller-id neighbours, taking the smallest colour none of them holds, so the
// result is exactly serial first fit in id order, with one colouring task per vertex and no
// recolouring.  gc_wait[v] starts at 1 + (smaller neighbours of v).  The virtual initial task v
// releases the 1; a coloured vertex decrements the count of each larger neighbour; whichever
// decrement reaches zero makes the vertex ready and (for a neighbour) pushes it as ~w.  Only one
// decrement reaches zero, so each vertex is coloured exactly once.
//
// A ready vertex reads no neighbour: its smaller neighbours push their colours to it.  Every
// vertex has a bitmap of at least (smaller neighbours + 1) colour bits, and a coloured vertex sets
// its colour's bit in the bitmap of each larger neighbour just before it decrements that
// neighbour's count.  When the count reaches zero the bitmap holds the colours of all smaller
// neighbours, and its first clear bit is the first-fit colour (at most `smaller neighbours` bits
// are set, so one of the first smaller + 1 is clear).  The rows (I.col) list each vertex's
// smaller-id neighbours first (I.gc_mid[v] of them), so the countdown walks only the larger part.
// Each bit is fenced before its decrement (release), and the decrement that completes a count is
// fenced before the vertex is pushed, kept or coloured (acquire), so the bitmap a ready vertex
// reads is complete.  A dependency chain's hop is then a bitmap read and a decrement, whatever the
// row lengths.
#pragma once

#include "engine.cuh"

namespace atos {

constexpr int kGcWindow = 64;  // colours examined per pass: two 32-bit words per item
constexpr int kGcHead = 32;    // dependency order: larger neighbours counted down in a batch's first pass
constexpr int kGcSegment = 2048;  // dependency order: entries of a tail segment task
constexpr int kGcSegChunk = 64;   // dependency order: segment-table entries a CTA claims at a time

template <int B>
struct GcExtra {
  unsigned bits[2 * B];  // per item: forbidden colours [base, base + 64) (assign) or
                         // (own colour, conflict flag) (check)
};

// Pushed colours.  Each vertex's bitmap is its word gc_forbid[v] (colours 0..31) followed, for a
// vertex with 32 or more smaller neighbours, by gc_fw[v].y overflow words at gc_forbid[gc_fw[v].x]
// (colours 32 and up): (smaller neighbours + 1) bits rounded up to whole words, and most vertices
// (and most colours) need the first word only, which is found without reading gc_fw.

// Records colour c in the bitmap of the larger neighbour w.  A colour of the first word is always
// recorded; a later one only if w's bitmap reaches it (first fit for w is at most its
// smaller-neighbour count, and a set bit beyond that count never hides the first clear one, as at
// most that many bits are set).
template <class Ctx>
__device__ __forceinline__ void gc_push_colour(const Instance& I, int w, int c, Ctx& ctx) {
  if (c < 32) {
    atomicOr(I.gc_forbid + w, 1u << c);
    return;
  }
  const int2 f = __ldg(I.gc_fw + w);
  const int k = (c >> 5) - 1;
  if (k < f.y) atomicOr(I.gc_forbid + ATOS_IX(f.x + k, I.gc_forbid_words, ctx, kSiteEntry), 1u << (c & 31));
}

// The first-fit colour of a ready vertex: the first clear bit of its bitmap.
template <class Ctx>
__device__ __forceinline__ int gc_first_free(const Instance& I, int v, Ctx& ctx) {
  const unsigned b0 = __ldcg(I.gc_forbid + v);
  if (~b0) return __ffs(~b0) - 1;
  const int2 f = __ldg(I.gc_fw + v);
  for (int w = 0; w < f.y; ++w) {
    const unsigned b = __ldcg(I.gc_forbid + ATOS_IX(f.x + w, I.gc_forbid_words, ctx, kSiteEntry));
    if (~b) return 32 * (w + 1) + __ffs(~b) - 1;
  }
  return 32 * (f.y + 1);  // not reached: at most (f.y + 1) * 32 - 1 bits are set
}

// Dependency order: item v >= 0 is the release task of v (its initial count), ~v a pushed vertex.
__device__ __forceinline__ bool item_is_release(int item) { return item >= 0; }

// Queues an assign task for u unless one is already queued.
__device__ __forceinline__ bool gc_claim_assign(const Instance& I, int u) {
  const unsigned bit = 1u << (u & 31);
  return !(atomicOr(I.qbits + (u >> 5), bit) & bit);
}

struct GcBody {
  template <int B>
  using Extra = GcExtra<B>;
  // 768 threads per SM leave ~80 registers: the colouring bodies keep their bitmap, countdown and
  // push state in registers instead of spilling (RMAT 22, 128-thread CTAs: 34 -> 29 ms in
  // dependency order, 13 -> 9 ms for Algorithm 6 on the spread layout)
  static constexpr int kResidentThreads = 768;
  // edges per thread of a load-balancing round (RMAT 22, dependency order: 2 beats 4 at 128-256
  // threads)
  template <int B>
  static constexpr int kLbsR = B <= 512 ? 2 : 1;

  // Dependency-ordered mode: item v >= 0 releases the initial count of v, item ~v is a vertex
  // made ready by its last smaller neighbour, an item below -n a tail segment.  A ready vertex
  // takes the first clear bit of its colour bitmap (its smaller neighbours' colours, pushed by
  // them), then counts down its larger neighbours (the row after its first gc_mid[v] entries):
  // each gets the colour's bit, then a decrement.  A vertex made ready is published as soon as
  // the round that made it ready ends, not at the end of the batch: a hub's row is long, and the
  // next vertex on the longest dependency path is often among the first it releases.
  //
  // Local continuation: the vertices the last countdown round made ready (up to FETCH_SIZE of
  // them) are not published but run by this CTA as its next batch, which takes the queue's
  // push-pop round trip off a dependency chain's hops; the rest are published.  While a CTA holds
  // such local work it leaves one task of the batch it popped unreported, so the instance cannot
  // look finished (completed = pushed) before the local work, and whatever it releases, is done.
  template <int BLOCK, class S>
  __device__ static void cta_batch_dependency(S& sm, int cnt, const Launch& L, unsigned long long* st) {
    const int keep_max = min(L.fetch, BLOCK);
    int from_queue = cnt;
    bool open = false;
    for (;;) {
      const int keep = cta_dependency_round<BLOCK>(sm, cnt, keep_max, L, st);
      int done = from_queue;
      if (keep && !open) done -= 1, open = true;  // from_queue >= 1 here: the first batch was popped
      else if (!keep && open) done += 1, open = false;
      const int item = (int)threadIdx.x < keep ? sm.push[threadIdx.x] : 0;
      cta_flush<BLOCK>(sm, sm.I, done, L, st, keep);  // publishes the rest
      if (!keep) return;
      if ((int)threadIdx.x < keep) sm.items[threadIdx.x] = item;
      __syncthreads();
      cnt = keep;
      from_queue = 0;
    }
  }

  // One batch of the dependency-ordered mode; returns how many of the vertices it made ready (the
  // first entries of the push buffer, which the caller publishes from there on) it keeps for local
  // continuation.
  //
  // The countdown runs in two passes.  The first covers the first kGcHead larger neighbours of
  // every ready vertex of the batch: the next vertex of a dependency chain is nearly always among a
  // vertex's first larger neighbours, so it is released in the first round whatever the other
  // rows hold.  The rest of the rows (the tails) follow in a second pass, together with the tail
  // segments in the batch; a tail longer than kGcSegment entries is cut into segment tasks
  // instead (table I.segs, item -(n + 1 + entry)), which idle CTAs count down in parallel, so a
  // hub's long row does not hold one CTA for its whole length.
  template <int BLOCK, class S>
  __device__ static int cta_dependency_round(S& sm, int cnt, int keep_max, const Launch& L, unsigned long long* st) {
    const Instance& I = sm.I;
    const int t = threadIdx.x;
    int item = 0, v = 0, head = 0, start = 0, tail = 0, colour = -1;
    bool ready = false, segment = false;
    if (t < cnt) {
      item = sm.items[t];
      segment = item < -I.n;
      if (segment) {  // a tail segment: entries [y, y + z) of x's row, x coloured w
        const int4 e = __ldcg(I.segs + ATOS_IX(-(item + I.n + 1), I.seg_cap, sm, kSiteItem));
        v = e.x, start = e.y, tail = e.z, colour = e.w;
      } else {
        v = item >= 0 ? item : ~item;
        ready = item < 0 || atomicSub(I.gc_wait + v, 1) == 1;
        const int s = ldg(I.row_ptr + v);
        if (ready) {
          const int lower = ldg(I.gc_mid + v);
          const int upper = ldg(I.row_ptr + v + 1) - s - lower;
          if (item_is_release(item) && lower > 0) __threadfence();  // the count's other decrements (and bits) come first
          colour = gc_first_free(I, v, sm);
          st_relaxed(I.color + v, colour);  // read after the run only: the neighbours get it by their bitmaps
          head = min(upper, kGcHead);
          start = s + lower;
          tail = upper - head;
        }
      }
      sm.aux[t] = colour;
    }
    // with tails to come, the first pass publishes everything it releases at once (other CTAs go on
    // with those vertices while this one walks the tails); otherwise its last round's are kept
    const bool more = __syncthreads_or(tail > 0);
    int total = countdown_pass<BLOCK>(sm, cnt, head, start, more, L, st);
    if (more) {
      // tails longer than a segment go to other CTAs as segments; the others follow inline
      const bool long_tail = ready && tail > kGcSegment;
      if (I.segs && __syncthreads_or(long_tail) &&
          split_tails<BLOCK>(sm, v, start + head, long_tail ? tail : 0, colour, sm.npush)) {
        if (long_tail) tail = 0;
        cta_flush<BLOCK>(sm, I, 0, L, st);  // the segments go out before the inline pass
      }
      total += countdown_pass<BLOCK>(sm, cnt, tail, ready ? start + head : start, false, L, st);
    }
    __syncthreads();
    const int front = sm.npush;  // the last round's vertices
    __syncthreads();
    if (t == 0) {
      st[kStatTasks] += cnt;
      st[kStatEdges] += total;
      // a failed launch stops here (the caller publishes, and nothing is kept)
      sm.keep = ld_relaxed(L.status) != 0 ? 0 : min(front, keep_max);
    }
    __syncthreads();
    return sm.keep;
  }

  // Appends to the push buffer, after its first `released` entries, the tail of a ready vertex
  // (entries [start, start + tail) of v's row, v coloured `colour`) as segments of up to kGcSegment
  // entries.  Table entries are claimed kGcSegChunk at a time per CTA.  Returns false (nothing
  // appended) when the table or the push buffer has no room.  Whole block.
  template <int BLOCK, class S>
  __device__ static bool split_tails(S& sm, int v, int start, int tail, int colour, int released) {
    const Instance& I = sm.I;
    const int parts = tail > 0 ? (tail + kGcSegment - 1) / kGcSegment : 0;
    int nseg;
    const int off = block_exclusive_scan<BLOCK>(parts, sm.tmp, nseg);  // ends with a barrier
    if (threadIdx.x == 0) {
      unsigned j0 = 0xffffffffu;
      if (released + nseg <= S::kPushCap) {
        if (sm.seg_hi - sm.seg_lo < (unsigned)nseg) {  // claim a new chunk (the rest of the old one is lost)
          const unsigned want = max((unsigned)nseg, (unsigned)kGcSegChunk);
          sm.seg_lo = atomicAdd(&I.ctl->seg_next, want);
          sm.seg_hi = sm.seg_lo + want;
        }
        if (sm.seg_hi <= I.seg_cap && sm.seg_lo <= sm.seg_hi) {
          j0 = sm.seg_lo;
          sm.seg_lo += (unsigned)nseg;
        } else {
          sm.seg_lo = sm.seg_hi = 0;
        }
      }
      sm.base = j0;
    }
    __syncthreads();
    const unsigned j0 = sm.base;
    if (j0 == 0xffffffffu) return false;  // uniform
    for (int k = 0; k < parts; ++k) {
      const int j = (int)j0 + off + k;
      const int first = k * kGcSegment;
      I.segs[j] = make_int4(v, start + first, min(kGcSegment, tail - first), colour);
      sm.push[ATOS_IX(released + off + k, S::kPushCap, sm, kSitePushBuffer)] = -(I.n + 1 + j);
    }
    __syncthreads();
    if (threadIdx.x == 0) sm.npush = released + nseg;
    __syncthreads();
    return true;
  }

  // One countdown pass over entries [start, start + count) of each batch item's row (the
  // neighbours' colour bits, then their counts).  Vertices made ready are published after every
  // round but the last, and after the last too if flush_last (else they stay in the push buffer
  // for the caller to keep or publish).  Returns the entries counted down.
  template <int BLOCK, class S>
  __device__ static int countdown_pass(S& sm, int cnt, int count, int start, bool flush_last, const Launch& L,
                                       unsigned long long* st) {
    const Instance& I = sm.I;
    const int t = threadIdx.x;
    constexpr int R = S::kR;
    int total;
    const int off = block_exclusive_scan<BLOCK>(count, sm.tmp, total);  // ends with a barrier
    if (t < cnt) {
      sm.off[t] = off;
      sm.start[t] = start;
    }
    __syncthreads();
    for (int r = 0; r < total; r += BLOCK * R) {
      int owner[R], nb[R];
      lbs_round<BLOCK>(sm, I.col, cnt, total, r, owner, nb);
      if (owner[0] >= 0) {  // a thread's entries are consecutive: none if the first is past the end
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (owner[j] >= 0) gc_push_colour(I, nb[j], sm.aux[owner[j]], sm);
        __threadfence();  // the colour bits are visible before the decrements
      }
      bool made_ready = false;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const bool go = owner[j] >= 0 && atomicSub(I.gc_wait + nb[j], 1) == 1;
        made_ready |= go;
        cta_push(sm, go, ~nb[j]);
      }
      if (made_ready) __threadfence();  // the count's other decrements (and their writes) come first
      __syncthreads();
      if (sm.npush > 0 && (flush_last || r + BLOCK * R < total)) cta_flush<BLOCK>(sm, I, 0, L, st);
    }
    return total;
  }

  template <int BLOCK, class S>
  __device__ static void cta_batch(S& sm, int cnt, const Launch& L, unsigned long long* st) {
    if (sm.I.gc_wait) {
      cta_batch_dependency<BLOCK>(sm, cnt, L, st);
      return;
    }
    const Instance& I = sm.I;
    const int t = threadIdx.x;
    int v = 0, deg = 0, s = 0;
    bool assign = false;
    if (t < cnt) {
      const int item = sm.items[t];
      assign = item >= 0;
      v = assign ? item : ~item;
      s = ldg(I.row_ptr + v);
      deg = ldg(I.row_ptr + v + 1) - s;
      sm.start[t] = s;
      sm.aux[t] = item;
      if (assign) {
        atomicAnd(I.qbits + (v >> 5), ~(1u << (v & 31)));  // requests from now on queue a new assign
        sm.x.bits[2 * t] = 0u;
        sm.x.bits[2 * t + 1] = 0u;
      } else {
        sm.x.bits[2 * t] = (unsigned)__ldcg(I.color + v);
        sm.x.bits[2 * t + 1] = 0u;
      }
    }
    __threadfence();  // order every earlier colour write of this CTA before the checks' reads
    __syncthreads();
    int64_t edges = 0;
    int colour = -1;  // result of an assign item (thread t)
    // pass 0 runs every item; later passes only assign items that found no free colour in the
    // window [base, base + 64).
    bool active = t < cnt;
    for (int base = 0;; base += kGcWindow) {
      const int mydeg = active ? deg : 0;
      int total;
      const int off = block_exclusive_scan<BLOCK>(mydeg, sm.tmp, total);
      // inactive items have degree 0 here, so the offsets stay non-decreasing and the owner
      // search never lands on them
      if (t < cnt) sm.off[t] = off;
      if (total == 0 && base > 0) break;
      __syncthreads();
      constexpr int R = S::kR;
      int rounds = 0;
      for (int r = 0; r < total; r += BLOCK * R) {
        int owner[R], nb[R], c[R];
        lbs_round<BLOCK>(sm, I.col, cnt, total, r, owner, nb);
#pragma unroll
        for (int j = 0; j < R; ++j) c[j] = owner[j] >= 0 ? __ldcg(I.color + nb[j]) : 0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
          bool push_nb = false;
          const int i = owner[j];
          if (i >= 0) {
            const int item = sm.aux[i];
            if (item >= 0) {
              const int rel = c[j] - base;
              if (rel >= 0 && rel < kGcWindow && (!I.gc_ordered || nb[j] < item))
                atomicOr(&sm.x.bits[2 * i + (rel >> 5)], 1u << (rel & 31));
            } else if (c[j] == (int)sm.x.bits[2 * i] && nb[j] != ~item) {
              if (nb[j] < ~item) sm.x.bits[2 * i + 1] = 1u;   // v is the larger: v recolours
              else push_nb = gc_claim_assign(I, nb[j]);       // the neighbour is the larger
            }
          }
          cta_push(sm, push_nb, nb[j]);
        }
        if (r + BLOCK * R < total && flush_round<S>(rounds)) cta_maybe_flush<BLOCK>(sm, I, L, st);
      }
      cta_maybe_flush<BLOCK>(sm, I, L, st);
      edges += total;
      __syncthreads();
      bool again = false;
      if (active && assign) {
        const unsigned lo = sm.x.bits[2 * t], hi = sm.x.bits[2 * t + 1];
        const unsigned long long used = ((unsigned long long)hi << 32) | lo;
        if (~used) {
          colour = base + __ffsll((long long)~used) - 1;
        } else {
          again = true;
          sm.x.bits[2 * t] = 0u;
          sm.x.bits[2 * t + 1] = 0u;
        }
      }
      active = again;
      if (!__syncthreads_or(again)) break;
    }
    // results: write colours, then push check tasks / recolourings
    bool want = false;
    int push_item = 0;
    if (t < cnt) {
      if (assign) {
        st_relaxed(I.color + v, colour);
        __threadfence();  // the colour is visible before the check task can be taken
        want = true;
        push_item = ~v;
      } else if (sm.x.bits[2 * t + 1] && gc_claim_assign(I, v)) {
        want = true;
        push_item = v;
      }
    }
    cta_push(sm, want, push_item);
    __syncthreads();
    if (t == 0) {
      st[kStatTasks] += cnt;
      st[kStatEdges] += edges;
    }
    cta_flush<BLOCK>(sm, I, cnt, L, st);
  }

  template <int BLOCK, class S>
  __device__ static int cta_idle(S& sm, const Launch&, unsigned long long*) {
    return threadIdx.x == 0 ? (instance_quiescent(sm.I) ? 1 : 0) : 0;
  }

  // Dependency-ordered mode for a warp worker (see cta_batch_dependency).
  __device__ static void warp_item_dependency(WarpSmem& ws, const Instance& I, int item, const Launch& L,
                                              unsigned long long* st) {
    const int lane = threadIdx.x & 31;
    const int v = item >= 0 ? item : ~item;
    int ready = 0;
    if (lane == 0) ready = item < 0 || atomicSub(I.gc_wait + v, 1) == 1;
    if (!__shfl_sync(0xffffffffu, ready, 0)) return;
    const int s = ldg(I.row_ptr + v), e = ldg(I.row_ptr + v + 1);
    const int m = s + ldg(I.gc_mid + v);  // [s, m): smaller neighbours, [m, e): larger ones
    int colour = 0;
    if (lane == 0) {
      if (item_is_release(item) && m > s) __threadfence();  // the count's other decrements (and bits) come first
      colour = gc_first_free(I, v, L);
      st_relaxed(I.color + v, colour);  // read after the run only
    }
    colour = __shfl_sync(0xffffffffu, colour, 0);
    __syncwarp();
    for (int k0 = m; k0 < e; k0 += 32) {
      const int k = k0 + lane;
      int w = 0;
      bool go = false;
      if (k < e) {
        w = nbr_at(I, k, L);
        gc_push_colour(I, w, colour, L);
        __threadfence();  // the colour bit is visible before the decrement
        go = atomicSub(I.gc_wait + w, 1) == 1;
        if (go) __threadfence();  // the count's other decrements (and their writes) come first
      }
      warp_push(ws, go, ~w);
      if (ws.npush > 0) warp_flush(ws, I, 0, L, st);  // publish a ready vertex right away
    }
    if (lane == 0) st[kStatEdges] += e - m;
  }

  __device__ static void warp_item(WarpSmem& ws, const Instance& I, int item, const Launch& L,
                                   unsigned long long* st) {
    if (I.gc_wait) {
      warp_item_dependency(ws, I, item, L, st);
      return;
    }
    const int lane = threadIdx.x & 31;
    const bool assign = item >= 0;
    const int v = assign ? item : ~item;
    const int s = ldg(I.row_ptr + v), e = ldg(I.row_ptr + v + 1);
    int64_t edges = 0;
    if (assign) {
      if (lane == 0) atomicAnd(I.qbits + (v >> 5), ~(1u << (v & 31)));
      __syncwarp();
      int colour = -1;
      for (int base = 0; colour < 0; base += kGcWindow) {
        unsigned lo = 0, hi = 0;
        for (int k = s + lane; k < e; k += 32) {
          const int u = nbr_at(I, k, L);
          if (I.gc_ordered && u > v) continue;
          const int rel = __ldcg(I.color + u) - base;
          if (rel >= 0 && rel < 32) lo |= 1u << rel;
          else if (rel >= 32 && rel < 64) hi |= 1u << (rel - 32);
        }
        edges += e - s;
        lo = __reduce_or_sync(0xffffffffu, lo);
        hi = __reduce_or_sync(0xffffffffu, hi);
        const unsigned long long used = ((unsigned long long)hi << 32) | lo;
        if (~used) colour = base + __ffsll((long long)~used) - 1;
      }
      if (lane == 0) {
        st_relaxed(I.color + v, colour);
        __threadfence();  // the colour is visible before the check task can be taken
      }
      __syncwarp();
      warp_push(ws, lane == 0, ~v);
    } else {
      __threadfence();  // store-buffering pattern with the assign's fence (see the file comment)
      int cv = 0;
      if (lane == 0) cv = __ldcg(I.color + v);
      cv = __shfl_sync(0xffffffffu, cv, 0);
      bool conflict = false;
      for (int k = s; k < e; k += 32) {
        const int j = k + lane;
        bool larger = false;
        int nb = 0;
        if (j < e) {
          nb = nbr_at(I, j, L);
          if (nb != v && __ldcg(I.color + nb) == cv) {
            if (nb < v) conflict = true;
            else larger = gc_claim_assign(I, nb);
          }
        }
        warp_push(ws, larger, nb);  // the larger neighbour recolours
        warp_maybe_flush(ws, I, L, st);
      }
      edges += e - s;
      conflict = __any_sync(0xffffffffu, conflict);
      warp_push(ws, lane == 0 && conflict && gc_claim_assign(I, v), v);
    }
    warp_maybe_flush(ws, I, L, st);
    if (lane == 0) st[kStatEdges] += edges;
  }

  // Thread worker (worker_size 1, Section 3.2's smallest worker): each lane runs its own task
  // (kEmpty: none), walking its row one entry per step with the warp stepping together; tasks
  // whose rows are longer than kLaneRowMax are run afterwards by the warp worker's path.
  static constexpr int kLaneRowMax = 32;
  __device__ static void lane_items(WarpSmem& ws, const Instance& I, int item, const Launch& L,
                                    unsigned long long* st) {
    bool have = item != kEmpty;
    const int v = !have ? 0 : (item >= 0 ? item : ~item);
    int s = 0, e = 0;
    bool longrow = false;
    if (have) {
      s = ldg(I.row_ptr + v), e = ldg(I.row_ptr + v + 1);
      longrow = e - s > kLaneRowMax;
      have = !longrow;
    }
    if (I.gc_wait) lane_dependency(ws, I, item, have, v, s, e, L, st);
    else lane_speculative(ws, I, item, have, v, s, e, L, st);
    for (unsigned big = __ballot_sync(0xffffffffu, longrow); big; big &= big - 1)
      warp_item(ws, I, __shfl_sync(0xffffffffu, item, __ffs(big) - 1), L, st);
  }

  // Algorithm 6 per lane: an assign task takes the first colour free among its neighbours'
  // (windows of 64 colours, the row walked again for each), writes it and pushes its check task;
  // a check task pushes the larger endpoint of each conflict (itself once if a smaller neighbour
  // shares its colour).
  __device__ static void lane_speculative(WarpSmem& ws, const Instance& I, int item, bool have, int v, int s, int e,
                                          const Launch& L, unsigned long long* st) {
    const bool assign = have && item >= 0;
    const bool check = have && item < 0;
    if (assign) atomicAnd(I.qbits + (v >> 5), ~(1u << (v & 31)));  // later requests queue a new assign
    if (__any_sync(0xffffffffu, check)) __threadfence();  // store-buffering pattern (see the file comment)
    unsigned long long edges = 0;
    int colour = -1;
    for (int base = 0; __any_sync(0xffffffffu, assign && colour < 0); base += kGcWindow) {
      const bool active = assign && colour < 0;
      unsigned long long used = 0;
      int k = active ? s : e;
      while (__any_sync(0xffffffffu, k < e)) {
        if (k < e) {
          const int u = nbr_at(I, k, L);
          if (!I.gc_ordered || u < v) {
            const int rel = __ldcg(I.color + u) - base;
            if (rel >= 0 && rel < kGcWindow) used |= 1ull << rel;
          }
          ++k;
        }
      }
      if (active) {
        edges += (unsigned long long)(e - s);
        if (~used) colour = base + __ffsll((long long)~used) - 1;
      }
    }
    if (assign) {
      st_relaxed(I.color + v, colour);
      __threadfence();  // the colour is visible before the check task can be taken
    }
    warp_push(ws, assign, ~v);
    // check tasks
    const int cv = check ? __ldcg(I.color + v) : 0;
    bool conflict = false;
    int k = check ? s : e;
    if (check) edges += (unsigned long long)(e - s);
    while (__any_sync(0xffffffffu, k < e)) {
      bool larger = false;
      int u = 0;
      if (k < e) {
        u = nbr_at(I, k, L);
        if (u != v && __ldcg(I.color + u) == cv) {
          if (u < v) conflict = true;
          else larger = gc_claim_assign(I, u);
        }
        ++k;
      }
      warp_push(ws, larger, u);  // the larger neighbour recolours
      warp_maybe_flush(ws, I, L, st);
    }
    warp_push(ws, check && conflict && gc_claim_assign(I, v), v);
    warp_maybe_flush(ws, I, L, st);
#pragma unroll
    for (int o = 16; o; o >>= 1) edges += __shfl_xor_sync(0xffffffffu, edges, o);
    if ((threadIdx.x & 31) == 0) st[kStatEdges] += edges;
  }

  // Dependency-ordered mode per lane (see cta_batch_dependency).
  __device__ static void lane_dependency(WarpSmem& ws, const Instance& I, int item, bool have, int v, int s, int e,
                                         const Launch& L, unsigned long long* st) {
    const bool ready = have && (item < 0 || atomicSub(I.gc_wait + v, 1) == 1);
    const int m = ready ? s + ldg(I.gc_mid + v) : s;  // [s, m): smaller neighbours, [m, e): larger
    unsigned long long edges = 0;
    int colour = -1;
    if (ready) {
      if (item_is_release(item) && m > s) __threadfence();  // the count's other decrements (and bits) come first
      colour = gc_first_free(I, v, L);
      st_relaxed(I.color + v, colour);
      __threadfence();  // not needed for the result; thread workers measured faster with it (RMAT 22)
      edges += (unsigned long long)(e - m);
    }
    int k = ready ? m : e;
    while (__any_sync(0xffffffffu, k < e)) {
      bool go = false;
      int w = 0;
      if (k < e) {
        w = nbr_at(I, k, L);
        gc_push_colour(I, w, colour, L);
        __threadfence();  // the colour bit is visible before the decrement
        go = atomicSub(I.gc_wait + w, 1) == 1;
        if (go) __threadfence();  // the count's other decrements (and their writes) come first
        ++k;
      }
      warp_push(ws, go, ~w);
      if (ws.npush > 0) warp_flush(ws, I, 0, L, st);  // publish a ready vertex right away
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) edges += __shfl_xor_sync(0xffffffffu, edges, o);
    if ((threadIdx.x & 31) == 0) st[kStatEdges] += edges;
  }

  __device__ static int warp_idle(WarpSmem&, const Instance& I, const Launch&, unsigned long long*) {
    return (threadIdx.x & 31) == 0 ? (instance_quiescent(I) ? 1 : 0) : 0;
  }
};

}  // namespace atos
