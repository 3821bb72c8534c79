// engine.cuh -- device worklist and worker engines of the task-parallel scheduler.
//
// The scheduling model is the one of Section 3 of the Atos paper: workers repeatedly pop a task
// from one shared queue, run the application function on it and push the tasks it creates
// (Listing 2), in a persistent kernel or in one discrete launch per queue generation
// (Section 3.4), with warp- or CTA-sized workers (Section 3.2) that fetch FETCH_SIZE items per
// pop (Section 4).  The queue itself is not specified by the paper; this is the GB300 design:
//
//   * one power-of-two ring per instance; a slot holds (ticket << 32 | item), all ones when free.
//     The ticket tag makes a slot match only the exact ticket that wrote it, so pops may reserve
//     tickets arbitrarily far ahead of the tail without ever reading a previous lap's item;
//   * a packed 64-bit control word: high half = tasks pushed (tail), low half = tasks completed.
//     A worker reserves its pushes and reports its finished tasks with ONE atomicAdd per batch,
//     and the instance has terminated exactly when the two halves are equal (nothing queued,
//     nothing running), which needs no barrier and no extra counter;
//   * pops reserve a range of ticket numbers with one atomicAdd on `head` and then wait (with a
//     bounded spin) for each reserved slot to be filled, so a pop never retries a CAS;
//   * the first `prefix_len` items are virtual (the BFS source, or every vertex for PageRank and
//     colouring) and are never written to memory;
//   * every wait is bounded by a wall-clock budget read from %globaltimer; on expiry the kernel
//     sets ATOS_ERR_TIMEOUT in the launch status word and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "atos.h"

namespace atos {

constexpr int32_t kEmpty = INT32_MIN;             // "no item" as returned by take_ticket
constexpr unsigned long long kFreeSlot = ~0ull;  // a free ring slot (tag 0xffffffff is no ticket)
constexpr int32_t kUnreached = INT32_MAX;

enum : int32_t { kAppBfs = 0, kAppPr = 1, kAppGc = 2 };

// Most hubs of the spread-id copy (the highest-degree vertices; PageRank CTAs combine their
// batch's updates to them in shared memory).
constexpr int kHubRegion = 16384;

// Where the hubs of the spread-id copy sit: the hub of rank i has the id 32 line(i), the first
// entry of a 128-byte line of every 4-byte state array, with line(i) = (mul i + add) mod 2^k
// (mask = 2^k - 1, mul odd, inv = mul^-1 mod 2^32), so the hubs are spread over the first 2^k
// lines and the rank of a line's hub is one multiplication away.
struct HubMap {
  uint32_t mask, mul, inv, add;
  __host__ __device__ __forceinline__ int32_t id_of(uint32_t i) const { return (int32_t)(((mul * i + add) & mask) << 5); }
  // Rank of the hub at id u, or a value >= 2^k (never a valid rank of fewer hubs) when no hub
  // could sit at u.
  __device__ __forceinline__ uint32_t rank_of(int32_t u) const {
    const uint32_t l = (uint32_t)u >> 5;
    if ((u & 31) || l > mask) return 0xffffffffu;
    return (inv * (l - add)) & mask;
  }
};

enum : int32_t { kStatTasks = 0, kStatEdges = 1, kStatPushes = 2, kStatIdle = 3, kStatBatches = 4, kNumStats = 5 };

// Per-instance queue control block; each hot counter sits on its own 128-byte line.
struct alignas(128) QueueCtl {
  unsigned long long word;  // [63:32] tasks pushed (tail), [31:0] tasks completed
  char pad0[120];
  unsigned int head;  // pop tickets handed out
  char pad1[124];
  unsigned int check;  // PageRank: Check_Size cursor (Algorithm 4)
  char pad2[124];
  unsigned long long vword;  // PageRank final sweep: [63:32] epoch (tail at quiescence), [31:0] next chunk
  unsigned long long vdone;  // [63:32] epoch, [31:0] vertices found clean in that epoch
  int finished;              // set once the instance has terminated
  int succ;                  // batched launch: instance that takes over this one's workers
  unsigned int gen_begin;    // discrete strategy: current generation [gen_begin, gen_end)
  unsigned int gen_end;
  unsigned int orphan_count[2];  // serving: pop tickets left pending by paused workers, per epoch parity
  unsigned int orphan_head;      // serving: orphans of the previous epoch handed out so far
  unsigned int seg_next;         // BFS row splitting: segment-table entries handed out
  char pad3[80];
};
static_assert(sizeof(QueueCtl) == 512, "QueueCtl layout");

// Everything a worker needs to run one instance (one BFS source, one PageRank, one colouring).
struct Instance {
  const int32_t* row_ptr;
  const int32_t* col;
  int32_t n;
  int32_t app;
  unsigned long long* ring;  // slots: (ticket << 32) | item, kFreeSlot when free
  uint32_t cap;          // ring slots (power of two)
  uint32_t prefix_len;   // items [0, prefix_len) are virtual
  int32_t prefix_item;   // >= 0: the single virtual item; < 0: virtual item i is vertex i
  int32_t hubs;          // PageRank on the spread-id copy: hubs of rank < hubs sit where `hub` says
  QueueCtl* ctl;
  int32_t* depth;        // BFS
  float* rank;           // PageRank
  float* res;
  uint32_t* qbits;       // PageRank: one bit per vertex, set while the vertex is queued
  float alpha;
  float eps;
  uint32_t check_size;
  int32_t pr_crossing;   // PageRank: 1 = threshold-crossing enqueue instead of the Check_Size scan
  int32_t* color;        // colouring
  unsigned long long* stats;  // kNumStats counters
  unsigned* orphans[2];  // serving: pending tickets recorded at a pause, by epoch parity
  uint32_t orphan_cap;
  int32_t gc_ordered;    // colouring: 1 = an assign avoids only the colours of smaller-id neighbours
  int32_t* gc_wait;      // colouring in dependency order: 1 + smaller-id neighbours not coloured yet
  const int32_t* gc_mid; // colouring in dependency order: smaller-id neighbours of each vertex, which
                         // `col` lists first in its row (the larger ones follow)
  const int2* gc_fw;     // colouring in dependency order: per vertex, (first word, words) of the
                         // overflow part of its bitmap (colours 32 and up) in gc_forbid
  unsigned* gc_forbid;   // the bitmaps: word v holds vertex v's colours 0..31, the overflow words
                         // follow; bit c set = a coloured smaller neighbour holds colour c
  uint32_t gc_forbid_words;  // words of gc_forbid
  double* cert_y;        // PageRank in batches and serving: FP64 scratch (n) of the output certificate
  int32_t* expanded;     // BFS (optional): the smallest depth at which each vertex has been expanded
  int4* segs;            // segment tasks (optional): BFS row splitting (vertex, first entry, depth, -);
                         // dependency-ordered colouring (vertex, first entry, entries, colour)
  uint32_t seg_cap;      // entries of segs
  double exact_sum;      // PageRank: n - alpha * (isolated vertices), the fixed point's sum
  HubMap hub;            // PageRank on the spread-id copy: the hubs' ids
};

struct Launch {
  Instance* insts;
  int32_t ninst;
  int32_t window;      // instances active at once (batched)
  int32_t fetch;       // FETCH_SIZE
  int32_t policy;      // ATOS_FETCH_*
  int32_t nworkers;    // workers in the grid (for ATOS_FETCH_SPREAD)
  uint32_t flags;
  int* status;         // first error of the launch (0 = OK)
  unsigned int* next_inst;
  long long spin_limit_ns;  // budget of any single wait
  long long lifetime_ns;    // budget of a worker's whole run (bounds livelock as well as waits)
  int* fail_site;           // which wait gave up first (diagnostics)
  long long slice_ns;       // serving: a worker pauses at its next safe point after this long (0 = never)
  unsigned epoch;           // serving: epoch number (its parity selects the orphan buffers)
  // throughput timeline (optional): per bucket of bucket_ns after *t_origin, tasks and neighbour
  // entries of the batches that ended in it (timeline[2 b], timeline[2 b + 1])
  unsigned long long* timeline;
  const unsigned long long* t_origin;
  long long bucket_ns;
  int32_t nbuckets;
};

// ------------------------------------------------------------------------------------ PTX

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ float ld_relaxed_f32(const float* p) {
  float v;
  asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// Fire-and-forget float add at L2 (no value returned, so the thread does not wait for it).
__device__ __forceinline__ void red_add_f32(float* p, float v) {
  asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
// Read-only CSR data: non-coherent cached loads.
__device__ __forceinline__ int ldg(const int32_t* p) { return __ldg(p); }

__device__ __forceinline__ void raise_status(int* status, int code) { atomicCAS(status, 0, code); }

// Sites of the bounded waits, recorded with the first timeout of a launch.
enum : int { kSiteSlotEmpty = 1, kSiteCtaIdle = 2, kSiteWarpIdle = 3, kSiteSuccessor = 4, kSiteLifetime = 5 };

// ------------------------------------------------------------------------------ wait budget

struct Waiter {
  unsigned long long start = 0;
  unsigned sleep_ns = 0;
  // Returns false once the wait has exceeded `limit` nanoseconds.
  __device__ __forceinline__ bool step(long long limit) {
    unsigned long long now = globaltimer();
    if (start == 0) start = now;
    if ((long long)(now - start) > limit) return false;
    if (sleep_ns) __nanosleep(sleep_ns);
    sleep_ns = sleep_ns ? min(sleep_ns * 2, 512u) : 32u;
    return true;
  }
  __device__ __forceinline__ void reset() { start = 0, sleep_ns = 0; }
};

__device__ __forceinline__ void raise_timeout(const Launch& L, int site) {
  if (atomicCAS(L.status, 0, ATOS_ERR_TIMEOUT) == 0 && L.fail_site) atomicExch(L.fail_site, site);
}

// ----------------------------------------------------------------- bounds-checked build
//
// Compiled with ATOS_CHECKED, the worker engines and task bodies check every popped item, every
// CSR entry index and neighbour id read from the CSR, and every push-buffer and shared-bitmap
// slot before use.  A violation records ATOS_ERR_BOUNDS in the launch status (the first one's
// site in fail_site) and the access goes to index 0 instead, so nothing outside the arrays is
// touched; the status stops the launch at its next check.  Ring slots need no check: their index
// is masked by the power-of-two capacity.  Without the macro every check compiles to nothing.
enum : int {
  kSiteItem = 101,        // a popped item outside the instance's vertices
  kSiteEntry = 102,       // a CSR entry index outside [0, nnz)
  kSiteNeighbour = 103,   // a neighbour id outside [0, n)
  kSitePushBuffer = 104,  // a CTA push-buffer slot
  kSiteWarpPush = 105,    // a warp push-buffer slot
  kSiteShared = 106,      // a shared-memory bitmap or accumulator slot
  kSiteFrontier = 107,    // a BSP frontier slot
  kSiteChunk = 108        // a BSP edge-chunk slot
};

#ifdef ATOS_CHECKED
static __device__ __noinline__ void record_bounds(int* status, int* fail_site, int site) {
  if (atomicCAS(status, 0, ATOS_ERR_BOUNDS) == 0 && fail_site) atomicExch(fail_site, site);
}
template <class T>
__device__ __forceinline__ T checked_ix(T i, long long limit, int* status, int* fail_site, int site) {
  if ((long long)i < 0 || (long long)i >= limit) {
    record_bounds(status, fail_site, site);
    return T(0);
  }
  return i;
}
// i if 0 <= i < limit; else the violation is recorded through `ctx` (anything with status and
// fail_site pointers: the Launch, a worker's shared state) and the result is 0
#define ATOS_IX(i, limit, ctx, site) ::atos::checked_ix((i), (long long)(limit), (ctx).status, (ctx).fail_site, (site))
#else
#define ATOS_IX(i, limit, ctx, site) (i)
#endif

// col[k] of an instance's CSR (the entry index and the neighbour id checked in checked builds).
__device__ __forceinline__ int nbr_at(const Instance& I, int k, const Launch& L) {
#ifdef ATOS_CHECKED
  const int nnz = ldg(I.row_ptr + I.n);
  return ATOS_IX(ldg(I.col + ATOS_IX(k, nnz, L, kSiteEntry)), I.n, L, kSiteNeighbour);
#else
  (void)L;
  return ldg(I.col + k);
#endif
}

// A popped item: a vertex of the instance, or (colouring) the check task ~v of one.
__device__ __forceinline__ int checked_item(const Instance& I, int item, const Launch& L) {
#ifdef ATOS_CHECKED
  const bool ok = (item >= 0 && item < I.n) || (I.app == kAppGc && item < 0 && ~item < I.n) ||
                  (I.app == kAppGc && I.segs && item < -I.n && (uint32_t)(-(item + I.n + 1)) < I.seg_cap) ||
                  (I.app == kAppBfs && I.segs && item < 0 && (uint32_t)(-(item + 1)) < I.seg_cap);
  if (!ok) {
    record_bounds(L.status, L.fail_site, kSiteItem);
    return 0;
  }
#else
  (void)I, (void)L;
#endif
  return item;
}

// Waits until a ring slot of the previous lap has been consumed.  Returns false on timeout or
// when the launch has failed.
__device__ __forceinline__ bool wait_slot_empty(unsigned long long* slot, const Launch& L) {
  Waiter w;
  while (ld_relaxed_u64(slot) != kFreeSlot) {
    if (ld_relaxed(L.status) != 0) return false;
    if (!w.step(L.spin_limit_ns)) {
      raise_timeout(L, kSiteSlotEmpty);
      return false;
    }
  }
  return true;
}

// Item of ticket `idx`: virtual prefix, or the ring slot once the push with that very ticket has
// written it (kEmpty before).  A taken slot is freed so the ring can be reused on the next lap.
__device__ __forceinline__ int take_ticket(const Instance& I, unsigned idx) {
  if (idx < I.prefix_len) return I.prefix_item >= 0 ? I.prefix_item : (int)idx;
  unsigned long long* slot = I.ring + (idx & (I.cap - 1));
  const unsigned long long v = ld_acquire_u64(slot);
  if ((unsigned)(v >> 32) != idx) return kEmpty;
  st_relaxed_u64(slot, kFreeSlot);
  return (int)(unsigned)v;
}

// Reserve `m` push tickets and report `done` finished tasks in one atomic.  Returns the first
// ticket, or 0xffffffff if the ring is full (status set).
__device__ __forceinline__ unsigned reserve_and_complete(const Instance& I, int m, int done, const Launch& L) {
  if (m == 0 && done == 0) return 0;
  unsigned long long old = atomicAdd(&I.ctl->word, ((unsigned long long)(unsigned)m << 32) + (unsigned)done);
  if (m == 0) return 0;
  long long base = (long long)(old >> 32);
  long long last = base + m - 1;
  bool ovf = last >= 0x7fffffffLL;
  long long prev = last - (long long)I.cap;  // previous-lap ticket of the last slot
  if (!ovf && prev >= (long long)I.prefix_len) {
    long long hd = (long long)ld_relaxed_u32(&I.ctl->head);
    if (hd <= prev) ovf = true;  // that ticket is not even reserved by a popper: ring full
  }
  if (ovf) {
    raise_status(L.status, ATOS_ERR_QUEUE_OVERFLOW);
    return 0xffffffffu;
  }
  return (unsigned)base;
}

// Writes one pushed item into its ticket's slot (waiting for the previous lap to drain).
__device__ __forceinline__ void publish(const Instance& I, unsigned idx, int item, const Launch& L) {
  unsigned long long* slot = I.ring + (idx & (I.cap - 1));
  if (idx >= I.cap && !wait_slot_empty(slot, L)) return;
  st_relaxed_u64(slot, ((unsigned long long)idx << 32) | (unsigned)item);
}

__device__ __forceinline__ bool instance_quiescent(const Instance& I) {
  unsigned long long w = ld_relaxed_u64(&I.ctl->word);
  return (unsigned)(w >> 32) == (unsigned)w;
}

// Number of tickets a pop reserves under the fetch policy.
__device__ __forceinline__ int pop_size(const Instance& I, const Launch& L, int fetch) {
  if (L.policy == ATOS_FETCH_FIXED) return fetch;
  unsigned long long w = ld_relaxed_u64(&I.ctl->word);
  int avail = (int)((unsigned)(w >> 32) - ld_relaxed_u32(&I.ctl->head));
  if (L.policy == ATOS_FETCH_SPREAD) avail = avail / max(1, L.nworkers);
  return max(1, min(fetch, avail));
}

// -------------------------------------------------------------------------- block helpers

// Exclusive prefix sum over the block; `total` receives the block sum.  `tmp` needs 33 ints.
template <int BLOCK>
__device__ __forceinline__ int block_exclusive_scan(int x, int* tmp, int& total) {
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) tmp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int s = lane < NW ? tmp[lane] : 0;
    int si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    if (lane < NW) tmp[lane] = si - s;
    if (lane == 31) tmp[32] = si;
  }
  __syncthreads();
  total = tmp[32];
  int r = tmp[wid] + inc - x;
  __syncthreads();  // tmp may be reused right away
  return r;
}

// Largest i in [0, cnt) with off[i] <= e (off non-decreasing, off[0] = 0 <= e).
__device__ __forceinline__ int owner_of(const int* off, int cnt, int e) {
  int lo = 0, hi = cnt - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Consecutive edges each thread handles per round of a CTA worker's load-balancing loop: one
// owner search per run, and R independent loads in flight per thread.
template <int BLOCK>
struct LbsRun {
  static constexpr int R = BLOCK <= 256 ? 4 : (BLOCK == 512 ? 2 : 1);
};

// Shared memory of a CTA worker.  `Extra` is the task body's own per-item state; R_ the edges per
// thread of its load-balancing rounds (the body's kLbsR).
template <int BLOCK, class Extra, int R_ = LbsRun<BLOCK>::R>
struct CtaSmem {
  static constexpr int kR = R_;
  static constexpr int kRoundPushes = R_ * BLOCK;  // most pushes one round can add
  // push buffer: room for several rounds, so the load-balancing loops check it (a block barrier)
  // only every kFlushEvery rounds
  static constexpr int kPushCap = 4 * kRoundPushes < 4096 ? 4 * kRoundPushes
                                  : (2 * kRoundPushes > 4096 ? 2 * kRoundPushes : 4096);
  static constexpr int kFlushEvery = kPushCap / kRoundPushes - 1;
  int items[BLOCK];
  int start[BLOCK];
  int off[BLOCK + 1];
  int aux[BLOCK];
  int push[kPushCap];
  unsigned tk[BLOCK];  // the pop tickets this CTA holds (a contiguous range or previous-epoch orphans)
  int tmp[33];
  int npush;
  int h, n, flag, cnt;
  int keep;        // a body's block-wide decision (colouring: local continuation)
  unsigned seg_lo, seg_hi;  // segment-table entries this CTA has claimed and not used yet
  unsigned base;
  int inst_id;
  int* status;     // the launch's status and failed-site words (checked builds record here)
  int* fail_site;
  Instance I;
  Extra x;
};

struct NoExtra {};

// Appends `item` (when `want`) to the CTA push buffer; every lane of the warp must call it.
template <class S>
__device__ __forceinline__ void cta_push(S& sm, bool want, int item) {
  unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&sm.npush, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (want) sm.push[ATOS_IX(base + __popc(m & lanemask_lt()), S::kPushCap, sm, kSitePushBuffer)] = item;
}

// Publishes the CTA push buffer from entry `from` on and reports `done` finished tasks (call with
// the whole block, after a __syncthreads that follows the last cta_push).  Leaves npush = 0.
template <int BLOCK, class S>
__device__ __forceinline__ void cta_flush(S& sm, const Instance& I, int done, const Launch& L,
                                          unsigned long long* st, int from = 0) {
  const int m = sm.npush - from;
  if (threadIdx.x == 0) {
    sm.base = reserve_and_complete(I, m, done, L);
    st[kStatPushes] += m;
  }
  __syncthreads();
  const unsigned base = sm.base;
  if (m && base != 0xffffffffu) {
    if ((int)threadIdx.x < m) __threadfence();  // order the task body's writes before the items
    for (int k = threadIdx.x; k < m; k += BLOCK) publish(I, base + k, sm.push[from + k], L);
  }
  __syncthreads();
  if (threadIdx.x == 0) sm.npush = 0;
  __syncthreads();
}

// Flush when the buffer could overflow within the next kFlushEvery rounds of appends.
template <int BLOCK, class S>
__device__ __forceinline__ void cta_maybe_flush(S& sm, const Instance& I, const Launch& L, unsigned long long* st) {
  __syncthreads();
  if (sm.npush > S::kPushCap - S::kFlushEvery * S::kRoundPushes) cta_flush<BLOCK>(sm, I, 0, L, st);
}

// Round counter of a load-balancing loop: true on the rounds after which the buffer is checked.
template <class S>
__device__ __forceinline__ bool flush_round(int& rounds) {
  if (++rounds < S::kFlushEvery) return false;
  rounds = 0;
  return true;
}

// One round of the load-balancing search: thread t takes the R consecutive flattened edges
// starting at e0 = base + t * R; for each it returns the owning item and the neighbour id.
template <int BLOCK, class S>
__device__ __forceinline__ void lbs_round(const S& sm, const int32_t* __restrict__ col, int cnt, int total,
                                          int base, int (&item)[S::kR], int (&nb)[S::kR]) {
  constexpr int R = S::kR;
  const int e0 = base + (int)threadIdx.x * R;
#pragma unroll
  for (int j = 0; j < R; ++j) item[j] = -1;
  if (e0 >= total) return;
  int i = owner_of(sm.off, cnt, e0);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int e = e0 + j;
    if (e < total) {
      while (i + 1 < cnt && sm.off[i + 1] <= e) ++i;
      item[j] = i;
#ifdef ATOS_CHECKED
      const int k = ATOS_IX(sm.start[i] + (e - sm.off[i]), ldg(sm.I.row_ptr + sm.I.n), sm, kSiteEntry);
      nb[j] = ATOS_IX(ldg(col + k), sm.I.n, sm, kSiteNeighbour);
#else
      nb[j] = ldg(col + sm.start[i] + (e - sm.off[i]));
#endif
    }
  }
}

// Adds a finished batch to the throughput timeline (one thread per worker).
__device__ __forceinline__ void timeline_add(const Launch& L, unsigned long long tasks, unsigned long long edges) {
  const long long dt = (long long)(globaltimer() - *L.t_origin);
  int b = dt < 0 ? 0 : (int)min(dt / L.bucket_ns, (long long)L.nbuckets - 1);
  atomicAdd(L.timeline + 2 * b, tasks);
  atomicAdd(L.timeline + 2 * b + 1, edges);
}

// After a batch: stop if the launch failed or this worker has outlived the launch budget.
__device__ __forceinline__ bool must_stop(const Launch& L, unsigned long long t0) {
  if (ld_relaxed(L.status) != 0) return true;
  if ((long long)(globaltimer() - t0) > L.lifetime_ns) {
    raise_timeout(L, kSiteLifetime);
    return true;
  }
  return false;
}

// ------------------------------------------------------------------------ instance choice

// Batched launches: CTA (or warp) `w` starts on instance w % window; when an instance ends, the
// first worker to see it claims a successor from next_inst for all of its workers, so at most
// `window` instances are active at a time (their state stays resident in L2).
__device__ __forceinline__ int successor_of(int inst, const Launch& L) {
  QueueCtl* c = L.insts[inst].ctl;
  int s = atomicCAS(&c->succ, -2, -3);
  if (s == -2) {
    unsigned k = atomicAdd(L.next_inst, 1u);
    s = k < (unsigned)L.ninst ? (int)k : -1;
    atomicExch(&c->succ, s);
    return s;
  }
  Waiter w;
  while ((s = ld_relaxed(&c->succ)) == -3) {
    if (!w.step(L.spin_limit_ns)) {
      raise_timeout(L, kSiteSuccessor);
      return -1;
    }
  }
  return s;
}

// When no successor is left, help any started instance that has not finished.
__device__ __forceinline__ int unfinished_instance(int from, const Launch& L) {
  unsigned started = min(ld_relaxed_u32(L.next_inst), (unsigned)L.ninst);
  for (unsigned k = 0; k < started; ++k) {
    int i = (int)((from + 1 + k) % started);
    if (!ld_relaxed(&L.insts[i].ctl->finished)) return i;
  }
  return -1;
}

__device__ __forceinline__ int next_instance(int inst, const Launch& L) {
  if (L.ninst == 1) return -1;
  int s = successor_of(inst, L);
  if (s >= 0) return s;
  return unfinished_instance(inst, L);
}

__device__ __forceinline__ void flush_stats(const Instance& I, unsigned long long* st) {
#pragma unroll
  for (int k = 0; k < kNumStats; ++k)
    if (st[k]) atomicAdd(&I.stats[k], st[k]), st[k] = 0;
}

// ------------------------------------------------------------------------ CTA worker engine
//
// Body must provide:
//   template <int B> using Extra;                 per-CTA shared state of a B-thread worker
//   template <int B, class S> static void cta_batch(S& sm, int cnt, const Launch&, st);
//       processes sm.items[0, cnt) of sm.I, pushes with cta_push / cta_maybe_flush and ends
//       with cta_flush(sm, I, cnt, ...) so the batch is reported complete;
//   template <int B, class S> static int cta_idle(S& sm, const Launch&, st);
//       called by the whole block when its reserved slots hold nothing: returns 1 when the
//       instance has terminated, 0 to keep waiting (it may push work, e.g. PageRank's f2).

// Serving: true once this worker's time slice is over (it then pauses at a safe point).
__device__ __forceinline__ bool slice_over(const Launch& L, unsigned long long t0) {
  return L.slice_ns > 0 && (long long)(globaltimer() - t0) > L.slice_ns;
}

// Serving pause: record the tickets this CTA still waits for, so that the next epoch's workers
// take them over (they may be filled later by a push of this epoch).
template <int BLOCK, class S>
__device__ __forceinline__ void cta_orphan_pending(S& sm, bool pending, const Launch& L) {
  const Instance& I = sm.I;
  if (pending) {
    const unsigned w = (L.epoch + 1) & 1;
    const unsigned idx = atomicAdd(&I.ctl->orphan_count[w], 1u);
    if (idx < I.orphan_cap) I.orphans[w][idx] = sm.tk[threadIdx.x];
    else raise_status(L.status, ATOS_ERR_QUEUE_OVERFLOW);
  }
}

// Returns 1 when the worker paused (serving slice over), 0 when the instance ended for it
// (terminated, or the launch failed).
template <class Body, int BLOCK>
__device__ int cta_run_instance(CtaSmem<BLOCK, typename Body::template Extra<BLOCK>, Body::template kLbsR<BLOCK>>& sm,
                                const Launch& L,
                                unsigned long long* st, unsigned long long t0) {
  const Instance& I = sm.I;
  Waiter wait;
  for (;;) {
    if (threadIdx.x == 0) {
      int n = pop_size(I, L, L.fetch);
      int from_orphans = 0;
      if (L.slice_ns > 0) {  // serving: the previous epoch's pending tickets come first
        const unsigned r = L.epoch & 1;
        const unsigned cnt = ld_relaxed_u32(&I.ctl->orphan_count[r]);
        if (ld_relaxed_u32(&I.ctl->orphan_head) < cnt) {
          const unsigned o = atomicAdd(&I.ctl->orphan_head, (unsigned)n);
          if (o < cnt) {
            n = (int)min((unsigned)n, cnt - o);
            sm.h = (int)o;
            from_orphans = 1;
          }
        }
      }
      if (!from_orphans) sm.h = (int)atomicAdd(&I.ctl->head, (unsigned)n);
      sm.n = n;
      sm.cnt = from_orphans;
    }
    __syncthreads();
    const int n = sm.n;
    if ((int)threadIdx.x < n)
      sm.tk[threadIdx.x] = sm.cnt ? I.orphans[L.epoch & 1][(unsigned)sm.h + threadIdx.x] : (unsigned)sm.h + threadIdx.x;
    bool pending = (int)threadIdx.x < n;
    for (;;) {
      int item = kEmpty;
      if (pending) {
        item = take_ticket(I, sm.tk[threadIdx.x]);
        if (item != kEmpty) pending = false, item = checked_item(I, item, L);
      }
      // compact the items taken this round into sm.items
      const bool got = item != kEmpty;
      int total;
      const int pos = block_exclusive_scan<BLOCK>(got ? 1 : 0, sm.tmp, total);
      if (got) sm.items[pos] = item;
      const int still = __syncthreads_count(pending);
      if (total > 0) {
        unsigned long long edges0 = 0;
        if (threadIdx.x == 0) st[kStatBatches]++, edges0 = st[kStatEdges];
        Body::template cta_batch<BLOCK>(sm, total, L, st);
        if (threadIdx.x == 0 && L.timeline) timeline_add(L, (unsigned long long)total, st[kStatEdges] - edges0);
        wait.reset();
        if (threadIdx.x == 0) sm.flag = must_stop(L, t0) ? 1 : (slice_over(L, t0) ? 2 : 0);
        __syncthreads();
        if (sm.flag == 1) return 0;
        if (sm.flag == 2) {
          cta_orphan_pending<BLOCK>(sm, pending, L);
          return 1;
        }
        if (still == 0) break;
        continue;
      }
      // nothing arrived: termination / failure / budget / end of the serving slice
      int verdict = Body::template cta_idle<BLOCK>(sm, L, st);
      if (threadIdx.x == 0) {
        int f = verdict;
        if (!f && ld_relaxed(L.status) != 0) f = 2;
        if (!f && slice_over(L, t0)) f = 3;
        if (!f && !wait.step(L.spin_limit_ns)) {
          raise_timeout(L, kSiteCtaIdle);
          f = 2;
        }
        st[kStatIdle]++;
        sm.flag = f;
      }
      __syncthreads();
      if (sm.flag == 3) {
        cta_orphan_pending<BLOCK>(sm, pending, L);
        return 1;
      }
      if (sm.flag) return 0;
      if (still == 0) break;
    }
  }
}

// Minimum resident CTAs per SM the compiler must allow: Body::kResidentThreads threads per SM.
// 1536 (75% of an SM's 2048 threads) caps registers near 42 per thread, trading per-thread ILP
// for resident warps; 1024 leaves 64 registers, so a body can keep more gathers in flight per
// thread instead.
template <class Body, int BLOCK>
struct MinBlocks {
  static constexpr int value = BLOCK >= Body::kResidentThreads ? 1 : Body::kResidentThreads / BLOCK;
};

template <class Body, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (MinBlocks<Body, BLOCK>::value)) cta_persistent_kernel(Launch L) {
  __shared__ CtaSmem<BLOCK, typename Body::template Extra<BLOCK>, Body::template kLbsR<BLOCK>> sm;
  unsigned long long st[kNumStats] = {};
  const unsigned long long t0 = globaltimer();
  int inst = (int)(blockIdx.x % (unsigned)min(L.window, L.ninst));
  if (threadIdx.x == 0) sm.npush = 0, sm.status = L.status, sm.fail_site = L.fail_site;
  while (inst >= 0) {
    if (threadIdx.x == 0) {
      sm.I = L.insts[inst];
      sm.inst_id = inst;
      sm.seg_lo = sm.seg_hi = 0;
      sm.flag = ld_relaxed(&sm.I.ctl->finished);  // one thread decides for the block
    }
    __syncthreads();
    int paused = 0;
    if (!sm.flag) paused = cta_run_instance<Body, BLOCK>(sm, L, st, t0);
    if (threadIdx.x == 0) {
      flush_stats(sm.I, st);
      int next = -1;
      if (!paused && ld_relaxed(L.status) == 0) {
        atomicExch(&sm.I.ctl->finished, 1);
        next = next_instance(inst, L);
      }
      sm.flag = next;  // a paused worker leaves the launch (serving epochs end this way)
    }
    __syncthreads();
    inst = sm.flag;
    __syncthreads();
  }
}

// Discrete strategy: one launch processes generation [gen_begin, gen_end) of every instance;
// blockIdx.y selects the instance, blockIdx.x a FETCH-sized slice.  Items are already written.
template <class Body, int BLOCK>
__global__ void __launch_bounds__(BLOCK) cta_discrete_kernel(Launch L) {
  __shared__ CtaSmem<BLOCK, typename Body::template Extra<BLOCK>, Body::template kLbsR<BLOCK>> sm;
  unsigned long long st[kNumStats] = {};
  const int inst = blockIdx.y;
  if (threadIdx.x == 0) {
    sm.I = L.insts[inst];
    sm.npush = 0;
    sm.seg_lo = sm.seg_hi = 0;
    sm.status = L.status;
    sm.fail_site = L.fail_site;
  }
  __syncthreads();
  const Instance& I = sm.I;
  const unsigned b = I.ctl->gen_begin, e = I.ctl->gen_end;
  const unsigned lo = b + blockIdx.x * (unsigned)L.fetch;
  if (lo >= e) return;
  const int span = (int)min((unsigned)L.fetch, e - lo);
  // every ticket of a generation was written by the previous launch; an EMPTY one can only
  // follow a failed push (the status is already set), and is skipped
  int item = (int)threadIdx.x < span ? take_ticket(I, lo + threadIdx.x) : kEmpty;
  if (item != kEmpty) item = checked_item(I, item, L);
  int cnt;
  const int pos = block_exclusive_scan<BLOCK>(item != kEmpty ? 1 : 0, sm.tmp, cnt);
  if (item != kEmpty) sm.items[pos] = item;
  __syncthreads();
  if (cnt > 0) Body::template cta_batch<BLOCK>(sm, cnt, L, st);
  if (threadIdx.x == 0 && cnt > 0 && L.timeline) timeline_add(L, (unsigned long long)cnt, st[kStatEdges]);
  if (threadIdx.x == 0) st[kStatBatches] += cnt > 0, flush_stats(I, st);
}

// ----------------------------------------------------------------------- warp worker engine
//
// Each warp is an independent worker (persist-32 of Section 6.2): it pops up to 32 tickets, and
// processes the items it got one after another, its 32 lanes striding each item's neighbours.
// Body must provide:
//   static void warp_item(WarpSmem&, const Instance&, int item, const Launch&, st)
//   static int warp_idle(WarpSmem&, const Instance&, const Launch&, st)  (lane-uniform result)

constexpr int kWarpPushCap = 128;
struct WarpSmem {
  int push[kWarpPushCap];
  int npush;
  unsigned bits[4];
  int* status;  // the launch's status and failed-site words (checked builds record here)
  int* fail_site;
};

// Appends (warp-wide call) and flushes when the buffer could overflow in the next round.
__device__ __forceinline__ void warp_push(WarpSmem& ws, bool want, int item) {
  unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  int base = ws.npush;
  if (want) ws.push[ATOS_IX(base + __popc(m & lanemask_lt()), kWarpPushCap, ws, kSiteWarpPush)] = item;
  __syncwarp();
  if (lane == 0) ws.npush = base + __popc(m);
  __syncwarp();
}

__device__ __forceinline__ void warp_flush(WarpSmem& ws, const Instance& I, int done, const Launch& L,
                                           unsigned long long* st) {
  const int lane = threadIdx.x & 31;
  const int m = ws.npush;
  unsigned base = 0;
  if (lane == 0) {
    base = reserve_and_complete(I, m, done, L);
    st[kStatPushes] += m;
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  if (m && base != 0xffffffffu) {
    if (lane < m) __threadfence();
    for (int k = lane; k < m; k += 32) publish(I, base + k, ws.push[k], L);
  }
  __syncwarp();
  if (lane == 0) ws.npush = 0;
  __syncwarp();
}

__device__ __forceinline__ void warp_maybe_flush(WarpSmem& ws, const Instance& I, const Launch& L,
                                                 unsigned long long* st) {
  if (ws.npush > kWarpPushCap - 32) warp_flush(ws, I, 0, L, st);
}

// kLanes: thread workers (worker_size 1) -- the warp pops up to 32 tasks as one, and each lane
// processes its own task (Body::lane_items) instead of the 32 lanes sharing each task in turn.
template <class Body, bool kLanes = false>
__device__ void warp_run_instance(WarpSmem& ws, const Instance& I, const Launch& L, unsigned long long* st,
                                  unsigned long long t0) {
  const int lane = threadIdx.x & 31;
  const int fetch = min(L.fetch, 32);
  Waiter wait;
  for (;;) {
    unsigned h = 0;
    int n = 0;
    if (lane == 0) {
      n = pop_size(I, L, fetch);
      h = atomicAdd(&I.ctl->head, (unsigned)n);
    }
    h = __shfl_sync(0xffffffffu, h, 0);
    n = __shfl_sync(0xffffffffu, n, 0);
    bool pending = lane < n;
    for (;;) {
      int item = kEmpty;
      if (pending) {
        item = take_ticket(I, h + lane);
        if (item != kEmpty) pending = false, item = checked_item(I, item, L);
      }
      unsigned got = __ballot_sync(0xffffffffu, item != kEmpty);
      const unsigned still = __ballot_sync(0xffffffffu, pending);
      if (got) {
        const int cnt = __popc(got);
        const unsigned long long edges0 = st[kStatEdges];
        if constexpr (kLanes) {
          Body::lane_items(ws, I, item, L, st);
        } else {
          while (got) {
            const int src = __ffs(got) - 1;
            got &= got - 1;
            const int it = __shfl_sync(0xffffffffu, item, src);
            Body::warp_item(ws, I, it, L, st);
          }
        }
        if (lane == 0) st[kStatTasks] += cnt, st[kStatBatches]++;
        if (lane == 0 && L.timeline) timeline_add(L, (unsigned long long)cnt, st[kStatEdges] - edges0);
        warp_flush(ws, I, cnt, L, st);
        wait.reset();
        int stop = 0;
        if (lane == 0) stop = must_stop(L, t0) ? 1 : 0;
        if (__shfl_sync(0xffffffffu, stop, 0)) return;
        if (!still) break;
        continue;
      }
      int f = Body::warp_idle(ws, I, L, st);
      if (lane == 0) {
        if (!f && ld_relaxed(L.status) != 0) f = 2;
        if (!f && !wait.step(L.spin_limit_ns)) {
          raise_timeout(L, kSiteWarpIdle);
          f = 2;
        }
        st[kStatIdle]++;
      }
      f = __shfl_sync(0xffffffffu, f, 0);
      if (f) return;
      if (!still) break;
    }
  }
}

constexpr int kWarpBlock = 256;

template <class Body, bool kLanes = false>
__global__ void __launch_bounds__(kWarpBlock) warp_persistent_kernel(Launch L) {
  __shared__ WarpSmem wsm[kWarpBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpSmem& ws = wsm[wid];
  unsigned long long st[kNumStats] = {};
  const int gw = blockIdx.x * (kWarpBlock / 32) + wid;
  const unsigned long long t0 = globaltimer();
  int inst = gw % min(L.window, L.ninst);
  if (lane == 0) ws.npush = 0, ws.status = L.status, ws.fail_site = L.fail_site;
  __syncwarp();
  while (inst >= 0) {
    const Instance I = L.insts[inst];
    int fin = 0;
    if (lane == 0) fin = ld_relaxed(&I.ctl->finished);  // one lane decides for the warp
    if (!__shfl_sync(0xffffffffu, fin, 0)) warp_run_instance<Body, kLanes>(ws, I, L, st, t0);
    int next = -1;
    if (lane == 0) {
      flush_stats(I, st);
      if (ld_relaxed(L.status) == 0) {
        atomicExch(&I.ctl->finished, 1);
        next = next_instance(inst, L);
      }
    }
    inst = __shfl_sync(0xffffffffu, next, 0);
  }
}

// Discrete warp strategy: warp w of the grid processes up to `fetch` items of the generation.
template <class Body, bool kLanes = false>
__global__ void __launch_bounds__(kWarpBlock) warp_discrete_kernel(Launch L) {
  __shared__ WarpSmem wsm[kWarpBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpSmem& ws = wsm[wid];
  unsigned long long st[kNumStats] = {};
  const Instance I = L.insts[blockIdx.y];
  const int fetch = min(L.fetch, 32);
  const unsigned b = I.ctl->gen_begin, e = I.ctl->gen_end;
  const unsigned lo = b + (blockIdx.x * (kWarpBlock / 32) + wid) * (unsigned)fetch;
  if (lo >= e) return;
  if (lane == 0) ws.npush = 0, ws.status = L.status, ws.fail_site = L.fail_site;
  __syncwarp();
  const int span = (int)min((unsigned)fetch, e - lo);
  int item = lane < span ? take_ticket(I, lo + lane) : kEmpty;
  if (item != kEmpty) item = checked_item(I, item, L);
  unsigned got = __ballot_sync(0xffffffffu, item != kEmpty);  // EMPTY only after a failed push
  const int cnt = __popc(got);
  if constexpr (kLanes) {
    Body::lane_items(ws, I, item, L, st);
  } else {
    while (got) {
      const int src = __ffs(got) - 1;
      got &= got - 1;
      Body::warp_item(ws, I, __shfl_sync(0xffffffffu, item, src), L, st);
    }
  }
  if (lane == 0) st[kStatTasks] += cnt, st[kStatBatches] += cnt > 0;
  if (lane == 0 && cnt > 0 && L.timeline) timeline_add(L, (unsigned long long)cnt, st[kStatEdges]);
  warp_flush(ws, I, cnt, L, st);
  if (lane == 0) flush_stats(I, st);
}

}  // namespace atos
