// state.cuh -- declarations shared by the host API and the bookkeeping kernels.
#pragma once

#include <cuda_runtime.h>

#include "engine.cuh"

namespace atos {

// Small device-side control block of one scratch area (mirrored to pinned host memory).
struct alignas(128) DevCtl {
  int status;          // first error of the last launch
  int dirty;           // rings may hold stale items (the last launch failed, or never used)
  unsigned next_inst;  // batched launch: next instance to start
  unsigned maxgen;     // discrete strategy: largest generation
  unsigned pushed;     // PageRank final sweep (discrete): items pushed
  int num_colors;
  int fail_site;       // first wait that timed out (kSite*), 0 if none
  int pad[1];
  double sum_rank;     // PageRank: FP64 sum of the ranks
  double sum_res;      // PageRank: FP64 sum of the residues left
  double cert_l1;      // PageRank: FP64 ||(1 - alpha) 1 + alpha P x - x||_1 on the exact scale
  unsigned long long t_origin;  // %globaltimer when the run's state was prepared (timeline origin)
};

cudaError_t launch_prepare(Instance* d_insts, int ninst, int max_n, DevCtl* d_ctl, uint32_t flags, unsigned window,
                           cudaStream_t s);
cudaError_t launch_pr_init(Instance* d_insts, int ninst, int64_t max_nnz, cudaStream_t s);
cudaError_t launch_next_generation(Instance* d_insts, int ninst, DevCtl* d_ctl, cudaStream_t s);
cudaError_t launch_finalize(const Instance* d_insts, int ninst, DevCtl* d_ctl, cudaStream_t s);

// Results computed on the spread-id copy of a graph, to be returned in the caller's ids:
// dst[v] = src[perm[v]] for 4-byte elements (perm: the copy's id of each vertex).
struct SpreadJob {
  const void* src;
  void* dst;
  int32_t n;
  int32_t pad;
  const int32_t* perm;
};
cudaError_t unspread_jobs(const SpreadJob* d_jobs, int njobs, int max_n, cudaStream_t s);

// FP64 certificate of normalised PageRank outputs (ranks summing to 1): for the instances
// d_insts[d_idx[j]], j < count, out[j] = ||(1 - alpha) 1 + alpha P x - x||_1 with x = exact_sum *
// rank, so the L1 distance of the output to the normalised fixed point is at most
// out[j] / ((1 - alpha) exact_sum).  Uses each instance's cert_y scratch.
cudaError_t pr_certify_outputs(const Instance* d_insts, const int* d_idx, int count, int max_n, int64_t max_nnz,
                               double* d_out, cudaStream_t s);

// Host loop of the discrete strategy (Section 3.4) over d_insts[0, ninst), after prepare: one
// launch of `fn` per queue generation (grid: generation slices x instances), until every queue is
// empty; PageRank instances (has_pr) also need a verification sweep that enqueues nothing.  Reads
// the generation size back after every launch (h_ctl: pinned mirror of d_ctl).  Returns a
// cudaError_t; *iterations receives the launches of `fn`.
cudaError_t discrete_loop(const void* fn, int threads, int per_block, Launch L, Instance* d_insts, int ninst,
                          int max_n, unsigned first_gen, bool has_pr, DevCtl* d_ctl, DevCtl* h_ctl, cudaStream_t st,
                          int64_t* iterations);

const void* bfs_persistent_kernel(int worker);
const void* bfs_discrete_kernel(int worker);

}  // namespace atos
