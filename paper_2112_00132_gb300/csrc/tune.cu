// tune.cu -- autotuner: picks worker size, fetch size, fetch policy, strategy and (BFS with many
// sources) the instance window for one application on one graph by timing the candidates, the
// sweep of Figure 4 (worker size x FETCH_SIZE, thread workers included) extended with
// the kernel strategy (Section 3.4) and, for PageRank and colouring, the spread-id layout of the
// graph.
//
// Candidates are run on the caller's graph through the public entry points (each run is checked:
// a candidate that fails, or a PageRank candidate whose FP64 error bound exceeds
// ATOS_TUNE_PR_MAX_ERROR, is skipped), timed with the library's own CUDA events, best of
// `repeats` runs.  A colouring qualifies only when its colour count is within
// ATOS_TUNE_GC_MAX_COLOR_RATIO of the fewest any candidate reached, so a fast colouring with many
// more colours does not win.  The winner is cached per graph class -- application, log2 of the vertex count,
// log2 of the average degree and log2 of the max/average degree ratio -- so graphs of the same
// shape reuse it through atos_tuned_config without a new sweep.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "atos.h"

namespace {

using ClassKey = std::tuple<int, int, int, int>;
std::mutex g_cache_mu;
std::map<ClassKey, std::pair<atos_config, double>> g_cache;

ClassKey class_of(atos_graph_t g, int app) {
  int32_t n = 0, maxd = 0;
  int64_t nnz = 0;
  atos_graph_info(g, &n, &nnz, &maxd);
  const double avg = n > 0 ? (double)nnz / n : 0.0;
  const int ln = n > 0 ? (int)floor(log2((double)n)) : 0;
  const int ld = avg > 0 ? (int)floor(log2(avg)) : -1;
  const int lr = avg > 0 ? (int)floor(log2(std::max(1.0, (double)maxd / avg))) : 0;
  return ClassKey(app, ln, ld, lr);
}

atos_config make(const char* preset, int worker, int fetch, int policy) {
  atos_config c;
  atos_queue_config(&c, preset);
  if (worker) c.worker_size = worker;
  if (fetch) c.fetch_size = fetch;
  if (policy >= 0) c.fetch_policy = policy;
  return c;
}

std::vector<atos_config> candidates(int app, int nsrc) {
  std::vector<atos_config> out;
  for (int w : {128, 256, 512, 1024}) out.push_back(make(nullptr, w, w, ATOS_FETCH_SPREAD));
  out.push_back(make(nullptr, 256, 256, ATOS_FETCH_FIXED));
  out.push_back(make(nullptr, 256, 64, ATOS_FETCH_GREEDY));
  out.push_back(make(nullptr, 32, 32, ATOS_FETCH_SPREAD));
  out.push_back(make("persist-warp", 0, 0, -1));
  out.push_back(make("discrete-cta", 0, 0, -1));
  out.push_back(make("bsp", 0, 0, -1));
  {
    atos_config c = make("bsp", 0, 0, -1);  // the level loop on the device (conditional graph node)
    c.flags |= ATOS_FLAG_BSP_DEVICE_LOOP;
    out.push_back(c);
  }
  if (app == ATOS_APP_COLOR) {
    // dependency-ordered colouring: exactly serial first fit in id order, one task per vertex
    for (int w : {128, 256, 512, 1024})
      for (int f : {w, w == 128 ? 32 : 64}) {  // small pops spread the long dependency chains' ready vertices
        atos_config c = make(nullptr, w, f, ATOS_FETCH_GREEDY);
        c.flags |= ATOS_FLAG_GC_DEPENDENCY;
        out.push_back(c);
      }
    atos_config c = make(nullptr, 32, 32, ATOS_FETCH_GREEDY);
    c.flags |= ATOS_FLAG_GC_DEPENDENCY;
    out.push_back(c);
  }
  if (app == ATOS_APP_PAGERANK) {
    for (int w : {512, 1024})
      for (int cs : {8, 16, 64}) {
        atos_config c = make(nullptr, w, w, ATOS_FETCH_SPREAD);
        c.check_size = cs;
        out.push_back(c);
      }
    for (int f : {128, 256, 512})  // greedy pops at 512 threads
      for (int cs : {8, 16}) {
        atos_config c = make(nullptr, 512, f, ATOS_FETCH_GREEDY);
        c.check_size = cs;
        out.push_back(c);
      }
    for (int w : {256, 512, 1024}) {  // threshold-crossing enqueue instead of the Check_Size scan
      atos_config c = make(nullptr, w, w, ATOS_FETCH_SPREAD);
      c.flags |= ATOS_FLAG_PR_CROSSING;
      out.push_back(c);
    }
  }
  if (app == ATOS_APP_BFS) {
    // small greedy pops: a search's late re-expansions of long rows spread over more workers
    for (int w : {512, 1024})
      for (int f : {64, 128}) out.push_back(make(nullptr, w, f, ATOS_FETCH_GREEDY));
  }
  if (app == ATOS_APP_BFS && nsrc > 1) {
    for (int w : {256, 512})
      for (int win : {1, 2, 4, 8, 16, 32}) {
        if (win >= nsrc) break;
        atos_config c = make(nullptr, w, w, ATOS_FETCH_SPREAD);
        c.window = win;
        out.push_back(c);
        if (w == 512 && win >= 4 && win <= 16) {
          c = make(nullptr, w, 64, ATOS_FETCH_GREEDY);
          c.window = win;
          out.push_back(c);
        }
      }
  }
  out.push_back(make(nullptr, 1, 32, ATOS_FETCH_SPREAD));  // thread workers
  if (app == ATOS_APP_BFS) {
    // the same shapes with expansion markers
    const size_t k = out.size();
    for (size_t i = 0; i < k; ++i)
      if (out[i].strategy != ATOS_BSP) {
        atos_config c = out[i];
        c.flags |= ATOS_FLAG_BFS_EXPAND_ONCE;
        out.push_back(c);
        if (c.worker_size > 32) {  // and with long rows split into segment tasks
          c.flags |= ATOS_FLAG_BFS_SPLIT_ROWS;
          out.push_back(c);
        }
      }
  }
  if (app == ATOS_APP_PAGERANK || app == ATOS_APP_COLOR) {
    // the same shapes on the spread-id copy of the graph
    const size_t k = out.size();
    for (size_t i = 0; i < k; ++i)
      if (!(out[i].flags & ATOS_FLAG_PR_CROSSING)) {
        atos_config c = out[i];
        c.flags |= ATOS_FLAG_SPREAD_IDS;
        out.push_back(c);
      }
  }
  return out;
}

}  // namespace

extern "C" {

int atos_autotune(atos_graph_t g, int32_t app, const int32_t* sources, int32_t nsrc, void* scratch_out,
                  int32_t repeats, atos_config* best, double* best_ms, void* stream) {
  if (!g || !best || !scratch_out || repeats < 1) return ATOS_ERR_INVALID_ARG;
  if (app == ATOS_APP_BFS && (!sources || nsrc < 1)) return ATOS_ERR_INVALID_ARG;
  if (app != ATOS_APP_BFS && app != ATOS_APP_PAGERANK && app != ATOS_APP_COLOR) return ATOS_ERR_INVALID_ARG;
  double best_t = INFINITY;
  atos_config best_c;
  atos_queue_config(&best_c, nullptr);
  struct Tried {
    atos_config c;
    double ms;
    int32_t colors;
  };
  std::vector<Tried> done;
  for (const atos_config& c : candidates(app, app == ATOS_APP_BFS ? nsrc : 1)) {
    double t = INFINITY;
    int32_t colors = 0;
    bool ok = true;
    for (int r = 0; r <= repeats && ok; ++r) {  // run 0 warms up
      atos_stats st = {};
      int rc;
      if (app == ATOS_APP_BFS) rc = atos_bfs(g, sources, nsrc, (int32_t*)scratch_out, &c, stream, &st);
      else if (app == ATOS_APP_PAGERANK) rc = atos_pagerank(g, 0.85f, 1e-9f, (float*)scratch_out, &c, stream, &st);
      else rc = atos_color(g, (int32_t*)scratch_out, nullptr, &c, stream, &st);
      colors = st.num_colors;
      if (rc != ATOS_OK) ok = false;
      else if (app == ATOS_APP_PAGERANK && !(st.error_bound <= ATOS_TUNE_PR_MAX_ERROR)) ok = false;
      else if (r > 0) t = std::min(t, st.ms);
      // the warm-up alone is far slower: not a contender (colourings are judged on their colour
      // count first, so every one of them is timed)
      else if (app != ATOS_APP_COLOR && st.ms > 4.0 * best_t) ok = false;
    }
    if (!ok) continue;
    done.push_back(Tried{c, t, colors});
    if (t < best_t) best_t = t;
  }
  if (done.empty()) return ATOS_ERR_CUDA;
  // colourings: only those within ATOS_TUNE_GC_MAX_COLOR_RATIO of the fewest colours qualify
  int32_t fewest = INT32_MAX;
  for (const Tried& d : done) fewest = std::min(fewest, d.colors);
  best_t = INFINITY;
  for (const Tried& d : done) {
    if (app == ATOS_APP_COLOR && (double)d.colors > ATOS_TUNE_GC_MAX_COLOR_RATIO * (double)fewest) continue;
    if (d.ms < best_t) best_t = d.ms, best_c = d.c;
  }
  *best = best_c;
  if (best_ms) *best_ms = best_t;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  g_cache[class_of(g, app)] = std::make_pair(best_c, best_t);
  return ATOS_OK;
}

int atos_batch_autotune(const atos_graph_t* graphs, int32_t ngraphs, const atos_instance* inst, int32_t ninst,
                        int32_t repeats, atos_config* best, double* best_ms, void* stream) {
  if (!graphs || ngraphs < 1 || !inst || ninst < 1 || !best || repeats < 1) return ATOS_ERR_INVALID_ARG;
  bool has_pr = false;
  for (int i = 0; i < ninst; ++i) has_pr |= inst[i].app == ATOS_APP_PAGERANK;
  std::vector<atos_config> cands;
  for (int w : {128, 256, 512, 1024}) cands.push_back(make(nullptr, w, w, ATOS_FETCH_SPREAD));
  cands.push_back(make(nullptr, 256, 64, ATOS_FETCH_GREEDY));
  cands.push_back(make(nullptr, 32, 32, ATOS_FETCH_SPREAD));
  for (int w : {256, 512})
    for (int win : {8, 64, 512}) {
      if (win >= ninst) break;
      atos_config c = make(nullptr, w, w, ATOS_FETCH_SPREAD);
      c.window = win;
      cands.push_back(c);
      if (has_pr && win == 512)
        for (int cs : {8, 16}) {  // PageRank's Check_Size at the widest window
          atos_config d = c;
          d.check_size = cs;
          cands.push_back(d);
        }
    }
  cands.push_back(make("discrete-cta", 0, 0, -1));
  {
    // the persistent shapes so far on the spread-id copies of the graphs
    const size_t k = cands.size();
    for (size_t i = 0; i < k; ++i)
      if (cands[i].strategy == ATOS_PERSISTENT) {
        atos_config c = cands[i];
        c.flags |= ATOS_FLAG_SPREAD_IDS;
        cands.push_back(c);
      }
  }
  if (has_pr)
    for (int w : {256, 512}) {
      atos_config c = make(nullptr, w, w, ATOS_FETCH_SPREAD);
      c.flags |= ATOS_FLAG_PR_CROSSING;
      cands.push_back(c);
    }
  std::vector<atos_stats> per((size_t)ninst);
  double best_t = INFINITY;
  atos_config best_c;
  atos_queue_config(&best_c, nullptr);
  int tried = 0;
  for (const atos_config& c : cands) {
    atos_batch_t b = nullptr;
    if (atos_batch_create(graphs, ngraphs, inst, ninst, &c, &b) != ATOS_OK) continue;
    const bool graph = c.strategy == ATOS_PERSISTENT;
    double t = INFINITY;
    bool ok = true;
    for (int r = 0; r <= repeats && ok; ++r) {  // run 0 warms up (and captures the graph)
      atos_stats total;
      int rc = graph ? atos_batch_run_graph(b, stream) : atos_batch_run(b, stream);
      if (rc == ATOS_OK) rc = atos_batch_stats(b, &total, per.data(), stream);
      if (rc != ATOS_OK) {
        ok = false;
        break;
      }
      for (int i = 0; i < ninst && ok; ++i)
        if (inst[i].app == ATOS_APP_PAGERANK && !(per[i].error_bound <= ATOS_TUNE_PR_MAX_ERROR)) ok = false;
      if (!ok) break;
      if (r > 0) t = std::min(t, total.ms);
      else if (total.ms > 4.0 * best_t) ok = false;  // the warm-up alone is far slower: not a contender
    }
    atos_batch_destroy(b);
    if (!ok) continue;
    tried++;
    if (t < best_t) {
      best_t = t;
      best_c = c;
    }
  }
  if (!tried) return ATOS_ERR_CUDA;
  *best = best_c;
  if (best_ms) *best_ms = best_t;
  return ATOS_OK;
}

int atos_tuned_config(atos_graph_t g, int32_t app, atos_config* cfg) {
  if (!g || !cfg) return ATOS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  auto it = g_cache.find(class_of(g, app));
  if (it == g_cache.end()) {
    atos_queue_config(cfg, nullptr);
    return ATOS_ERR_UNSUPPORTED;
  }
  *cfg = it->second.first;
  return ATOS_OK;
}

}  // extern "C"
