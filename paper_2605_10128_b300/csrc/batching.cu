// Mixed-grid batching and sweep tile autotuning.
//
// tto_grid_autotune times every sweep tile variant of one precision mode on a
// grid (a batch of unsplit topologies costs the same sweep work as any other
// batch, since the sweep has no data-dependent loops) and keeps the fastest
// for later evaluation calls on that grid.
//
// tto_evaluate_multi evaluates several (grid, topology batch) jobs as one unit
// of work.  In graph mode the first call with a given set of jobs runs them
// eagerly on forked streams and records the same fork/join launch sequence into
// a CUDA graph; later calls with the same jobs replay that graph with one
// cudaGraphLaunch, each grid's kernels on their own branch so that small grids
// fill the SMs that large ones leave idle.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <new>
#include <mutex>
#include <vector>

#include "sweep.cuh"
#include "tto_internal.h"

namespace tto {
namespace {

constexpr int kMaxJobs = kMaxMultiJobs;

struct StreamPool {
  std::vector<cudaStream_t> side;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  // graph mode records and replays on this stream (a legacy default stream,
  // which callers often pass, cannot be captured), joined to the caller's
  cudaStream_t cap = nullptr;
  cudaEvent_t cap_in = nullptr, cap_out = nullptr;
};

std::recursive_mutex g_mu;  // recursive: workspace growth drops graphs while a call holds it
StreamPool g_pool[64];

int stream_pool(int dev, int n, StreamPool** out) {
  if (dev < 0 || dev >= 64) return set_error(TTO_E_ARG, "device %d out of range", dev);
  StreamPool& p = g_pool[dev];
  if (!p.fork) TTO_CUDA_TRY(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming));
  if (!p.cap) {
    TTO_CUDA_TRY(cudaStreamCreateWithFlags(&p.cap, cudaStreamNonBlocking));
    TTO_CUDA_TRY(cudaEventCreateWithFlags(&p.cap_in, cudaEventDisableTiming));
    TTO_CUDA_TRY(cudaEventCreateWithFlags(&p.cap_out, cudaEventDisableTiming));
  }
  while ((int)p.side.size() < n) {
    cudaStream_t st;
    TTO_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    p.side.push_back(st);
    cudaEvent_t ev;
    TTO_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    p.join.push_back(ev);
  }
  *out = &p;
  return TTO_OK;
}

struct GraphKey {
  std::vector<uint64_t> words;
  bool operator<(const GraphKey& o) const { return words < o.words; }
};

struct GraphEntry {
  cudaGraphExec_t exec;
  std::vector<uint64_t> grids;  // uids of the grids the graph reads and writes
  unsigned int* counter = nullptr;  // persistent mode: the graph's own work-list counter
};

void drop_entry(GraphEntry& e) {
  cudaGraphExecDestroy(e.exec);
  if (e.counter) cudaFree(e.counter);
}

std::map<GraphKey, GraphEntry> g_graphs;

GraphKey make_key(const tto_eval_job* jobs, int n, const tto_eval_opts* o, int mode) {
  GraphKey k;
  k.words.push_back((uint64_t)mode);
  k.words.push_back(((uint64_t)o->precision << 48) | ((uint64_t)o->fitness_kind << 32) |
                    ((uint64_t)o->d_split << 16) | (uint64_t)o->d_moved);
  k.words.push_back((uint64_t)(uint32_t)o->d_disc);
  for (int i = 0; i < n; ++i) {
    const tto_eval_job& j = jobs[i];
    k.words.push_back(j.grid->uid);
    k.words.push_back(j.grid->ws_epoch);
    k.words.push_back((uint64_t)j.grid->tuned_shape[o->precision] + 1);
    k.words.push_back((uint64_t)(uintptr_t)j.topo);
    k.words.push_back((uint64_t)j.B);
    k.words.push_back((uint64_t)j.n_t);
    for (int t = 0; t < (j.timesteps ? j.n_t : 0); ++t) k.words.push_back((uint64_t)j.timesteps[t]);
    k.words.push_back((uint64_t)(uintptr_t)j.fitness);
    k.words.push_back((uint64_t)(uintptr_t)j.desc);
    k.words.push_back((uint64_t)(uintptr_t)j.cell);
    k.words.push_back((uint64_t)(uintptr_t)j.island);
    k.words.push_back((uint64_t)(uintptr_t)j.metrics);
  }
  return k;
}

int run_job(const tto_eval_job& j, const tto_eval_opts* o, cudaStream_t s) {
  return evaluate_impl(j.grid, j.topo, j.B, j.timesteps, j.n_t, o, j.fitness, j.desc, j.cell, j.island,
                       j.metrics, nullptr, s);
}

// Fork the jobs onto side streams after `s` and join them back into `s`.
int run_forked(const tto_eval_job* jobs, int n, const tto_eval_opts* o, cudaStream_t s, StreamPool* p) {
  TTO_CUDA_TRY(cudaEventRecord(p->fork, s));
  for (int i = 0; i < n; ++i) {
    TTO_CUDA_TRY(cudaStreamWaitEvent(p->side[i], p->fork, 0));
    int rc = run_job(jobs[i], o, p->side[i]);
    if (rc) return rc;
    TTO_CUDA_TRY(cudaEventRecord(p->join[i], p->side[i]));
    TTO_CUDA_TRY(cudaStreamWaitEvent(s, p->join[i], 0));
  }
  return TTO_OK;
}

// ------------------------------------------------------- persistent work list
unsigned int* g_counter[64] = {};  // per device: the eager persistent mode's work-list counter

// Arguments of the one-launch-per-stage evaluation of jobs (FP32 only): every
// job's evaluation arguments (no launches), its sweep items of G topologies x
// one 128-row tile, the jobs ordered by the cost of one item (largest first).
int build_multi(const tto_eval_job* jobs, int n, const tto_eval_opts* o, cudaStream_t s, unsigned int* counter,
                MultiArgs* m) {
  if (o->precision != TTO_PREC_FP32)
    return set_error(TTO_E_ARG, "the persistent work list runs the FP32 sweep (TTO_PREC_FP32) only");
  if (o->fitness_kind == TTO_FIT_F2) return set_error(TTO_E_ARG, "the persistent work list has no busbar outages");
  std::vector<EvalArgs> args(n);
  std::vector<double> cost(n);
  std::vector<unsigned long long> items(n);
  for (int i = 0; i < n; ++i) {
    const tto_eval_job& j = jobs[i];
    memset(&args[i], 0, sizeof(EvalArgs));
    int rc = evaluate_impl(j.grid, j.topo, j.B, j.timesteps, j.n_t, o, j.fitness, j.desc, j.cell, j.island,
                           j.metrics, nullptr, s, &args[i], false, true);
    if (rc) return rc;
    EvalArgs& a = args[i];
    a.n_parts = a.n_rowtiles;  // as the FP32 sweep launcher sets it
    const int G = fp32_item_group(a.TT);
    items[i] = (unsigned long long)a.n_rowtiles * ((a.B + G - 1) / G);
    cost[i] = (double)G * a.O_pad * ((a.KP <= 4 ? 4 : 8) + 2.0 * a.TT);
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  memset(m, 0, sizeof(MultiArgs));
  m->n = n;
  m->counter = counter;
  unsigned long long it = 0;
  long long blk = 0;
  for (int k = 0; k < n; ++k) {
    const int i = order[k];
    m->job[k] = args[i];
    m->item_start[k] = (unsigned int)it;
    m->blk_start[k] = (int)blk;
    it += items[i];
    blk += args[i].B;
    if (it >= 0xFFFFFFFFull || blk > 0x7FFFFFFFll) return set_error(TTO_E_ARG, "mixed batch too large for one work list");
  }
  m->item_start[n] = (unsigned int)it;
  m->blk_start[n] = (int)blk;
  m->n_items = (unsigned int)it;
  return TTO_OK;
}

int run_persistent(const MultiArgs& m, int dev, cudaStream_t s) {
  int rc = launch_split_update_multi(m, s);
  if (rc) return rc;
  if ((rc = launch_sweep_persistent(m, dev, s))) return rc;
  return launch_fitness_multi(m, s);
}

}  // namespace

void forget_grid_graphs(const tto_grid* g) {
  std::lock_guard<std::recursive_mutex> lock(g_mu);
  for (auto it = g_graphs.begin(); it != g_graphs.end();) {
    bool uses = false;
    for (uint64_t u : it->second.grids) uses = uses || u == g->uid;
    if (uses) {
      drop_entry(it->second);
      it = g_graphs.erase(it);
    } else {
      ++it;
    }
  }
}

}  // namespace tto

using namespace tto;

extern "C" int tto_grid_autotune(tto_grid* g, int32_t B, int32_t n_t, int32_t precision,
                                 int32_t* shape_out, float* ms_out, void* stream) {
  if (!g || B < 1 || n_t < 1 || n_t > TTO_MAX_T || n_t > g->T) return set_error(TTO_E_ARG, "bad autotune arguments");
  if (precision < TTO_PREC_FP32 || precision > TTO_PREC_FP16X3) return set_error(TTO_E_ARG, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  int rc = ensure_workspace(g, B, padded_T(n_t));
  if (rc) return rc;
  Workspace& w = g->ws;
  TTO_CUDA_TRY(cudaMemsetAsync(w.topo, 0xFF, (size_t)B * g->gw * sizeof(int32_t), s));
  std::vector<int32_t> tsel(n_t);
  for (int t = 0; t < n_t; ++t) tsel[t] = t;
  tto_eval_opts o{};
  o.precision = precision;
  o.fitness_kind = TTO_FIT_WORKLOAD;
  o.d_split = 8;
  o.d_moved = 8;
  cudaEvent_t e0, e1;
  TTO_CUDA_TRY(cudaEventCreate(&e0));
  TTO_CUDA_TRY(cudaEventCreate(&e1));
  const int n_shapes = sweep_shapes(precision);
  const int saved = g->tuned_shape[precision];
  int best = 0;
  float best_ms = 0.f;
  for (int sh = 0; sh < n_shapes && rc == TTO_OK; ++sh) {
    g->tuned_shape[precision] = sh;
    rc = evaluate_impl(g, w.topo, B, tsel.data(), n_t, &o, w.fit, w.desc, w.cell, w.island, nullptr, nullptr, s);
    if (rc) break;
    cudaError_t e = cudaEventRecord(e0, s);
    for (int r = 0; r < 2 && rc == TTO_OK && e == cudaSuccess; ++r)
      rc = evaluate_impl(g, w.topo, B, tsel.data(), n_t, &o, w.fit, w.desc, w.cell, w.island, nullptr, nullptr, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) rc = cuda_error(e, "autotune timing");
    ms *= 0.5f;
    if (ms_out) ms_out[sh] = ms;
    if (sh == 0 || ms < best_ms) {
      best = sh;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    g->tuned_shape[precision] = saved;
    return rc;
  }
  g->tuned_shape[precision] = best;
  if (shape_out) *shape_out = best;
  return TTO_OK;
}

extern "C" int tto_grid_set_sweep_shape(tto_grid* g, int32_t precision, int32_t shape) {
  if (!g || precision < TTO_PREC_FP32 || precision > TTO_PREC_FP16X3) return set_error(TTO_E_ARG, "bad arguments");
  if (shape < -1 || shape >= sweep_shapes(precision)) return set_error(TTO_E_ARG, "unknown sweep shape %d", shape);
  g->tuned_shape[precision] = shape;
  return TTO_OK;
}

extern "C" int tto_evaluate_multi(const tto_eval_job* jobs, int32_t n, const tto_eval_opts* opts,
                                  int32_t mode, void* stream) {
  if (!jobs || !opts || n < 1 || n > kMaxJobs) return set_error(TTO_E_ARG, "need 1..%d jobs", kMaxJobs);
  if (mode < TTO_MULTI_SEQUENTIAL || mode > TTO_MULTI_PERSISTENT_GRAPH) return set_error(TTO_E_ARG, "unknown multi mode");
  const int dev = jobs[0].grid ? jobs[0].grid->device : -1;
  for (int i = 0; i < n; ++i) {
    const tto_eval_job& j = jobs[i];
    if (!j.grid || j.grid->device != dev) return set_error(TTO_E_ARG, "job %d: grids must share one device", i);
    if (j.B < 1 || !j.topo || !j.fitness) return set_error(TTO_E_ARG, "job %d: empty batch or null buffer", i);
    for (int k = 0; k < i; ++k)
      if (jobs[k].grid == j.grid) return set_error(TTO_E_ARG, "job %d: a grid may appear once (its workspace is shared)", i);
  }
  cudaStream_t s = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(dev));
  if (mode == TTO_MULTI_SEQUENTIAL) {
    for (int i = 0; i < n; ++i) {
      int rc = run_job(jobs[i], opts, s);
      if (rc) return rc;
    }
    return TTO_OK;
  }
  std::lock_guard<std::recursive_mutex> lock(g_mu);
  if (mode == TTO_MULTI_PERSISTENT) {
    if (dev < 0 || dev >= 64) return set_error(TTO_E_ARG, "device %d out of range", dev);
    if (!g_counter[dev]) TTO_CUDA_TRY(cudaMalloc(&g_counter[dev], sizeof(unsigned int)));
    MultiArgs* m = new (std::nothrow) MultiArgs;
    if (!m) return set_error(TTO_E_NOMEM, "host allocation");
    int rc = build_multi(jobs, n, opts, s, g_counter[dev], m);
    if (rc == TTO_OK) rc = run_persistent(*m, dev, s);
    delete m;
    return rc;
  }
  StreamPool* pool = nullptr;
  int rc = stream_pool(dev, n, &pool);
  if (rc) return rc;
  if (mode == TTO_MULTI_STREAMS) return run_forked(jobs, n, opts, s, pool);

  // graph mode: replay a recorded graph of exactly these jobs, or run them
  // eagerly once and record the graph for the next call
  for (int i = 0; i < n; ++i) {
    const tto_eval_job& j = jobs[i];
    const int nt = j.timesteps ? j.n_t : j.grid->T;
    if (nt < 1 || nt > TTO_MAX_T) return set_error(TTO_E_ARG, "job %d: n_t must be in [1, %d]", i, TTO_MAX_T);
    rc = ensure_workspace(j.grid, j.B, padded_T(nt));
    if (rc) return rc;
    if (opts->precision != TTO_PREC_FP32) {
      rc = ensure_fragment_N(j.grid, s);
      if (rc) return rc;
    }
  }
  GraphKey key = make_key(jobs, n, opts, mode);
  cudaStream_t cs = pool->cap;
  TTO_CUDA_TRY(cudaEventRecord(pool->cap_in, s));
  TTO_CUDA_TRY(cudaStreamWaitEvent(cs, pool->cap_in, 0));
  auto it = g_graphs.find(key);
  if (it != g_graphs.end()) {
    TTO_CUDA_TRY(cudaGraphLaunch(it->second.exec, cs));
    TTO_CUDA_TRY(cudaEventRecord(pool->cap_out, cs));
    TTO_CUDA_TRY(cudaStreamWaitEvent(s, pool->cap_out, 0));
    return TTO_OK;
  }
  // the launch sequence of these jobs: per-grid launches on forked streams,
  // or the persistent work list (which owns a counter of its own)
  GraphEntry entry;
  MultiArgs* m = nullptr;
  if (mode == TTO_MULTI_PERSISTENT_GRAPH) {
    TTO_CUDA_TRY(cudaMalloc(&entry.counter, sizeof(unsigned int)));
    m = new (std::nothrow) MultiArgs;
    if (!m) rc = set_error(TTO_E_NOMEM, "host allocation");
    if (rc == TTO_OK) rc = build_multi(jobs, n, opts, cs, entry.counter, m);
  }
  auto record = [&]() { return m ? run_persistent(*m, dev, cs) : run_forked(jobs, n, opts, cs, pool); };
  if (rc == TTO_OK) rc = record();  // this call's results, run eagerly
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaSuccess;
  if (rc == TTO_OK) {
    e = cudaEventRecord(pool->cap_out, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, pool->cap_out, 0);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = record();
      e = cudaStreamEndCapture(cs, &graph);
    }
  }
  delete m;
  cudaGraphExec_t exec = nullptr;
  if (rc == TTO_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (rc != TTO_OK || e != cudaSuccess) {
    if (entry.counter) cudaFree(entry.counter);
    return rc != TTO_OK ? rc : cuda_error(e, "recording the mixed batch as a graph");
  }
  entry.exec = exec;
  for (int i = 0; i < n; ++i) entry.grids.push_back(jobs[i].grid->uid);
  g_graphs[key] = entry;
  return TTO_OK;
}
