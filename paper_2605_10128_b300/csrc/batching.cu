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

#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "sweep.cuh"
#include "tto_internal.h"

namespace tto {
namespace {

constexpr int kMaxJobs = 16;

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
};

std::map<GraphKey, GraphEntry> g_graphs;

GraphKey make_key(const tto_eval_job* jobs, int n, const tto_eval_opts* o) {
  GraphKey k;
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

}  // namespace

void forget_grid_graphs(const tto_grid* g) {
  std::lock_guard<std::recursive_mutex> lock(g_mu);
  for (auto it = g_graphs.begin(); it != g_graphs.end();) {
    bool uses = false;
    for (uint64_t u : it->second.grids) uses = uses || u == g->uid;
    if (uses) {
      cudaGraphExecDestroy(it->second.exec);
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
  if (mode < TTO_MULTI_SEQUENTIAL || mode > TTO_MULTI_GRAPH) return set_error(TTO_E_ARG, "unknown multi mode");
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
  GraphKey key = make_key(jobs, n, opts);
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
  rc = run_forked(jobs, n, opts, cs, pool);
  if (rc) return rc;
  TTO_CUDA_TRY(cudaEventRecord(pool->cap_out, cs));
  TTO_CUDA_TRY(cudaStreamWaitEvent(s, pool->cap_out, 0));
  TTO_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  rc = run_forked(jobs, n, opts, cs, pool);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
  GraphEntry entry;
  entry.exec = exec;
  for (int i = 0; i < n; ++i) entry.grids.push_back(jobs[i].grid->uid);
  g_graphs[key] = entry;
  return TTO_OK;
}
