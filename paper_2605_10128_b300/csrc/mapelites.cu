// MapElites on the device: Philox-driven split mutation (Algorithm 1, action
// part), deterministic scatter insert into a one-elite-per-cell archive
// (Algorithm 3), and the fused iteration.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
// (word block, candidate, iteration lo, iteration hi).  Every decision compares
// one 32-bit word with an integer threshold computed on the host in FP64 from
// the mutation probabilities, so the draws are reproducible bit for bit by any
// implementation that follows the same word order:
//   parent word, N_mut word, then per mutation round one operation word and the
//   operation's own words (Add: slot, action; Remove: slot; Change: slot, new
//   action), and a final forced Add (slot, action) if the genome ended empty.
#include <math.h>
#include <string.h>

#include "philox.cuh"
#include "sweep.cuh"
#include "tto_internal.h"

namespace tto {

namespace {

enum { kAdd = 0, kRemove = 1, kChange = 2, kIdentity = 3 };

struct Words {
  uint2 key;
  uint32_t cand, it_lo, it_hi, block, idx;
  uint4 buf;
  __device__ uint32_t next() {
    if (idx == 4) {
      buf = philox4x32_10(make_uint4(block, cand, it_lo, it_hi), key);
      ++block;
      idx = 0;
    }
    const uint32_t w = idx == 0 ? buf.x : (idx == 1 ? buf.y : (idx == 2 ? buf.z : buf.w));
    ++idx;
    return w;
  }
};

__device__ __forceinline__ int uniform_index(uint32_t w, int n) {
  return (int)(((uint64_t)w * (uint32_t)n) >> 32);
}

struct MutArgs {
  const int32_t* parents;     // archive genomes [cells][k_max]
  const int32_t* filled_list; // count, then filled cells
  const int* act_off;         // [S+1]
  const int* act_st;          // [A]
  int A, k_max;
  uint2 key;
  uint32_t it_lo, it_hi;
  int B;
  unsigned long long op_thr[16][4];
  unsigned long long poi_thr[TTO_MAX_K];
  int32_t* out;               // [B][k_max]
};

__device__ int sample_allowed(const int* g, int k, const MutArgs& a, uint32_t w) {
  int ex[TTO_MAX_K];
  int ne = 0, allowed = a.A;
  for (int i = 0; i < k; ++i) {
    if (g[i] < 0) continue;
    const int s = a.act_st[g[i]];
    int j = ne++;
    while (j > 0 && ex[j - 1] > s) {
      ex[j] = ex[j - 1];
      --j;
    }
    ex[j] = s;
    allowed -= a.act_off[s + 1] - a.act_off[s];
  }
  int pos = uniform_index(w, allowed);
  for (int i = 0; i < ne; ++i) {
    const int s = ex[i];
    if (pos >= a.act_off[s]) pos += a.act_off[s + 1] - a.act_off[s];
    else break;
  }
  return pos;
}

__device__ void do_add(int* g, int k, const MutArgs& a, Words& ws) {
  int empty[TTO_MAX_K], ne = 0;
  for (int i = 0; i < k; ++i)
    if (g[i] < 0) empty[ne++] = i;
  const int slot = empty[uniform_index(ws.next(), ne)];
  g[slot] = sample_allowed(g, k, a, ws.next());
}

__global__ void propose_kernel(MutArgs a) {
  const int cand = blockIdx.x * blockDim.x + threadIdx.x;
  if (cand >= a.B) return;
  Words ws;
  ws.key = a.key;
  ws.cand = (uint32_t)cand;
  ws.it_lo = a.it_lo;
  ws.it_hi = a.it_hi;
  ws.block = 0;
  ws.idx = 4;
  const int k = a.k_max;
  int g[TTO_MAX_K];
  const int nf = a.filled_list[0];
  const uint32_t wp = ws.next();
  if (nf > 0) {
    const int cell = a.filled_list[1 + uniform_index(wp, nf)];
    for (int i = 0; i < k; ++i) g[i] = a.parents[(size_t)cell * k + i];
  } else {
    for (int i = 0; i < k; ++i) g[i] = -1;
  }
  // N_mut ~ clip(Poisson(mean), 1, k_max) by inversion
  const uint32_t wn = ws.next();
  int nmut = k;
  for (int j = 0; j < k; ++j)
    if ((unsigned long long)wn < a.poi_thr[j]) {
      nmut = j;
      break;
    }
  nmut = max(1, min(nmut, k));
  for (int r = 0; r < nmut; ++r) {
    int filled[TTO_MAX_K], nfl = 0, chg[TTO_MAX_K], nch = 0, nempty = 0, allowed = a.A;
    for (int i = 0; i < k; ++i) {
      if (g[i] < 0) {
        ++nempty;
        continue;
      }
      filled[nfl++] = i;
      const int s = a.act_st[g[i]];
      const int cnt = a.act_off[s + 1] - a.act_off[s];
      allowed -= cnt;
      if (cnt >= 2) chg[nch++] = i;
    }
    int feas = 1 << kIdentity;
    if (nempty > 0 && allowed > 0) feas |= 1 << kAdd;
    if (nfl > 0) feas |= 1 << kRemove;
    if (nch > 0) feas |= 1 << kChange;
    const unsigned long long w = ws.next();
    int op = kIdentity;
    for (int i = 0; i < 4; ++i)
      if (w < a.op_thr[feas][i]) {
        op = i;
        break;
      }
    if (op == kAdd) {
      do_add(g, k, a, ws);
    } else if (op == kRemove) {
      g[filled[uniform_index(ws.next(), nfl)]] = -1;
    } else if (op == kChange) {
      const int slot = chg[uniform_index(ws.next(), nch)];
      const int s = a.act_st[g[slot]];
      const int off = a.act_off[s], cnt = a.act_off[s + 1] - off;
      const int cur = g[slot] - off;
      const int rr = uniform_index(ws.next(), cnt - 1);
      g[slot] = off + rr + (rr >= cur ? 1 : 0);
    }
  }
  bool empty = true;
  for (int i = 0; i < k; ++i) empty = empty && g[i] < 0;
  if (empty) do_add(g, k, a, ws);
  for (int i = 0; i < k; ++i) a.out[(size_t)cand * k + i] = g[i];
}

__global__ void philox_blocks_kernel(uint2 key, uint32_t cand, uint32_t it_lo, uint32_t it_hi,
                                     uint32_t block, int n, uint32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox4x32_10(make_uint4(block + (uint32_t)i, cand, it_lo, it_hi), key);
  out[4 * i + 0] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

__device__ __forceinline__ uint32_t orderable(float f) {
  const uint32_t u = __float_as_uint(f + 0.0f);  // -0 -> +0
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void key_reset_kernel(unsigned long long* key, int cells) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cells) key[i] = 0ull;
}

__global__ void insert_key_kernel(const float* fit, const int32_t* cell, int B, int cells,
                                  unsigned long long* key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const float f = fit[i];
  const int c = cell[i];
  if (!isfinite(f) || c < 0 || c >= cells) return;
  const unsigned long long k = ((unsigned long long)orderable(f) << 32) | (0xFFFFFFFFu - (uint32_t)i);
  atomicMax(key + c, k);
}

__global__ void insert_apply_kernel(const float* fit, const int32_t* cell, const int32_t* topo,
                                    int B, int cells, int k_max, const unsigned long long* key,
                                    float* afit, int32_t* agen, uint8_t* afilled) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const float f = fit[i];
  const int c = cell[i];
  if (!isfinite(f) || c < 0 || c >= cells) return;
  const unsigned long long k = ((unsigned long long)orderable(f) << 32) | (0xFFFFFFFFu - (uint32_t)i);
  if (key[c] != k) return;  // not this cell's batch winner
  if (afilled[c] && !(f > afit[c])) return;
  afit[c] = f;
  for (int j = 0; j < k_max; ++j) agen[(size_t)c * k_max + j] = topo[(size_t)i * k_max + j];
  afilled[c] = 1;
}

__global__ void filled_list_kernel(const uint8_t* filled, int cells, int32_t* list) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int n = 0;
  for (int c = 0; c < cells; ++c)
    if (filled[c]) list[1 + n++] = c;
  list[0] = n;
}

// Cumulative uint32 thresholds (2^32 for the last feasible operation) of the
// operation draw, for each feasibility subset of {Add, Remove, Change, Identity}.
void op_thresholds(const tto_mut_params* mp, unsigned long long thr[16][4]) {
  const double p[4] = {mp->p_add, mp->p_remove, mp->p_change, mp->p_identity};
  for (int f = 0; f < 16; ++f) {
    double w[4], cum[4], acc = 0.0;
    int last = -1;
    for (int i = 0; i < 4; ++i) {
      w[i] = ((f >> i) & 1) ? p[i] : 0.0;
      acc = acc + w[i];
      cum[i] = acc;
      if (w[i] > 0.0) last = i;
    }
    const double total = cum[3];
    for (int i = 0; i < 4; ++i) {
      if (last < 0 || i >= last)
        thr[f][i] = 1ull << 32;
      else
        thr[f][i] = (unsigned long long)floor(cum[i] / total * 4294967296.0);
    }
  }
}

// floor(CDF(j) * 2^32) of Poisson(mean), pmf by p_0 = e^-mean, p_j = p_{j-1} mean / j.
void poisson_thresholds(double mean, int k, unsigned long long* thr) {
  double pmf = exp(-mean), cdf = pmf;
  thr[0] = (unsigned long long)floor(cdf * 4294967296.0);
  for (int j = 1; j < k; ++j) {
    pmf = pmf * mean / j;
    cdf = cdf + pmf;
    thr[j] = (unsigned long long)floor(cdf * 4294967296.0);
  }
}

int check_mut(const tto_mut_params* mp) {
  if (!mp) return set_error(TTO_E_ARG, "null mutation parameters");
  const double p[4] = {mp->p_add, mp->p_remove, mp->p_change, mp->p_identity};
  for (double x : p)
    if (!(x >= 0.0) || !isfinite(x)) return set_error(TTO_E_ARG, "mutation probabilities must be >= 0");
  if (!(mp->p_identity > 0.0) && !(mp->p_add > 0.0 && mp->p_remove > 0.0))
    return set_error(TTO_E_ARG, "some operation must be feasible for every genome (p_identity > 0, or p_add and p_remove > 0)");
  if (!(mp->n_mut_mean >= 0.0) || !isfinite(mp->n_mut_mean)) return set_error(TTO_E_ARG, "n_mut_mean must be >= 0");
  return TTO_OK;
}

}  // namespace

int propose_impl(tto_archive* ar, uint64_t seed, uint64_t it, int B, const tto_mut_params* mp,
                 int32_t* out, cudaStream_t s) {
  int rc = check_mut(mp);
  if (rc) return rc;
  tto_grid* g = ar->g;
  if (g->A < 1) return set_error(TTO_E_ARG, "the grid has no actions");
  MutArgs a;
  memset(&a, 0, sizeof(a));
  a.parents = ar->d_genome;
  a.filled_list = ar->d_filled_list;
  a.act_off = g->d_act_off;
  a.act_st = g->d_act_st;
  a.A = g->A;
  a.k_max = g->k_max;
  a.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  a.it_lo = (uint32_t)it;
  a.it_hi = (uint32_t)(it >> 32);
  a.B = B;
  op_thresholds(mp, a.op_thr);
  poisson_thresholds(mp->n_mut_mean, g->k_max, a.poi_thr);
  a.out = out;
  if (B > 0) {
    propose_kernel<<<(B + 127) / 128, 128, 0, s>>>(a);
    TTO_CUDA_TRY(cudaGetLastError());
  }
  return TTO_OK;
}

int insert_impl(tto_archive* ar, const int32_t* topo, int B, const float* fit, const int32_t* cell,
                cudaStream_t s) {
  if (B <= 0) return TTO_OK;
  const int cells = ar->cells;
  key_reset_kernel<<<(cells + 255) / 256, 256, 0, s>>>(ar->d_key, cells);
  insert_key_kernel<<<(B + 255) / 256, 256, 0, s>>>(fit, cell, B, cells, ar->d_key);
  insert_apply_kernel<<<(B + 255) / 256, 256, 0, s>>>(fit, cell, topo, B, cells, ar->g->k_max,
                                                      ar->d_key, ar->d_fit, ar->d_genome,
                                                      ar->d_filled);
  filled_list_kernel<<<1, 32, 0, s>>>(ar->d_filled, cells, ar->d_filled_list);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

}  // namespace tto

using namespace tto;

extern "C" {

int tto_archive_create(tto_grid* g, int32_t d_split, int32_t d_moved, tto_archive** out) {
  if (!g || !out || d_split < 1 || d_moved < 1) return set_error(TTO_E_ARG, "bad archive arguments");
  *out = nullptr;
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  tto_archive* a = new (std::nothrow) tto_archive();
  if (!a) return set_error(TTO_E_NOMEM, "host allocation failed");
  a->g = g;
  a->d_split = d_split;
  a->d_moved = d_moved;
  a->cells = d_split * d_moved;
  const size_t C = a->cells;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&a->d_fit, C * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&a->d_genome, C * g->k_max * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&a->d_filled, C);
  if (e == cudaSuccess) e = cudaMalloc(&a->d_key, C * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&a->d_filled_list, (C + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(a->d_filled, 0, C);
  if (e == cudaSuccess) e = cudaMemset(a->d_filled_list, 0, (C + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(a->d_genome, 0xFF, C * g->k_max * sizeof(int32_t));
  if (e == cudaSuccess) {
    std::vector<float> ninf(C, -INFINITY);
    e = cudaMemcpy(a->d_fit, ninf.data(), C * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    tto_archive_destroy(a);
    return cuda_error(e, "archive allocation");
  }
  *out = a;
  return TTO_OK;
}

int tto_archive_destroy(tto_archive* a) {
  if (!a) return TTO_OK;
  cudaSetDevice(a->g->device);
  void* ptrs[] = {a->d_fit, a->d_genome, a->d_filled, a->d_key, a->d_filled_list};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete a;
  return TTO_OK;
}

int tto_archive_export(const tto_archive* a, float* fitness, int32_t* genome, uint8_t* filled) {
  if (!a) return set_error(TTO_E_ARG, "null archive");
  TTO_CUDA_TRY(cudaSetDevice(a->g->device));
  TTO_CUDA_TRY(cudaDeviceSynchronize());
  const size_t C = a->cells;
  if (fitness) TTO_CUDA_TRY(cudaMemcpy(fitness, a->d_fit, C * sizeof(float), cudaMemcpyDeviceToHost));
  if (genome) TTO_CUDA_TRY(cudaMemcpy(genome, a->d_genome, C * a->g->k_max * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (filled) TTO_CUDA_TRY(cudaMemcpy(filled, a->d_filled, C, cudaMemcpyDeviceToHost));
  return TTO_OK;
}

int tto_archive_import(tto_archive* a, const float* fitness, const int32_t* genome,
                       const uint8_t* filled) {
  if (!a || !fitness || !genome || !filled) return set_error(TTO_E_ARG, "null argument");
  const size_t C = a->cells;
  const int k = a->g->k_max;
  for (size_t c = 0; c < C; ++c) {
    if (!filled[c]) continue;
    if (!isfinite(fitness[c])) return set_error(TTO_E_ARG, "filled cell %zu has non-finite fitness", c);
    for (int j = 0; j < k; ++j) {
      int act = genome[c * k + j];
      if (act < -1 || act >= a->g->A) return set_error(TTO_E_ARG, "cell %zu holds invalid action %d", c, act);
    }
  }
  TTO_CUDA_TRY(cudaSetDevice(a->g->device));
  TTO_CUDA_TRY(cudaDeviceSynchronize());
  TTO_CUDA_TRY(cudaMemcpy(a->d_fit, fitness, C * sizeof(float), cudaMemcpyHostToDevice));
  TTO_CUDA_TRY(cudaMemcpy(a->d_genome, genome, C * k * sizeof(int32_t), cudaMemcpyHostToDevice));
  TTO_CUDA_TRY(cudaMemcpy(a->d_filled, filled, C, cudaMemcpyHostToDevice));
  filled_list_kernel<<<1, 32>>>(a->d_filled, (int)C, a->d_filled_list);
  TTO_CUDA_TRY(cudaGetLastError());
  TTO_CUDA_TRY(cudaDeviceSynchronize());
  return TTO_OK;
}

int tto_archive_insert(tto_archive* a, const int32_t* topo, int32_t B, const float* fitness,
                       const int32_t* cell, void* stream) {
  if (!a || B < 0 || (B > 0 && (!topo || !fitness || !cell))) return set_error(TTO_E_ARG, "bad insert arguments");
  TTO_CUDA_TRY(cudaSetDevice(a->g->device));
  return insert_impl(a, topo, B, fitness, cell, (cudaStream_t)stream);
}

int tto_mapelites_propose(tto_archive* a, uint64_t seed, uint64_t iteration, int32_t B,
                          const tto_mut_params* mp, int32_t* topo_out, void* stream) {
  if (!a || B < 0 || (B > 0 && !topo_out)) return set_error(TTO_E_ARG, "bad propose arguments");
  TTO_CUDA_TRY(cudaSetDevice(a->g->device));
  return propose_impl(a, seed, iteration, B, mp, topo_out, (cudaStream_t)stream);
}

int tto_mapelites_step(tto_archive* a, uint64_t seed, uint64_t iteration, int32_t B,
                       const tto_mut_params* mp, const tto_eval_opts* opts, int32_t* topo_out,
                       float* fitness_out, void* stream) {
  if (!a || !opts || B < 1) return set_error(TTO_E_ARG, "bad step arguments");
  if (opts->d_split != a->d_split || opts->d_moved != a->d_moved)
    return set_error(TTO_E_ARG, "evaluation cell extents differ from the archive's");
  tto_grid* g = a->g;
  cudaStream_t s = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  if (g->T > TTO_MAX_T) return set_error(TTO_E_ARG, "grid has more than %d timesteps", TTO_MAX_T);
  int rc = ensure_workspace(g, B, padded_T(g->T));
  if (rc) return rc;
  Workspace& w = g->ws;
  rc = propose_impl(a, seed, iteration, B, mp, w.topo, s);
  if (rc) return rc;
  rc = evaluate_impl(g, w.topo, B, nullptr, g->T, opts, w.fit, w.desc, w.cell, w.island, nullptr,
                     nullptr, s);
  if (rc) return rc;
  rc = insert_impl(a, w.topo, B, w.fit, w.cell, s);
  if (rc) return rc;
  if (topo_out)
    TTO_CUDA_TRY(cudaMemcpyAsync(topo_out, w.topo, (size_t)B * g->k_max * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (fitness_out)
    TTO_CUDA_TRY(cudaMemcpyAsync(fitness_out, w.fit, (size_t)B * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return TTO_OK;
}

int tto_philox_blocks(uint64_t seed, uint64_t iteration, uint32_t cand, uint32_t block, int32_t n,
                      uint32_t* out, void* stream) {
  if (n < 0 || (n > 0 && !out)) return set_error(TTO_E_ARG, "bad philox arguments");
  if (n == 0) return TTO_OK;
  philox_blocks_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), cand, (uint32_t)iteration,
      (uint32_t)(iteration >> 32), block, n, out);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

}  // extern "C"
