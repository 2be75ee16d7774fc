// MapElites on the device: Philox-driven mutation (Algorithm 1, split and
// disconnection parts) and crossover (Algorithm 2), deterministic scatter
// insert into a one-elite-per-cell archive (Algorithm 3), and the fused
// iteration.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
// (word block, candidate, iteration lo, iteration hi).  Every decision compares
// one 32-bit word with an integer threshold computed on the host in FP64 from
// the mutation probabilities, so the draws are reproducible bit for bit by any
// implementation that follows the same word order:
//   mutation: parent word, N_mut word, then per mutation round one operation
//   word and the operation's own words (Add: slot, action; Remove: slot;
//   Change: slot, new action); then, with disconnection slots, one operation
//   word and its words (Add: slot, branch; Remove: slot; Change: branch, slot),
//   else a forced split Add (slot, action) if the genome ended empty;
//   crossover: two parent words, then per child slot (splits, then
//   disconnections) a parent word and an entry word until a part runs dry.
// The batch's mutation/crossover split b_mc is candidate 0xFFFFFFFF's first
// word.
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
  const int32_t* parents;     // archive genomes [cells][gw]
  const int32_t* filled_list; // count, then filled cells
  const int* act_off;         // [S+1]
  const int* act_st;          // [A]
  int A, k_max, n_dslot, n_disc, gw;
  uint2 key;
  uint32_t it_lo, it_hi;
  int B;
  int crossover;
  unsigned long long t_c1;    // parent-1 threshold floor(p_c1 2^32) (2^32 at p_c1 = 1)
  unsigned long long op_thr[16][4];
  unsigned long long dop_thr[16][4];
  unsigned long long poi_thr[TTO_MAX_K];
  int32_t* out;               // [B][gw]
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

// Uniform disconnection index among those not in d[0 .. nd).
__device__ int sample_free(const int* d, int nd, int n_disc, uint32_t w) {
  int ex[TTO_MAX_K], ne = 0;
  for (int i = 0; i < nd; ++i) {
    if (d[i] < 0) continue;
    int j = ne++;
    while (j > 0 && ex[j - 1] > d[i]) {
      ex[j] = ex[j - 1];
      --j;
    }
    ex[j] = d[i];
  }
  int pos = uniform_index(w, n_disc - ne);
  for (int i = 0; i < ne; ++i) {
    if (pos >= ex[i]) ++pos;
    else break;
  }
  return pos;
}

// The disconnection part of Algorithm 1 on slots d[0 .. nd), after the split
// rounds left the split slots g[0 .. k).
__device__ void mutate_disc(const int* g, int k, int* d, int nd, const MutArgs& a, Words& ws) {
  int filled[TTO_MAX_K], nfl = 0, empty[TTO_MAX_K], nem = 0;
  for (int i = 0; i < nd; ++i) {
    if (d[i] >= 0) filled[nfl++] = i;
    else empty[nem++] = i;
  }
  const int free = a.n_disc - nfl;
  int feas = 1 << kIdentity;
  if (nem > 0 && free > 0) feas |= 1 << kAdd;
  if (nfl > 0) feas |= 1 << kRemove;
  if (nfl > 0 && free > 0) feas |= 1 << kChange;
  const unsigned long long w = ws.next();
  int op = kIdentity;
  for (int i = 0; i < 4; ++i)
    if (w < a.dop_thr[feas][i]) {
      op = i;
      break;
    }
  bool no_split = true;
  for (int i = 0; i < k; ++i) no_split = no_split && g[i] < 0;
  if (nfl == 0 && no_split && ((feas >> kAdd) & 1)) op = kAdd;  // never the unchanged default
  if (op == kAdd) {
    const int slot = empty[uniform_index(ws.next(), nem)];
    d[slot] = sample_free(d, nd, a.n_disc, ws.next());
  } else if (op == kRemove) {
    d[filled[uniform_index(ws.next(), nfl)]] = -1;
  } else if (op == kChange) {
    const int x = sample_free(d, nd, a.n_disc, ws.next());
    d[filled[uniform_index(ws.next(), nfl)]] = x;
  }
}

// One part of Algorithm 2: child slots take, in turn, an entry of the
// parents' union that is feasible for the child (distinct stations for
// splits, distinct branches for disconnections); parent 1 with probability
// p_c1 when both parents offer one, a parent whose weight is zero never; the
// first slot with nothing to take ends the part.  An entry both parents hold
// counts as parent 1's.
__device__ void cross_part(const int* x1, const int* x2, int width, bool split, const MutArgs& a, Words& ws,
                           int* child) {
  int n = 0;
  for (int slot = 0; slot < width; ++slot) {
    int r1[TTO_MAX_K], n1 = 0, r2[TTO_MAX_K], n2 = 0;
    for (int pass = 0; pass < 2; ++pass) {
      const int* x = pass == 0 ? x1 : x2;
      for (int i = 0; i < width; ++i) {
        const int v = x[i];
        if (v < 0) continue;
        if (pass == 1) {
          bool in1 = false;
          for (int j = 0; j < width; ++j) in1 = in1 || x1[j] == v;
          if (in1) continue;
        }
        bool taken = false;
        for (int j = 0; j < n; ++j)
          taken = taken || (split ? a.act_st[child[j]] == a.act_st[v] : child[j] == v);
        if (taken) continue;
        if (pass == 0) r1[n1++] = v;
        else r2[n2++] = v;
      }
    }
    if (n1 == 0 && n2 == 0) break;
    const unsigned long long w = ws.next();
    bool from1;
    if (n1 > 0 && n2 > 0) {
      from1 = w < a.t_c1;
    } else if (n1 > 0) {
      if (a.t_c1 == 0) break;
      from1 = true;
    } else {
      if (a.t_c1 >= (1ull << 32)) break;
      from1 = false;
    }
    child[n++] = from1 ? r1[uniform_index(ws.next(), n1)] : r2[uniform_index(ws.next(), n2)];
  }
  for (int i = n; i < width; ++i) child[i] = -1;
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
  const int k = a.k_max, nd = a.n_dslot, gw = a.gw;
  int g[TTO_MAX_K];  // split slots, then disconnection slots
  const int nf = a.filled_list[0];
  int b_mc = a.B;
  if (a.crossover) {
    Words wr = ws;
    wr.cand = 0xFFFFFFFFu;
    b_mc = uniform_index(wr.next(), a.B + 1);
  }
  if (cand >= b_mc) {
    int p1[TTO_MAX_K], p2[TTO_MAX_K];
    const uint32_t w1 = ws.next(), w2 = ws.next();
    for (int i = 0; i < gw; ++i) {
      p1[i] = nf > 0 ? a.parents[(size_t)a.filled_list[1 + uniform_index(w1, nf)] * gw + i] : -1;
      p2[i] = nf > 0 ? a.parents[(size_t)a.filled_list[1 + uniform_index(w2, nf)] * gw + i] : -1;
    }
    cross_part(p1, p2, k, true, a, ws, g);
    if (nd > 0) cross_part(p1 + k, p2 + k, nd, false, a, ws, g + k);
    for (int i = 0; i < gw; ++i) a.out[(size_t)cand * gw + i] = g[i];
    return;
  }
  const uint32_t wp = ws.next();
  if (nf > 0) {
    const int cell = a.filled_list[1 + uniform_index(wp, nf)];
    for (int i = 0; i < gw; ++i) g[i] = a.parents[(size_t)cell * gw + i];
  } else {
    for (int i = 0; i < gw; ++i) g[i] = -1;
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
  if (nd > 0 && a.n_disc > 0) {
    mutate_disc(g, k, g + k, nd, a, ws);
  } else {
    bool empty = true;
    for (int i = 0; i < k; ++i) empty = empty && g[i] < 0;
    if (empty) do_add(g, k, a, ws);
  }
  for (int i = 0; i < gw; ++i) a.out[(size_t)cand * gw + i] = g[i];
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
                                    int B, int cells, int gw, const unsigned long long* key,
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
  for (int j = 0; j < gw; ++j) agen[(size_t)c * gw + j] = topo[(size_t)i * gw + j];
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
// With identity_fallback, a subset where no feasible operation has weight
// draws Identity.
void op_thresholds(const double p[4], bool identity_fallback, unsigned long long thr[16][4]) {
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
    if (last < 0 && identity_fallback) {
      for (int i = 0; i < 4; ++i) thr[f][i] = i == kIdentity ? 1ull << 32 : 0ull;
      continue;
    }
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
  const double dp[4] = {mp->dp_add, mp->dp_remove, mp->dp_change, mp->dp_identity};
  for (double x : dp)
    if (!(x >= 0.0) || !isfinite(x)) return set_error(TTO_E_ARG, "disconnection probabilities must be >= 0");
  if (mp->crossover != 0 && mp->crossover != 1) return set_error(TTO_E_ARG, "crossover must be 0 or 1");
  if (!(mp->p_c1 >= 0.0 && mp->p_c1 <= 1.0)) return set_error(TTO_E_ARG, "p_c1 must be in [0, 1]");
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
  a.n_dslot = g->n_dslot;
  a.n_disc = g->n_disc;
  a.gw = g->gw;
  a.crossover = mp->crossover;
  a.t_c1 = mp->p_c1 >= 1.0 ? (1ull << 32) : (unsigned long long)floor(mp->p_c1 * 4294967296.0);
  a.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  a.it_lo = (uint32_t)it;
  a.it_hi = (uint32_t)(it >> 32);
  a.B = B;
  const double p[4] = {mp->p_add, mp->p_remove, mp->p_change, mp->p_identity};
  const double dp[4] = {mp->dp_add, mp->dp_remove, mp->dp_change, mp->dp_identity};
  op_thresholds(p, false, a.op_thr);
  op_thresholds(dp, true, a.dop_thr);
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
  insert_apply_kernel<<<(B + 255) / 256, 256, 0, s>>>(fit, cell, topo, B, cells, ar->g->gw,
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
  return tto_archive_create_ex(g, d_split, d_moved, 1, out);
}

int tto_archive_create_ex(tto_grid* g, int32_t d_split, int32_t d_moved, int32_t d_disc, tto_archive** out) {
  if (!g || !out || d_split < 1 || d_moved < 1 || d_disc < 1) return set_error(TTO_E_ARG, "bad archive arguments");
  if ((int64_t)d_split * d_moved * d_disc > (1 << 24)) return set_error(TTO_E_ARG, "more than 2^24 archive cells");
  *out = nullptr;
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  tto_archive* a = new (std::nothrow) tto_archive();
  if (!a) return set_error(TTO_E_NOMEM, "host allocation failed");
  a->g = g;
  a->d_split = d_split;
  a->d_moved = d_moved;
  a->d_disc = d_disc;
  a->cells = d_split * d_moved * d_disc;
  const size_t C = a->cells;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&a->d_fit, C * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&a->d_genome, C * g->gw * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&a->d_filled, C);
  if (e == cudaSuccess) e = cudaMalloc(&a->d_key, C * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&a->d_filled_list, (C + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(a->d_filled, 0, C);
  if (e == cudaSuccess) e = cudaMemset(a->d_filled_list, 0, (C + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(a->d_genome, 0xFF, C * g->gw * sizeof(int32_t));
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
  free_epoch(a);
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
  if (genome) TTO_CUDA_TRY(cudaMemcpy(genome, a->d_genome, C * a->g->gw * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (filled) TTO_CUDA_TRY(cudaMemcpy(filled, a->d_filled, C, cudaMemcpyDeviceToHost));
  return TTO_OK;
}

int tto_archive_import(tto_archive* a, const float* fitness, const int32_t* genome,
                       const uint8_t* filled) {
  if (!a || !fitness || !genome || !filled) return set_error(TTO_E_ARG, "null argument");
  const size_t C = a->cells;
  const int k = a->g->gw;
  for (size_t c = 0; c < C; ++c) {
    if (!filled[c]) continue;
    if (!isfinite(fitness[c])) return set_error(TTO_E_ARG, "filled cell %zu has non-finite fitness", c);
    for (int j = 0; j < k; ++j) {
      const int v = genome[c * k + j];
      const int hi = j < a->g->k_max ? a->g->A : a->g->n_disc;
      if (v < -1 || v >= hi) return set_error(TTO_E_ARG, "cell %zu slot %d holds invalid id %d", c, j, v);
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
  if (opts->d_split != a->d_split || opts->d_moved != a->d_moved || (opts->d_disc > 1 ? opts->d_disc : 1) != a->d_disc)
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
    TTO_CUDA_TRY(cudaMemcpyAsync(topo_out, w.topo, (size_t)B * g->gw * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
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
