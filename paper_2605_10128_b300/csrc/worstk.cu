// Worst-k N-1 export for the AC validation stage (Sec. "AC-Validator": the DC
// optimiser computes every N-1 case's overload energy and writes out the worst
// k cases so that the AC loadflows can start with them).
//
// After the split update of the requested topologies (U, V, f', g in the
// evaluation workspace, as for tto_evaluate_batch):
//   1. outage_energy_kernel: for every (topology, outage c)
//        E_c = sum_t sum_l max(|F_lc[t]| - lim_l, 0),
//        F_lc[t] = f'_l[t] - (N_lc - U_l . V_c) g_c[t]   (FP32, CUDA cores),
//      NaN for an outage that islands the topology or whose branch it opened
//      (g = NaN there).  One thread per outage column and kEG topologies walks
//      all monitored rows in a fixed order (deterministic sums); the rows' U,
//      f' and limits are staged in shared memory per tile, the thread's V and g
//      stay in registers, and N_lc is read coalesced along c.
//   2. worst_k_kernel: per topology, k rounds of a block-wide selection of the
//      next outage in the order (energy descending, index ascending), each
//      round taking the best entry that follows the previous pick in that
//      order; NaN never qualifies, missing picks are -1 / NaN.
// Both kernels are plain loops with no waits; the export is meant for the
// archive's elites at the end of an epoch, not for every candidate.
#include <math.h>

#include "sweep.cuh"
#include "tto_internal.h"

namespace tto {

namespace {

constexpr int kEG = 4;         // topologies per thread
constexpr int kEThreads = 128;  // outage columns per CTA
constexpr int kERows = 32;     // monitored rows staged per tile

template <int TT>
__global__ void __launch_bounds__(kEThreads) outage_energy_kernel(EvalArgs a, float* energy, const uint8_t* use) {
  __shared__ __align__(16) float sU[kEG][kERows][8];
  __shared__ float sF[kEG][kERows][TT];
  __shared__ float sL[kERows];
  const int tid = threadIdx.x;
  const int c = blockIdx.x * kEThreads + tid;
  const int b0 = blockIdx.y * kEG;
  const float qnan = __int_as_float(0x7fc00000);
  if (use) {  // CTA-uniform: a group of topologies that are all unused writes NaN and leaves
    bool any = false;
    for (int gi = 0; gi < kEG && b0 + gi < a.B; ++gi) any = any || use[b0 + gi];
    if (!any) {
      for (int gi = 0; gi < kEG && b0 + gi < a.B && c < a.O; ++gi) energy[(size_t)(b0 + gi) * a.O + c] = qnan;
      return;
    }
  }
  const int Ep = a.E_mon_pad, Op = a.O_pad;
  const int cc = c < Op ? c : Op - 1;  // idle columns still join the staging
  float v[kEG][8], g[kEG][TT], e[kEG];
#pragma unroll
  for (int gi = 0; gi < kEG; ++gi) {
    const int bb = min(b0 + gi, a.B - 1);
    const float* vr = a.V + ((size_t)bb * Op + cc) * 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) v[gi][j] = vr[j];
#pragma unroll
    for (int t = 0; t < TT; ++t) g[gi][t] = a.gg[((size_t)bb * Op + cc) * TT + t];
    e[gi] = 0.f;
  }
  for (int l0 = 0; l0 < a.E_mon; l0 += kERows) {
    const int nr = min(kERows, a.E_mon - l0);
    __syncthreads();
    for (int i = tid; i < kEG * kERows * 8; i += kEThreads) {
      const int gi = i / (kERows * 8), r = (i / 8) % kERows, j = i % 8;
      const int bb = min(b0 + gi, a.B - 1);
      sU[gi][r][j] = r < nr ? a.U[((size_t)bb * Ep + l0 + r) * 8 + j] : 0.f;
    }
    for (int i = tid; i < kEG * kERows * TT; i += kEThreads) {
      const int gi = i / (kERows * TT), r = (i / TT) % kERows, t = i % TT;
      const int bb = min(b0 + gi, a.B - 1);
      sF[gi][r][t] = r < nr ? a.fp[((size_t)bb * TT + t) * Ep + l0 + r] : 0.f;
    }
    if (tid < kERows) sL[tid] = tid < nr ? a.lim[l0 + tid] : 1.f;
    __syncthreads();
#pragma unroll 4  // several rows' N loads in flight at once
    for (int r = 0; r < nr; ++r) {
      const float n = a.Nmo[(size_t)(l0 + r) * Op + cc];
      const float lim = sL[r];
#pragma unroll
      for (int gi = 0; gi < kEG; ++gi) {
        float d = n;
#pragma unroll
        for (int j = 0; j < 8; ++j) d = fmaf(-sU[gi][r][j], v[gi][j], d);
#pragma unroll
        for (int t = 0; t < TT; ++t) e[gi] += fmaxf(fabsf(fmaf(-d, g[gi][t], sF[gi][r][t])) - lim, 0.f);
      }
    }
  }
  if (c >= a.O) return;
#pragma unroll
  for (int gi = 0; gi < kEG; ++gi) {
    const int b = b0 + gi;
    if (b < a.B) energy[(size_t)b * a.O + c] = (isnan(g[gi][0]) || (use && !use[b])) ? qnan : e[gi];
  }
}

// (v1, i1) precedes (v2, i2): larger energy first, lower index among equals.
__device__ __forceinline__ bool before(float v1, int i1, float v2, int i2) {
  return v1 > v2 || (v1 == v2 && i1 < i2);
}

__global__ void __launch_bounds__(256) worst_k_kernel(const float* energy, int O, int k, int32_t* idx_out,
                                                      float* val_out) {
  __shared__ float sv[8];
  __shared__ int si[8];
  __shared__ float last_v;
  __shared__ int last_i;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* e = energy + (size_t)b * O;
  if (tid == 0) {
    last_v = INFINITY;
    last_i = -1;
  }
  __syncthreads();
  for (int r = 0; r < k; ++r) {
    const float lv = last_v;
    const int li = last_i;
    float bv = -INFINITY;
    int bi = -1;
    for (int c = tid; c < O; c += blockDim.x) {
      const float x = e[c];
      if (isnan(x) || !before(lv, li, x, c)) continue;  // only entries after the previous pick
      if (bi < 0 || before(x, c, bv, bi)) {
        bv = x;
        bi = c;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi >= 0 && (bi < 0 || before(ov, oi, bv, bi))) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      sv[warp] = bv;
      si[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      float v = -INFINITY;
      int i = -1;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        if (si[w] >= 0 && (i < 0 || before(sv[w], si[w], v, i))) {
          v = sv[w];
          i = si[w];
        }
      idx_out[(size_t)b * k + r] = i;
      val_out[(size_t)b * k + r] = i >= 0 ? v : __int_as_float(0x7fc00000);
      if (i >= 0) {
        last_v = v;
        last_i = i;
      } else {
        last_v = -INFINITY;  // nothing left: later rounds find nothing either
        last_i = 0x7fffffff;
      }
    }
    __syncthreads();
  }
}

template <int TT>
int launch_energy(const EvalArgs& a, float* energy, const uint8_t* use, cudaStream_t s) {
  if ((a.B + kEG - 1) / kEG > 65535) return set_error(TTO_E_ARG, "at most %d topologies per worst-k call", 65535 * kEG);
  const dim3 grid((unsigned)((a.O_pad + kEThreads - 1) / kEThreads), (unsigned)((a.B + kEG - 1) / kEG));
  outage_energy_kernel<TT><<<grid, kEThreads, 0, s>>>(a, energy, use);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

}  // namespace

// use (device, may be NULL): topologies b with use[b] == 0 are skipped (their
// energies NaN, their lists -1), as the epoch export does for empty cells.
int worst_k_impl(tto_grid* g, const int32_t* topo, int32_t n, const int32_t* timesteps, int32_t n_t, int32_t k,
                 int32_t* outage_out, float* energy_out, float* all_energy, const uint8_t* use, cudaStream_t s);

}  // namespace tto

using namespace tto;

extern "C" int tto_worst_k(tto_grid* g, const int32_t* topo, int32_t n, const int32_t* timesteps, int32_t n_t,
                           int32_t k, int32_t* outage_out, float* energy_out, float* all_energy, void* stream) {
  return worst_k_impl(g, topo, n, timesteps, n_t, k, outage_out, energy_out, all_energy, nullptr,
                      (cudaStream_t)stream);
}

int tto::worst_k_impl(tto_grid* g, const int32_t* topo, int32_t n, const int32_t* timesteps, int32_t n_t,
                      int32_t k, int32_t* outage_out, float* energy_out, float* all_energy, const uint8_t* use,
                      cudaStream_t s) {
  if (!g) return set_error(TTO_E_ARG, "null grid");
  if (n < 0 || k < 1 || k > 1024) return set_error(TTO_E_ARG, "need n >= 0 and 1 <= k <= 1024");
  if (n > 0 && (!topo || !outage_out || !energy_out)) return set_error(TTO_E_ARG, "null buffer");
  if (n == 0) return TTO_OK;
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  const int TT = padded_T(timesteps ? n_t : g->T);
  if (TT < 0) return set_error(TTO_E_ARG, "at most %d timesteps", TTO_MAX_T);
  int rc = ensure_workspace(g, n, TT);  // the same size evaluate_impl asks for: no reallocation there
  if (rc) return rc;
  tto_eval_opts o{};
  o.precision = TTO_PREC_FP32;
  o.fitness_kind = TTO_FIT_WORKLOAD;
  o.d_split = 1;
  o.d_moved = 1;
  EvalArgs a;
  rc = evaluate_impl(g, topo, n, timesteps, n_t, &o, g->ws.fit, nullptr, nullptr, nullptr, nullptr, nullptr, s, &a);
  if (rc) return rc;
  // all_energy (caller's [n][n_outage]) or scratch: the tensor-core sweep's g
  // staging buffer (B x O_pad x TT floats), which the FP32 split update leaves unused
  float* energy = all_energy ? all_energy : g->ws.gq;
  switch (a.TT) {
    case 1: rc = launch_energy<1>(a, energy, use, s); break;
    case 2: rc = launch_energy<2>(a, energy, use, s); break;
    case 4: rc = launch_energy<4>(a, energy, use, s); break;
    case 8: rc = launch_energy<8>(a, energy, use, s); break;
    case 16: rc = launch_energy<16>(a, energy, use, s); break;
    case 24: rc = launch_energy<24>(a, energy, use, s); break;
    case 32: rc = launch_energy<32>(a, energy, use, s); break;
    default: return set_error(TTO_E_ARG, "unsupported timestep count %d", a.TT);
  }
  if (rc) return rc;
  worst_k_kernel<<<n, 256, 0, s>>>(energy, a.O, k, outage_out, energy_out);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}
