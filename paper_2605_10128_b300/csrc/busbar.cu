// Busbar outage sweep (Sec. "Fitness function heuristics": lambda_b =
// sum_e Pi(max_{b in O_b} |f_e^(b)| - fbar_e); lambda_f2 in Sec. "High-level
// Genetic Algorithm loop").
//
// The split update writes one record per (topology, busbar node) (see
// busbar_setup in evaluate.cu): station s, the N columns of the node's other
// branches R', the node's injection p_v[t], and z[t], y[t] of
//   F_l[t] = f'_l[t] - p_v[t] pi_s,l - sum_j N_{l r_j} z_j[t] - U_l . y[t].
// This kernel evaluates F for every monitored row and keeps the running
// maximum over the busbar outages per (row, timestep), on the CUDA cores in
// FP32.  A thread takes R adjacent rows of G topologies (R = 2, G = 1 up to 8
// timesteps: CTA = 64 threads = 128 rows x 1 topology).  The records are
// staged kBVB at a time in shared memory as float4s, and each record's
// broadcast loads (indices, p_v, z, y) then serve the thread's R rows.  The
// thread's U rows and f' stay in registers.  N_{l r_j} and pi_s,l are read
// R rows at a time from column-major FP32 tables, coalesced along the rows.
// Each CTA reduces its rows to one partial lambda_b per topology in a fixed
// order (no atomics).
#include <math.h>

#include "sweep.cuh"
#include "tto_internal.h"

namespace tto {

namespace {

constexpr int kBRows = 128;
constexpr int kBVB = 16;  // busbar records staged per round

// R adjacent monitored rows per thread (R = 1 or 2): the per-record shared
// loads (indices, p_v, z, y) serve R rows, and the N and pi reads become
// R-wide vector loads.
template <int R>
struct RowVec;
template <>
struct RowVec<1> {
  __device__ static void load(const float* p, float* x) { x[0] = *p; }
  __device__ static void store(float* p, const float* x) { *p = x[0]; }
};
template <>
struct RowVec<2> {
  __device__ static void load(const float* p, float* x) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    x[0] = v.x;
    x[1] = v.y;
  }
  __device__ static void store(float* p, const float* x) { *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]); }
};

template <int TT, int G, int R>
__global__ void __launch_bounds__(kBRows / R) busbar_sweep_kernel(EvalArgs a) {
  constexpr int kThreads = kBRows / R, kWarps = kThreads / 32;
  extern __shared__ __align__(16) float srec[];  // [G][kBVB][kRec]
  __shared__ float sred[kWarps][G];
  // topology groups vary fastest along the grid: the CTAs resident at one time
  // share a row tile, so the N and pi_s segments that their records name
  // (mostly the same stations in every topology) are re-read from L1 and L2
  const int tid = threadIdx.x, tile = blockIdx.y;
  const int l = tile * kBRows + tid * R;  // rows l .. l + R - 1 (the padded row count is a multiple of 128)
  const int b0 = blockIdx.x * G;
  const int Ep = a.E_mon_pad;
  constexpr int kRec = bb_record_floats(TT), kRec4 = kRec / 4;  // records are whole float4s
  static_assert(kRec % 4 == 0, "busbar records must be 16-byte multiples");
  float u[G][R][8], fpv[G][TT][R], m[G][TT][R];
#pragma unroll
  for (int gi = 0; gi < G; ++gi) {
    const int bb = min(b0 + gi, a.B - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4* ur = reinterpret_cast<const float4*>(a.U + ((size_t)bb * Ep + l + r) * 8);
      const float4 u0 = ur[0], u1 = ur[1];
      u[gi][r][0] = u0.x, u[gi][r][1] = u0.y, u[gi][r][2] = u0.z, u[gi][r][3] = u0.w;
      u[gi][r][4] = u1.x, u[gi][r][5] = u1.y, u[gi][r][6] = u1.z, u[gi][r][7] = u1.w;
    }
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      RowVec<R>::load(a.fp + ((size_t)bb * TT + t) * Ep + l, fpv[gi][t]);
#pragma unroll
      for (int r = 0; r < R; ++r) m[gi][t][r] = 0.f;
    }
  }
  for (int v0 = 0; v0 < a.NB; v0 += kBVB) {
    const int nv = min(kBVB, a.NB - v0);
    __syncthreads();
    // a topology's records v0 .. v0 + nv - 1 are contiguous: float4 copies with
    // compile-time divisors
    for (int i = tid; i < G * kBVB * kRec4; i += kThreads) {
      const int gi = i / (kBVB * kRec4), q = i % (kBVB * kRec4);
      const int bb = min(b0 + gi, a.B - 1);
      float4 x = make_float4(0.f, __int_as_float(-1), 0.f, 0.f);  // slot past the end: |R'| = -1 marks it unused
      if (q < nv * kRec4) x = reinterpret_cast<const float4*>(a.bbrec + ((size_t)bb * a.NB + v0) * kRec)[q];
      reinterpret_cast<float4*>(srec)[i] = x;
    }
    __syncthreads();
    // unrolled so that later records' gathers of N and pi_s are issued while
    // earlier records' arithmetic runs (the loop is bound by their latency)
#pragma unroll 4
    for (int vv = 0; vv < nv; ++vv) {
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        const float* rec = srec + (gi * kBVB + vv) * kRec;
        const int* irec = reinterpret_cast<const int*>(rec);
        const int nr = irec[1];
        if (nr < 0) continue;
        float pi[R];
        RowVec<R>::load(a.Pm + (size_t)irec[0] * Ep + l, pi);
        const float* pr = rec + kBBHead;
        const float* zr = pr + TT;
        const float* yr = zr + kMaxBB * TT;
        float F[TT][R];
        if constexpr (TT % 4 == 0) {  // records are 16-byte aligned: four timesteps per load
#pragma unroll
          for (int t4 = 0; t4 < TT; t4 += 4) {
            const float4 p4 = *reinterpret_cast<const float4*>(pr + t4);
            const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
            for (int d = 0; d < 4; ++d)
#pragma unroll
              for (int r = 0; r < R; ++r) F[t4 + d][r] = fmaf(-pv[d], pi[r], fpv[gi][t4 + d][r]);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float4 y4 = *reinterpret_cast<const float4*>(yr + i * TT + t4);
              const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
              for (int d = 0; d < 4; ++d)
#pragma unroll
                for (int r = 0; r < R; ++r) F[t4 + d][r] = fmaf(-u[gi][r][i], yv[d], F[t4 + d][r]);
            }
          }
          // the gathers of up to 4 columns are issued together, ahead of their
          // arithmetic (2 or 8 at a time measured slower)
          for (int j0 = 0; j0 < nr; j0 += 4) {
            float n[4][R];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
              if (j0 + d < nr) {
                RowVec<R>::load(a.Nswm + (size_t)irec[2 + j0 + d] * Ep + l, n[d]);
              } else {
#pragma unroll
                for (int r = 0; r < R; ++r) n[d][r] = 0.f;
              }
            }
#pragma unroll
            for (int d = 0; d < 4; ++d) {
              if (j0 + d >= nr) break;
              const int jj = j0 + d;
#pragma unroll
              for (int t4 = 0; t4 < TT; t4 += 4) {
                const float4 z4 = *reinterpret_cast<const float4*>(zr + jj * TT + t4);
                const float zv[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
#pragma unroll
                  for (int r = 0; r < R; ++r) F[t4 + e][r] = fmaf(-n[d][r], zv[e], F[t4 + e][r]);
              }
            }
          }
        } else {
#pragma unroll
          for (int t = 0; t < TT; ++t) {
            const float pt = pr[t];
#pragma unroll
            for (int r = 0; r < R; ++r) F[t][r] = fmaf(-pt, pi[r], fpv[gi][t][r]);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float yt = yr[i * TT + t];
#pragma unroll
              for (int r = 0; r < R; ++r) F[t][r] = fmaf(-u[gi][r][i], yt, F[t][r]);
            }
          }
          for (int jj = 0; jj < nr; ++jj) {
            float n[R];
            RowVec<R>::load(a.Nswm + (size_t)irec[2 + jj] * Ep + l, n);
#pragma unroll
            for (int t = 0; t < TT; ++t) {
              const float zt = zr[jj * TT + t];
#pragma unroll
              for (int r = 0; r < R; ++r) F[t][r] = fmaf(-n[r], zt, F[t][r]);
            }
          }
        }
#pragma unroll
        for (int t = 0; t < TT; ++t)
#pragma unroll
          for (int r = 0; r < R; ++r) m[gi][t][r] = fmaxf(m[gi][t][r], fabsf(F[t][r]));
      }
    }
  }
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int gi = 0; gi < G; ++gi) {
    const int bb = b0 + gi;
    float over = 0.f;
    if (bb < a.B) {
#pragma unroll
      for (int t = 0; t < TT; ++t) {  // fixed trip count: m stays in registers
        if (t >= a.n_t) break;
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (l + r < a.E_mon) over += fmaxf(m[gi][t][r] - a.lim[l + r], 0.f);
        if (a.bmax) {
          float* out = a.bmax + ((size_t)bb * a.n_t + t) * a.E_mon + l;
          if (R > 1 && l + R - 1 < a.E_mon && a.E_mon % R == 0 && (reinterpret_cast<uintptr_t>(a.bmax) & (4 * R - 1)) == 0) {
            RowVec<R>::store(out, m[gi][t]);
          } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
              if (l + r < a.E_mon) out[r] = m[gi][t][r];
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) over += __shfl_xor_sync(0xffffffffu, over, o);
    if (lane == 0) sred[warp][gi] = over;
  }
  __syncthreads();
  if (tid < G && b0 + tid < a.B) {
    float s = 0.f;
    for (int w = 0; w < kWarps; ++w) s += sred[w][tid];
    a.bbpart[(size_t)(b0 + tid) * a.n_rowtiles + tile] = s;
  }
}

__global__ void build_nswm_kernel(const double* Nsw, const int* mon, int E, int E_mon, int Ep, int n_sw, float* out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n_sw * Ep) return;
  const int q = (int)(i / Ep), l = (int)(i % Ep);
  out[i] = l < E_mon ? (float)Nsw[(size_t)q * E + mon[l]] : 0.f;
}

// lambda_b and the islanding count per topology (fixed-order sum of the row tiles)
__global__ void busbar_metrics_kernel(EvalArgs a, float* lambda_b, int32_t* n_island) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.B) return;
  const TopoInfo inf = a.info[b];
  double s = 0.0;
  for (int r = 0; r < a.n_rowtiles; ++r) s += (double)a.bbpart[(size_t)b * a.n_rowtiles + r];
  if (lambda_b) lambda_b[b] = inf.island_base ? __int_as_float(0x7fc00000) : (float)s;
  if (n_island) n_island[b] = inf.island_base ? -1 : inf.nbisl;
}

template <int TT, int G, int R>
int launch_tt(const EvalArgs& a, cudaStream_t s) {
  if (a.kRec != bb_record_floats(TT)) return set_error(TTO_E_ARG, "busbar record size mismatch");
  const size_t smem = (size_t)G * kBVB * a.kRec * sizeof(float);
  static bool attr[64] = {};
  int dev = 0;
  TTO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    TTO_CUDA_TRY(cudaFuncSetAttribute(busbar_sweep_kernel<TT, G, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    attr[dev] = true;
  }
  if (a.E_mon_pad / kBRows > 65535) return set_error(TTO_E_ARG, "too many monitored rows for the busbar sweep");
  const dim3 grid((unsigned)((a.B + G - 1) / G), (unsigned)(a.E_mon_pad / kBRows));
  busbar_sweep_kernel<TT, G, R><<<grid, kBRows / R, smem, s>>>(a);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

}  // namespace

int ensure_busbar(tto_grid* g, int B, int TT, cudaStream_t s) {
  if (kRowTile != kBRows) return set_error(TTO_E_ARG, "busbar sweep tile mismatch");
  if (!g->d_Nswm) {
    const size_t n = (size_t)std::max(g->n_sw, 1) * g->E_mon_pad;
    TTO_CUDA_TRY(cudaMalloc(&g->d_Nswm, n * sizeof(float)));
    build_nswm_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->d_Nsw, g->d_mon, g->E, g->E_mon, g->E_mon_pad,
                                                                   g->n_sw, g->d_Nswm);
    TTO_CUDA_TRY(cudaGetLastError());
  }
  const int NB = g->S + g->k_max;
  if (B > g->bb_cap_B || TT > g->bb_cap_T) {
    const int nB = std::max(B, g->bb_cap_B), nT = std::max(TT, g->bb_cap_T);
    TTO_CUDA_TRY(cudaStreamSynchronize(s));
    if (g->d_bbrec) cudaFree(g->d_bbrec);
    if (g->d_bbpart) cudaFree(g->d_bbpart);
    if (g->d_bbstate) cudaFree(g->d_bbstate);
    g->d_bbrec = nullptr;
    g->d_bbpart = nullptr;
    g->d_bbstate = nullptr;
    g->bb_cap_B = g->bb_cap_T = 0;
    TTO_CUDA_TRY(cudaMalloc(&g->d_bbrec, (size_t)nB * NB * bb_record_floats(nT) * sizeof(float)));
    TTO_CUDA_TRY(cudaMalloc(&g->d_bbpart, (size_t)nB * g->n_rowtiles * sizeof(float)));
    TTO_CUDA_TRY(cudaMalloc(&g->d_bbstate, (size_t)nB * sizeof(SplitState)));
    g->bb_cap_B = nB;
    g->bb_cap_T = nT;
    forget_grid_graphs(g);
    ++g->ws_epoch;
  }
  return TTO_OK;
}

void fill_busbar_args(tto_grid* g, EvalArgs& a) {
  a.busbar = 1;
  a.S = g->S;
  a.NB = g->S + g->k_max;
  a.kRec = bb_record_floats(a.TT);
  a.Pst = g->d_Pst;
  a.Pm = g->d_Pm;
  a.Nswm = g->d_Nswm;
  a.bbrec = g->d_bbrec;
  a.bbstate = static_cast<SplitState*>(g->d_bbstate);
  a.bbpart = g->d_bbpart;
  a.lbpre = g->d_lbpre;
}

int launch_busbar_sweep(const EvalArgs& a, cudaStream_t s) {
  switch (a.TT) {
    case 1: return launch_tt<1, 1, 2>(a, s);
    case 2: return launch_tt<2, 1, 2>(a, s);
    case 4: return launch_tt<4, 1, 2>(a, s);
    case 8: return launch_tt<8, 1, 2>(a, s);
    case 16: return launch_tt<16, 2, 1>(a, s);
    case 24: return launch_tt<24, 1, 1>(a, s);
    case 32: return launch_tt<32, 1, 1>(a, s);
    default: return set_error(TTO_E_ARG, "unsupported timestep count %d", a.TT);
  }
}

int launch_busbar_metrics(const EvalArgs& a, float* lambda_b, int32_t* n_island, cudaStream_t s) {
  busbar_metrics_kernel<<<(a.B + 127) / 128, 128, 0, s>>>(a, lambda_b, n_island);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

}  // namespace tto

using namespace tto;

extern "C" int tto_evaluate_busbar(tto_grid* g, const int32_t* topo, int32_t B, const int32_t* timesteps, int32_t n_t,
                                   float* lambda_b, int32_t* n_island, float* bmax, void* stream) {
  if (!g || B < 0) return set_error(TTO_E_ARG, "bad busbar arguments");
  if (B == 0) return TTO_OK;
  if (!topo) return set_error(TTO_E_ARG, "null topology buffer");
  if (g->S < 1) return set_error(TTO_E_ARG, "the grid has no stations, so no busbar outages");
  cudaStream_t s = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  const int TT = padded_T(timesteps ? n_t : g->T);
  if (TT < 0) return set_error(TTO_E_ARG, "at most %d timesteps", TTO_MAX_T);
  int rc = ensure_workspace(g, B, TT);
  if (rc) return rc;
  rc = ensure_busbar(g, B, TT, s);
  if (rc) return rc;
  tto_eval_opts o{};
  o.precision = TTO_PREC_FP32;
  o.fitness_kind = TTO_FIT_WORKLOAD;
  o.d_split = 1;
  o.d_moved = 1;
  EvalArgs a;
  rc = evaluate_impl(g, topo, B, timesteps, n_t, &o, g->ws.fit, nullptr, nullptr, nullptr, nullptr, nullptr, s, &a,
                     /*busbar_setup=*/true);
  if (rc) return rc;
  a.bmax = bmax;
  rc = launch_busbar_sweep(a, s);
  if (rc) return rc;
  return launch_busbar_metrics(a, lambda_b, n_island, s);
}

extern "C" int tto_grid_busbar_reference(tto_grid* g, const int32_t* timesteps, int32_t n_t, void* stream) {
  if (!g) return set_error(TTO_E_ARG, "null grid");
  cudaStream_t s = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  const int nt = timesteps ? n_t : g->T;
  if (nt < 1 || nt > TTO_MAX_T) return set_error(TTO_E_ARG, "n_t must be in [1, %d]", TTO_MAX_T);
  if (!g->d_lbpre) TTO_CUDA_TRY(cudaMalloc(&g->d_lbpre, sizeof(float)));
  if (!g->d_empty) {
    TTO_CUDA_TRY(cudaMalloc(&g->d_empty, TTO_MAX_K * sizeof(int32_t)));
    TTO_CUDA_TRY(cudaMemset(g->d_empty, 0xFF, TTO_MAX_K * sizeof(int32_t)));
  }
  const int rc = tto_evaluate_busbar(g, g->d_empty, 1, timesteps, n_t, g->d_lbpre, nullptr, nullptr, stream);
  if (rc) return rc;
  g->lbpre_nt = nt;
  for (int t = 0; t < nt; ++t) g->lbpre_tsel[t] = timesteps ? timesteps[t] : t;
  (void)s;
  return TTO_OK;
}
