// Fused N-1 sweep on the CUDA cores (FP32 throughout; TTO_PREC_FP32).
//
// CTA = one tile of 128 monitored rows x a group of G topologies; thread = row.
// The CTA walks all outage columns in chunks of 32: the per-topology column
// factors V and g of the chunk are staged in shared memory, the thread keeps
// its row of N for the chunk in registers and reuses it for all G topologies.
// Per (row l, outage c, topology):  n' = N_lc - U_l . V_c  (KP FMAs), then for
// every timestep  F = f'_l[t] - n' g_c[t],  m[t] = max(m[t], |F|).  The running
// maxima live in registers for the whole column walk, so each CTA owns complete
// rows and reduces them straight to per-row-tile partial metrics (no atomics,
// fixed reduction order).
#include "sweep.cuh"

namespace tto {

constexpr int kCC = 32;  // outage columns per staged chunk

template <int TT, int G, int KP>
__global__ void __launch_bounds__(kRowTile) sweep_fp32_kernel(EvalArgs a) {
  __shared__ __align__(16) float sU[G][kRowTile][KP];
  __shared__ __align__(16) float sV[G][kCC][KP];
  __shared__ __align__(16) float sg[G][kCC][TT];
  __shared__ float sred[kRowTile / 32][G][3];
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int l = tile * kRowTile + tid;
  const int b0 = blockIdx.y * G;
  const int nG = min(G, a.B - b0);
  const int Ep = a.E_mon_pad, Op = a.O_pad;

  float fpv[G][TT];
  float m[G][TT];
#pragma unroll
  for (int gi = 0; gi < G; ++gi) {
    const int bb = min(b0 + gi, a.B - 1);
    const float* ur = a.U + ((size_t)bb * Ep + l) * 8;
#pragma unroll
    for (int j = 0; j < KP; ++j) sU[gi][tid][j] = ur[j];
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      fpv[gi][t] = a.fp[((size_t)bb * TT + t) * Ep + l];
      m[gi][t] = 0.f;
    }
  }

  for (int c0 = 0; c0 < Op; c0 += kCC) {
    __syncthreads();
    for (int i = tid; i < G * kCC * KP; i += kRowTile) {
      const int gi = i / (kCC * KP), r = i % (kCC * KP);
      const int bb = min(b0 + gi, a.B - 1);
      (&sV[gi][0][0])[r] = a.V[((size_t)bb * Op + c0 + r / KP) * 8 + r % KP];
    }
    for (int i = tid; i < G * kCC * TT; i += kRowTile) {
      const int gi = i / (kCC * TT), r = i % (kCC * TT);
      const int bb = min(b0 + gi, a.B - 1);
      (&sg[gi][0][0])[r] = a.gg[((size_t)bb * Op + c0) * TT + r];
    }
    float nrow[kCC];
    const float4* np = reinterpret_cast<const float4*>(a.Nmo + (size_t)l * Op + c0);
#pragma unroll
    for (int q = 0; q < kCC / 4; ++q) {
      const float4 v = __ldg(np + q);
      nrow[4 * q + 0] = v.x;
      nrow[4 * q + 1] = v.y;
      nrow[4 * q + 2] = v.z;
      nrow[4 * q + 3] = v.w;
    }
    __syncthreads();
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      if (gi < nG) {
        float u[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) u[j] = sU[gi][tid][j];
#pragma unroll
        for (int c = 0; c < kCC; ++c) {
          float nn = nrow[c];
#pragma unroll
          for (int j = 0; j < KP; ++j) nn = fmaf(-u[j], sV[gi][c][j], nn);
#pragma unroll
          for (int t = 0; t < TT; ++t) {
            const float F = fmaf(-nn, sg[gi][c][t], fpv[gi][t]);
            m[gi][t] = fmaxf(m[gi][t], fabsf(F));
          }
        }
      }
    }
  }

  // per-row metrics, then a fixed-order CTA reduction per topology
  const bool live = l < a.E_mon;
  const float lim = live ? a.lim[l] : 1.f;
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int gi = 0; gi < G; ++gi) {
    float over = 0.f, cnt = 0.f, ml = 0.f;
    if (live && gi < nG) {
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        if (t < a.n_t) {
          const float mm = m[gi][t];
          over += fmaxf(mm - lim, 0.f);
          cnt += mm > lim ? 1.f : 0.f;
          ml = fmaxf(ml, fmaxf(fabsf(fpv[gi][t]), mm) / lim);
          if (a.fmax) a.fmax[((size_t)(b0 + gi) * a.n_t + t) * a.E_mon + l] = mm;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      over += __shfl_xor_sync(0xffffffffu, over, o);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      ml = fmaxf(ml, __shfl_xor_sync(0xffffffffu, ml, o));
    }
    if (lane == 0) {
      sred[warp][gi][0] = over;
      sred[warp][gi][1] = cnt;
      sred[warp][gi][2] = ml;
    }
  }
  __syncthreads();
  if (tid < nG) {
    float over = 0.f, cnt = 0.f, ml = 0.f;
#pragma unroll
    for (int w = 0; w < kRowTile / 32; ++w) {
      over += sred[w][tid][0];
      cnt += sred[w][tid][1];
      ml = fmaxf(ml, sred[w][tid][2]);
    }
    float* pp = a.part + ((size_t)(b0 + tid) * a.n_parts + tile) * 4;
    pp[0] = over;
    pp[1] = cnt;
    pp[2] = ml;
    pp[3] = 0.f;
  }
}

template <int TT, int KP, int G>
static int launch_fp32_g(const EvalArgs& a, cudaStream_t s) {
  if ((a.B + G - 1) / G > 65535) return set_error(TTO_E_ARG, "batch too large for one FP32 sweep launch");
  dim3 grid(a.n_rowtiles, (a.B + G - 1) / G);
  sweep_fp32_kernel<TT, G, KP><<<grid, kRowTile, 0, s>>>(a);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

// Tile variants: shape 0 keeps G topologies per CTA (G x TT <= 32 registers of
// running maxima), shape 1 halves G (more CTAs, fewer registers).
template <int TT, int KP>
static int launch_fp32_tt(const EvalArgs& a, cudaStream_t s) {
  constexpr int G = TT <= 4 ? 8 : (TT <= 8 ? 4 : (TT <= 16 ? 2 : 1));
  constexpr int G2 = G > 1 ? G / 2 : 1;
  return a.shape == 1 ? launch_fp32_g<TT, KP, G2>(a, s) : launch_fp32_g<TT, KP, G>(a, s);
}

template <int KP>
static int launch_fp32_k(const EvalArgs& a, cudaStream_t s) {
  switch (a.TT) {
    case 1: return launch_fp32_tt<1, KP>(a, s);
    case 2: return launch_fp32_tt<2, KP>(a, s);
    case 4: return launch_fp32_tt<4, KP>(a, s);
    case 8: return launch_fp32_tt<8, KP>(a, s);
    case 16: return launch_fp32_tt<16, KP>(a, s);
    case 24: return launch_fp32_tt<24, KP>(a, s);
    case 32: return launch_fp32_tt<32, KP>(a, s);
  }
  return set_error(TTO_E_ARG, "unsupported padded timestep count %d", a.TT);
}

int launch_sweep_fp32(const EvalArgs& a, cudaStream_t s) {
  switch (a.KP) {
    case 2: return launch_fp32_k<2>(a, s);
    case 4: return launch_fp32_k<4>(a, s);
    case 8: return launch_fp32_k<8>(a, s);
  }
  return set_error(TTO_E_ARG, "unsupported padded rank %d", a.KP);
}

int sweep_shapes(int precision) {
  return precision == TTO_PREC_FP32 ? 2 : (precision == TTO_PREC_TF32X3 ? kUmmaShape + 1 : 4);
}

int launch_sweep(EvalArgs& a, cudaStream_t s) {
  if (a.shape < 0 || a.shape >= sweep_shapes(a.precision)) return set_error(TTO_E_ARG, "unknown sweep shape %d", a.shape);
  if (a.precision == TTO_PREC_FP32) {
    a.n_parts = a.n_rowtiles;
    return launch_sweep_fp32(a, s);
  }
  return launch_sweep_tc(a, s);
}

}  // namespace tto
