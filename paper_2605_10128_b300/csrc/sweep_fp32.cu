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
//
// The same tile body serves the persistent work-list sweep of mixed-grid
// batches (sweep_fp32_persistent_kernel): there each CTA takes (job, row tile,
// topology group) items from a shared counter until the list is exhausted.
#include "sweep.cuh"

namespace tto {

constexpr int kCC = 32;  // outage columns per staged chunk

// The grid and batch fields one CTA of the FP32 sweep reads, copied out of the
// job's arguments once per tile.
struct Fp32Tile {
  const float* U;
  const float* V;
  const float* gg;
  const float* fp;
  const float* Nmo;
  const float* lim;
  float* fmax;
  float* part;
  int B, E_mon, E_mon_pad, O_pad, n_t, n_parts;
};

__device__ __forceinline__ Fp32Tile fp32_tile(const EvalArgs& a) {
  return Fp32Tile{a.U, a.V, a.gg, a.fp, a.Nmo, a.lim, a.fmax, a.part, a.B, a.E_mon, a.E_mon_pad, a.O_pad, a.n_t,
                  a.n_parts};
}

template <int TT, int G, int KP>
struct Fp32Smem {
  float sU[G][kRowTile][KP];
  float sV[G][kCC][KP];
  float sg[G][kCC][TT];
  float sred[kRowTile / 32][G][3];
};

// One CTA's share of the sweep: row tile `tile` (128 rows) x topologies
// G grp .. G grp + G - 1, all outage columns.
template <int TT, int G, int KP>
__device__ __forceinline__ void fp32_sweep_tile(const Fp32Tile& a, int tile, int grp, Fp32Smem<TT, G, KP>& sm) {
  auto& sU = sm.sU;
  auto& sV = sm.sV;
  auto& sg = sm.sg;
  auto& sred = sm.sred;
  const int tid = threadIdx.x;
  const int l = tile * kRowTile + tid;
  const int b0 = grp * G;
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

template <int TT, int G, int KP>
__global__ void __launch_bounds__(kRowTile) sweep_fp32_kernel(EvalArgs a) {
  __shared__ __align__(16) Fp32Smem<TT, G, KP> sm;
  fp32_sweep_tile<TT, G, KP>(fp32_tile(a), blockIdx.x, blockIdx.y, sm);
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
  constexpr int G = fp32_group(TT);
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

// ------------------------------------------------------- persistent work list
// Mixed-grid batches (tto_evaluate_multi, TTO_MULTI_PERSISTENT): one launch of
// four CTAs per SM; every CTA takes the next (job, row tile, topology group)
// item from a shared counter and runs the FP32 tile body above for it, until
// the list is exhausted.  One kernel holds the bodies of every timestep count
// and rank, so it needs the registers of the largest; items therefore take the
// smaller topology group of the two FP32 tile variants (fp32_item_group),
// which keeps every body within 128 registers at four CTAs per SM.  Items are
// numbered job by job, the jobs ordered by the cost of one item (largest
// first), so the large items start first and the small ones fill the tail.
// Each item writes its own partial metrics, so the result does not depend on
// which CTA took it.  Rank 2 genomes run the rank-4 body (U and V are stored
// 8 wide, zero beyond the genome's rank).
template <int TT, int G, int KP>
__device__ __forceinline__ void persistent_item(const EvalArgs& a, int tile, int grp, unsigned char* dsm) {
  fp32_sweep_tile<TT, G, KP>(fp32_tile(a), tile, grp, *reinterpret_cast<Fp32Smem<TT, G, KP>*>(dsm));
}

template <int TT, int KP>
__device__ __forceinline__ void persistent_tt(const EvalArgs& a, int tile, int grp, unsigned char* dsm) {
  persistent_item<TT, fp32_item_group(TT), KP>(a, tile, grp, dsm);
}

template <int KP>
__device__ __forceinline__ void persistent_kp(const EvalArgs& a, int tile, int grp, unsigned char* dsm) {
  switch (a.TT) {
    case 1: persistent_tt<1, KP>(a, tile, grp, dsm); break;
    case 2: persistent_tt<2, KP>(a, tile, grp, dsm); break;
    case 4: persistent_tt<4, KP>(a, tile, grp, dsm); break;
    case 8: persistent_tt<8, KP>(a, tile, grp, dsm); break;
    case 16: persistent_tt<16, KP>(a, tile, grp, dsm); break;
    case 24: persistent_tt<24, KP>(a, tile, grp, dsm); break;
    case 32: persistent_tt<32, KP>(a, tile, grp, dsm); break;
  }
}

__global__ void __launch_bounds__(kRowTile, 4) sweep_fp32_persistent_kernel(const __grid_constant__ MultiArgs m) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ unsigned int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(m.counter, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    if (it >= m.n_items) break;  // the same for every thread of the CTA
    int j = 0;
    for (int q = 1; q < m.n; ++q)
      if (it >= m.item_start[q]) j = q;
    const EvalArgs& a = m.job[j];
    const int r = (int)(it - m.item_start[j]);
    const int tile = r % a.n_rowtiles, grp = r / a.n_rowtiles;
    if (a.KP <= 4)
      persistent_kp<4>(a, tile, grp, dsm);
    else
      persistent_kp<8>(a, tile, grp, dsm);
    __syncthreads();  // shared memory and s_item are reused by the next item
  }
}

template <int TT, int KP>
constexpr size_t fp32_smem_tt() {
  return sizeof(Fp32Smem<TT, fp32_item_group(TT), KP>);
}

template <int KP>
constexpr size_t fp32_smem_kp() {
  size_t m = 0;
  const size_t v[] = {fp32_smem_tt<1, KP>(),  fp32_smem_tt<2, KP>(),  fp32_smem_tt<4, KP>(), fp32_smem_tt<8, KP>(),
                      fp32_smem_tt<16, KP>(), fp32_smem_tt<24, KP>(), fp32_smem_tt<32, KP>()};
  for (size_t x : v) m = x > m ? x : m;
  return m;
}

constexpr size_t kPersistentSmem = fp32_smem_kp<4>() > fp32_smem_kp<8>() ? fp32_smem_kp<4>() : fp32_smem_kp<8>();

int launch_sweep_persistent(const MultiArgs& m, int device, cudaStream_t s) {
  static int blocks_per_sm[64] = {};
  if (device < 0 || device >= 64) return set_error(TTO_E_ARG, "device %d out of range", device);
  if (blocks_per_sm[device] == 0) {
    TTO_CUDA_TRY(cudaFuncSetAttribute(sweep_fp32_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kPersistentSmem));
    int nb = 0;
    TTO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_fp32_persistent_kernel, kRowTile,
                                                               kPersistentSmem));
    blocks_per_sm[device] = nb > 0 ? nb : 1;
  }
  int sms = 0;
  TTO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const unsigned int slots = (unsigned int)(sms * blocks_per_sm[device]);
  const unsigned int grid = m.n_items < slots ? m.n_items : slots;
  if (grid == 0) return TTO_OK;
  TTO_CUDA_TRY(cudaMemsetAsync(m.counter, 0, sizeof(unsigned int), s));
  sweep_fp32_persistent_kernel<<<grid, kRowTile, kPersistentSmem, s>>>(m);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

}  // namespace tto
