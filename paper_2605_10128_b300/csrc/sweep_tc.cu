// Fused N-1 sweep with the low-rank term on the tensor cores.
//
// For every (monitored l, outage c) the post-split response is
//     N'_lc = N_lc - U_l . V_c        (rank k <= 8)
// and the post-contingency flow of every timestep is
//     F_lc[t] = f'_l[t] - N'_lc g_c[t],     fmax_l[t] = max_c |F_lc[t]|.
// Per 16 x 8 tile, mma.sync accumulates the split products of U and V onto an
// accumulator preloaded with -N (stored once per grid in C-fragment order), so
// D = U V^T - N = -N'.  Modes: TF32X3 = three m16n8k8 tf32 products
// U_hi V_hi + U_lo V_hi + U_hi V_lo (about 2^-22 relative error of the low-rank
// term); BF16X3 = two m16n8k16 bf16 products [U_hi|U_lo][V_hi;V_hi] and
// [U_hi|U_lo][V_lo;0] (about 2^-16); BF16 = U_hi V_hi only.  The
// accumulator registers hold each lane's four (l, c) entries, and the epilogue
// runs on them directly: F = fma(D, g_c[t], f'_l[t]) and a max of |F| per row
// and timestep, two FP32 instructions per (l, c, t).  Islanding outages carry
// g = NaN, which fmaxf ignores.
//
// CTA = 8 warps = 8 topologies on one band of 16*MW monitored rows; each warp
// walks every outage column of its topology, so the running maxima stay in
// registers and every warp reduces its own rows at the end (no atomics).  The
// 8 warps of a CTA read the same -N tiles (L1 hits after the first), and the
// launch order is tiled (16 row bands x 16 topology groups) so that the -N
// band and the column factors of the co-resident CTAs stay in L2.
#include <cuda_bf16.h>

#include "sweep.cuh"

namespace tto {

constexpr int kTCWarps = 8;           // topologies per CTA
constexpr int kSwB = 16, kSwG = 16;   // launch-order tile: row bands x topology groups
constexpr int kMaxTChunk = 8;         // timesteps per sweep pass

__device__ __forceinline__ void mma_bf16(float4& d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d.x), "+f"(d.y), "+f"(d.z), "+f"(d.w)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_tf32(float4& d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d.x), "+f"(d.y), "+f"(d.z), "+f"(d.w)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Low-rank modes of the tensor-core sweep.
enum { kModeBF16x3 = 0, kModeBF16 = 1, kModeTF32x3 = 2 };

template <int BW>
__device__ __forceinline__ void load_b(uint32_t (&vb)[BW], const uint32_t* p) {
  if constexpr (BW == 2) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    vb[0] = v.x;
    vb[1] = v.y;
  } else {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    vb[0] = v.x;
    vb[1] = v.y;
    vb[2] = v.z;
    vb[3] = v.w;
  }
}

template <int TC>
__device__ __forceinline__ void load_g(float (&gv)[2 * TC], const float* p) {
  if constexpr (TC == 1) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    gv[0] = v.x;
    gv[1] = v.y;
  } else {
#pragma unroll
    for (int i = 0; i < TC / 2; ++i) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
      gv[4 * i + 0] = v.x;
      gv[4 * i + 1] = v.y;
      gv[4 * i + 2] = v.z;
      gv[4 * i + 3] = v.w;
    }
  }
}

template <int TC, int MW, int MODE>
__global__ void __launch_bounds__(kTCWarps * 32, 2)
    sweep_tc_kernel(EvalArgs a, int t0, int tci, int n_tchunks, int n_bands, int n_groups) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int tiles_b = (n_bands + kSwB - 1) / kSwB;
  const int tile = blockIdx.x / (kSwB * kSwG), within = blockIdx.x % (kSwB * kSwG);
  const int band = (tile % tiles_b) * kSwB + within % kSwB;
  const int grp = (tile / tiles_b) * kSwG + within / kSwB;
  if (band >= n_bands || grp >= n_groups) return;
  const int b = grp * kTCWarps + warp;
  if (b >= a.B) return;  // warp-uniform; the kernel has no block barrier
  const int TT = a.TT;
  const int n_mt = a.E_mon_pad >> 4, n_nt = a.O_pad >> 3;
  const int mt0 = band * MW;
  const size_t Ep = a.E_mon_pad;

  constexpr bool TF = MODE == kModeTF32x3;
  constexpr int AW = TF ? 8 : 4;  // A-fragment words per lane
  constexpr int BW = TF ? 4 : 2;  // B-fragment words per lane
  uint32_t A[MW][AW];
  float f[MW][2][TC], m[MW][2][TC];
  const uint4* Ua = reinterpret_cast<const uint4*>(a.U);
#pragma unroll
  for (int i = 0; i < MW; ++i) {
#pragma unroll
    for (int w = 0; w < AW / 4; ++w) {
      const uint4 u = __ldg(Ua + (((size_t)b * n_mt + mt0 + i) * 32 + lane) * (AW / 4) + w);
      A[i][4 * w + 0] = u.x;
      A[i][4 * w + 1] = u.y;
      A[i][4 * w + 2] = u.z;
      A[i][4 * w + 3] = u.w;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = (mt0 + i) * 16 + g + 8 * h;
#pragma unroll
      for (int t = 0; t < TC; ++t) {
        f[i][h][t] = a.fp[((size_t)b * TT + t0 + t) * Ep + row];
        m[i][h][t] = 0.f;
      }
    }
  }
  const float4* Nf = a.Nf + (size_t)mt0 * n_nt * 32 + lane;
  const uint32_t* Vb = reinterpret_cast<const uint32_t*>(a.V) + ((size_t)b * n_nt * 32 + lane) * BW;
  const float* gq = a.gg + ((size_t)b * n_nt * 4 + q) * TT * 2 + t0 * 2;
  const size_t gstride = (size_t)4 * TT * 2;

  float4 nf_n[MW];
  uint32_t vb_n[BW];
  float gv_n[2 * TC];
#pragma unroll
  for (int i = 0; i < MW; ++i) nf_n[i] = __ldg(Nf + (size_t)i * n_nt * 32);
  load_b<BW>(vb_n, Vb);
  load_g<TC>(gv_n, gq);

  for (int nt = 0; nt < n_nt; ++nt) {
    float4 nf[MW];
#pragma unroll
    for (int i = 0; i < MW; ++i) nf[i] = nf_n[i];
    uint32_t vb[BW];
#pragma unroll
    for (int j = 0; j < BW; ++j) vb[j] = vb_n[j];
    float gv[2 * TC];
#pragma unroll
    for (int j = 0; j < 2 * TC; ++j) gv[j] = gv_n[j];
    if (nt + 1 < n_nt) {
#pragma unroll
      for (int i = 0; i < MW; ++i) nf_n[i] = __ldg(Nf + ((size_t)i * n_nt + nt + 1) * 32);
      load_b<BW>(vb_n, Vb + (size_t)(nt + 1) * 32 * BW);
      load_g<TC>(gv_n, gq + (nt + 1) * gstride);
    }
#pragma unroll
    for (int i = 0; i < MW; ++i) {
      float4 d = nf[i];
      if (MODE == kModeTF32x3) {
        mma_tf32(d, &A[i][0], vb[0], vb[1]);  // U_hi V_hi
        mma_tf32(d, &A[i][4], vb[0], vb[1]);  // U_lo V_hi
        mma_tf32(d, &A[i][0], vb[2], vb[3]);  // U_hi V_lo
      } else if (MODE == kModeBF16x3) {
        mma_bf16(d, &A[i][0], vb[0], vb[0]);  // [U_hi | U_lo] [V_hi ; V_hi]
        mma_bf16(d, &A[i][0], vb[1], 0u);     // [U_hi | U_lo] [V_lo ; 0]
      } else {
        mma_bf16(d, &A[i][0], vb[0], 0u);     // U_hi V_hi
      }
#pragma unroll
      for (int t = 0; t < TC; ++t) {
        const float g0 = gv[2 * t], g1 = gv[2 * t + 1];
        m[i][0][t] = fmaxf(fmaxf(m[i][0][t], fabsf(fmaf(d.x, g0, f[i][0][t]))), fabsf(fmaf(d.y, g1, f[i][0][t])));
        m[i][1][t] = fmaxf(fmaxf(m[i][1][t], fabsf(fmaf(d.z, g0, f[i][1][t]))), fabsf(fmaf(d.w, g1, f[i][1][t])));
      }
    }
  }

  // rows: combine the four lanes that share a row, then per-row metrics
  float over = 0.f, cnt = 0.f, ml = 0.f;
#pragma unroll
  for (int i = 0; i < MW; ++i) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = (mt0 + i) * 16 + g + 8 * h;
#pragma unroll
      for (int t = 0; t < TC; ++t) {
        float v = m[i][h][t];
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 2));
        m[i][h][t] = v;
      }
      if (q == 0 && row < a.E_mon) {
        const float lim = a.lim[row];
#pragma unroll
        for (int t = 0; t < TC; ++t) {
          const int tt = t0 + t;
          if (tt < a.n_t) {
            const float mm = m[i][h][t];
            over += fmaxf(mm - lim, 0.f);
            cnt += mm > lim ? 1.f : 0.f;
            ml = fmaxf(ml, fmaxf(fabsf(f[i][h][t]), mm) / lim);
            if (a.fmax) a.fmax[((size_t)b * a.n_t + tt) * a.E_mon + row] = mm;
          }
        }
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
    float* pp = a.part + ((size_t)b * a.n_parts + (size_t)band * n_tchunks + tci) * 4;
    pp[0] = over;
    pp[1] = cnt;
    pp[2] = ml;
    pp[3] = 0.f;
  }
}

// -N in mma C-fragment order: tile (mt, nt), lane (g, q) holds
// (-N[16mt+g][8nt+2q], -N[16mt+g][8nt+2q+1], -N[16mt+g+8][8nt+2q], -N[16mt+g+8][8nt+2q+1]).
__global__ void fragment_N_kernel(const float* __restrict__ Nmo, float4* __restrict__ Nf, int n_mt,
                                  int n_nt, int O_pad) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)n_mt * n_nt * 32;
  if (i >= total) return;
  const int lane = (int)(i & 31);
  const size_t tile = i >> 5;
  const int nt = (int)(tile % n_nt), mt = (int)(tile / n_nt);
  const int g = lane >> 2, q = lane & 3;
  const size_t r0 = (size_t)(16 * mt + g) * O_pad, r1 = r0 + (size_t)8 * O_pad;
  const int c = 8 * nt + 2 * q;
  Nf[i] = make_float4(-Nmo[r0 + c], -Nmo[r0 + c + 1], -Nmo[r1 + c], -Nmo[r1 + c + 1]);
}

int ensure_fragment_N(tto_grid* g, cudaStream_t s) {
  if (g->d_Nf) return TTO_OK;
  const size_t n = (size_t)g->E_mon_pad * g->O_pad;
  TTO_CUDA_TRY(cudaMalloc(&g->d_Nf, n * sizeof(float)));
  const int n_mt = g->E_mon_pad >> 4, n_nt = g->O_pad >> 3;
  const size_t threads = (size_t)n_mt * n_nt * 32;
  fragment_N_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(g->d_Nmo, g->d_Nf, n_mt, n_nt, g->O_pad);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

size_t max_parts(const tto_grid* g) {
  const size_t fp32 = g->n_rowtiles;
  const size_t tc = (size_t)(g->E_mon_pad >> 4) * ((TTO_MAX_T + kMaxTChunk - 1) / kMaxTChunk);
  return fp32 > tc ? fp32 : tc;
}

template <int TC, int MW, int MODE>
static int launch_tc(EvalArgs& a, int t0, int tci, int n_tchunks, cudaStream_t s) {
  const int n_bands = a.E_mon_pad / (16 * MW);
  const int n_groups = (a.B + kTCWarps - 1) / kTCWarps;
  const int tiles_b = (n_bands + kSwB - 1) / kSwB, tiles_g = (n_groups + kSwG - 1) / kSwG;
  const size_t blocks = (size_t)tiles_b * tiles_g * kSwB * kSwG;
  if (blocks > 0x7fffffffu) return set_error(TTO_E_ARG, "batch too large for one sweep launch");
  sweep_tc_kernel<TC, MW, MODE><<<(unsigned)blocks, kTCWarps * 32, 0, s>>>(a, t0, tci, n_tchunks, n_bands, n_groups);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

template <int MODE>
static int launch_tc_chunk(EvalArgs& a, int tc, int t0, int tci, int n_tchunks, cudaStream_t s) {
  switch (tc) {
    case 1: return launch_tc<1, 2, MODE>(a, t0, tci, n_tchunks, s);
    case 2: return launch_tc<2, 2, MODE>(a, t0, tci, n_tchunks, s);
    case 4: return launch_tc<4, 2, MODE>(a, t0, tci, n_tchunks, s);
    case 8: return launch_tc<8, 1, MODE>(a, t0, tci, n_tchunks, s);
  }
  return set_error(TTO_E_ARG, "unsupported timestep chunk %d", tc);
}

int launch_sweep_tc(EvalArgs& a, cudaStream_t s) {
  const int TT = a.TT;
  const int tc = TT <= 4 ? TT : kMaxTChunk;
  const int n_tchunks = (TT + tc - 1) / tc;
  const int mw = tc <= 4 ? 2 : 1;
  a.n_parts = (a.E_mon_pad / (16 * mw)) * n_tchunks;
  for (int ci = 0; ci < n_tchunks; ++ci) {
    int rc;
    if (a.precision == TTO_PREC_TF32X3)
      rc = launch_tc_chunk<kModeTF32x3>(a, tc, ci * tc, ci, n_tchunks, s);
    else if (a.precision == TTO_PREC_BF16)
      rc = launch_tc_chunk<kModeBF16>(a, tc, ci * tc, ci, n_tchunks, s);
    else
      rc = launch_tc_chunk<kModeBF16x3>(a, tc, ci * tc, ci, n_tchunks, s);
    if (rc) return rc;
  }
  return TTO_OK;
}

}  // namespace tto
