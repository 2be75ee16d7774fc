// Fused N-1 sweep with the low-rank term on the tensor cores.
//
// For every (monitored l, outage c) the post-split response is
//     N'_lc = N_lc - U_l . V_c        (rank k <= 8)
// and the post-contingency flow of every timestep is
//     F_lc[t] = f'_l[t] - N'_lc g_c[t],     fmax_l[t] = max_c |F_lc[t]|.
// Per 16 x 8 tile, mma.sync accumulates split products of U and V onto an
// accumulator preloaded with -N (stored once per grid in C-fragment order), so
// D = U V^T - N = -N'.  Modes (hi/lo = leading and residual part of a split):
//   FP16X3: [U_hi|U_lo][V_hi;V_hi] + [U_hi|U_lo][V_lo;0], two m16n8k16 fp16
//           products, about 2^-21 relative error of the low-rank term; U and V
//           are first balanced by a power-of-two scale per topology (exact),
//           which keeps both inside the fp16 range;
//   TF32X3: U_hi V_hi + U_lo V_hi + U_hi V_lo, three m16n8k8 tf32 products,
//           about 2^-21;
//   BF16X3: as FP16X3 in bf16, about 2^-16;  BF16: U_hi V_hi only.
// The accumulator registers hold each lane's four (l, c) entries and the
// epilogue runs on them directly: F = fma(D, g_c[t], f'_l[t]) and a max of |F|
// per row and timestep, two FP32 instructions per (l, c, t).  Islanding
// outages carry g = NaN, which fmaxf ignores.
//
// CTA = TOPO topologies x HALVES row groups (default 4 x 2: a band of 32*MW
// monitored rows per CTA), one warp each, two CTAs per SM.  Each warp walks every outage column of its topology for 16*MW rows,
// so its running maxima stay in registers and it reduces its own rows at the
// end (no atomics).  Operands stream through a three-slot shared-memory ring
// filled by TMA bulk copies (cp.async.bulk, completion counted on an mbarrier):
// per stage of 8 outage tiles, the -N slab of the band (shared by the 4
// topologies) and each topology's column factors V and g (shared by its two
// warps).  The last warp to release a slot (a shared counter) refills it, its
// lanes issuing the stage's copies in parallel.  Every wait is bounded; a wait that gives up sets the
// status word to TTO_E_TIMEOUT, lets the copies already issued land, and ends
// the kernel.  The launch order is tiled (16 row bands x 16 topology groups)
// so that the -N band and the column factors of co-resident CTAs stay in L2.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sweep.cuh"


namespace tto {

// CTA shapes: TOPO topologies x HALVES row groups of 16*MW rows, one warp
// each, SLOTS pipeline slots, CTAS resident CTAs per SM (the register budget
// per thread follows: 128 at two, 80 at three).  The autotuner picks one per
// grid.
template <int TOPO, int HALVES, int SLOTS, int CTAS>
struct CtaShape {
  static constexpr int kTopo = TOPO, kHalves = HALVES, kWarps = TOPO * HALVES, kSlots = SLOTS, kCtas = CTAS;
};
using Shape0 = CtaShape<4, 2, 3, 2>;  // default: 64 rows x 4 topologies
using Shape1 = CtaShape<8, 1, 2, 2>;  // 32 rows x 8 topologies
using Shape2 = CtaShape<2, 4, 2, 2>;  // 128 rows x 2 topologies
using Shape3 = CtaShape<4, 2, 2, 3>;  // as Shape0, three CTAs (24 warps) per SM
constexpr int kNumShapes = 4;
constexpr int kSwB = 16, kSwG = 16;   // launch-order tile: row bands x topology groups
constexpr int kMaxTChunk = 8;         // timesteps per sweep pass
constexpr int kSN = 8;                // outage tiles (8 columns each) per pipeline stage
constexpr long long kWaitCycles = 1ll << 31;  // give up after ~1 s at 2 GHz

enum { kModeBF16x3 = 0, kModeBF16 = 1, kModeTF32x3 = 2, kModeFP16x3 = 3 };

__device__ __forceinline__ void mma_bf16(float4& d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d.x), "+f"(d.y), "+f"(d.z), "+f"(d.w)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_fp16(float4& d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
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

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete: a test, then
// short sleeps between tests so that waiting warps leave the issue slots to
// the warps that compute.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    __nanosleep(64);  // yield issue slots to the warps that have data
    if (mbar_test(bar, parity)) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

template <int MODE>
struct TCMode {
  static constexpr int AW = MODE == kModeTF32x3 ? 8 : 4;  // A-fragment words per lane and m-tile
  static constexpr int BW = MODE == kModeTF32x3 ? 4 : 2;  // B-fragment words per lane and n-tile
};

// Shared-memory layout of one pipeline slot.
template <int MW, int MODE, int TC, class SH>
struct Slot {
  static constexpr int kTopo = SH::kTopo, kHalves = SH::kHalves;
  static constexpr uint32_t kNf = kHalves * MW * kSN * 512;           // -N tiles of the band
  static constexpr uint32_t kVb = kSN * 32 * TCMode<MODE>::BW * 4;    // per topology
  static constexpr uint32_t kG = kSN * 4 * TC * 2 * 4;                // per topology
  static constexpr uint32_t kTopoBytes = kVb + kG;
  static constexpr uint32_t kBytes = kNf + kTopo * kTopoBytes;
};

template <int TC, int MW, int MODE, class SH>
__global__ void __launch_bounds__(SH::kWarps * 32, SH::kCtas)
    sweep_tc_kernel(EvalArgs a, int tci, int n_bands, int n_groups) {
  using S = Slot<MW, MODE, TC, SH>;
  constexpr int AW = TCMode<MODE>::AW, BW = TCMode<MODE>::BW;
  constexpr int kSlots = SH::kSlots, kTopo = SH::kTopo, kHalves = SH::kHalves;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kSlots];
  __shared__ int released[kSlots];  // warps done with the slot's current stage
  __shared__ int s_issued;          // stages issued so far

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int tw = warp / kHalves, half = warp % kHalves;
  const int tiles_b = (n_bands + kSwB - 1) / kSwB;
  const int tile = blockIdx.x / (kSwB * kSwG), within = blockIdx.x % (kSwB * kSwG);
  const int band = (tile % tiles_b) * kSwB + within % kSwB;
  const int grp = (tile / tiles_b) * kSwG + within / kSwB;
  if (band >= n_bands || grp >= n_groups) return;  // CTA-uniform
  const int n_topo = min(kTopo, a.B - grp * kTopo);
  const int b = grp * kTopo + tw;
  const int TT = a.TT;
  const int t0 = tci * TC;
  const int n_mt = a.E_mon_pad >> 4, n_nt = a.O_pad >> 3;
  const int n_stages = n_nt / kSN;
  const int mt_band = band * kHalves * MW;  // first m-tile of the band
  const int mt0 = mt_band + half * MW;      // first m-tile of this warp
  const size_t Ep = a.E_mon_pad;
  const bool producer = threadIdx.x == 0;

  if (producer) {
    for (int sl = 0; sl < kSlots; ++sl) {
      mbar_init(&full[sl], 1);
      released[sl] = 0;
    }
    s_issued = kSlots < n_stages ? kSlots : n_stages;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // stage s -> slot s % kSlots; run by all lanes of warp 0, one copy per lane
  auto issue = [&](int s) {
    const int sl = s % kSlots;
    unsigned char* base = smem + (size_t)sl * S::kBytes;
    if (lane == 0) mbar_expect_tx(&full[sl], S::kNf + n_topo * S::kTopoBytes);
    __syncwarp();
    const int nt0 = s * kSN;
    const int n_copies = kHalves * MW + 2 * n_topo;
    for (int c = lane; c < n_copies; c += 32) {
      if (c < kHalves * MW) {
        bulk_copy(base + c * (kSN * 512), a.Nf + ((size_t)(mt_band + c) * n_nt + nt0) * 32, kSN * 512, &full[sl]);
      } else {
        const int w = (c - kHalves * MW) >> 1;
        const size_t bw = (size_t)grp * kTopo + w;
        unsigned char* wb = base + S::kNf + w * S::kTopoBytes;
        if (((c - kHalves * MW) & 1) == 0)
          bulk_copy(wb, a.Vb + (bw * n_nt + nt0) * 32 * BW, S::kVb, &full[sl]);
        else
          bulk_copy(wb + S::kVb, a.gq + ((bw * a.n_tch + tci) * n_nt + nt0) * 4 * TC * 2, S::kG, &full[sl]);
      }
    }
  };
  if (warp == 0)
    for (int s = 0; s < kSlots && s < n_stages; ++s) issue(s);
  __syncthreads();  // stages 0.. are in flight and the release counters are set

  if (tw >= n_topo) return;  // past the batch end; not counted by the empty barriers

  uint32_t A[MW][AW];
  float f[MW][2][TC], m[MW][2][TC];
  const uint4* Ua = reinterpret_cast<const uint4*>(a.Ua);
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

  bool ok = true;
  int pending = 0;  // first stage whose copies may still be in flight
  for (int s = 0; s < n_stages; ++s) {
    const int sl = s % kSlots;
    const uint32_t par = (uint32_t)(s / kSlots) & 1u;
    // every lane observes the stage's completion; the decision is warp-uniform
    if (!__all_sync(0xffffffffu, mbar_wait(&full[sl], par))) {
      ok = false;
      break;
    }
    pending = s + 1;
    const unsigned char* base = smem + (size_t)sl * S::kBytes;
    const float4* nfs = reinterpret_cast<const float4*>(base) + half * MW * kSN * 32 + lane;
    const uint32_t* vbs = reinterpret_cast<const uint32_t*>(base + S::kNf + tw * S::kTopoBytes) + lane * BW;
    const float* gs = reinterpret_cast<const float*>(base + S::kNf + tw * S::kTopoBytes + S::kVb) + q * TC * 2;
#pragma unroll
    for (int j = 0; j < kSN; ++j) {
      uint32_t vb[BW];
      if constexpr (BW == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(vbs + j * 32 * BW);
        vb[0] = v.x;
        vb[1] = v.y;
      } else {
        const uint4 v = *reinterpret_cast<const uint4*>(vbs + j * 32 * BW);
        vb[0] = v.x;
        vb[1] = v.y;
        vb[2] = v.z;
        vb[3] = v.w;
      }
      float gv[2 * TC];
      if constexpr (TC == 1) {
        const float2 v = *reinterpret_cast<const float2*>(gs + j * 8 * TC);
        gv[0] = v.x;
        gv[1] = v.y;
      } else {
#pragma unroll
        for (int x = 0; x < TC / 2; ++x) {
          const float4 v = *reinterpret_cast<const float4*>(gs + j * 8 * TC + 4 * x);
          gv[4 * x + 0] = v.x;
          gv[4 * x + 1] = v.y;
          gv[4 * x + 2] = v.z;
          gv[4 * x + 3] = v.w;
        }
      }
#pragma unroll
      for (int i = 0; i < MW; ++i) {
        float4 d = nfs[(i * kSN + j) * 32];
        if (MODE == kModeTF32x3) {
          mma_tf32(d, &A[i][0], vb[0], vb[1]);  // U_hi V_hi
          mma_tf32(d, &A[i][4], vb[0], vb[1]);  // U_lo V_hi
          mma_tf32(d, &A[i][0], vb[2], vb[3]);  // U_hi V_lo
        } else if (MODE == kModeFP16x3) {
          mma_fp16(d, &A[i][0], vb[0], vb[0]);  // [U_hi | U_lo] [V_hi ; V_hi]
          mma_fp16(d, &A[i][0], vb[1], 0u);     // [U_hi | U_lo] [V_lo ; 0]
        } else if (MODE == kModeBF16x3) {
          mma_bf16(d, &A[i][0], vb[0], vb[0]);
          mma_bf16(d, &A[i][0], vb[1], 0u);
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
    // release the slot; the last warp to release it issues the refill
    __syncwarp();
    int last = 0;
    if (lane == 0) {
      __threadfence_block();  // this warp's reads of the slot precede the release
      last = atomicAdd(&released[sl], 1) == kHalves * n_topo - 1;
      if (last) {
        atomicExch(&released[sl], 0);
        __threadfence_block();  // the reset precedes the refill that other warps wait for
      }
    }
    if (__shfl_sync(0xffffffffu, last, 0) && s + kSlots < n_stages) {
      issue(s + kSlots);
      if (lane == 0) atomicMax(&s_issued, s + kSlots + 1);
    }
  }

  if (!ok) {
    atomicExch(a.status, TTO_E_TIMEOUT);
    if (lane == 0) {
      // let the copies already in flight land before the CTA releases its
      // shared memory (bounded like every other wait)
      const int issued = atomicAdd(&s_issued, 0);
      for (int s = pending; s < issued; ++s) mbar_wait(&full[s % kSlots], (uint32_t)(s / kSlots) & 1u);
    }
    return;
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
    float* pp = a.part + ((size_t)b * a.n_parts + (size_t)(band * kHalves + half) * a.n_tch + tci) * 4;
    pp[0] = over;
    pp[1] = cnt;
    pp[2] = ml;
    pp[3] = 0.f;
  }
}

// ------------------------------------------------------------ fragment packing
// Rows l of U (FP32 [B][E_mon_pad][8]) go to A fragments of 16-row tiles, lane
// = 4 g + q with g = l % 8:
//   16-bit modes (m16n8k16, K = [hi 0..7 | lo 0..7]): word (l % 16) / 8 holds
//     (hi[2q], hi[2q+1]), word 2 + (l % 16) / 8 holds (lo[2q], lo[2q+1]);
//   tf32 (m16n8k8): words (l%16)/8 and 2+(l%16)/8 hold hi[q], hi[q+4], words
//     4+... and 6+... the same for lo.
// Columns c of V go to B fragments of 8-outage tiles, lane = 4 (c % 8) + q:
//   16-bit modes: (hi[2q], hi[2q+1]), (lo[2q], lo[2q+1]); tf32: hi[q], hi[q+4], lo[q], lo[q+4].
// g [B][O_pad][TT] goes to [B][n_tch][O_pad/8][q][TC][2].
__device__ __forceinline__ uint32_t pack_half2(float lo_elem, float hi_elem, bool fp16) {
  uint32_t a, b;
  if (fp16) {
    a = __half_as_ushort(__float2half_rn(lo_elem));
    b = __half_as_ushort(__float2half_rn(hi_elem));
  } else {
    a = __bfloat16_as_ushort(__float2bfloat16_rn(lo_elem));
    b = __bfloat16_as_ushort(__float2bfloat16_rn(hi_elem));
  }
  return a | (b << 16);
}

__device__ __forceinline__ void split16(float x, bool fp16, float& hi, float& lo) {
  hi = fp16 ? __half2float(__float2half_rn(x)) : __bfloat162float(__float2bfloat16_rn(x));
  lo = x - hi;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Power-of-two exponent that balances max|U| 2^e and max|V| 2^-e.
__device__ __forceinline__ int balance_exponent(float umax, float vmax) {
  if (!(umax > 0.f) || !(vmax > 0.f)) return 0;
  int eu, ev;
  frexpf(umax, &eu);
  frexpf(vmax, &ev);
  return (ev - eu) / 2;
}

__global__ void pack_factors_kernel(EvalArgs a, int mode) {
  const int rows = a.E_mon_pad, cols = a.O_pad;
  const size_t per = (size_t)rows + cols;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per * a.B) return;
  const int b = (int)(i / per);
  const int x = (int)(i % per);
  const TopoInfo inf = a.info[b];
  const bool fp16 = mode == kModeFP16x3;
  const int e = fp16 ? balance_exponent(inf.umax, inf.vmax) : 0;
  if (fp16 && (ldexpf(inf.umax, e) > 16384.f || ldexpf(inf.vmax, -e) > 16384.f))
    atomicExch(a.status, TTO_E_ARG);  // low-rank factors beyond the fp16 range
  if (x < rows) {
    const int l = x;
    const float4* ur = reinterpret_cast<const float4*>(a.U + ((size_t)b * rows + l) * 8);
    const float4 u0 = ur[0], u1 = ur[1];
    float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    const int mt = l >> 4, r = l & 15, gg = r & 7, hf = r >> 3;
    if (mode == kModeTF32x3) {
      uint32_t hi[8], lo[8];
      for (int j = 0; j < 8; ++j) {
        hi[j] = to_tf32(u[j]);
        lo[j] = to_tf32(u[j] - __uint_as_float(hi[j]));
      }
      uint32_t* base = a.Ua + ((size_t)b * (rows >> 4) + mt) * 256;
      for (int q = 0; q < 4; ++q) {
        uint32_t* w = base + (gg * 4 + q) * 8;
        w[hf] = hi[q];
        w[2 + hf] = hi[q + 4];
        w[4 + hf] = lo[q];
        w[6 + hf] = lo[q + 4];
      }
    } else {
      float hi[8], lo[8];
      for (int j = 0; j < 8; ++j) split16(ldexpf(u[j], e), fp16, hi[j], lo[j]);
      uint32_t* base = a.Ua + ((size_t)b * (rows >> 4) + mt) * 128;
      for (int q = 0; q < 4; ++q) {
        uint32_t* w = base + (gg * 4 + q) * 4;
        w[hf] = pack_half2(hi[2 * q], hi[2 * q + 1], fp16);
        w[2 + hf] = pack_half2(lo[2 * q], lo[2 * q + 1], fp16);
      }
    }
    return;
  }
  const int c = x - rows;
  const float4* vr = reinterpret_cast<const float4*>(a.V + ((size_t)b * cols + c) * 8);
  const float4 v0 = vr[0], v1 = vr[1];
  float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
  const int ntl = c >> 3, cc = c & 7, n_nt = cols >> 3;
  const size_t tl = (size_t)b * n_nt + ntl;
  if (mode == kModeTF32x3) {
    uint32_t hi[8], lo[8];
    for (int j = 0; j < 8; ++j) {
      hi[j] = to_tf32(v[j]);
      lo[j] = to_tf32(v[j] - __uint_as_float(hi[j]));
    }
    uint32_t* vb = a.Vb + tl * 128;
    for (int q = 0; q < 4; ++q) {
      uint32_t* w = vb + (cc * 4 + q) * 4;
      w[0] = hi[q];
      w[1] = hi[q + 4];
      w[2] = lo[q];
      w[3] = lo[q + 4];
    }
  } else {
    float hi[8], lo[8];
    for (int j = 0; j < 8; ++j) split16(ldexpf(v[j], -e), fp16, hi[j], lo[j]);
    uint32_t* vb = a.Vb + tl * 64;
    for (int q = 0; q < 4; ++q) {
      vb[(cc * 4 + q) * 2 + 0] = pack_half2(hi[2 * q], hi[2 * q + 1], fp16);
      vb[(cc * 4 + q) * 2 + 1] = pack_half2(lo[2 * q], lo[2 * q + 1], fp16);
    }
  }
  const float* gr = a.gg + ((size_t)b * cols + c) * a.TT;
  for (int t = 0; t < a.TT; ++t) {
    const int ci = t / a.TC, tt = t - ci * a.TC;
    const size_t slab = ((size_t)b * a.n_tch + ci) * n_nt + ntl;
    a.gq[((slab * 4 + (cc >> 1)) * a.TC + tt) * 2 + (cc & 1)] = gr[t];
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

template <int TC, int MW, int MODE, class SH>
static int launch_tc(EvalArgs& a, int tci, cudaStream_t s) {
  using S = Slot<MW, MODE, TC, SH>;
  const size_t smem = (size_t)SH::kSlots * S::kBytes;
  static bool attr_set[64] = {};  // per device; set once, outside any stream capture that follows
  int dev = 0;
  TTO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(TTO_E_ARG, "device %d out of range", dev);
  if (!attr_set[dev]) {
    TTO_CUDA_TRY(cudaFuncSetAttribute(sweep_tc_kernel<TC, MW, MODE, SH>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set[dev] = true;
  }
  const int n_bands = a.E_mon_pad / (16 * SH::kHalves * MW);
  const int n_groups = (a.B + SH::kTopo - 1) / SH::kTopo;
  const int tiles_b = (n_bands + kSwB - 1) / kSwB, tiles_g = (n_groups + kSwG - 1) / kSwG;
  const size_t blocks = (size_t)tiles_b * tiles_g * kSwB * kSwG;
  if (blocks > 0x7fffffffu) return set_error(TTO_E_ARG, "batch too large for one sweep launch");
  sweep_tc_kernel<TC, MW, MODE, SH><<<(unsigned)blocks, SH::kWarps * 32, smem, s>>>(a, tci, n_bands, n_groups);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

template <int MODE, class SH>
static int launch_tc_chunk(EvalArgs& a, int tci, cudaStream_t s) {
  switch (a.TC) {
    case 1: return launch_tc<1, 2, MODE, SH>(a, tci, s);
    case 2: return launch_tc<2, 2, MODE, SH>(a, tci, s);
    case 4: return launch_tc<4, 2, MODE, SH>(a, tci, s);
    case 8: return launch_tc<8, 1, MODE, SH>(a, tci, s);
  }
  return set_error(TTO_E_ARG, "unsupported timestep chunk %d", a.TC);
}

template <int MODE>
static int launch_tc_shape(EvalArgs& a, int tci, cudaStream_t s) {
  switch (a.shape) {
    case 1: return launch_tc_chunk<MODE, Shape1>(a, tci, s);
    case 2: return launch_tc_chunk<MODE, Shape2>(a, tci, s);
    case 3: return launch_tc_chunk<MODE, Shape3>(a, tci, s);
    default: return launch_tc_chunk<MODE, Shape0>(a, tci, s);
  }
}

static int tc_mode(int precision) {
  switch (precision) {
    case TTO_PREC_TF32X3: return kModeTF32x3;
    case TTO_PREC_FP16X3: return kModeFP16x3;
    case TTO_PREC_BF16: return kModeBF16;
    default: return kModeBF16x3;
  }
}

int launch_sweep_tc(EvalArgs& a, cudaStream_t s) {
  if (a.shape == kUmmaShape) return launch_sweep_umma(a, s);
  if ((a.O_pad >> 3) % kSN != 0) return set_error(TTO_E_ARG, "outage padding is not a multiple of the stage width");
  if ((a.E_mon_pad >> 4) % 8 != 0) return set_error(TTO_E_ARG, "monitored padding is not a multiple of the band");
  if (a.shape < 0 || a.shape >= kNumShapes) return set_error(TTO_E_ARG, "unknown sweep shape %d", a.shape);
  const int mode = tc_mode(a.precision);
  const size_t threads = ((size_t)a.E_mon_pad + a.O_pad) * a.B;
  pack_factors_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a, mode);
  TTO_CUDA_TRY(cudaGetLastError());
  const int mw = a.TC <= 4 ? 2 : 1;
  a.n_parts = (a.E_mon_pad / (16 * mw)) * a.n_tch;
  for (int ci = 0; ci < a.n_tch; ++ci) {
    int rc;
    switch (mode) {
      case kModeTF32x3: rc = launch_tc_shape<kModeTF32x3>(a, ci, s); break;
      case kModeFP16x3: rc = launch_tc_shape<kModeFP16x3>(a, ci, s); break;
      case kModeBF16: rc = launch_tc_shape<kModeBF16>(a, ci, s); break;
      default: rc = launch_tc_shape<kModeBF16x3>(a, ci, s); break;
    }
    if (rc) return rc;
  }
  return TTO_OK;
}

}  // namespace tto
