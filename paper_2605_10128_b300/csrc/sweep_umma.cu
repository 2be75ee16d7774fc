// Fused N-1 sweep on the fifth-generation tensor cores (tcgen05, sm_100 family).
//
// Same arithmetic as the mma.sync sweep (sweep_tc.cu): for every monitored row
// l, outage c and timestep t,
//     F_lc[t] = f'_l[t] + (U_l . V_c - N_lc) g_c[t],   fmax_l[t] = max_c |F_lc[t]|,
// with the rank-k product split into TF32 parts, U V^T = U_hi V_hi + U_lo V_hi +
// U_hi V_lo (about 2^-21 relative error), and F never stored.
//
// CTA = one band of 128 monitored rows x 4 topologies, all outage columns in
// chunks of 64.  Roles:
//   warp 0 (one lane)   streams each chunk's operands into a 3-slot shared-memory
//                       ring with bulk copies (cp.async.bulk, completion counted
//                       on an mbarrier): the -N tile of the band in mma
//                       C-fragment order (shared by the four topologies) and
//                       per topology the V_hi / V_lo tiles and the g values;
//   warp 1 (one lane)   per chunk and topology, issues three tcgen05.mma
//                       (M = 128, N = 64, K = 8, kind::tf32) computing U V^T
//                       into that topology's accumulator in tensor memory (two
//                       64-column buffers per topology, 512 columns in all) and
//                       commits them to an mbarrier;
//   warps 2, 3          idle: they complete warpgroup 0, whose registers
//                       (setmaxnreg) go to the epilogue;
//   warps 4..19         four epilogue warpgroups, one per topology: each warp
//                       reads its 32 accumulator lanes with tcgen05.ld.16x256b,
//                       whose register layout is the mma C fragment (a thread
//                       holds 4 rows x 2 columns of every 8-column block, so
//                       one g value serves 4 rows and one 16-byte load brings
//                       the matching -N values), adds -N, and keeps the running
//                       maxima of every timestep in registers; the 4 lanes that
//                       share rows combine theirs at the end.
// (Copying -N into each accumulator with tcgen05.cp instead measured slower:
// the copies of four topologies' accumulators per chunk became the critical
// path.)
// The U tiles of the four topologies stay in shared memory for the whole
// sweep.  Operand tiles use the canonical K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes, 128 bytes apart along K and 256 bytes apart
// along M/N.  Every wait is bounded (about a second): a wait that gives
// up raises a CTA-wide abort flag and sets the status word to TTO_E_TIMEOUT;
// before the CTA exits, the copies and MMAs it issued are waited for (again
// bounded) and the tensor memory is released.
#include <stdint.h>

#include "sweep.cuh"

namespace tto {

namespace {

constexpr int kUTopo = 4;                 // topologies per CTA (one epilogue warpgroup each)
constexpr int kUNC = 64;                  // outage columns per chunk (MMA N)
constexpr int kUStages = 3;               // shared-memory ring slots
constexpr int kUTileB = 16, kUTileG = 64;  // launch order: tiles of 16 bands x 64 topology groups
constexpr int kUEpiWarps = 4 * kUTopo;    // 16 epilogue warps
// warpgroup 0: producer (warp 0), MMA issuer (warp 1), two idle warps;
// warpgroups 1-4: the epilogue
constexpr int kUThreads = 32 * (4 + kUEpiWarps);
// Register split (setmaxnreg): the block is launched at 96 registers per
// thread (640 x 96 = 61440, five warps per sub-partition), warpgroup 0 gives
// back down to 56 and the epilogue warps grow to 104: 128 x 56 + 512 x 104 =
// 60416 registers, within the launch's 61440, so no increase can wait.
constexpr int kULaunchRegs = 96, kUCtlRegs = 56, kUEpiRegs = 104;
static_assert(128 * kUCtlRegs + 32 * kUEpiWarps * kUEpiRegs <= kUThreads * kULaunchRegs,
              "register split exceeds the launch allocation");
static_assert((kUThreads / 32 + 3) / 4 * 32 * kULaunchRegs <= 16384, "launch registers exceed a sub-partition");
constexpr uint32_t kUTmemCols = 512;      // 4 topologies x 2 buffers x 64 columns
constexpr uint32_t kUA = 2 * 128 * 8 * 4;        // U_hi + U_lo tiles of one topology (8 KB)
constexpr uint32_t kUN = 128 * kUNC * 4;         // -N tile of a chunk (32 KB)
constexpr uint32_t kUV = 2 * kUNC * 8 * 4;       // V_hi + V_lo tiles of a chunk (4 KB)
constexpr long long kUWaitCycles = 1ll << 31;    // ~1 s at 2 GHz

template <int TC>
struct UCfg {
  static constexpr uint32_t kG = kUNC * TC * 4;           // g values of a chunk
  static constexpr uint32_t kTopoBytes = kUV + kG;
  static constexpr uint32_t kStage = kUN + kUTopo * kTopoBytes;
  static constexpr uint32_t kSmem = kUTopo * kUA + kUStages * kStage + 1024;  // + alignment slack
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
// mbarrier.try_wait: returns once the phase completed or after a
// hardware-chosen suspension, so polling warps leave the issue slots free.
__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false when it gave up, when another role of the CTA raised
// the abort flag, or when another CTA already timed out (status word), so that
// one timeout ends the whole launch within about a second.
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                                         const volatile int* status, long long limit = kUWaitCycles) {
  if (bar_try(b, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (bar_try(b, parity)) return true;
    if (*abort_flag || *status == TTO_E_TIMEOUT) return false;
    if (clock64() - t0 > limit) return false;
  }
}

// One thread waits, through the sweep's bounded wait, on an mbarrier that
// nothing completes; when the wait gives up it records TTO_E_TIMEOUT exactly
// as a sweep does.
__global__ void bounded_wait_probe_kernel(int* status, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_abort;
  bar_init(&bar, 1);
  s_abort = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!bar_wait(&bar, 0, &s_abort, status, limit)) atomicExch(status, TTO_E_TIMEOUT);
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(b))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// start address, leading (K) byte offset, stride (M/N) byte offset, the fixed
// descriptor version 1 at bit 46, base offset 0, swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = su32(p);
  return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::tf32: F32 accumulator (bits 4-5 = 1), A and B
// TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdescTF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kUNC >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(kIdescTF32), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}

// Two 16-lane x 8-column blocks (16x256b.x2): thread i gets lanes base + i/4
// and base + i/4 + 8, columns 2 (i % 4) and 2 (i % 4) + 1 of each block, in
// r[4 blk + {0, 1}] (first lane) and r[4 blk + {2, 3}] (second lane).
__device__ __forceinline__ void tmem_ld_2blk(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
// Wait for the thread's outstanding tcgen05.ld; the registers are tied to the
// wait so that no use of them moves above it.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r0)[8], uint32_t (&r1)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r0[0]), "+r"(r0[1]), "+r"(r0[2]), "+r"(r0[3]), "+r"(r0[4]), "+r"(r0[5]), "+r"(r0[6]),
                 "+r"(r0[7]), "+r"(r1[0]), "+r"(r1[1]), "+r"(r1[2]), "+r"(r1[3]), "+r"(r1[4]), "+r"(r1[5]),
                 "+r"(r1[6]), "+r"(r1[7])
               :
               : "memory");
}

// Packed pairs of FP32 values in one 64-bit register (sm_100 family):
// add.rn.f32x2 / fma.rn.f32x2 process two elements per instruction, and the
// three-input max takes both absolute values at once.
__device__ __forceinline__ uint64_t pack2(float x, float y) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// max(m, |v.x|, |v.y|)
__device__ __forceinline__ float max_abs_pair(float m, uint64_t v) {
  float r;
  asm("{\n .reg .f32 x, y;\n mov.b64 {x, y}, %2;\n abs.f32 x, x;\n abs.f32 y, y;\n max.f32 %0, %1, x, y;\n}"
      : "=f"(r)
      : "f"(m), "l"(v));
  return r;
}

// One step of 16 columns (two 8-column blocks): A holds U V^T of rows {r,
// r+8} and B of rows {r+16, r+24} of the warp's 32 (r = lane / 4), columns
// 2 (lane % 4) + {0, 1} of each block, adjacent registers; nf points at this
// lane's -N fragment of the first 16-row tile and block (the second 16-row
// tile is 8 fragment tiles further on); gs holds g of column pairs with the
// two columns interleaved per timestep, so each 64-bit load is the g pair of
// one timestep.  f2 holds (f', f') per row and timestep.
template <int TC>
__device__ __forceinline__ void epilogue_step(const uint32_t (&A)[8], const uint32_t (&B)[8], const float4* nf,
                                              const float* gs, int c0, const uint64_t (&f2)[4][TC],
                                              float (&m)[4][TC]) {
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    const ulonglong2 na = *reinterpret_cast<const ulonglong2*>(nf + (c0 / 8 + blk) * 32);
    const ulonglong2 nb = *reinterpret_cast<const ulonglong2*>(nf + (8 + c0 / 8 + blk) * 32);
    const int pair = (c0 + 8 * blk) / 2 + (threadIdx.x & 3);
    uint64_t g[TC];  // (g[c][t], g[c + 1][t])
    if constexpr (TC >= 2) {
#pragma unroll
      for (int x = 0; x < TC / 2; ++x) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(gs + pair * 2 * TC + 4 * x);
        g[2 * x] = v.x;
        g[2 * x + 1] = v.y;
      }
    } else {
      g[0] = *reinterpret_cast<const uint64_t*>(gs + pair * 2);
    }
    const uint64_t d[4] = {add2(pack2(__uint_as_float(A[4 * blk]), __uint_as_float(A[4 * blk + 1])), na.x),
                           add2(pack2(__uint_as_float(A[4 * blk + 2]), __uint_as_float(A[4 * blk + 3])), na.y),
                           add2(pack2(__uint_as_float(B[4 * blk]), __uint_as_float(B[4 * blk + 1])), nb.x),
                           add2(pack2(__uint_as_float(B[4 * blk + 2]), __uint_as_float(B[4 * blk + 3])), nb.y)};
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int t = 0; t < TC; ++t) m[r][t] = max_abs_pair(m[r][t], fma2(d[r], g[t], f2[r][t]));
  }
}

// Launched at 96 registers per thread (five warps per sub-partition allow no
// more); the split above then moves registers from warpgroup 0 to the
// epilogue, which at 96 spilled.
template <int TC>
__global__ void __launch_bounds__(kUThreads, 1)
    sweep_umma_kernel(EvalArgs a, int tci, int n_bands, int n_groups) {
  using C = UCfg<TC>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar_a, full[kUStages], empty[kUStages], tfull[kUTopo][2], tempty[kUTopo][2],
      mma_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  volatile int* abort_flag = &s_abort;
  auto give_up = [&]() {
    atomicExch(a.status, TTO_E_TIMEOUT);
    *abort_flag = 1;
  };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CTAs walk tiles of kUTileB bands x kUTileG groups, bands fastest: the
  // groups that share a band's -N tile run close together in time (16 x 64
  // moved 51 GB from DRAM per benchmark launch, 16 x 16 83 GB, at equal time)
  const int tiles_b = (n_bands + kUTileB - 1) / kUTileB;
  const int tile = blockIdx.x / (kUTileB * kUTileG), within = blockIdx.x % (kUTileB * kUTileG);
  const int band = (tile % tiles_b) * kUTileB + within % kUTileB;
  const int grp = (tile / tiles_b) * kUTileG + within / kUTileB;
  if (band >= n_bands || grp >= n_groups) return;  // CTA-uniform, before any barrier or allocation
  // an earlier CTA gave up: end at once, every warp alike (one thread reads
  // the status word: the register split below needs all warps present)
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = *(const volatile int*)a.status == TTO_E_TIMEOUT;
  __syncthreads();
  if (s_skip) return;
  const int n_topo = min(kUTopo, a.B - grp * kUTopo);
  const int n_chunks = a.O_pad / kUNC;
  unsigned char* smA = smem;                          // [topo][hi, lo][128 x 8]
  unsigned char* smS = smem + kUTopo * kUA;           // ring slots

  if (threadIdx.x == 0) {
    bar_init(&bar_a, 1);
    for (int s = 0; s < kUStages; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 4 * n_topo);
    }
    for (int b = 0; b < kUTopo; ++b)
      for (int x = 0; x < 2; ++x) {
        bar_init(&tfull[b][x], 1);
        bar_init(&tempty[b][x], 4);
      }
    bar_init(&mma_done, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(kUTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  int issued = 0;  // producer: stages issued
  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kUCtlRegs) : "memory");
    if (warp == 0 && lane == 0) {
      // U tiles of the group's topologies, then the ring
      bar_expect_tx(&bar_a, n_topo * kUA);
      for (int b = 0; b < n_topo; ++b)
        bulk_g2s(smA + b * kUA, a.Ua + (((size_t)(grp * kUTopo + b) * n_bands + band) * (kUA / 4)), kUA, &bar_a);
      for (int s = 0; s < n_chunks; ++s) {
        const int slot = s % kUStages;
        if (s >= kUStages && !bar_wait(&empty[slot], (uint32_t)((s / kUStages) - 1) & 1u, abort_flag, a.status)) {
          give_up();
          break;
        }
        unsigned char* st = smS + (size_t)slot * C::kStage;
        bar_expect_tx(&full[slot], kUN + n_topo * C::kTopoBytes);
        // -N fragments of the band's 8 16-row tiles x the chunk's 8 column blocks
        for (int i = 0; i < 8; ++i)
          bulk_g2s(st + i * (kUN / 8), a.Nf + ((size_t)(band * 8 + i) * (a.O_pad / 8) + (size_t)s * (kUNC / 8)) * 32,
                   kUN / 8, &full[slot]);
        for (int b = 0; b < n_topo; ++b) {
          const size_t bt = (size_t)grp * kUTopo + b;
          unsigned char* tb = st + kUN + b * C::kTopoBytes;
          bulk_g2s(tb, a.Vb + (bt * n_chunks + s) * (kUV / 4), kUV, &full[slot]);
          bulk_g2s(tb + kUV, a.gq + ((bt * a.n_tch + tci) * a.O_pad + (size_t)s * kUNC) * TC, C::kG, &full[slot]);
        }
        issued = s + 1;
      }
    } else if (warp == 1 && lane == 0) {
      if (!bar_wait(&bar_a, 0, abort_flag, a.status)) {
        give_up();
      } else {
        // This thread shares its sub-partition with four busy epilogue warps,
        // so its per-chunk work is kept to a few instructions: descriptors of
        // the first U and V tiles are built once and the others reached by
        // adding offsets to the start-address field (16-byte units; every
        // offset is a multiple of 16 bytes and all of shared memory lies below
        // 2^14 units, so the field never carries into its neighbours).
        const uint64_t a_d0 = smem_desc(smA, 128, 256), v_d0 = smem_desc(smS + kUN, 128, 256);
        constexpr uint32_t kDA = kUA >> 4, kDAlo = (kUA / 2) >> 4, kDV = C::kTopoBytes >> 4, kDVlo = (kUV / 2) >> 4,
                           kDS = C::kStage >> 4;
        int slot = 0;
        uint32_t ring_ph = 0;
        uint64_t v_ds = v_d0;
        for (int s = 0; s < n_chunks; ++s) {
          const int buf = s & 1;
          if (!bar_wait(&full[slot], ring_ph, abort_flag, a.status)) {
            give_up();
            break;
          }
          bool ok = true;
          for (int b = 0; b < n_topo; ++b) {
            if (s >= 2 && !bar_wait(&tempty[b][buf], (uint32_t)((s >> 1) - 1) & 1u, abort_flag, a.status)) {
              give_up();
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t a_hi = a_d0 + (uint64_t)(b * kDA), v_hi = v_ds + (uint64_t)(b * kDV);
            const uint32_t d = tmem + (uint32_t)(b * 2 * kUNC + buf * kUNC);
            umma_tf32(d, a_hi, v_hi, 0u);
            umma_tf32(d, a_hi + kDAlo, v_hi, 1u);
            umma_tf32(d, a_hi, v_hi + kDVlo, 1u);
            umma_commit(&tfull[b][buf]);
          }
          if (!ok) break;
          if (++slot == kUStages) {
            slot = 0;
            ring_ph ^= 1u;
            v_ds = v_d0;
          } else {
            v_ds += kDS;
          }
        }
      }
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kUEpiRegs) : "memory");
    const int e = warp - 4, b = e >> 2, q = warp & 3;  // q: this warp's tensor-memory lane quarter
    if (b < n_topo) {
      const size_t bt = (size_t)grp * kUTopo + b;
      const int t0 = tci * TC;
      // rows of this thread within the band: 32 q + lane / 4 + {0, 8, 16, 24}
      const int rb = 32 * q + (lane >> 2);
      float m[4][TC];
      uint64_t f2[4][TC];  // (f', f') of every row and timestep
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int t = 0; t < TC; ++t) {
          const float fv = a.fp[(bt * a.TT + t0 + t) * (size_t)a.E_mon_pad + band * 128 + rb + 8 * r];
          f2[r][t] = pack2(fv, fv);
          m[r][t] = 0.f;
        }
      bool ok = true;
      // ring slot, its phase and the slot's shared-memory base advance
      // incrementally; the tensor-memory base of the topology is fixed
      int slot = 0;
      uint32_t ring_ph = 0;
      const unsigned char* st = smS;
      const uint32_t lo_base = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 2 * kUNC);
      const int noff = (2 * q) * 8 * 32 + lane;         // this lane's fragment, 16-row tile 2 q, block 0
      const int goff = kUN + b * C::kTopoBytes + kUV;   // g of this topology within a slot
      for (int s = 0; s < n_chunks && ok; ++s) {
        const int buf = s & 1;
        ok = __all_sync(0xffffffffu, bar_wait(&full[slot], ring_ph, abort_flag, a.status) &&
                                         bar_wait(&tfull[b][buf], (uint32_t)(s >> 1) & 1u, abort_flag, a.status));
        if (!ok) break;
        tc_fence_after();
        const float* gs = reinterpret_cast<const float*>(st + goff);
        const float4* nf = reinterpret_cast<const float4*>(st) + noff;
        const uint32_t lo = lo_base + (uint32_t)(buf * kUNC), hi = lo + (16u << 16);
        uint32_t A0[8], B0[8], A1[8], B1[8];
        tmem_ld_2blk(lo, A0);
        tmem_ld_2blk(hi, B0);
        tmem_wait_ld(A0, B0);
        tmem_ld_2blk(lo + 16, A1);
        tmem_ld_2blk(hi + 16, B1);
        epilogue_step<TC>(A0, B0, nf, gs, 0, f2, m);
        tmem_wait_ld(A1, B1);
        tmem_ld_2blk(lo + 32, A0);
        tmem_ld_2blk(hi + 32, B0);
        epilogue_step<TC>(A1, B1, nf, gs, 16, f2, m);
        tmem_wait_ld(A0, B0);
        tmem_ld_2blk(lo + 48, A1);
        tmem_ld_2blk(hi + 48, B1);
        epilogue_step<TC>(A0, B0, nf, gs, 32, f2, m);
        tmem_wait_ld(A1, B1);
        epilogue_step<TC>(A1, B1, nf, gs, 48, f2, m);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          bar_arrive(&tempty[b][buf]);
          bar_arrive(&empty[slot]);
        }
        if (++slot == kUStages) {
          slot = 0;
          ring_ph ^= 1u;
          st = smS;
        } else {
          st += C::kStage;
        }
      }
      if (!ok) {
        give_up();
      } else {
        // combine the 4 lanes that share rows, then per-row metrics and one
        // partial record per warp (its 32 rows)
        float over = 0.f, cnt = 0.f, ml = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int row = band * 128 + rb + 8 * r;
#pragma unroll
          for (int t = 0; t < TC; ++t) {
            float v = m[r][t];
            v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
            v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 2));
            m[r][t] = v;
          }
          if ((lane & 3) == 0 && row < a.E_mon) {
            const float lim = a.lim[row];
#pragma unroll
            for (int t = 0; t < TC; ++t) {
              const int tt = t0 + t;
              if (tt < a.n_t) {
                over += fmaxf(m[r][t] - lim, 0.f);
                cnt += m[r][t] > lim ? 1.f : 0.f;
                ml = fmaxf(ml, fmaxf(fabsf(__uint_as_float((uint32_t)f2[r][t])), m[r][t]) / lim);
                if (a.fmax) a.fmax[(bt * a.n_t + tt) * a.E_mon + row] = m[r][t];
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
          float* pp = a.part + (bt * a.n_parts + (size_t)(band * 4 + q) * a.n_tch + tci) * 4;
          pp[0] = over;
          pp[1] = cnt;
          pp[2] = ml;
          pp[3] = 0.f;
        }
      }
    }
  }
  __syncthreads();
  // drain: no copy or MMA of this CTA may still be in flight when it exits
  if (warp == 0 && lane == 0) {
    for (int s = issued > kUStages ? issued - kUStages : 0; s < issued; ++s) {
      int dummy = 0;
      bar_wait(&full[s % kUStages], (uint32_t)(s / kUStages) & 1u, &dummy, &dummy);
    }
  } else if (warp == 1 && lane == 0) {
    int dummy = 0;
    umma_commit(&mma_done);
    bar_wait(&mma_done, 0, &dummy, &dummy);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUTmemCols) : "memory");
  }
}

// U rows -> [B][band][hi, lo][128 x 8]; V columns -> [B][chunk][hi, lo][64 x 8];
// g -> [B][t-chunk][O_pad / 2][TC][2], column pairs interleaved (zero beyond
// the padded timesteps).
__global__ void pack_umma_kernel(EvalArgs a) {
  const int rows = a.E_mon_pad, cols = a.O_pad;
  const size_t per = (size_t)rows + cols;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per * a.B) return;
  const int b = (int)(i / per);
  const int x = (int)(i % per);
  if (x < rows) {
    const int l = x, band = l >> 7, r = l & 127;
    const float4* ur = reinterpret_cast<const float4*>(a.U + ((size_t)b * rows + l) * 8);
    const float4 u0 = ur[0], u1 = ur[1];
    const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    uint32_t* base = a.Ua + ((size_t)b * (rows >> 7) + band) * 2048;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t hi = tf32_bits(u[k]);
      base[canon(r, k)] = hi;
      base[1024 + canon(r, k)] = tf32_bits(u[k] - __uint_as_float(hi));
    }
  } else {
    const int c = x - rows, chunk = c / kUNC, n = c % kUNC;
    const float4* vr = reinterpret_cast<const float4*>(a.V + ((size_t)b * cols + c) * 8);
    const float4 v0 = vr[0], v1 = vr[1];
    const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint32_t* base = a.Vb + ((size_t)b * (cols / kUNC) + chunk) * 1024;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t hi = tf32_bits(v[k]);
      base[canon(n, k)] = hi;
      base[512 + canon(n, k)] = tf32_bits(v[k] - __uint_as_float(hi));
    }
    // g of column pairs, the two columns interleaved per timestep:
    // [B][t-pass][O_pad / 2][TC][2]
    for (int ci = 0; ci < a.n_tch; ++ci)
      for (int t = 0; t < a.TC; ++t) {
        const int tt = ci * a.TC + t;
        a.gq[((((size_t)b * a.n_tch + ci) * (cols / 2) + c / 2) * a.TC + t) * 2 + (c & 1)] =
            tt < a.TT ? a.gg[((size_t)b * cols + c) * a.TT + tt] : 0.f;
      }
  }
}

template <int TC>
int launch_umma_tc(EvalArgs& a, int tci, cudaStream_t s) {
  using C = UCfg<TC>;
  static bool attr_set[64] = {};
  int dev = 0;
  TTO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(TTO_E_ARG, "device %d out of range", dev);
  if (!attr_set[dev]) {
    TTO_CUDA_TRY(cudaFuncSetAttribute(sweep_umma_kernel<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem));
    // the register split is sized for a launch at exactly kULaunchRegs per
    // thread; with fewer, an increase could wait for registers that never come
    cudaFuncAttributes fa{};
    TTO_CUDA_TRY(cudaFuncGetAttributes(&fa, sweep_umma_kernel<TC>));
    if (fa.numRegs != kULaunchRegs)
      return set_error(TTO_E_CUDA, "tcgen05 sweep built with %d registers per thread, its register split needs %d",
                       fa.numRegs, kULaunchRegs);
    attr_set[dev] = true;
  }
  const int n_bands = a.E_mon_pad / 128;
  const int n_groups = (a.B + kUTopo - 1) / kUTopo;
  const int tiles_b = (n_bands + kUTileB - 1) / kUTileB, tiles_g = (n_groups + kUTileG - 1) / kUTileG;
  const size_t blocks = (size_t)tiles_b * tiles_g * (kUTileB * kUTileG);
  if (blocks > 0x7fffffffu) return set_error(TTO_E_ARG, "batch too large for one sweep launch");
  sweep_umma_kernel<TC><<<(unsigned)blocks, kUThreads, C::kSmem, s>>>(a, tci, n_bands, n_groups);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, sweep_umma_kernel<TC>);
    return set_error(TTO_E_CUDA,
                     "tcgen05 sweep launch: %s (threads %d, regs %d, max threads %d, static smem %zu, dynamic %u "
                     "of max %d, local %zu)",
                     cudaGetErrorString(e), kUThreads, fa.numRegs, fa.maxThreadsPerBlock, fa.sharedSizeBytes,
                     C::kSmem, fa.maxDynamicSharedSizeBytes, fa.localSizeBytes);
  }
  return TTO_OK;
}

}  // namespace

int bounded_wait_probe(int* status, long long cycles, cudaStream_t s) {
  bounded_wait_probe_kernel<<<1, 1, 0, s>>>(status, cycles);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

int launch_sweep_umma(EvalArgs& a, cudaStream_t s) {
  if (a.precision != TTO_PREC_TF32X3) return set_error(TTO_E_ARG, "the tcgen05 sweep runs in TF32X3 only");
  if (a.E_mon_pad % 128 != 0 || a.O_pad % kUNC != 0) return set_error(TTO_E_ARG, "padding does not fit the tcgen05 tiles");
  if (!a.Nf) return set_error(TTO_E_ARG, "fragment-ordered -N missing");
  // at most 4 timesteps per pass (the running maxima of 4 rows x 4 timesteps
  // stay in registers); more timesteps take more passes
  a.TC = a.TT < 4 ? a.TT : 4;
  a.n_tch = a.TT / a.TC;
  if (!a.umma_packed) {  // the split update did not write the operand layouts itself
    const size_t threads = ((size_t)a.E_mon_pad + a.O_pad) * a.B;
    pack_umma_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    TTO_CUDA_TRY(cudaGetLastError());
  }
  a.n_parts = (a.E_mon_pad / 32) * a.n_tch;
  for (int ci = 0; ci < a.n_tch; ++ci) {
    int rc;
    switch (a.TC) {
      case 1: rc = launch_umma_tc<1>(a, ci, s); break;
      case 2: rc = launch_umma_tc<2>(a, ci, s); break;
      case 4: rc = launch_umma_tc<4>(a, ci, s); break;
      default: return set_error(TTO_E_ARG, "unsupported timestep chunk %d", a.TC);
    }
    if (rc) return rc;
  }
  return TTO_OK;
}

}  // namespace tto
