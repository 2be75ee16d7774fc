// Learned surrogate screen for MapElites proposals (the paper has no
// counterpart; the network, its inputs and its online training are this
// library's own).
//
// An MLP with three hidden ReLU layers predicts log1p(-fitness) of a topology
// from (a) eight values of every split station and (b) the post-split N-0
// loading |f'_l| / fbar_l at timestep 0 of the R branches that are most loaded
// in the unsplit grid.  The screened MapElites step proposes many more
// candidates than it evaluates, scores them all, evaluates exactly only the
// best-scored ones, and trains the network online (mean squared error, Adam)
// on the exact pairs it has produced, kept in a replay ring.  The network
// learns the targets standardised by the mean and standard deviation of the
// ring's targets (recomputed after every append): the fitness of most splits of
// a large grid differs by a fraction of a percent, which an unscaled target
// would leave below the training noise.  Scores are returned unscaled.
//
// Numerics: parameters and Adam moments are FP32; every product rounds both
// operands to BF16 and accumulates in FP32 (tcgen05.mma kind::f16 with the
// accumulator in tensor memory for the dense products).  The station block of the input holds at most k_max non-zero
// 8-value slices per genome, so the first layer adds those slices of W1
// directly instead of multiplying a mostly-zero matrix, and its gradient is a
// per-station segmented sum.  Every reduction runs in a fixed order (no
// floating-point atomics), so results are reproducible call for call.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "philox.cuh"
#include "sweep.cuh"
#include "tto_internal.h"

struct tto_surrogate {
  tto_grid* g = nullptr;
  int H = 0, R = 0, S = 0, D = 0, k = 0;
  int cap = 0, mb = 0;
  double lr = 1e-3, beta1 = 0.9, beta2 = 0.999, eps = 1e-8;
  uint64_t seed = 0;
  long long step = 0;  // Adam steps taken
  size_t n_params = 0, oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, ow4 = 0, ob4 = 0;
  float* P = nullptr;     // packed parameters (FP32)
  float* G = nullptr;     // packed gradient
  float* Am = nullptr;    // Adam first moment
  float* Av = nullptr;    // Adam second moment
  float* W1sT = nullptr;  // [8S][H] station block of W1, transposed (refreshed after every update)
  float* wsk = nullptr;   // split-K partials of the weight gradients
  int* rows = nullptr;    // [R] branch ids of the loading features
  double* row_lim = nullptr;  // [R] their thermal limits
  double* Nsr = nullptr;  // [n_sw][R] N[rows[r]][movable branch] (the movable columns at those rows)
  double psum = 1.0;      // sum |p(t=0)|
  // per-batch buffers (capacity bcap rows)
  int bcap = 0;
  int* SI = nullptr;      // [bcap][k] station of each genome slot, -1 = empty
  uint32_t* SM = nullptr; // [S][ceil(bcap / 32)] bit r of word w: row 32 w + r splits the station
  float* SF = nullptr;    // [bcap][k][8] that station's eight values
  float* XD = nullptr;    // [bcap][R] loadings
  int* valid = nullptr;   // [bcap] 0 = the split islands the grid (or the genome is invalid)
  int2* nsm = nullptr;    // [bcap] descriptors: split stations, moved assets
  float *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *Y = nullptr;
  float *dH1 = nullptr, *dH2 = nullptr, *dH3 = nullptr, *dY = nullptr, *T = nullptr;
  int32_t* mb_topo = nullptr;  // [bcap][k] genomes of a training minibatch
  float* loss = nullptr;       // [2]: sum of squared errors, rows counted
  float* stats = nullptr;      // [3]: mean, standard deviation, 1 / deviation of the ring's targets
  // replay ring
  int rep_n = 0, rep_head = 0;
  int32_t* rep_genome = nullptr;  // [cap][k]
  float* rep_xd = nullptr;        // [cap][R]
  float* rep_t = nullptr;         // [cap] log1p(-fitness), NaN = no target
  // screening
  int pcap = 0;
  int32_t* prop = nullptr;              // [pcap][k] proposals
  unsigned long long* keys = nullptr;   // [keys_n] (score, index) sort keys
  int keys_n = 0;
  int32_t* sel = nullptr;               // [pcap] proposals chosen for exact evaluation
};

namespace tto {
namespace {

constexpr int kMaxHidden = 1024;
constexpr int kSortChunk = 2048;  // keys sorted per CTA in shared memory

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ------------------------------------------------------------------ GEMM
// C[M][N] (ldc) = opA(A) opB(B) + bias[n], then zeroed where mask[m][n] <= 0
// (mask has C's layout) and/or clamped at 0 (relu);
// opA(m, k) = TA ? A[k lda + m] : A[m lda + k];
// opB(k, n) = TB ? B[n ldb + k] : B[k ldb + n].
// On the fifth-generation tensor cores: a CTA of 128 threads owns a 128 x 128
// output tile whose FP32 accumulator lives in 128 columns of tensor memory.
// K advances 64 at a time through two shared-memory stages: all threads load
// the FP32 operands (all of a stage's loads issued at once, 32 float4 per
// thread), round them to BF16 and store them in the canonical
// K-major layout without swizzle (core matrices of 8 rows x 16 bytes: 128
// bytes apart along K, 1024 bytes apart along M / N), then one thread issues
// four tcgen05.mma kind::f16 (M = 128, N = 128, K = 16, BF16 x BF16 -> FP32)
// and commits them to the stage's mbarrier, so the loads of the next stage
// overlap these products.  The epilogue reads the accumulator with
// tcgen05.ld (thread = row).  Split K: blockIdx.z covers k in [z kc, z kc +
// kc) and writes its partial product to C + z c_split (bias, mask and relu
// only without a split).  Every mbarrier wait is bounded (about a second):
// one that gives up sets TTO_E_TIMEOUT, and the CTA still waits (bounded) for
// the products it issued before it frees the tensor memory.
constexpr int kGM = 128, kGN = 128, kGK = 64, kGStages = 2;
constexpr uint32_t kGTile = kGM * kGK * 2;                  // one BF16 operand tile, 16 KB
constexpr uint32_t kGSmem = kGStages * 2 * kGTile + 1024;   // + alignment slack
constexpr long long kGWait = 1ll << 31;
// instruction descriptor, kind::f16: F32 accumulator (bit 4), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdescBF16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGN >> 3) << 17) |
                                ((uint32_t)(kGM >> 4) << 24);

__device__ __forceinline__ uint32_t g_su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool g_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(g_su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false when it gave up or another thread of the CTA already did.
__device__ __forceinline__ bool g_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  if (g_try(b, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (g_try(b, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kGWait) return false;
  }
}
// canonical K-major no-swizzle position of element (r, k) of a 128 x 64 tile
__device__ __forceinline__ uint32_t g_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
// shared-memory descriptor of such a tile: start, LBO 128 B (along K), SBO
// 1024 B (along M / N), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t g_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46);
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Stage rows r0 .. r0 + 127 and k k0 .. k0 + 63 of op(X) into a tile:
// op(r, k) = KMAJ ? X[r ld + k] : X[k ld + r], zero outside [0, R) x [k0, ke).
// KMAJ: eight threads per row read 32 contiguous floats (16 float4 per
// thread); otherwise a thread reads four rows at four consecutive k and
// transposes them in registers (4 blocks of 4 float4 per thread).  vec:
// float4 reads allowed (ld and X 16-byte aligned).
__device__ __forceinline__ float4 g_ld4(const float* __restrict__ X, size_t o, int valid, bool vec) {
  if (vec && valid >= 4) return __ldg(reinterpret_cast<const float4*>(X + o));
  float4 x;
  x.x = valid > 0 ? __ldg(X + o) : 0.f;
  x.y = valid > 1 ? __ldg(X + o + 1) : 0.f;
  x.z = valid > 2 ? __ldg(X + o + 2) : 0.f;
  x.w = valid > 3 ? __ldg(X + o + 3) : 0.f;
  return x;
}

// Loads (g_load, into registers) and stores (g_store, rounded to BF16 into
// the tile) are split so that a stage's loads of both operands are all in
// flight before any of them is used, and before the thread waits for the
// products that last read the stage.
template <bool KMAJ>
__device__ __forceinline__ void g_load(float4 (&x)[16], const float* __restrict__ X, int ld, int r0, int R, int k0,
                                       int ke, bool vec) {
  const int tid = threadIdx.x;
  if (KMAJ) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int idx = i * 128 + tid;
      const int r = (idx >> 3) & 127, k = ((idx >> 10) << 5) + ((idx & 7) << 2);
      const int gr = r0 + r, gk = k0 + k;
      x[i] = gr < R ? g_ld4(X, (size_t)gr * ld + gk, ke - gk, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  } else {
#pragma unroll
    for (int b = 0; b < 4; ++b) {  // four 4 x 4 blocks: x[4 b + j] = rows r .. r + 3 at k + j
      const int idx = b * 128 + tid;
      const int r = (idx & 31) << 2, k = (idx >> 5) << 2;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gk = k0 + k + j, gr = r0 + r;
        x[4 * b + j] = gk < ke ? g_ld4(X, (size_t)gk * ld + gr, R - gr, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

template <bool KMAJ>
__device__ __forceinline__ void g_store(unsigned char* tile, const float4 (&x)[16]) {
  const int tid = threadIdx.x;
  if (KMAJ) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int idx = i * 128 + tid;
      const int r = (idx >> 3) & 127, k = ((idx >> 10) << 5) + ((idx & 7) << 2);
      uint2 w;
      w.x = pack_bf16x2(x[i].x, x[i].y);
      w.y = pack_bf16x2(x[i].z, x[i].w);
      *reinterpret_cast<uint2*>(tile + g_off(r, k)) = w;
    }
  } else {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int idx = b * 128 + tid;
      const int r = (idx & 31) << 2, k = (idx >> 5) << 2;
      const float4* v = x + 4 * b;
      uint2 w;
      w.x = pack_bf16x2(v[0].x, v[1].x), w.y = pack_bf16x2(v[2].x, v[3].x);
      *reinterpret_cast<uint2*>(tile + g_off(r, k)) = w;
      w.x = pack_bf16x2(v[0].y, v[1].y), w.y = pack_bf16x2(v[2].y, v[3].y);
      *reinterpret_cast<uint2*>(tile + g_off(r + 1, k)) = w;
      w.x = pack_bf16x2(v[0].z, v[1].z), w.y = pack_bf16x2(v[2].z, v[3].z);
      *reinterpret_cast<uint2*>(tile + g_off(r + 2, k)) = w;
      w.x = pack_bf16x2(v[0].w, v[1].w), w.y = pack_bf16x2(v[2].w, v[3].w);
      *reinterpret_cast<uint2*>(tile + g_off(r + 3, k)) = w;
    }
  }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) gemm_umma_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                        const float* __restrict__ B, int ldb, float* C, int ldc,
                                                        const float* __restrict__ bias,
                                                        const float* __restrict__ mask, int relu, int kc,
                                                        size_t c_split, int* status) {
  extern __shared__ unsigned char g_smem_raw[];
  unsigned char* smem = g_smem_raw + ((1024u - (g_su32(g_smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t mbar[kGStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  volatile int* abort_flag = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * kGN;
  const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
  const int nk = ke > kb ? (ke - kb + kGK - 1) / kGK : 0;
  C += blockIdx.z * c_split;
  const bool vecA = ((lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const bool vecB = ((ldb & 3) == 0) && ((reinterpret_cast<uintptr_t>(B) & 15) == 0);
  if (tid == 0) {
    for (int i = 0; i < kGStages; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(g_su32(&mbar[i])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(g_su32(&done)) : "memory");
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(g_su32(&s_tmem)),
                 "r"(kGN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  bool ok = true;
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    unsigned char* sa = smem + st * 2 * kGTile;
    unsigned char* sb = sa + kGTile;
    const int k0 = kb + kt * kGK;
    float4 xa[16], xb[16];
    g_load<!TA>(xa, A, lda, m0, M, k0, ke, vecA);
    g_load<TB>(xb, B, ldb, n0, N, k0, ke, vecB);
    // the products that read this stage two steps ago must be complete
    if (kt >= kGStages) ok = g_wait(&mbar[st], (uint32_t)((kt >> 1) - 1) & 1u, abort_flag);
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    g_store<!TA>(sa, xa);
    g_store<TB>(sb, xb);
    // the generic-proxy stores must be visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = g_desc(g_su32(sa)), db = g_desc(g_su32(sb));
#pragma unroll
      for (int kk = 0; kk < kGK / 16; ++kk) {
        // K = 16 per product: two core matrices, 256 bytes (16 units) along K
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(da + (uint64_t)(16 * kk)), "l"(db + (uint64_t)(16 * kk)), "r"(kIdescBF16), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       g_su32(&mbar[st]))
                   : "memory");
    }
  }
  // every product issued by this CTA, complete (also on the error path)
  if (tid == 0 && nk > 0)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(g_su32(&done))
                 : "memory");
  if (nk > 0) {
    int dummy = 0;
    const bool fin = g_wait(&done, 0, &dummy);
    ok = ok && fin;
  }
  if (!__syncthreads_and(ok)) {
    if (tid == 0) atomicExch(status, TTO_E_TIMEOUT);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    const bool vecC = ((ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0) &&
                      (!mask || (reinterpret_cast<uintptr_t>(mask) & 15) == 0);
#pragma unroll 1
    for (int c0 = 0; c0 < kGN; c0 += 32) {
      uint32_t r[32];
      if (nk > 0) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
            "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = 0u;
      }
      if (row >= M) continue;
      float* crow = C + (size_t)row * ldc;
      const float* mrow = mask ? mask + (size_t)row * ldc : nullptr;
#pragma unroll
      for (int j4 = 0; j4 < 32; j4 += 4) {
        const int n = n0 + c0 + j4;
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          v[j] = __uint_as_float(r[j4 + j]);
          if (bias && n + j < N) v[j] += bias[n + j];
        }
        if (vecC && n + 3 < N) {
          if (mrow) {
            const float4 mk = *reinterpret_cast<const float4*>(mrow + n);
            v[0] = mk.x > 0.f ? v[0] : 0.f, v[1] = mk.y > 0.f ? v[1] : 0.f;
            v[2] = mk.z > 0.f ? v[2] : 0.f, v[3] = mk.w > 0.f ? v[3] : 0.f;
          }
          if (relu)
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = fmaxf(v[j], 0.f);
          *reinterpret_cast<float4*>(crow + n) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (n + j >= N) continue;
            float x = v[j];
            if (mrow && !(mrow[n + j] > 0.f)) x = 0.f;
            if (relu) x = fmaxf(x, 0.f);
            crow[n + j] = x;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGN) : "memory");
  }
}

template <bool TA, bool TB>
int launch_gemm(dim3 grid, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                const float* bias, const float* mask, bool relu, int kc, size_t c_split, int* status,
                cudaStream_t s) {
  static bool attr[64] = {};
  int dev = 0;
  TTO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(TTO_E_ARG, "device %d out of range", dev);
  if (!attr[dev]) {
    TTO_CUDA_TRY(cudaFuncSetAttribute(gemm_umma_kernel<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kGSmem));
    attr[dev] = true;
  }
  gemm_umma_kernel<TA, TB><<<grid, 128, kGSmem, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, relu ? 1 : 0, kc,
                                                     c_split, status);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

template <bool TA, bool TB>
int gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
         const float* bias, const float* mask, bool relu, int* status, cudaStream_t s) {
  if (M <= 0 || N <= 0) return TTO_OK;
  const dim3 grid((N + kGN - 1) / kGN, (M + kGM - 1) / kGM);
  if (grid.y > 65535) return set_error(TTO_E_ARG, "surrogate batch too large for one product");
  return launch_gemm<TA, TB>(grid, M, N, K, A, lda, B, ldb, C, ldc, bias, mask, relu, K, 0, status, s);
}

// out[m][n] (ldo) = sum over z in order of part[z][m][n]
__global__ void splitk_reduce_kernel(int M, int N, int splits, const float* part, float* out, int ldo) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)M * N) return;
  float v = 0.f;
  for (int z = 0; z < splits; ++z) v += part[(size_t)z * M * N + i];
  out[(i / N) * ldo + i % N] = v;
}

constexpr int kMaxSplitK = 16;

// Weight gradient C[M][N] (ldc) = A^T B over K batch rows (A [K][M], B [K][N]):
// few output tiles and a long K, so K is split over up to 16 CTAs per tile
// whose partials (in ws, kMaxSplitK * M * N floats) are summed in a fixed order.
int gemm_wgrad(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc, float* ws,
               int* status, cudaStream_t s) {
  if (M <= 0 || N <= 0) return TTO_OK;
  const int tiles = ((N + kGN - 1) / kGN) * ((M + kGM - 1) / kGM);
  int splits = std::max(1, std::min(kMaxSplitK, (3 * 148 + tiles - 1) / tiles));
  splits = std::max(1, std::min(splits, (K + 255) / 256));
  const int kc = ((K + splits - 1) / splits + kGK - 1) / kGK * kGK;
  splits = (K + kc - 1) / kc;
  if (splits <= 1) return gemm<true, false>(M, N, K, A, lda, B, ldb, C, ldc, nullptr, nullptr, false, status, s);
  const dim3 grid((N + kGN - 1) / kGN, (M + kGM - 1) / kGM, splits);
  int rc = launch_gemm<true, false>(grid, M, N, K, A, lda, B, ldb, ws, N, nullptr, nullptr, false, kc, (size_t)M * N,
                                    status, s);
  if (rc) return rc;
  const size_t n = (size_t)M * N;
  splitk_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M, N, splits, ws, C, ldc);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

// ------------------------------------------------------------------ features
struct FeatArgs {
  const int32_t* topo;
  int k, A, R, E;
  const int* act_st;
  const uint32_t* act_mask;
  const int* station_bus;
  const int* asset_off;
  const int* asset_br;
  const int* from;
  const double* b;
  const double* p;    // [T][n_bus]; timestep 0 is used
  const double* f0;   // [T][E]
  const double* Nsw;  // [n_sw][E]
  const int* swcol;   // [E]
  const double* Nsr;  // [n_sw][R]
  const int* rows;
  const double* row_lim;
  double psum;
  int with_loads;     // 0: station values only (the loadings come from the replay ring)
  int* SI;
  float* SF;
  float* XD;
  int* valid;
  int2* nsm;
};

// One CTA per genome.  Decodes the genome as the evaluation does (an
// out-of-range action or a station split twice makes it invalid), writes the
// station values, and with_loads solves the split at timestep 0 --
// K = S^T N D S in FP64, LDL^T with the same islanding pivot test,
// psi = K^-1 (p_M - S^T f0) -- for f'_r = f0_r + sum_j W_rj psi_j on the R
// loading rows.
__global__ void __launch_bounds__(128) features_kernel(FeatArgs a) {
  const int bi = blockIdx.x, tid = threadIdx.x;
  __shared__ int s_k, s_isl, s_nm;
  __shared__ int s_slot[TTO_MAX_K + 1];
  __shared__ int s_e[kMaxMoved], s_sw[kMaxMoved];
  __shared__ double s_sign[kMaxMoved], s_coef[kMaxMoved];
  __shared__ int s_injbus[TTO_MAX_K];
  __shared__ double s_K[TTO_MAX_K][TTO_MAX_K], s_rhs[TTO_MAX_K], s_psi[TTO_MAX_K], s_sb[TTO_MAX_K];
  if (tid == 0) {
    int k = 0, ne = 0, bad = 0, nm = 0;
    int seen[TTO_MAX_K];
    s_slot[0] = 0;
    for (int j = 0; j < a.k; ++j) {
      a.SI[(size_t)bi * a.k + j] = -1;
      float* sf = a.SF + ((size_t)bi * a.k + j) * 8;
      for (int c = 0; c < 8; ++c) sf[c] = 0.f;
    }
    for (int j = 0; j < a.k; ++j) {
      const int act = a.topo[(size_t)bi * a.k + j];
      if (act < 0) continue;
      if (act >= a.A) {
        bad = 1;
        break;
      }
      const int st = a.act_st[act];
      for (int q = 0; q < k; ++q)
        if (seen[q] == st) bad = 1;
      if (bad) break;
      seen[k] = st;
      const uint32_t mask = a.act_mask[act];
      const int bus = a.station_bus[st], a0 = a.asset_off[st], m = a.asset_off[st + 1] - a0;
      const int nb = __popc(mask);
      nm += min(nb, m - nb);
      double b_all = 0.0, b_b = 0.0, pb = 0.0;
      int br = 0, br_b = 0;
      s_injbus[k] = -1;
      for (int i = 0; i < m; ++i) {
        const int e = a.asset_br[a0 + i];
        const bool onb = (mask >> i) & 1u;
        if (e < 0) {
          if (onb) {
            pb += a.p[bus];
            s_injbus[k] = bus;
          }
          continue;
        }
        ++br;
        b_all += a.b[e];
        if (!onb) continue;
        ++br_b;
        b_b += a.b[e];
        const double sg = (a.from[e] == bus) ? 1.0 : -1.0;
        s_e[ne] = e;
        s_sw[ne] = a.swcol[e];
        s_sign[ne] = sg;
        s_coef[ne] = sg * a.b[e];
        ++ne;
      }
      a.SI[(size_t)bi * a.k + j] = st;
      float* sf = a.SF + ((size_t)bi * a.k + j) * 8;
      sf[0] = 1.f;
      sf[1] = (float)((double)min(nb, m - nb) / m);
      sf[2] = (float)(b_b / b_all);
      sf[3] = (float)(pb / a.psum);
      sf[4] = (float)((double)br_b / br);
      sf[5] = (float)((double)nb / m);
      ++k;
      s_slot[k] = ne;
    }
    if (bad)
      for (int j = 0; j < a.k; ++j) a.SI[(size_t)bi * a.k + j] = -1;
    s_k = bad ? 0 : k;
    s_isl = bad;
    s_nm = nm;
  }
  __syncthreads();
  if (tid == 0) a.nsm[bi] = make_int2(s_k, s_nm);
  if (!a.with_loads) {
    if (tid == 0) a.valid[bi] = s_isl ? 0 : 1;
    return;
  }
  const int k = s_k;
  if (tid < k * k) {
    const int i = tid / k, j = tid % k;
    double acc = 0.0;
    for (int q = s_slot[i]; q < s_slot[i + 1]; ++q) {
      double w = 0.0;
      for (int r = s_slot[j]; r < s_slot[j + 1]; ++r) w += s_coef[r] * a.Nsw[(size_t)s_sw[r] * a.E + s_e[q]];
      acc += s_sign[q] * w;
    }
    s_K[i][j] = acc;
  }
  if (tid < k) {
    double st = 0.0, sb = 0.0;
    for (int q = s_slot[tid]; q < s_slot[tid + 1]; ++q) {
      st += s_sign[q] * a.f0[s_e[q]];
      sb += a.b[s_e[q]];
    }
    s_rhs[tid] = (s_injbus[tid] >= 0 ? a.p[s_injbus[tid]] : 0.0) - st;
    s_sb[tid] = sb;
  }
  __syncthreads();
  if (tid == 0 && k > 0 && !s_isl) {
    double L[TTO_MAX_K][TTO_MAX_K], Dg[TTO_MAX_K], x[TTO_MAX_K];
    int isl = 0;
    for (int j = 0; j < k; ++j) {
      double dj = s_K[j][j];
      for (int q = 0; q < j; ++q) dj -= L[j][q] * L[j][q] * Dg[q];
      Dg[j] = dj;
      if (!(dj > kIslandTol * s_sb[j])) {
        isl = 1;
        break;
      }
      for (int i = j + 1; i < k; ++i) {
        double v = s_K[i][j];
        for (int q = 0; q < j; ++q) v -= L[i][q] * L[j][q] * Dg[q];
        L[i][j] = v / dj;
      }
    }
    if (!isl) {
      for (int i = 0; i < k; ++i) {
        double v = s_rhs[i];
        for (int q = 0; q < i; ++q) v -= L[i][q] * x[q];
        x[i] = v;
      }
      for (int i = 0; i < k; ++i) x[i] /= Dg[i];
      for (int i = k - 1; i >= 0; --i) {
        double v = x[i];
        for (int q = i + 1; q < k; ++q) v -= L[q][i] * x[q];
        x[i] = v;
      }
      for (int i = 0; i < k; ++i) s_psi[i] = x[i];
    }
    s_isl = isl;
  }
  __syncthreads();
  const bool dead = s_isl != 0;
  if (tid == 0) a.valid[bi] = dead ? 0 : 1;
  for (int r = tid; r < a.R; r += blockDim.x) {
    float v = 0.f;
    if (!dead) {
      double f = a.f0[a.rows[r]];
      for (int j = 0; j < k; ++j) {
        double w = 0.0;
        for (int q = s_slot[j]; q < s_slot[j + 1]; ++q) w += s_coef[q] * a.Nsr[(size_t)s_sw[q] * a.R + r];
        f += w * s_psi[j];
      }
      v = (float)(fabs(f) / a.row_lim[r]);
    }
    a.XD[(size_t)bi * a.R + r] = v;
  }
}

// Nsr[sw][r] = Nsw[sw][rows[r]]
__global__ void gather_rows_kernel(int n_sw, int E, int R, const double* Nsw, const int* rows, double* Nsr) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n_sw * R) return;
  const size_t sw = i / R;
  Nsr[i] = Nsw[sw * E + rows[i % R]];
}

// out[c][h] = W1[h][c] for the station columns c < C (32x32 tiles).
__global__ void transpose_station_kernel(int H, int D, int C, const float* W1, float* out) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, h0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int h = h0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (h < H && c < C) ? W1[(size_t)h * D + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, h = h0 + threadIdx.x;
    if (c < C && h < H) out[(size_t)c * H + h] = t[threadIdx.x][y];
  }
}

// ------------------------------------------------------------------ layers
// H1[row][h] = relu(Z1[row][h] + sum over split stations s of the row, c < 8,
// of W1[h][8 s + c] f_c), in place (Z1 holds the dense part and the bias).
__global__ void station_terms_relu_kernel(int M, int H, int k, const int* SI, const float* SF,
                                          const float* W1sT, float* Z) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)M * H) return;
  const int row = (int)(i / H), h = (int)(i % H);
  float v = Z[i];
  for (int j = 0; j < k; ++j) {
    const int st = SI[(size_t)row * k + j];
    if (st < 0) continue;
    const float* f = SF + ((size_t)row * k + j) * 8;
#pragma unroll
    for (int c = 0; c < 8; ++c) v += bf(W1sT[(size_t)(8 * st + c) * H + h]) * bf(f[c]);
  }
  Z[i] = fmaxf(v, 0.f);
}

// y = w4 . h3 + b4 (one warp per row); with stats, mean + deviation * y and
// +inf where valid is 0.
__global__ void output_kernel(int M, int H, const float* H3, const float* w4, const float* b4, const int* valid,
                              const float* stats, float* Y) {
  const int row = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= M) return;
  float s = 0.f;
  for (int h = lane; h < H; h += 32) s += bf(H3[(size_t)row * H + h]) * bf(w4[h]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const float y = s + b4[0];
    Y[row] = (valid && !valid[row]) ? INFINITY : (stats ? fmaf(stats[1], y, stats[0]) : y);
  }
}

// Y = 0 where valid, +inf elsewhere (ranking before the network has data).
__global__ void valid_only_kernel(int M, const int* valid, float* Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) Y[i] = valid[i] ? 0.f : INFINITY;
}

// loss[0] = sum (y - t)^2 and loss[1] = rows, over the rows with a finite
// target; dY = 2 (y - t) / loss[1] there, 0 elsewhere.  One CTA, fixed order.
__global__ void __launch_bounds__(1024) loss_kernel(int M, const float* Y, const float* T, float* dY,
                                                    float* loss) {
  __shared__ float s_sum[32], s_cnt[32];
  __shared__ float s_n;
  float sum = 0.f, cnt = 0.f;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const float t = T[i], y = Y[i];
    if (isfinite(t) && isfinite(y)) {
      const float r = y - t;
      sum += r * r;
      cnt += 1.f;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_sum[threadIdx.x >> 5] = sum;
    s_cnt[threadIdx.x >> 5] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, c = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += s_sum[w];
      c += s_cnt[w];
    }
    loss[0] = a;
    loss[1] = c;
    s_n = c;
  }
  __syncthreads();
  const float n = fmaxf(s_n, 1.f);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const float t = T[i], y = Y[i];
    dY[i] = (isfinite(t) && isfinite(y)) ? 2.f * (y - t) / n : 0.f;
  }
}

// dH3[row][h] = dY[row] w4[h] where h3 > 0.
__global__ void out_back_kernel(int M, int H, const float* dY, const float* w4, const float* H3, float* dH3) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)M * H) return;
  const int row = (int)(i / H), h = (int)(i % H);
  dH3[i] = H3[i] > 0.f ? dY[row] * bf(w4[h]) : 0.f;
}

// out[n] = sum_m A[m][n] (w ? w[m] : 1), fixed order: 32 columns x 32 row
// groups per CTA, then the groups summed in order.
__global__ void __launch_bounds__(1024) colsum_kernel(int M, int N, const float* A, const float* w, float* out) {
  __shared__ float s[32][33];
  const int n = blockIdx.x * 32 + threadIdx.x;
  float acc = 0.f;
  if (n < N)
    for (int m = threadIdx.y; m < M; m += 32) acc += A[(size_t)m * N + n] * (w ? w[m] : 1.f);
  s[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && n < N) {
    float t = 0.f;
    for (int y = 0; y < 32; ++y) t += s[y][threadIdx.x];
    out[n] = t;
  }
}

// Gradient of the station block of W1: one CTA per station s,
// G1[h][8 s + c] = sum over genome slots holding s (in slot order, i.e. row
// order) of dH1[row][h] f_c.  The hits are staged in shared memory 1024 at a
// time and accumulated by all threads, two hidden units each (H <= 1024:
// four).
constexpr int kGradList = 1024;
// Row masks of the batch per station (SM zeroed before): one thread per
// genome slot sets its row's bit in the word of its station.  A genome names
// a station at most once (a repeat marks the whole genome invalid, every slot
// -1), so a station's set rows are exactly its (row, slot) entries.
__global__ void station_mask_kernel(int n_ent, int k, int words, const int* SI, uint32_t* SM) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_ent) return;
  const int st = SI[e];
  if (st < 0) return;
  const int row = e / k;
  atomicOr(SM + (size_t)st * words + (row >> 5), 1u << (row & 31));
}

// Gradient of the station block of W1 (columns 8 s .. 8 s + 7): for every
// hidden unit h, the sum over the batch rows that split station s, in row
// order, of dH1[row][h] times the station's eight values (rounded to BF16 as
// in the forward product).  One CTA per station: its rows come from the
// station's mask words (each thread a run of words, a prefix sum over the
// threads gives every row its place), kGradList rows at a time.
__global__ void __launch_bounds__(256) station_grad_kernel(int H, int D, int k, int words, const int* SI,
                                                           const float* SF, const uint32_t* SM,
                                                           const float* dH1, float* G1) {
  const int s = blockIdx.x, tid = threadIdx.x;
  __shared__ int s_row[kGradList];
  __shared__ float s_f[kGradList][8];
  __shared__ int s_cnt[256];
  __shared__ int s_total;
  const uint32_t* sm = SM + (size_t)s * words;
  const int per = (words + 255) / 256;
  const int w0 = min(words, tid * per), w1 = min(words, w0 + per);
  int cnt = 0;
  for (int w = w0; w < w1; ++w) cnt += __popc(sm[w]);
  s_cnt[tid] = cnt;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int i = 0; i < 256; ++i) {
      const int c = s_cnt[i];
      s_cnt[i] = run;
      run += c;
    }
    s_total = run;
  }
  __syncthreads();
  const int total = s_total, off = s_cnt[tid];
  float acc[kMaxHidden / 256][8];
#pragma unroll
  for (int u = 0; u < kMaxHidden / 256; ++u)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[u][c] = 0.f;
  for (int base = 0; base < total; base += kGradList) {
    if (cnt > 0 && off < base + kGradList && off + cnt > base) {
      int pos = off;
      for (int w = w0; w < w1 && pos < base + kGradList; ++w) {
        uint32_t bits = sm[w];
        while (bits && pos < base + kGradList) {
          const int row = 32 * w + __ffs(bits) - 1;
          bits &= bits - 1;
          if (pos >= base) {
            int j = 0;
            while (j < k - 1 && SI[(size_t)row * k + j] != s) ++j;
            const float* f = SF + ((size_t)row * k + j) * 8;
            s_row[pos - base] = row;
#pragma unroll
            for (int c = 0; c < 8; ++c) s_f[pos - base][c] = bf(f[c]);
          }
          ++pos;
        }
      }
    }
    __syncthreads();
    const int nl = min(kGradList, total - base);
    for (int i = 0; i < nl; ++i) {
      const float* dr = dH1 + (size_t)s_row[i] * H;
#pragma unroll
      for (int u = 0; u < kMaxHidden / 256; ++u) {
        const int h = tid + 256 * u;
        if (h < H) {
          const float dv = dr[h];
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[u][c] += dv * s_f[i][c];
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kMaxHidden / 256; ++u) {
    const int h = tid + 256 * u;
    if (h < H)
#pragma unroll
      for (int c = 0; c < 8; ++c) G1[(size_t)h * D + 8 * s + c] = acc[u][c];
  }
}

// Adam with bias correction: c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void adam_kernel(size_t n, float* P, const float* G, float* m, float* v, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = G[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------ top-k
// Unsigned integer with the order of the float (after -0 -> +0).
__device__ __forceinline__ uint32_t orderable(float f) {
  const uint32_t u = __float_as_uint(f + 0.0f);  // -0 -> +0
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Screening keys (ascending = evaluated first), 64 bits: a flag, the
// orderable bits of a float, and the proposal index (31 bits).
// by_gain = 0: flag 0 and the predicted log1p(-fitness);
// by_gain = 1: flag 0 and the predicted log1p(-fitness) for a proposal whose
// descriptors map to an empty archive cell, flag 1 and the predicted
// improvement over the cell's elite, y - log1p(-fitness_elite) (FP64, then
// rounded), for a filled one.
// Either way +inf with flag 1 for a proposal that islands the grid or equals
// its cell's elite slot for slot (evaluated already; its score is reported as
// +inf).  Padding entries are all ones.
__global__ void screen_keys_kernel(int n, int npad, int k, int by_gain, const int32_t* prop, const int2* nsm,
                                   int d_split, int d_moved, const int32_t* elite, const float* elite_fit,
                                   const uint8_t* filled, float* Y, unsigned long long* keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  if (i >= n) {
    keys[i] = ~0ull;
    return;
  }
  float y = Y[i];
  unsigned long long flag = 1;
  float key = INFINITY;
  if (!isnan(y) && isfinite(y)) {
    const int2 d = nsm[i];
    const int cell = min(d.x, d_split - 1) * d_moved + min(d.y, d_moved - 1);
    if (!filled[cell]) {
      flag = 0;
      key = y;
    } else {
      bool same = true;
      for (int j = 0; j < k && same; ++j) same = prop[(size_t)i * k + j] == elite[(size_t)cell * k + j];
      if (same) {
        Y[i] = INFINITY;
      } else if (by_gain) {
        key = (float)((double)y - log1p(-(double)elite_fit[cell]));
      } else {
        flag = 0;
        key = y;
      }
    }
  }
  keys[i] = (flag << 63) | ((unsigned long long)orderable(key) << 31) | (unsigned long long)(uint32_t)i;
}

// One compare-exchange stage (kk, jj) of the bitonic network over the array.
__global__ void bitonic_global_kernel(int npad, int kk, int jj, unsigned long long* keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  const int p = i ^ jj;
  if (p <= i) return;
  const unsigned long long x = keys[i], y = keys[p];
  if ((x > y) == ((i & kk) == 0)) {
    keys[i] = y;
    keys[p] = x;
  }
}

// The stages of the bitonic network that stay inside one 2048-key chunk: for
// kk_from = 0, every stage with kk <= 2048; else the stages jj = 1024 .. 1 of
// kk = kk_from.  1024 threads, one pair each per stage.
__global__ void __launch_bounds__(1024) bitonic_shared_kernel(int kk_from, unsigned long long* keys) {
  __shared__ unsigned long long s[kSortChunk];
  const int base = blockIdx.x * kSortChunk, t = threadIdx.x;
  s[t] = keys[base + t];
  s[t + 1024] = keys[base + t + 1024];
  __syncthreads();
  const int kk_lo = kk_from ? kk_from : 2, kk_hi = kk_from ? kk_from : kSortChunk;
  for (int kk = kk_lo; kk <= kk_hi; kk <<= 1) {
    for (int jj = min(kk >> 1, kSortChunk >> 1); jj > 0; jj >>= 1) {
      const int i = 2 * jj * (t / jj) + (t % jj), p = i + jj;
      const unsigned long long x = s[i], y = s[p];
      if ((x > y) == (((base + i) & kk) == 0)) {
        s[i] = y;
        s[p] = x;
      }
      __syncthreads();
    }
  }
  keys[base + t] = s[t];
  keys[base + t + 1024] = s[t + 1024];
}

__global__ void gather_topo_kernel(int n, int k, const int32_t* sel, const int32_t* src, int32_t* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t j = (size_t)sel[i];
  for (int c = 0; c < k; ++c) dst[(size_t)i * k + c] = src[j * k + c];
}

__global__ void gather_score_kernel(int n, const int32_t* sel, const float* Y, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = Y[sel[i]];
}

__device__ __forceinline__ uint32_t key_index(unsigned long long key) { return (uint32_t)(key & 0x7fffffffull); }

__device__ __forceinline__ bool same_genome(const int32_t* prop, int k, uint32_t x, uint32_t y) {
  for (int j = 0; j < k; ++j)
    if (prop[(size_t)x * k + j] != prop[(size_t)y * k + j]) return false;
  return true;
}

// One CTA: walks the sorted keys and writes to sel the proposal indices of the
// first n_keep entries of the stable partition [entries whose genome differs
// from their predecessor's | the repeats].  Equal genomes have equal keys
// (apart from the index), so repeats are adjacent in the sorted order.
__global__ void __launch_bounds__(1024) select_kernel(int n, int n_keep, int k, const unsigned long long* keys,
                                                      const int32_t* prop, int32_t* sel) {
  __shared__ int s_cnt[1024];
  __shared__ int s_total;
  const int t = threadIdx.x, per = (n + 1023) / 1024;
  const int p0 = min(n, t * per), p1 = min(n, p0 + per);
  int uniq = 0;
  for (int p = p0; p < p1; ++p)
    uniq += (p == 0 || !same_genome(prop, k, key_index(keys[p]), key_index(keys[p - 1]))) ? 1 : 0;
  s_cnt[t] = uniq;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int i = 0; i < 1024; ++i) {
      const int c = s_cnt[i];
      s_cnt[i] = run;
      run += c;
    }
    s_total = run;
  }
  __syncthreads();
  int u = s_cnt[t], r = s_total + (p0 - s_cnt[t]);  // repeats before p0 = p0 - uniques before p0
  for (int p = p0; p < p1; ++p) {
    const bool first = p == 0 || !same_genome(prop, k, key_index(keys[p]), key_index(keys[p - 1]));
    const int dst = first ? u++ : r++;
    if (dst < n_keep) sel[dst] = (int32_t)key_index(keys[p]);
  }
}

// ------------------------------------------------------------------ replay
// Target of an exact fitness: log1p(-fitness) (NaN when not finite).
__device__ __forceinline__ float raw_target(float f) {
  return isfinite(f) ? log1pf(-f) : __int_as_float(0x7fc00000);
}

// Standardised target: (t - mean) / deviation.
__device__ __forceinline__ float scaled_target(float t, const float* stats) { return (t - stats[0]) * stats[2]; }

// stats = mean, population standard deviation and its reciprocal over the
// finite entries of rt[0 .. n) (FP64, fixed order); (0, 1, 1) when there are
// none, deviation 1 when they are all equal.
__global__ void __launch_bounds__(1024) target_stats_kernel(int n, const float* rt, float* stats) {
  __shared__ double s_a[32], s_b[32];
  __shared__ double s_mean;
  double sum = 0.0, cnt = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float t = rt[i];
    if (isfinite(t)) {
      sum += t;
      cnt += 1.0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_a[threadIdx.x >> 5] = sum;
    s_b[threadIdx.x >> 5] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += s_a[w];
      c += s_b[w];
    }
    s_mean = c > 0.0 ? a / c : 0.0;
    s_b[0] = c;
  }
  __syncthreads();
  const double mean = s_mean, count = s_b[0];
  __syncthreads();
  double sq = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float t = rt[i];
    if (isfinite(t)) sq += ((double)t - mean) * ((double)t - mean);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) s_a[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += s_a[w];
    double sd = count > 0.0 ? sqrt(a / count) : 1.0;
    if (!(sd > 0.0)) sd = 1.0;
    stats[0] = (float)mean;
    stats[1] = (float)sd;
    stats[2] = (float)(1.0 / sd);
  }
}

// T[i] = standardised target of fitness fit[i].
__global__ void targets_kernel(int n, const float* fit, const float* stats, float* T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) T[i] = scaled_target(raw_target(fit[i]), stats);
}

// Append n pairs at the ring head: genome i, the loadings of batch row
// (idx ? idx[i] : i), target log1p(-fitness) or NaN.
__global__ void replay_append_kernel(int n, int k, int R, int cap, int head, const int32_t* topo,
                                     const int32_t* idx, const float* XD, const float* fit,
                                     int32_t* rg, float* rx, float* rt) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const size_t slot = (size_t)((head + i) % cap);
  const size_t src = idx ? (size_t)idx[i] : (size_t)i;
  for (int r = threadIdx.x; r < R; r += blockDim.x) rx[slot * R + r] = XD[src * R + r];
  if (threadIdx.x < k) rg[slot * k + threadIdx.x] = topo[(size_t)i * k + threadIdx.x];
  if (threadIdx.x == 0) rt[slot] = raw_target(fit[i]);
}

// Minibatch row i: ring entry i when the ring holds at most M pairs, else a
// uniform draw from Philox4x32-10 (key = seed, counter = (i, ~0, step));
// its target standardised.
__global__ void sample_kernel(int M, int n_rep, int k, int R, uint2 key, uint32_t st_lo, uint32_t st_hi,
                              const int32_t* rg, const float* rx, const float* rt, const float* stats,
                              int32_t* topo, float* XD, float* T) {
  const int i = blockIdx.x;
  if (i >= M) return;
  size_t src = (size_t)i;
  if (n_rep > M) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, 0xffffffffu, st_lo, st_hi), key);
    src = (size_t)(((uint64_t)w.x * (uint32_t)n_rep) >> 32);
  }
  for (int r = threadIdx.x; r < R; r += blockDim.x) XD[(size_t)i * R + r] = rx[src * R + r];
  if (threadIdx.x < k) topo[(size_t)i * k + threadIdx.x] = rg[src * k + threadIdx.x];
  if (threadIdx.x == 0) T[i] = scaled_target(rt[src], stats);
}

// ------------------------------------------------------------------ host side
int alloc_batch(tto_surrogate* s, int B) {
  if (B <= s->bcap) return TTO_OK;
  void* old[] = {s->SI, s->SM, s->SF, s->XD, s->valid, s->nsm, s->H1, s->H2, s->H3, s->Y, s->dH1, s->dH2, s->dH3, s->dY,
                 s->T, s->mb_topo};
  for (void* p : old)
    if (p) cudaFree(p);
  s->SI = nullptr;
  s->SM = nullptr;
  s->SF = s->XD = s->H1 = s->H2 = s->H3 = s->Y = s->dH1 = s->dH2 = s->dH3 = s->dY = s->T = nullptr;
  s->valid = nullptr;
  s->nsm = nullptr;
  s->mb_topo = nullptr;
  s->bcap = 0;
  const size_t b = B, H = s->H;
  TTO_CUDA_TRY(cudaMalloc(&s->SI, b * s->k * sizeof(int)));
  TTO_CUDA_TRY(cudaMalloc(&s->SM, (size_t)s->S * ((b + 31) / 32) * sizeof(uint32_t)));
  TTO_CUDA_TRY(cudaMalloc(&s->SF, b * s->k * 8 * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->XD, b * s->R * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->valid, b * sizeof(int)));
  TTO_CUDA_TRY(cudaMalloc(&s->nsm, b * sizeof(int2)));
  TTO_CUDA_TRY(cudaMalloc(&s->H1, b * H * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->H2, b * H * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->H3, b * H * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->Y, b * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->dH1, b * H * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->dH2, b * H * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->dH3, b * H * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->dY, b * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->T, b * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&s->mb_topo, b * s->k * sizeof(int32_t)));
  s->bcap = B;
  return TTO_OK;
}

FeatArgs feat_args(const tto_surrogate* s, const int32_t* topo, int with_loads) {
  const tto_grid* g = s->g;
  FeatArgs a;
  a.topo = topo;
  a.k = s->k;
  a.A = g->A;
  a.R = s->R;
  a.E = g->E;
  a.act_st = g->d_act_st;
  a.act_mask = g->d_act_mask;
  a.station_bus = g->d_station_bus;
  a.asset_off = g->d_asset_off;
  a.asset_br = g->d_asset_br;
  a.from = g->d_from;
  a.b = g->d_b;
  a.p = g->d_p;
  a.f0 = g->d_f0;
  a.Nsw = g->d_Nsw;
  a.swcol = g->d_swcol;
  a.Nsr = s->Nsr;
  a.rows = s->rows;
  a.row_lim = s->row_lim;
  a.psum = s->psum;
  a.with_loads = with_loads;
  a.SI = s->SI;
  a.SF = s->SF;
  a.XD = s->XD;
  a.valid = s->valid;
  a.nsm = s->nsm;
  return a;
}

int features(tto_surrogate* s, const int32_t* topo, int B, int with_loads, cudaStream_t st) {
  if (B <= 0) return TTO_OK;
  features_kernel<<<B, 128, 0, st>>>(feat_args(s, topo, with_loads));
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

int refresh_station_weights(tto_surrogate* s, cudaStream_t st) {
  const int C = 8 * s->S;
  const dim3 grid((C + 31) / 32, (s->H + 31) / 32);
  transpose_station_kernel<<<grid, dim3(32, 8), 0, st>>>(s->H, s->D, C, s->P + s->oW1, s->W1sT);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

// Forward pass over the first B rows of the batch buffers (SI, SF, XD).
int forward(tto_surrogate* s, int B, const int* valid, cudaStream_t st) {
  const float* P = s->P;
  const int H = s->H, D = s->D, R = s->R;
  int rc = gemm<false, true>(B, H, R, s->XD, R, P + s->oW1 + 8 * (size_t)s->S, D, s->H1, H, P + s->ob1, nullptr,
                             false, s->g->d_status, st);
  if (rc) return rc;
  const size_t n = (size_t)B * H;
  station_terms_relu_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(B, H, s->k, s->SI, s->SF, s->W1sT, s->H1);
  TTO_CUDA_TRY(cudaGetLastError());
  if ((rc = gemm<false, true>(B, H, H, s->H1, H, P + s->oW2, H, s->H2, H, P + s->ob2, nullptr, true, s->g->d_status, st))) return rc;
  if ((rc = gemm<false, true>(B, H, H, s->H2, H, P + s->oW3, H, s->H3, H, P + s->ob3, nullptr, true, s->g->d_status, st))) return rc;
  output_kernel<<<(unsigned)(((size_t)B * 32 + 255) / 256), 256, 0, st>>>(B, H, s->H3, P + s->ow4, P + s->ob4, valid,
                                                                         valid ? s->stats : nullptr, s->Y);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

// Loss of the first M rows against s->T and the packed gradient into s->G
// (after a forward pass over the same rows).  Every gradient entry is written.
int backward(tto_surrogate* s, int M, cudaStream_t st) {
  const float* P = s->P;
  float* G = s->G;
  const int H = s->H, D = s->D, R = s->R;
  const unsigned nb = (unsigned)(((size_t)M * H + 255) / 256);
  const unsigned ncs = (unsigned)((H + 31) / 32);
  const dim3 cs(32, 32);
  loss_kernel<<<1, 1024, 0, st>>>(M, s->Y, s->T, s->dY, s->loss);
  colsum_kernel<<<ncs, cs, 0, st>>>(M, H, s->H3, s->dY, G + s->ow4);
  colsum_kernel<<<1, cs, 0, st>>>(M, 1, s->dY, nullptr, G + s->ob4);
  out_back_kernel<<<nb, 256, 0, st>>>(M, H, s->dY, P + s->ow4, s->H3, s->dH3);
  TTO_CUDA_TRY(cudaGetLastError());
  int rc;
  if ((rc = gemm_wgrad(H, H, M, s->dH3, H, s->H2, H, G + s->oW3, H, s->wsk, s->g->d_status, st))) return rc;
  colsum_kernel<<<ncs, cs, 0, st>>>(M, H, s->dH3, nullptr, G + s->ob3);
  if ((rc = gemm<false, false>(M, H, H, s->dH3, H, P + s->oW3, H, s->dH2, H, nullptr, s->H2, false, s->g->d_status, st))) return rc;
  if ((rc = gemm_wgrad(H, H, M, s->dH2, H, s->H1, H, G + s->oW2, H, s->wsk, s->g->d_status, st))) return rc;
  colsum_kernel<<<ncs, cs, 0, st>>>(M, H, s->dH2, nullptr, G + s->ob2);
  if ((rc = gemm<false, false>(M, H, H, s->dH2, H, P + s->oW2, H, s->dH1, H, nullptr, s->H1, false, s->g->d_status, st))) return rc;
  if ((rc = gemm_wgrad(H, R, M, s->dH1, H, s->XD, R, G + s->oW1 + 8 * (size_t)s->S, D, s->wsk, s->g->d_status, st))) return rc;
  colsum_kernel<<<ncs, cs, 0, st>>>(M, H, s->dH1, nullptr, G + s->ob1);
  const int words = (M + 31) / 32;
  TTO_CUDA_TRY(cudaMemsetAsync(s->SM, 0, (size_t)s->S * words * sizeof(uint32_t), st));
  station_mask_kernel<<<(unsigned)(((size_t)M * s->k + 255) / 256), 256, 0, st>>>(M * s->k, s->k, words, s->SI, s->SM);
  station_grad_kernel<<<s->S, 256, 0, st>>>(H, D, s->k, words, s->SI, s->SF, s->SM, s->dH1, G + s->oW1);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

int adam(tto_surrogate* s, cudaStream_t st) {
  ++s->step;
  const double c1 = 1.0 - pow(s->beta1, (double)s->step), c2 = 1.0 - pow(s->beta2, (double)s->step);
  adam_kernel<<<(unsigned)((s->n_params + 255) / 256), 256, 0, st>>>(s->n_params, s->P, s->G, s->Am, s->Av,
                                                                     (float)s->lr, (float)s->beta1, (float)s->beta2,
                                                                     (float)s->eps, (float)c1, (float)c2);
  TTO_CUDA_TRY(cudaGetLastError());
  return refresh_station_weights(s, st);
}

int score(tto_surrogate* s, const int32_t* topo, int B, cudaStream_t st) {
  int rc = alloc_batch(s, B);
  if (rc) return rc;
  if ((rc = features(s, topo, B, 1, st))) return rc;
  return forward(s, B, s->valid, st);
}

int train(tto_surrogate* s, int steps, float* loss_host, cudaStream_t st) {
  if (s->rep_n == 0) return set_error(TTO_E_ARG, "the replay ring is empty");
  const int M = std::min(s->mb, s->rep_n);
  int rc = alloc_batch(s, M);
  if (rc) return rc;
  const uint2 key = make_uint2((uint32_t)s->seed, (uint32_t)(s->seed >> 32));
  for (int it = 0; it < steps; ++it) {
    const uint64_t step = (uint64_t)s->step;
    sample_kernel<<<M, 128, 0, st>>>(M, s->rep_n, s->k, s->R, key, (uint32_t)step, (uint32_t)(step >> 32),
                                     s->rep_genome, s->rep_xd, s->rep_t, s->stats, s->mb_topo, s->XD, s->T);
    TTO_CUDA_TRY(cudaGetLastError());
    if ((rc = features(s, s->mb_topo, M, 0, st))) return rc;
    if ((rc = forward(s, M, nullptr, st))) return rc;
    if ((rc = backward(s, M, st))) return rc;
    if ((rc = adam(s, st))) return rc;
  }
  if (loss_host) {
    float l[2];
    TTO_CUDA_TRY(cudaMemcpyAsync(l, s->loss, sizeof(l), cudaMemcpyDeviceToHost, st));
    TTO_CUDA_TRY(cudaStreamSynchronize(st));
    *loss_host = l[1] > 0.f ? l[0] / l[1] : 0.f;
  }
  return TTO_OK;
}

int sort_pad(int n) {
  int npad = kSortChunk;
  while (npad < n) npad <<= 1;
  return npad;
}

int ensure_keys(tto_surrogate* s, int n) {
  const int npad = sort_pad(n);
  if (npad > s->keys_n) {
    if (s->keys) cudaFree(s->keys);
    s->keys = nullptr;
    s->keys_n = 0;
    TTO_CUDA_TRY(cudaMalloc(&s->keys, (size_t)npad * sizeof(unsigned long long)));
    s->keys_n = npad;
  }
  return TTO_OK;
}

// Sort the first sort_pad(n) keys in s->keys (ascending).
int sort_keys(tto_surrogate* s, int n, cudaStream_t st) {
  const int npad = sort_pad(n);
  const int chunks = npad / kSortChunk;
  bitonic_shared_kernel<<<chunks, 1024, 0, st>>>(0, s->keys);
  for (int kk = 2 * kSortChunk; kk <= npad; kk <<= 1) {
    for (int jj = kk >> 1; jj >= kSortChunk; jj >>= 1)
      bitonic_global_kernel<<<(npad + 255) / 256, 256, 0, st>>>(npad, kk, jj, s->keys);
    bitonic_shared_kernel<<<chunks, 1024, 0, st>>>(kk, s->keys);
  }
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

// Append n pairs (genomes topo [n][k], fitness fit [n]) whose loadings are
// batch rows idx[i] (or i) of XD.
int append(tto_surrogate* s, const int32_t* topo, int n, const int32_t* idx, const float* XD, const float* fit,
           cudaStream_t st) {
  n = std::min(n, s->cap);
  if (n <= 0) return TTO_OK;
  replay_append_kernel<<<n, 128, 0, st>>>(n, s->k, s->R, s->cap, s->rep_head, topo, idx, XD, fit, s->rep_genome,
                                          s->rep_xd, s->rep_t);
  TTO_CUDA_TRY(cudaGetLastError());
  s->rep_head = (s->rep_head + n) % s->cap;
  s->rep_n = std::min(s->cap, s->rep_n + n);
  target_stats_kernel<<<1, 1024, 0, st>>>(s->rep_n, s->rep_t, s->stats);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

void release(tto_surrogate* s) {
  void* ptrs[] = {s->P,  s->G,     s->Am, s->Av, s->W1sT, s->wsk, s->rows, s->row_lim, s->Nsr, s->SI, s->SM, s->SF,
                  s->XD, s->valid, s->nsm, s->H1, s->H2, s->H3, s->Y,    s->dH1,     s->dH2, s->dH3, s->dY,
                  s->T,  s->mb_topo, s->loss, s->stats, s->rep_genome, s->rep_xd, s->rep_t, s->prop, s->keys, s->sel};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete s;
}

}  // namespace
}  // namespace tto

using namespace tto;

extern "C" {

int tto_surrogate_create(tto_grid* g, const tto_surrogate_cfg* cfg, tto_surrogate** out) {
  if (!g || !cfg || !out) return set_error(TTO_E_ARG, "null argument");
  *out = nullptr;
  if (cfg->hidden < 16 || cfg->hidden > kMaxHidden || cfg->hidden % 16 != 0)
    return set_error(TTO_E_ARG, "hidden must be a multiple of 16 in [16, %d]", kMaxHidden);
  if (cfg->n_load < 1 || cfg->n_load > g->E) return set_error(TTO_E_ARG, "n_load must be in [1, n_branch]");
  if (cfg->replay < 1 || cfg->minibatch < 1) return set_error(TTO_E_ARG, "replay and minibatch must be >= 1");
  if (!(cfg->lr > 0.0) || !(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0) || !(cfg->beta2 >= 0.0 && cfg->beta2 < 1.0) ||
      !(cfg->eps > 0.0))
    return set_error(TTO_E_ARG, "Adam needs lr > 0, 0 <= beta < 1, eps > 0");
  if (g->S < 1 || g->k_max < 1) return set_error(TTO_E_ARG, "the grid has no splittable stations");
  if (g->n_dslot > 0) return set_error(TTO_E_ARG, "the surrogate screens split-only genomes (grid has disconnection slots)");
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  tto_surrogate* s = new (std::nothrow) tto_surrogate();
  if (!s) return set_error(TTO_E_NOMEM, "host allocation failed");
  s->g = g;
  s->H = cfg->hidden;
  s->R = cfg->n_load;
  s->S = g->S;
  s->D = 8 * g->S + s->R;
  s->k = g->k_max;
  s->cap = cfg->replay;
  s->mb = cfg->minibatch;
  s->lr = cfg->lr;
  s->beta1 = cfg->beta1;
  s->beta2 = cfg->beta2;
  s->eps = cfg->eps;
  s->seed = cfg->seed;
  const size_t H = s->H, D = s->D;
  s->oW1 = 0;
  s->ob1 = s->oW1 + H * D;
  s->oW2 = s->ob1 + H;
  s->ob2 = s->oW2 + H * H;
  s->oW3 = s->ob2 + H;
  s->ob3 = s->oW3 + H * H;
  s->ow4 = s->ob3 + H;
  s->ob4 = s->ow4 + H;
  s->n_params = s->ob4 + 1;
  // loading rows: highest |f0(t=0)| / limit first, ties by branch id
  std::vector<int> order(g->E);
  std::vector<double> load(g->E);
  for (int l = 0; l < g->E; ++l) {
    order[l] = l;
    load[l] = fabs(g->f0[l]) / g->limit[l];
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return load[x] > load[y]; });
  std::vector<int> rows(order.begin(), order.begin() + s->R);
  std::vector<double> rl(s->R);
  for (int r = 0; r < s->R; ++r) rl[r] = g->limit[rows[r]];
  double psum = 0.0;
  for (int i = 0; i < g->n_bus; ++i) psum += fabs(g->p[i]);
  s->psum = psum > 0.0 ? psum : 1.0;
  // He-uniform weights U(-sqrt(6/fan_in), +sqrt(6/fan_in)) from a xorshift64
  // stream seeded by cfg->seed; zero biases
  std::vector<float> P(s->n_params, 0.f);
  uint64_t x = cfg->seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;
  auto uni = [&]() {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](size_t off, size_t n_out, size_t n_in) {
    const double lim = sqrt(6.0 / (double)n_in);
    for (size_t i = 0; i < n_out * n_in; ++i) P[off + i] = (float)((2.0 * uni() - 1.0) * lim);
  };
  fill(s->oW1, H, D);
  fill(s->oW2, H, H);
  fill(s->oW3, H, H);
  fill(s->ow4, 1, H);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  A((void**)&s->P, s->n_params * 4);
  A((void**)&s->G, s->n_params * 4);
  A((void**)&s->Am, s->n_params * 4);
  A((void**)&s->Av, s->n_params * 4);
  A((void**)&s->W1sT, (size_t)8 * s->S * H * 4);
  A((void**)&s->wsk, (size_t)kMaxSplitK * H * std::max(H, (size_t)s->R) * 4);
  A((void**)&s->rows, s->R * sizeof(int));
  A((void**)&s->row_lim, s->R * sizeof(double));
  A((void**)&s->Nsr, (size_t)std::max(g->n_sw, 1) * s->R * sizeof(double));
  A((void**)&s->loss, 2 * sizeof(float));
  A((void**)&s->stats, 3 * sizeof(float));
  A((void**)&s->rep_genome, (size_t)s->cap * s->k * sizeof(int32_t));
  A((void**)&s->rep_xd, (size_t)s->cap * s->R * sizeof(float));
  A((void**)&s->rep_t, (size_t)s->cap * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(s->P, P.data(), s->n_params * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->G, 0, s->n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(s->Am, 0, s->n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(s->Av, 0, s->n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(s->loss, 0, 2 * sizeof(float));
  const float unit[3] = {0.f, 1.f, 1.f};
  if (e == cudaSuccess) e = cudaMemcpy(s->stats, unit, sizeof(unit), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->rows, rows.data(), s->R * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->row_lim, rl.data(), s->R * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && g->n_sw > 0) {
    const size_t n = (size_t)g->n_sw * s->R;
    gather_rows_kernel<<<(unsigned)((n + 255) / 256), 256>>>(g->n_sw, g->E, s->R, g->d_Nsw, s->rows, s->Nsr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int rc = refresh_station_weights(s, 0);
    if (rc) {
      release(s);
      return rc;
    }
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    release(s);
    return cuda_error(e, "surrogate allocation");
  }
  *out = s;
  return TTO_OK;
}

int tto_surrogate_destroy(tto_surrogate* s) {
  if (!s) return TTO_OK;
  cudaSetDevice(s->g->device);
  cudaDeviceSynchronize();
  release(s);
  return TTO_OK;
}

int tto_surrogate_info(const tto_surrogate* s, int64_t* n_params, int32_t* input_dim, int32_t* replay_fill,
                       int32_t* rows_out, float* target_stats) {
  if (!s) return set_error(TTO_E_ARG, "null surrogate");
  if (n_params) *n_params = (int64_t)s->n_params;
  if (input_dim) *input_dim = s->D;
  if (replay_fill) *replay_fill = s->rep_n;
  if (rows_out || target_stats) {
    TTO_CUDA_TRY(cudaSetDevice(s->g->device));
    TTO_CUDA_TRY(cudaDeviceSynchronize());
  }
  if (rows_out) TTO_CUDA_TRY(cudaMemcpy(rows_out, s->rows, s->R * sizeof(int), cudaMemcpyDeviceToHost));
  if (target_stats) TTO_CUDA_TRY(cudaMemcpy(target_stats, s->stats, 2 * sizeof(float), cudaMemcpyDeviceToHost));
  return TTO_OK;
}

int tto_surrogate_params(tto_surrogate* s, float* get_host, const float* set_host) {
  if (!s) return set_error(TTO_E_ARG, "null surrogate");
  TTO_CUDA_TRY(cudaSetDevice(s->g->device));
  TTO_CUDA_TRY(cudaDeviceSynchronize());
  if (set_host) {
    TTO_CUDA_TRY(cudaMemcpy(s->P, set_host, s->n_params * 4, cudaMemcpyHostToDevice));
    TTO_CUDA_TRY(cudaMemset(s->Am, 0, s->n_params * 4));
    TTO_CUDA_TRY(cudaMemset(s->Av, 0, s->n_params * 4));
    s->step = 0;
    const int rc = refresh_station_weights(s, 0);
    if (rc) return rc;
    TTO_CUDA_TRY(cudaDeviceSynchronize());
  }
  if (get_host) TTO_CUDA_TRY(cudaMemcpy(get_host, s->P, s->n_params * 4, cudaMemcpyDeviceToHost));
  return TTO_OK;
}

int tto_surrogate_score(tto_surrogate* s, const int32_t* topo, int32_t B, float* score_out, void* stream) {
  if (!s || B < 0 || (B > 0 && (!topo || !score_out))) return set_error(TTO_E_ARG, "bad score arguments");
  if (B == 0) return TTO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(s->g->device));
  const int rc = score(s, topo, B, st);
  if (rc) return rc;
  TTO_CUDA_TRY(cudaMemcpyAsync(score_out, s->Y, (size_t)B * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return TTO_OK;
}

int tto_surrogate_features(tto_surrogate* s, int32_t B, int32_t* si, float* sf, float* xd, int32_t* valid) {
  if (!s || B < 0 || B > s->bcap) return set_error(TTO_E_ARG, "B exceeds the last batch");
  TTO_CUDA_TRY(cudaSetDevice(s->g->device));
  TTO_CUDA_TRY(cudaDeviceSynchronize());
  const size_t b = B;
  if (si) TTO_CUDA_TRY(cudaMemcpy(si, s->SI, b * s->k * sizeof(int), cudaMemcpyDeviceToHost));
  if (sf) TTO_CUDA_TRY(cudaMemcpy(sf, s->SF, b * s->k * 8 * sizeof(float), cudaMemcpyDeviceToHost));
  if (xd) TTO_CUDA_TRY(cudaMemcpy(xd, s->XD, b * s->R * sizeof(float), cudaMemcpyDeviceToHost));
  if (valid) TTO_CUDA_TRY(cudaMemcpy(valid, s->valid, b * sizeof(int), cudaMemcpyDeviceToHost));
  return TTO_OK;
}

int tto_surrogate_trace(tto_surrogate* s, int32_t B, float* h, float* y, float* t, float* dy, float* dh) {
  if (!s || B < 0 || B > s->bcap) return set_error(TTO_E_ARG, "B exceeds the last batch");
  TTO_CUDA_TRY(cudaSetDevice(s->g->device));
  TTO_CUDA_TRY(cudaDeviceSynchronize());
  const size_t bh = (size_t)B * s->H * sizeof(float);
  const float* hs[3] = {s->H1, s->H2, s->H3};
  const float* ds[3] = {s->dH1, s->dH2, s->dH3};
  for (int l = 0; l < 3; ++l) {
    if (h) TTO_CUDA_TRY(cudaMemcpy((char*)h + l * bh, hs[l], bh, cudaMemcpyDeviceToHost));
    if (dh) TTO_CUDA_TRY(cudaMemcpy((char*)dh + l * bh, ds[l], bh, cudaMemcpyDeviceToHost));
  }
  if (y) TTO_CUDA_TRY(cudaMemcpy(y, s->Y, (size_t)B * sizeof(float), cudaMemcpyDeviceToHost));
  if (t) TTO_CUDA_TRY(cudaMemcpy(t, s->T, (size_t)B * sizeof(float), cudaMemcpyDeviceToHost));
  if (dy) TTO_CUDA_TRY(cudaMemcpy(dy, s->dY, (size_t)B * sizeof(float), cudaMemcpyDeviceToHost));
  return TTO_OK;
}

int tto_surrogate_add(tto_surrogate* s, const int32_t* topo, int32_t B, const float* fitness, void* stream) {
  if (!s || B < 0 || (B > 0 && (!topo || !fitness))) return set_error(TTO_E_ARG, "bad add arguments");
  if (B == 0) return TTO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(s->g->device));
  int rc = alloc_batch(s, B);
  if (rc) return rc;
  if ((rc = features(s, topo, B, 1, st))) return rc;
  // a batch larger than the ring leaves its last `cap` pairs
  const int skip = std::max(0, B - s->cap);
  return append(s, topo + (size_t)skip * s->k, B - skip, nullptr, s->XD + (size_t)skip * s->R, fitness + skip, st);
}

int tto_surrogate_train(tto_surrogate* s, int32_t steps, float* loss, void* stream) {
  if (!s || steps < 0) return set_error(TTO_E_ARG, "bad train arguments");
  if (steps == 0) return TTO_OK;
  TTO_CUDA_TRY(cudaSetDevice(s->g->device));
  return train(s, steps, loss, (cudaStream_t)stream);
}

int tto_surrogate_grad(tto_surrogate* s, const int32_t* topo, int32_t B, const float* fitness, float* loss,
                       float* grad, void* stream) {
  if (!s || B < 1 || !topo || !fitness) return set_error(TTO_E_ARG, "bad grad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(s->g->device));
  int rc = alloc_batch(s, B);
  if (rc) return rc;
  if ((rc = features(s, topo, B, 1, st))) return rc;
  targets_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, fitness, s->stats, s->T);
  TTO_CUDA_TRY(cudaGetLastError());
  if ((rc = forward(s, B, nullptr, st))) return rc;
  if ((rc = backward(s, B, st))) return rc;
  float l[2];
  TTO_CUDA_TRY(cudaMemcpyAsync(l, s->loss, sizeof(l), cudaMemcpyDeviceToHost, st));
  TTO_CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = l[1] > 0.f ? l[0] / l[1] : 0.f;
  if (grad) TTO_CUDA_TRY(cudaMemcpy(grad, s->G, s->n_params * 4, cudaMemcpyDeviceToHost));
  return TTO_OK;
}

int tto_mapelites_step_screened(tto_archive* a, tto_surrogate* s, uint64_t seed, uint64_t iteration,
                                int32_t n_propose, int32_t n_exact, int32_t rank_by, const tto_mut_params* mp,
                                const tto_eval_opts* opts, int32_t train_steps, int32_t* topo_out,
                                float* fitness_out, float* score_out, void* stream) {
  if (!a || !s || !mp || !opts || a->g != s->g) return set_error(TTO_E_ARG, "bad screened-step arguments");
  if (n_exact < 1 || n_propose < n_exact) return set_error(TTO_E_ARG, "need 1 <= n_exact <= n_propose");
  if (n_propose > (1 << 30)) return set_error(TTO_E_ARG, "n_propose must be at most 2^30");
  if (train_steps < 0) return set_error(TTO_E_ARG, "train_steps must be >= 0");
  if (rank_by != TTO_SCREEN_SCORE && rank_by != TTO_SCREEN_CELL_GAIN) return set_error(TTO_E_ARG, "unknown rank_by");
  if (opts->d_split != a->d_split || opts->d_moved != a->d_moved || a->d_disc != 1 || opts->d_disc > 1)
    return set_error(TTO_E_ARG, "evaluation cell extents differ from the archive's");
  tto_grid* g = a->g;
  cudaStream_t st = (cudaStream_t)stream;
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  if (g->T > TTO_MAX_T) return set_error(TTO_E_ARG, "grid has more than %d timesteps", TTO_MAX_T);
  int rc = ensure_workspace(g, n_exact, padded_T(g->T));
  if (rc) return rc;
  if (n_propose > s->pcap) {
    if (s->prop) cudaFree(s->prop);
    if (s->sel) cudaFree(s->sel);
    s->prop = nullptr;
    s->sel = nullptr;
    s->pcap = 0;
    TTO_CUDA_TRY(cudaMalloc(&s->prop, (size_t)n_propose * g->k_max * sizeof(int32_t)));
    TTO_CUDA_TRY(cudaMalloc(&s->sel, (size_t)n_propose * sizeof(int32_t)));
    s->pcap = n_propose;
  }
  // one allocation for scoring and training, so neither invalidates the other
  if ((rc = alloc_batch(s, std::max(n_propose, s->mb)))) return rc;
  Workspace& w = g->ws;
  if ((rc = propose_impl(a, seed, iteration, n_propose, mp, s->prop, st))) return rc;
  if (s->rep_n > 0) {
    if ((rc = score(s, s->prop, n_propose, st))) return rc;
  } else {
    if ((rc = features(s, s->prop, n_propose, 1, st))) return rc;
    valid_only_kernel<<<(n_propose + 255) / 256, 256, 0, st>>>(n_propose, s->valid, s->Y);
    TTO_CUDA_TRY(cudaGetLastError());
  }
  if ((rc = ensure_keys(s, n_propose))) return rc;
  const int npad = sort_pad(n_propose);
  screen_keys_kernel<<<(npad + 255) / 256, 256, 0, st>>>(n_propose, npad, g->k_max, rank_by, s->prop, s->nsm,
                                                         a->d_split, a->d_moved, a->d_genome, a->d_fit,
                                                         a->d_filled, s->Y, s->keys);
  TTO_CUDA_TRY(cudaGetLastError());
  if ((rc = sort_keys(s, n_propose, st))) return rc;
  select_kernel<<<1, 1024, 0, st>>>(n_propose, n_exact, g->k_max, s->keys, s->prop, s->sel);
  gather_topo_kernel<<<(n_exact + 255) / 256, 256, 0, st>>>(n_exact, g->k_max, s->sel, s->prop, w.topo);
  if (score_out) gather_score_kernel<<<(n_exact + 255) / 256, 256, 0, st>>>(n_exact, s->sel, s->Y, score_out);
  TTO_CUDA_TRY(cudaGetLastError());
  rc = evaluate_impl(g, w.topo, n_exact, nullptr, g->T, opts, w.fit, w.desc, w.cell, w.island, nullptr, nullptr, st);
  if (rc) return rc;
  if ((rc = insert_impl(a, w.topo, n_exact, w.fit, w.cell, st))) return rc;
  if ((rc = append(s, w.topo, n_exact, s->sel, s->XD, w.fit, st))) return rc;
  if (train_steps > 0 && (rc = train(s, train_steps, nullptr, st))) return rc;
  if (topo_out)
    TTO_CUDA_TRY(cudaMemcpyAsync(topo_out, w.topo, (size_t)n_exact * g->k_max * sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, st));
  if (fitness_out)
    TTO_CUDA_TRY(cudaMemcpyAsync(fitness_out, w.fit, (size_t)n_exact * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return TTO_OK;
}

}  // extern "C"
