// Evaluation entry point that allocates nothing.
//
// tto_evaluate_batch keeps its per-batch workspace in device memory that the
// library allocates (and grows) with cudaMalloc.  Some callers cannot allow
// that: a host process whose device memory is entirely owned by another
// allocator (for example a framework's caching allocator that reserved the
// device up front, or a fixed memory partition), or a long-running service
// that must not change its device-memory footprint once it has started.  For
// them, tto_evaluate_batch_static runs the same FP32 evaluation kernels with
// their workspace carved out of one file-scope __device__ array of fixed size,
// which exists on every device that loads this library until the process
// exits.  The array's device address is looked up once per device with
// cudaGetSymbolAddress (host code must not use the array's name as a device
// pointer); the first call on a device does that lookup and caches it for the
// life of the process, so the entry point must not be used across a
// cudaDeviceReset of that device (the cached address would be stale).
#include <string.h>

#include <mutex>

#include "sweep.cuh"
#include "tto_internal.h"

namespace tto {

__global__ void __launch_bounds__(256) split_update_kernel(EvalArgs a);
__global__ void fitness_kernel(EvalArgs a);

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device (looked up once).
int static_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return set_error(TTO_E_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TTO_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

}  // namespace tto

using namespace tto;

extern "C" int tto_evaluate_batch_static(tto_grid* g, const int32_t* topo, int32_t B,
                                         const int32_t* timesteps, int32_t n_t,
                                         const tto_eval_opts* o, float* fitness, int32_t* desc,
                                         int32_t* cell, uint8_t* island, float* metrics, float* fmax,
                                         void* stream) {
  if (!g || !o) return set_error(TTO_E_ARG, "null argument");
  if (B < 0) return set_error(TTO_E_ARG, "negative batch");
  if (B > 0 && (!topo || !fitness)) return set_error(TTO_E_ARG, "null topology or fitness buffer");
  if (o->precision != TTO_PREC_FP32)
    return set_error(TTO_E_ARG, "the static-scratch entry point evaluates with TTO_PREC_FP32 only");
  if (o->d_split < 1 || o->d_moved < 1 || o->d_disc < 0) return set_error(TTO_E_ARG, "archive extents must be >= 1");
  if (o->fitness_kind != TTO_FIT_WORKLOAD && o->fitness_kind != TTO_FIT_F1)
    return set_error(TTO_E_ARG, "unknown fitness kind");
  EvalArgs a;
  memset(&a, 0, sizeof(a));
  if (timesteps == nullptr) {
    if (g->T > TTO_MAX_T) return set_error(TTO_E_ARG, "n_t must be in [1, %d]", TTO_MAX_T);
    n_t = g->T;
    for (int t = 0; t < n_t; ++t) a.tsel[t] = t;
  } else {
    if (n_t < 1 || n_t > TTO_MAX_T) return set_error(TTO_E_ARG, "n_t must be in [1, %d]", TTO_MAX_T);
    for (int t = 0; t < n_t; ++t) {
      if (timesteps[t] < 0 || timesteps[t] >= g->T) return set_error(TTO_E_ARG, "timestep %d out of range", timesteps[t]);
      a.tsel[t] = timesteps[t];
    }
  }
  if (B == 0) return TTO_OK;
  const int TT = padded_T(n_t);
  const size_t Ep = g->E_mon_pad, Op = g->O_pad;
  const size_t bU = align256((size_t)B * Ep * 8 * sizeof(float));
  const size_t bV = align256((size_t)B * Op * 8 * sizeof(float));
  const size_t bF = align256((size_t)B * TT * Ep * sizeof(float));
  const size_t bG = align256((size_t)B * Op * TT * sizeof(float));
  const size_t bI = align256((size_t)B * sizeof(TopoInfo));
  const size_t bP = align256((size_t)B * g->n_rowtiles * 4 * sizeof(float));
  const size_t need = bU + bV + bF + bG + bI + bP;
  if (need > kStaticScratchBytes)
    return set_error(TTO_E_ARG,
                     "batch of %d topologies needs %zu bytes of scratch; the static scratch holds %zu "
                     "(use a smaller batch or tto_evaluate_batch)",
                     B, need, (size_t)kStaticScratchBytes);
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  unsigned char* base = nullptr;
  int rc = static_scratch(g->device, &base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  a.Nmo = g->d_Nmo;
  a.Nsw = g->d_Nsw;
  a.Nsw32 = g->d_Nsw32;
  a.swcol = g->d_swcol;
  a.f0 = g->d_f0;
  a.p = g->d_p;
  a.b = g->d_b;
  a.invb = g->d_invb;
  a.lim = g->d_lim;
  a.mon = g->d_mon;
  a.out = g->d_out;
  a.Ncc = g->d_Ncc;
  a.from = g->d_from;
  a.station_bus = g->d_station_bus;
  a.asset_off = g->d_asset_off;
  a.asset_br = g->d_asset_br;
  a.act_st = g->d_act_st;
  a.act_mask = g->d_act_mask;
  a.disc = g->d_disc;
  a.status = g->d_status;
  a.E = g->E;
  a.n_bus = g->n_bus;
  a.E_mon = g->E_mon;
  a.O = g->O;
  a.E_mon_pad = g->E_mon_pad;
  a.O_pad = g->O_pad;
  a.A = g->A;
  a.k_max = g->k_max;
  a.n_disc = g->n_disc;
  a.n_dslot = g->n_dslot;
  a.gw = g->gw;
  a.n_t = n_t;
  a.TT = TT;
  a.TC = TT <= 4 ? TT : 8;
  a.n_tch = (TT + a.TC - 1) / a.TC;
  a.KP = g->gw <= 2 ? 2 : (g->gw <= 4 ? 4 : 8);
  a.d_split = o->d_split;
  a.d_moved = o->d_moved;
  a.d_disc = o->d_disc > 1 ? o->d_disc : 1;
  a.precision = TTO_PREC_FP32;
  a.shape = g->tuned_shape[TTO_PREC_FP32] >= 0 ? g->tuned_shape[TTO_PREC_FP32] : 0;  // the autotuned variant
  a.fitness_kind = o->fitness_kind;
  a.n_rowtiles = g->n_rowtiles;
  a.n_parts = g->n_rowtiles;
  a.topo = topo;
  a.B = B;
  // every scratch array below is fully written before it is read within the
  // call, so nothing needs clearing between calls
  size_t off = 0;
  a.U = reinterpret_cast<float*>(base + off);
  off += bU;
  a.V = reinterpret_cast<float*>(base + off);
  off += bV;
  a.fp = reinterpret_cast<float*>(base + off);
  off += bF;
  a.gg = reinterpret_cast<float*>(base + off);
  off += bG;
  a.info = reinterpret_cast<TopoInfo*>(base + off);
  off += bI;
  a.part = reinterpret_cast<float*>(base + off);
  a.fitness = fitness;
  a.desc = desc;
  a.cell = cell;
  a.island = island;
  a.metrics = metrics;
  a.fmax = fmax;

  split_update_kernel<<<B, 256, 0, s>>>(a);
  TTO_CUDA_TRY(cudaGetLastError());
  rc = launch_sweep_fp32(a, s);
  if (rc) return rc;
  fitness_kernel<<<(B + 127) / 128, 128, 0, s>>>(a);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}
