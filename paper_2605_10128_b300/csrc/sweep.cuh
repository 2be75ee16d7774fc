// Kernel arguments shared by the evaluation kernels, and the sweep launcher.
#pragma once

#include <stdint.h>

#include "tto_internal.h"

namespace tto {

// busbar outage records: [station, |R'|, N columns of R' x kMaxBB, pad to a
// multiple of 4 floats], then p_v[TT], z[kMaxBB][TT], y[8][TT] (16-byte
// aligned rows, so timesteps load as float4)
constexpr int kMaxBB = TTO_MAX_ASSETS - 1;
constexpr int kBBHead = (2 + kMaxBB + 3) / 4 * 4;
constexpr int bb_record_floats(int TT) { return kBBHead + TT * (1 + kMaxBB + 8); }

// What the busbar setup needs from a topology's split update: the split
// slots, the moved branch ends (with the switchable column of each), K^-1 and
// psi per timestep.  k = -1 marks a topology without busbar records.
struct SplitState {
  int k, ns, nd, pad;
  int slot[TTO_MAX_K + 1];
  int st[TTO_MAX_K];
  uint32_t mask[TTO_MAX_K];
  int dis[TTO_MAX_K];
  int e[kMaxMoved];
  int col[kMaxMoved];
  double sign[kMaxMoved];
  double coef[kMaxMoved];
  double Ki[TTO_MAX_K][TTO_MAX_K];
  double psi[TTO_MAX_T][TTO_MAX_K];
};

struct EvalArgs {
  // grid (device)
  const float* Nmo;
  const float4* Nf;  // -N in mma C-fragment order (tensor-core sweep)
  const double* Nsw;
  const float* Nsw32;  // FP32 copy of Nsw
  const int* swcol;
  const double* f0;
  const double* p;
  const double* b;
  const double* invb;  // 1 / b
  const float* lim;
  const int* mon;
  const int* out;
  const double* Ncc;
  const int* from;
  const int* station_bus;
  const int* asset_off;
  const int* asset_br;
  const int* act_st;
  const uint32_t* act_mask;
  const int* disc;  // [n_disc] branches a genome may open
  int* status;
  int E, n_bus, E_mon, O, E_mon_pad, O_pad, A, k_max;
  int n_disc, n_dslot, gw;  // disconnection set and slots; genome width k_max + n_dslot
  int n_t, TT, KP;
  int TC, n_tch;  // tensor-core sweep: timesteps per pass and number of passes
  int tsel[TTO_MAX_T];
  int d_split, d_moved, d_disc;
  // busbar outages (lambda_b, lambda_f2)
  int busbar;            // compute them
  int S, NB, kRec;       // stations, busbar slots per topology (S + k_max), record floats
  const double* Pst;     // [S][E] unsplit responses to +1 at each station bus
  const float* Pm;       // [S][E_mon_pad] the same at the monitored rows
  const float* Nswm;     // [n_sw][E_mon_pad] switchable N columns at the monitored rows
  float* bbrec;          // [B][NB][kRec]
  SplitState* bbstate;   // [B] split state for the busbar setup
  float* bbpart;         // [B][n_rowtiles] partial lambda_b
  float* bmax;           // [B][n_t][E_mon] max over busbar outages of |flow|, or NULL
  const float* lbpre;    // lambda_b of the unsplit topology
  int precision;
  int fitness_kind;
  int n_rowtiles;
  int n_parts;  // partial-metric records per topology (set by the sweep launcher)
  int shape;    // sweep tile variant chosen by the autotuner (0 = default)
  int umma_packed;  // the split update writes the tcgen05 operand layouts (Ua, Vb, gq) instead of U, V, g
  // batch
  const int32_t* topo;
  int B;
  // workspace
  float* U;
  float* V;
  float* fp;
  float* gg;
  uint32_t* Ua;
  uint32_t* Vb;
  float* gq;
  TopoInfo* info;
  float* part;
  // outputs
  float* fitness;
  int32_t* desc;
  int32_t* cell;
  uint8_t* island;
  float* metrics;
  float* fmax;
};

// Topologies per CTA of the FP32 sweep at padded timestep count TT (the
// running maxima of G topologies x TT timesteps stay in registers).
constexpr int fp32_group(int TT) { return TT <= 4 ? 8 : (TT <= 8 ? 4 : (TT <= 16 ? 2 : 1)); }
// Topologies per item of the persistent work-list sweep: the smaller group of
// the FP32 sweep's two tile variants.
constexpr int fp32_item_group(int TT) { return fp32_group(TT) > 1 ? fp32_group(TT) / 2 : 1; }

// Several jobs (grid, topology batch) evaluated by one launch per stage:
// the split update over all jobs' topologies, the persistent FP32 sweep over
// (job, row tile, topology group) items, and the metric reduction.  Passed by
// value as a kernel parameter.
constexpr int kMaxMultiJobs = 16;
struct MultiArgs {
  int n;                                        // jobs
  unsigned int n_items;                         // sweep items in all
  unsigned int item_start[kMaxMultiJobs + 1];   // first sweep item of each job
  int blk_start[kMaxMultiJobs + 1];             // first topology of each job, counted over all jobs
  unsigned int* counter;                        // next sweep item (zeroed before the launch)
  EvalArgs job[kMaxMultiJobs];
};

// TF32 operand layouts of the tcgen05 sweep: the round-to-nearest TF32 bits of
// x, and the canonical K-major no-swizzle position of element (row, k) in a
// tile of 8-column rows: core matrix (row / 8, k / 4) at 256 (row / 8) +
// 128 (k / 4) bytes, 16 bytes per core-matrix row (in 32-bit words).
__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ int canon(int row, int k) { return (row >> 3) * 64 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3); }

// Launch the fused N-1 sweep for the precision in a.precision; sets a.n_parts.
int launch_sweep(EvalArgs& a, cudaStream_t s);
int launch_sweep_fp32(const EvalArgs& a, cudaStream_t s);
int launch_sweep_tc(EvalArgs& a, cudaStream_t s);
// Number of sweep tile variants for a precision mode (FP32 or tensor cores).
int sweep_shapes(int precision);
// Partial-metric records per topology the workspace must hold.
size_t max_parts(const tto_grid* g);
// Build the fragment-ordered copy of -N used by the tensor-core sweep (once).
int ensure_fragment_N(tto_grid* g, cudaStream_t s);
// One bounded wait on an mbarrier nothing completes (timeout-path test).
int bounded_wait_probe(int* status, long long cycles, cudaStream_t s);
// Mixed-grid batches: the persistent FP32 sweep over m's work list, and the
// split update and metric reduction of all of m's jobs in one launch each.
int launch_sweep_persistent(const MultiArgs& m, int device, cudaStream_t s);
int launch_split_update_multi(const MultiArgs& m, cudaStream_t s);
int launch_fitness_multi(const MultiArgs& m, cudaStream_t s);
// The tcgen05 sweep (TF32X3 only); sets a.n_parts.
int launch_sweep_umma(EvalArgs& a, cudaStream_t s);
// Sweep tile variant of TF32X3 that runs the tcgen05 kernel.
constexpr int kUmmaShape = 4;

}  // namespace tto
