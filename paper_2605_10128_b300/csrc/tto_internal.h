// Internal state of the DC N-1 topology evaluator (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tto.h"

namespace tto {

constexpr int kRowTile = 128;   // monitored-branch rows per sweep CTA
constexpr int kColPad = 64;     // outage columns are padded to this multiple
constexpr int kMaxMoved = TTO_MAX_K * TTO_MAX_ASSETS;
constexpr int kProfileCalls = 256;  // evaluation calls timed per profiling window
constexpr int kProfileEvents = 5;   // CUDA events per timed call
constexpr double kIslandTol = 1e-6;  // N'_cc (and normalised split pivot) at or below: islanded

int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);

#define TTO_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return ::tto::cuda_error(_e, #expr); \
  } while (0)

// Per-topology scalars written by the prep kernel.
struct TopoInfo {
  int island_base;   // the split disconnects the grid
  int n_islanded;    // outages that island the split grid
  int ns;            // split stations
  int nm;            // moved assets
  float lambda_c0;   // N-0 critical branches (summed over timesteps)
  float umax, vmax;  // largest |U| (monitored rows) and |V| (outage columns)
  int nd;            // opened branches (disconnection slots in use)
  int nbisl;         // busbar outages that island the topology
};

// Evaluation workspace, grown on demand (or once by tto_grid_reserve).
struct Workspace {
  int cap_B = 0;
  int cap_T = 0;
  float* U = nullptr;        // [B][E_mon_pad][8] FP32 row factors U = W K^-1
  float* V = nullptr;        // [B][O_pad][8]     FP32 column factors V_c = W_c / b_c
  uint32_t* Ua = nullptr;    // [B][E_mon_pad/16][lane][<=8] A fragments (tensor-core sweep)
  uint32_t* Vb = nullptr;    // [B][O_pad/8][lane][<=4]      B fragments (tensor-core sweep)
  float* gq = nullptr;       // [B][n_tch][O_pad/8][q][TC][2] g in lane order (tensor-core sweep)
  float* fp = nullptr;       // [B][TT][E_mon_pad]  post-split N-0 flows
  float* gg = nullptr;       // [B][O_pad][TT]      f'_c / N'_cc (NaN: outage islands)
  TopoInfo* info = nullptr;  // [B]
  float* part = nullptr;     // [B][parts][4]        per row-band partial metrics
  float* fit = nullptr;      // [B] scratch fitness (MapElites step)
  int32_t* cell = nullptr;   // [B]
  int32_t* desc = nullptr;   // [B][2]
  uint8_t* island = nullptr; // [B]
  int32_t* topo = nullptr;   // [B][gw] proposed genomes (MapElites step)
};

}  // namespace tto

struct tto_grid {
  uint64_t uid = 0;       // unique per created grid (keys recorded evaluation graphs)
  uint64_t ws_epoch = 0;  // bumped whenever the workspace is reallocated
  int device = 0;
  int n_bus = 0, E = 0, slack = 0, T = 0, E_mon = 0, O = 0, S = 0, A = 0, k_max = 0;
  int n_disc = 0, n_dslot = 0, gw = 0;  // disconnection set, its slots, genome width k_max + n_dslot
  int E_mon_pad = 0, O_pad = 0, n_sw = 0, n_rowtiles = 0;
  std::vector<int> from, to, mon, out, station_bus, asset_off, asset_br, act_st, act_off, disc;
  std::vector<uint32_t> act_mask;
  std::vector<double> b, p, limit, f0;
  // device copies
  float* d_Nmo = nullptr;      // [E_mon_pad][O_pad] N[mon l][out c], FP32
  float4* d_Nf = nullptr;      // -N in mma C-fragment order, built on first tensor-core use
  double* d_Nsw = nullptr;     // [n_sw][E] full N columns of movable branches, FP64
  float* d_Nsw32 = nullptr;    // [n_sw][E] FP32 copy (monitored rows of the split update)
  int* d_swcol = nullptr;      // [E] column of a movable branch in d_Nsw, else -1
  std::vector<int> swlist;     // branch of each d_Nsw column
  double* d_Pst = nullptr;     // [S][E] flows for +1 at station bus s, -1 at the slack (FP64)
  float* d_Pm = nullptr;       // [S][E_mon_pad] the same at the monitored rows, FP32
  float* d_Nswm = nullptr;     // [n_sw][E_mon_pad] d_Nsw at the monitored rows, FP32 (busbar outages; built on first use)
  float* d_lbpre = nullptr;    // lambda_b of the unsplit topology (tto_grid_busbar_reference)
  int lbpre_nt = 0;            // its timestep selection (lambda_f2 needs the same)
  int lbpre_tsel[TTO_MAX_T] = {};
  int32_t* d_empty = nullptr;  // one all-empty genome (the unsplit topology)
  float* d_bbrec = nullptr;    // busbar outage records [B][S + k_max][record]
  float* d_bbpart = nullptr;   // partial lambda_b [B][row tiles]
  void* d_bbstate = nullptr;   // split state per topology for the busbar setup [B]
  int bb_cap_B = 0, bb_cap_T = 0;
  double* d_f0 = nullptr;      // [T][E] base flows
  double* d_p = nullptr;       // [T][n_bus]
  double* d_b = nullptr;       // [E]
  double* d_invb = nullptr;    // [E] 1 / b (IEEE division, the same bits as on the device)
  float* d_lim = nullptr;      // [E_mon] limits of monitored branches
  int* d_mon = nullptr;        // [E_mon]
  int* d_out = nullptr;        // [O]
  double* d_Ncc = nullptr;     // [O] N[c][c]
  int* d_from = nullptr;       // [E]
  int* d_station_bus = nullptr;
  int* d_asset_off = nullptr;
  int* d_asset_br = nullptr;
  int* d_act_st = nullptr;
  int* d_act_off = nullptr;
  uint32_t* d_act_mask = nullptr;
  int* d_disc = nullptr;       // [n_disc] branches a genome may open
  int* d_status = nullptr;
  tto::Workspace ws;
  // sweep tile variant per precision mode chosen by tto_grid_autotune (-1: default)
  int tuned_shape[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  // optional per-stage timing (tto_grid_profile)
  int prof_on = 0, prof_n = 0;
  std::vector<cudaEvent_t> prof_ev;  // kProfileEvents per recorded call
};

namespace tto {
struct EpochSnap;  // epoch hand-over snapshot (epoch.cu)
}

struct tto_archive {
  tto_grid* g = nullptr;
  tto::EpochSnap* epoch = nullptr;  // created by the first tto_epoch_export
  int d_split = 0, d_moved = 0, d_disc = 1, cells = 0;
  float* d_fit = nullptr;         // [cells]
  int32_t* d_genome = nullptr;    // [cells][gw]
  uint8_t* d_filled = nullptr;    // [cells]
  unsigned long long* d_key = nullptr;  // [cells] batch winner keys
  int32_t* d_filled_list = nullptr;     // [cells + 1]: count, then filled cells ascending
};

namespace tto {
int ensure_workspace(tto_grid* g, int B, int T);
int padded_T(int n_t);  // timesteps rounded up to a compiled sweep width (-1 if > TTO_MAX_T)
void free_workspace(tto_grid* g);
// Drop recorded multi-grid evaluation graphs that use this grid.
void forget_grid_graphs(const tto_grid* g);
struct EvalArgs;
// Exact evaluation; with split_only set, stop after the split update (U, V,
// f', g in the workspace) and return the launch arguments there; with
// prepare_only as well, launch nothing (validation, workspace and arguments
// only; a batch of 0 topologies leaves *split_only untouched).
int evaluate_impl(tto_grid* g, const int32_t* topo, int B, const int32_t* tsel, int n_t,
                  const tto_eval_opts* o, float* fitness, int32_t* desc, int32_t* cell,
                  uint8_t* island, float* metrics, float* fmax, cudaStream_t s,
                  EvalArgs* split_only = nullptr, bool busbar_setup = false, bool prepare_only = false);
// Busbar outages (busbar.cu): tables and record workspace, launch arguments,
// the sweep and the per-topology lambda_b.
int ensure_busbar(tto_grid* g, int B, int TT, cudaStream_t s);
void fill_busbar_args(tto_grid* g, EvalArgs& a);
int launch_busbar_sweep(const EvalArgs& a, cudaStream_t s);
// MapElites building blocks shared by the plain and the surrogate-screened step.
int propose_impl(tto_archive* ar, uint64_t seed, uint64_t it, int B, const tto_mut_params* mp,
                 int32_t* out, cudaStream_t s);
int insert_impl(tto_archive* ar, const int32_t* topo, int B, const float* fit, const int32_t* cell,
                cudaStream_t s);
void free_epoch(tto_archive* a);  // waits for a pending epoch copy, frees the snapshot
// tto_worst_k with an optional device mask: topologies with use[b] == 0 are
// skipped (energies NaN, lists -1).
int worst_k_impl(tto_grid* g, const int32_t* topo, int32_t n, const int32_t* timesteps, int32_t n_t, int32_t k,
                 int32_t* outage_out, float* energy_out, float* all_energy, const uint8_t* use, cudaStream_t s);
}  // namespace tto
