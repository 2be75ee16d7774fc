// Exact DC N-1 evaluation of a batch of split topologies.
//
// Three kernels per call, all on the caller's stream:
//  1. split_update_kernel (one CTA per topology): decodes the genome into the
//     moved branch ends S (E x k, +-1) and moved injections, forms the split
//     matrix K = S^T N D S in FP64, factorises it (a pivot at or below
//     1e-6 * the moved susceptance marks a split that islands the grid), and
//     writes per topology
//        f'[t] = f0[t] + W psi[t],  psi[t] = K^-1 (p_M[t] - S^T f0[t]),  W = N D S,
//        U = W K^-1 (monitored rows),  V_c = W_c / b_c (outage rows),
//        g_c[t] = f'_c[t] / N'_cc  with  N'_cc = N_cc - U_c . V_c  in FP64
//     and g = NaN for an outage that islands the split grid (N'_cc <= 1e-6).
//     This is the bus split written as a phase shift on the moved branch ends
//     plus KCL at the new busbar: post-split flow responses are
//     N' = N - U V^T, the low-rank topology update of Sec. "DC-Optimizer".
//  2. the N-1 sweep (sweep_*.cu): for every (monitored l, outage c, t)
//        F = f'_l[t] - (N_lc - U_l . V_c) g_c[t],   fmax_l[t] = max_c |F|
//     (the LODF outage formula on the split grid), reduced on the fly to the
//     overload metrics; F is never stored.  fmaxf ignores a NaN operand, so
//     islanding outages drop out of the maximum for free.
//  3. fitness_kernel: fixed-order reduction of the per-row-tile partial
//     metrics into lambda_o, lambda_c, max loading and the fitness, plus the
//     descriptors and archive cell.
#include <math.h>
#include <stdio.h>

#include "sweep.cuh"
#include "tto_internal.h"

namespace tto {

// ------------------------------------------------------- factor layouts
// U [B][E_mon_pad][8], V [B][O_pad][8], g [B][O_pad][TT] in FP32; the
// tensor-core sweep repacks them into mma fragment order (sweep_tc.cu).
// With a.umma_packed (the tcgen05 sweep follows) the factors go straight into
// that sweep's operand layouts: U rows -> [B][band][hi, lo][128 x 8] and V
// columns -> [B][64-column chunk][hi, lo][64 x 8] as TF32 hi/lo splits in the
// canonical K-major layout, g -> [B][t-pass][O_pad / 2][TC][2] with the two
// columns of a pair interleaved per timestep (and U rows in plain order too
// when the busbar sweep follows).
__device__ __forceinline__ void store_row_factors(const EvalArgs& a, int b, int l, const float* u) {
  if (a.umma_packed) {
    uint32_t* base = a.Ua + ((size_t)b * (a.E_mon_pad >> 7) + (l >> 7)) * 2048;
    const int r = l & 127;
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      hi[k] = tf32_bits(u[k]);
      lo[k] = tf32_bits(u[k] - __uint_as_float(hi[k]));
    }
    // k = 0-3 and 4-7 of a row are 16 contiguous bytes each in the canonical layout
    *reinterpret_cast<uint4*>(base + canon(r, 0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(base + canon(r, 4)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
    *reinterpret_cast<uint4*>(base + 1024 + canon(r, 0)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<uint4*>(base + 1024 + canon(r, 4)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
    if (!a.busbar) return;  // the busbar sweep reads the plain U rows as well
  }
  float4* Urow = reinterpret_cast<float4*>(a.U + ((size_t)b * a.E_mon_pad + l) * 8);
  Urow[0] = make_float4(u[0], u[1], u[2], u[3]);
  Urow[1] = make_float4(u[4], u[5], u[6], u[7]);
}

__device__ __forceinline__ void store_col_v(const EvalArgs& a, int b, int c, const float* v) {
  if (a.umma_packed) {
    uint32_t* base = a.Vb + ((size_t)b * (a.O_pad >> 6) + (c >> 6)) * 1024;
    const int n = c & 63;
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      hi[k] = tf32_bits(v[k]);
      lo[k] = tf32_bits(v[k] - __uint_as_float(hi[k]));
    }
    *reinterpret_cast<uint4*>(base + canon(n, 0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(base + canon(n, 4)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
    *reinterpret_cast<uint4*>(base + 512 + canon(n, 0)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<uint4*>(base + 512 + canon(n, 4)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
    return;
  }
  float4* Vrow = reinterpret_cast<float4*>(a.V + ((size_t)b * a.O_pad + c) * 8);
  Vrow[0] = make_float4(v[0], v[1], v[2], v[3]);
  Vrow[1] = make_float4(v[4], v[5], v[6], v[7]);
}

// g of column c at padded timestep t = ci TC + tt (timestep pass ci, position
// tt within it; the packed layout's passes, the plain layout ignores them).
__device__ __forceinline__ void store_col_g(const EvalArgs& a, int b, int c, int t, int ci, int tt, float g) {
  if (a.umma_packed)
    a.gq[((((size_t)b * a.n_tch + ci) * (a.O_pad / 2) + c / 2) * a.TC + tt) * 2 + (c & 1)] = g;
  else
    a.gg[((size_t)b * a.O_pad + c) * a.TT + t] = g;
}

// ------------------------------------------------------ busbar outage setup
// Busbar outages (Sec. "Fitness function heuristics": lambda_b over the
// busbar outage set O_b): every splittable station's node, and both nodes of a
// split station, taken out of service (branches opened, injection dropped, the
// slack balances).  Per topology and busbar node v, with R_v its live branches
// and p_v its injection, the post-outage flows on the post-topology grid are
//   F = f' - p_v rho - N'[:, R'] z,   N'_{R'R'} z = f'_{R'} - p_v rho_{R'},
// rho = pi_s + U kappa (the post-topology response to +1 at v, -1 at the
// slack; pi_s the unsplit response at the station bus, kappa = dp_M - S^T pi_s
// with dp_M = e_j for busbar B of split slot j) and R' = R_v without its first
// branch: once p_v is gone, v hangs on that branch with no injection and
// carries no flow.  N'_{R'R'} is singular exactly when the rest of the grid
// falls apart without v (the busbar outage islands).  With N' = N - U V^T the
// monitored rows need only
//   F_l[t] = f'_l[t] - p_v[t] pi_s,l - sum_j N_{l r_j} z_j[t] - U_l . y[t],
//   y[t] = p_v[t] kappa - sum_j z_j[t] V_{r_j},
// so each (topology, busbar) record holds s, |R'|, the N columns of R', p_v,
// z and y.  The small system is solved in FP64 as D^-1 N'_{R'R'} (symmetric:
// D^-1 N and D^-1 U V^T = D^-1 W K^-1 W^T D^-1 are) by LDL^T, with the
// islanding test pivot x b_r <= 1e-6 as for single outages.
__device__ void busbar_record(const EvalArgs& a, int b, int v, const SplitState& ss, int* n_island) {
  const int TT = a.TT, nt = a.n_t;
  const int k = ss.k, ns = ss.ns, nd = ss.nd;
  const int* s_st = ss.st;
  const uint32_t* s_mask = ss.mask;
  const int* s_dis = ss.dis;
  const int* s_slot = ss.slot;
  const int* s_e = ss.e;
  const double* s_sign = ss.sign;
  const double* s_coef = ss.coef;
  const double(*s_Ki)[TTO_MAX_K] = ss.Ki;
  const double(*s_psi)[TTO_MAX_K] = ss.psi;
  {
    float* rec = a.bbrec + ((size_t)b * a.NB + v) * a.kRec;
    int* irec = reinterpret_cast<int*>(rec);
    int s, side, js = -1;
    if (v < a.S) {
      s = v;
      side = 0;
    } else {
      const int j = v - a.S;
      if (j >= ns) {
        irec[0] = 0;
        irec[1] = -1;  // no such busbar in this topology
        return;
      }
      s = s_st[j];
      side = 1;
    }
    for (int j = 0; j < ns; ++j)
      if (s_st[j] == s) js = j;
    const uint32_t mask = js >= 0 ? s_mask[js] : 0u;
    const int a0 = a.asset_off[s], m = a.asset_off[s + 1] - a0, bus = a.station_bus[s];
    int R[TTO_MAX_ASSETS], nrv = 0;
    bool inj = false;
    for (int i = 0; i < m; ++i) {
      const bool on_b = (mask >> i) & 1u;
      if (side == 1 ? !on_b : on_b) continue;  // the asset sits on the other node
      const int e = a.asset_br[a0 + i];
      if (e < 0) {
        inj = true;
        continue;
      }
      bool open = false;
      for (int q = 0; q < nd; ++q) open = open || s_dis[q] == e;
      if (!open) R[nrv++] = e;
    }
    irec[0] = s;
    if (nrv == 0) {  // a node without live branches: the topology itself islands (not reached)
      irec[1] = -2;
      atomicAdd(n_island, 1);
      return;
    }
    float* prec = rec + kBBHead;
    float* zrec = prec + TT;
    float* yrec = zrec + kMaxBB * TT;
    double kap[TTO_MAX_K];
    for (int i = 0; i < k; ++i) {
      double st = 0.0;
      for (int q = s_slot[i]; q < s_slot[i + 1]; ++q) st += s_sign[q] * a.Pst[(size_t)s * a.E + s_e[q]];
      kap[i] = (side == 1 && i == js ? 1.0 : 0.0) - st;
    }
    const int nrp = nrv - 1;
    // Per branch r_j of R': its W row, 1 / b_r, rho_r, and row j of
    // Q = D^-1 N'_{R'R'} (lower triangle, packed by rows: Q(i, j) at
    // i (i + 1) / 2 + j) from the branch's U row, which is not kept.
    double W[kMaxBB][TTO_MAX_K], Q[kMaxBB * (kMaxBB + 1) / 2], rho[kMaxBB], ib[kMaxBB];
    for (int ii = 0; ii < nrp; ++ii) {
      const int r = R[1 + ii];
      ib[ii] = a.invb[r];
      for (int i = 0; i < k; ++i) {
        double w = 0.0;
        for (int q = s_slot[i]; q < s_slot[i + 1]; ++q) w += s_coef[q] * a.Nsw[(size_t)ss.col[q] * a.E + r];
        W[ii][i] = w;
      }
      double U[TTO_MAX_K], rh = a.Pst[(size_t)s * a.E + r];
      for (int i = 0; i < k; ++i) {
        double u = 0.0;
        for (int i2 = 0; i2 < k; ++i2) u += W[ii][i2] * s_Ki[i2][i];
        U[i] = u;
        rh += u * kap[i];
      }
      rho[ii] = rh;
      for (int jj = 0; jj <= ii; ++jj) {
        double uv = 0.0;
        for (int i = 0; i < k; ++i) uv += U[i] * W[jj][i];
        Q[ii * (ii + 1) / 2 + jj] = (a.Nsw[(size_t)a.swcol[R[1 + jj]] * a.E + r] - uv * ib[jj]) * ib[ii];
      }
    }
    // LDL^T in place (L below the diagonal, D on it); idg = 1 / D
    bool isl = false;
    double idg[kMaxBB];
    for (int j = 0; j < nrp && !isl; ++j) {
      const int jr = j * (j + 1) / 2;
      double dj = Q[jr + j];
      for (int q = 0; q < j; ++q) dj -= Q[jr + q] * Q[jr + q] * Q[q * (q + 1) / 2 + q];
      if (!(dj * a.b[R[1 + j]] > kIslandTol)) isl = true;
      Q[jr + j] = dj;
      idg[j] = 1.0 / dj;
      for (int i = j + 1; i < nrp && !isl; ++i) {
        const int ir = i * (i + 1) / 2;
        double x = Q[ir + j];
        for (int q = 0; q < j; ++q) x -= Q[ir + q] * Q[jr + q] * Q[q * (q + 1) / 2 + q];
        Q[ir + j] = x * idg[j];
      }
    }
    if (isl) {
      irec[1] = -2;
      atomicAdd(n_island, 1);
      return;
    }
    // per timestep: rhs_j = (f'_{r_j} - p_v rho_j) / b_j, z from L D L^T, then y
    for (int t = 0; t < TT; ++t) {
      const double pvt = (inj && t < nt) ? a.p[(size_t)a.tsel[t] * a.n_bus + bus] : 0.0;
      prec[t] = (float)pvt;
      double z[kMaxBB];
      for (int i = 0; i < nrp; ++i) {
        double f = 0.0;
        if (t < nt) {
          f = a.f0[(size_t)a.tsel[t] * a.E + R[1 + i]];
          for (int q = 0; q < k; ++q) f += W[i][q] * s_psi[t][q];
        }
        const int ir = i * (i + 1) / 2;
        double x = (f - pvt * rho[i]) * ib[i];
        for (int q = 0; q < i; ++q) x -= Q[ir + q] * z[q];
        z[i] = x;
      }
      for (int i = 0; i < nrp; ++i) z[i] *= idg[i];
      for (int i = nrp - 1; i >= 0; --i) {
        double x = z[i];
        for (int q = i + 1; q < nrp; ++q) x -= Q[q * (q + 1) / 2 + i] * z[q];
        z[i] = x;
      }
      for (int jj = 0; jj < kMaxBB; ++jj) zrec[jj * TT + t] = jj < nrp ? (float)z[jj] : 0.f;
      for (int jj = 0; jj < nrp; ++jj) z[jj] *= ib[jj];  // z_j / b_j for y
      for (int i = 0; i < TTO_MAX_K; ++i) {
        double y = 0.0;
        if (i < k) {
          y = pvt * kap[i];
          for (int jj = 0; jj < nrp; ++jj) y -= z[jj] * W[jj][i];
        }
        yrec[i * TT + t] = (float)y;
      }
    }
    irec[1] = nrp;
    for (int jj = 0; jj < kMaxBB; ++jj) irec[2 + jj] = jj < nrp ? a.swcol[R[1 + jj]] : 0;
  }
}

// One thread per (topology, busbar node): the busbar outage record from the
// topology's split state, which its split update saved (records of a topology
// whose split islands the grid, or whose genome is invalid, are marked unused).
__global__ void __launch_bounds__(128) busbar_setup_kernel(EvalArgs a) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)a.B * a.NB) return;
  const int b = (int)(i / a.NB), v = (int)(i % a.NB);
  const SplitState& ss = a.bbstate[b];
  if (ss.k < 0) {
    int* irec = reinterpret_cast<int*>(a.bbrec + ((size_t)b * a.NB + v) * a.kRec);
    irec[0] = 0;
    irec[1] = -1;
    return;
  }
  busbar_record(a, b, v, ss, &a.info[b].nbisl);
}

// ---------------------------------------------------------------- split update
template <bool BB>
__device__ __forceinline__ void split_update_body(const EvalArgs& a, const int b) {
  const int tid = threadIdx.x;
  __shared__ int s_k, s_island, s_ns, s_nm;
  __shared__ int s_slot[TTO_MAX_K + 1];
  __shared__ int s_e[kMaxMoved];
  __shared__ double s_sign[kMaxMoved];
  __shared__ double s_coef[kMaxMoved];
  __shared__ const double* s_col[kMaxMoved];
  __shared__ const float* s_col32[kMaxMoved];
  __shared__ float s_coef32[kMaxMoved];
  __shared__ int s_injbus[TTO_MAX_K];
  __shared__ double s_K[TTO_MAX_K][TTO_MAX_K];
  __shared__ double s_Ki[TTO_MAX_K][TTO_MAX_K];
  __shared__ double s_Ki2[TTO_MAX_K][TTO_MAX_K];  // Ki_ji + Ki_ij for i > j
  __shared__ float s_Kif[TTO_MAX_K][TTO_MAX_K];  // FP32 copy for the monitored rows' U
  __shared__ double s_rhs[TTO_MAX_T][TTO_MAX_K];
  __shared__ double s_psi[TTO_MAX_T][TTO_MAX_K];
  __shared__ float s_psi32[TTO_MAX_T][TTO_MAX_K];
  __shared__ double s_sb[TTO_MAX_K];
  __shared__ int s_cnt_c0, s_cnt_isl;
  __shared__ float s_umax, s_vmax;
  __shared__ int s_dis[TTO_MAX_K], s_nd;  // branches the genome opens
  __shared__ int s_st[TTO_MAX_K];          // station of each split slot
  __shared__ uint32_t s_mk[TTO_MAX_K];     // its busbar-B mask

  if (tid == 0) {
    int k = 0, ne = 0, bad = 0, ns = 0, nm = 0, nd = 0;
    int stations[TTO_MAX_K];
    const int32_t* row = a.topo + (size_t)b * a.gw;
    // opened branches first: a split does not move a branch that is open
    for (int j = 0; j < a.n_dslot; ++j) {
      const int dj = row[a.k_max + j];
      if (dj < 0) continue;
      if (dj >= a.n_disc) {
        bad = 1;
        break;
      }
      const int e = a.disc[dj];
      for (int q = 0; q < nd; ++q)
        if (s_dis[q] == e) bad = 1;
      if (bad) break;
      s_dis[nd++] = e;
    }
    s_slot[0] = 0;
    for (int j = 0; j < a.k_max && !bad; ++j) {
      int act = row[j];
      if (act < 0) continue;
      if (act >= a.A) {
        bad = 1;
        break;
      }
      int st = a.act_st[act];
      for (int q = 0; q < k; ++q)
        if (stations[q] == st) bad = 1;
      if (bad) break;
      stations[k] = st;
      uint32_t mask = a.act_mask[act];
      s_st[k] = st;
      s_mk[k] = mask;
      int bus = a.station_bus[st];
      int a0 = a.asset_off[st], m = a.asset_off[st + 1] - a0;
      int onb = __popc(mask);
      ++ns;
      nm += min(onb, m - onb);
      s_injbus[k] = -1;
      for (int i = 0; i < m; ++i) {
        if (!((mask >> i) & 1u)) continue;
        int e = a.asset_br[a0 + i];
        if (e < 0) {
          s_injbus[k] = bus;
          continue;
        }
        bool open = false;
        for (int q = 0; q < nd; ++q) open = open || s_dis[q] == e;
        if (open) continue;  // busbar B keeps only open branches: zero pivot, islanded
        double sg = (a.from[e] == bus) ? 1.0 : -1.0;
        s_e[ne] = e;
        s_sign[ne] = sg;
        s_coef[ne] = sg * a.b[e];
        s_col[ne] = a.Nsw + (size_t)a.swcol[e] * a.E;
        s_coef32[ne] = (float)(sg * a.b[e]);
        s_col32[ne] = a.Nsw32 + (size_t)a.swcol[e] * a.E;
        ++ne;
      }
      ++k;
      s_slot[k] = ne;
    }
    // an opened branch is a phase shift across it whose constraint holds its
    // flow at zero: one more slot with S = e_l (its from end) and no injection
    for (int q = 0; q < nd && !bad; ++q) {
      const int e = s_dis[q];
      s_injbus[k] = -1;
      s_e[ne] = e;
      s_sign[ne] = 1.0;
      s_coef[ne] = a.b[e];
      s_col[ne] = a.Nsw + (size_t)a.swcol[e] * a.E;
      s_coef32[ne] = (float)a.b[e];
      s_col32[ne] = a.Nsw32 + (size_t)a.swcol[e] * a.E;
      ++ne;
      ++k;
      s_slot[k] = ne;
    }
    s_k = bad ? 0 : k;
    s_ns = ns;
    s_nm = nm;
    s_nd = bad ? 0 : nd;
    s_island = bad;
    s_cnt_c0 = 0;
    s_cnt_isl = 0;
    s_umax = 0.f;
    s_vmax = 0.f;
    if (bad) atomicExch(a.status, TTO_E_TOPOLOGY);
  }
  __syncthreads();
  const int k = s_k;
  const int nt = a.n_t;
  // K = S^T W, rhs = p_M - S^T f0 (sequential sums: deterministic)
  if (tid < k * k) {
    int i = tid / k, j = tid % k;
    double acc = 0.0;
    for (int q = s_slot[i]; q < s_slot[i + 1]; ++q) {
      double w = 0.0;
      for (int r = s_slot[j]; r < s_slot[j + 1]; ++r) w += s_coef[r] * s_col[r][s_e[q]];
      acc += s_sign[q] * w;
    }
    s_K[i][j] = acc;
  }
  if (tid < k * nt) {
    int j = tid / nt, t = tid % nt;
    int tt = a.tsel[t];
    double st = 0.0;
    for (int q = s_slot[j]; q < s_slot[j + 1]; ++q) st += s_sign[q] * a.f0[(size_t)tt * a.E + s_e[q]];
    double pm = s_injbus[j] >= 0 ? a.p[(size_t)tt * a.n_bus + s_injbus[j]] : 0.0;
    s_rhs[t][j] = pm - st;
  }
  if (tid < k) {
    double sb = 0.0;
    for (int q = s_slot[tid]; q < s_slot[tid + 1]; ++q) sb += a.b[s_e[q]];
    s_sb[tid] = sb;
  }
  __syncthreads();
  if (tid == 0 && k > 0) {
    // LDL^T of the SPD split matrix; a vanishing pivot means the split islands
    double L[TTO_MAX_K][TTO_MAX_K], D[TTO_MAX_K];
    int isl = 0;
    for (int j = 0; j < k; ++j) {
      double d = s_K[j][j];
      for (int q = 0; q < j; ++q) d -= L[j][q] * L[j][q] * D[q];
      D[j] = d;
      if (!(d > kIslandTol * s_sb[j])) {
        isl = 1;
        break;
      }
      for (int i = j + 1; i < k; ++i) {
        double v = s_K[i][j];
        for (int q = 0; q < j; ++q) v -= L[i][q] * L[j][q] * D[q];
        L[i][j] = v / d;
      }
      L[j][j] = 1.0;
    }
    s_island = isl;
    if (!isl) {
      for (int c = 0; c < k; ++c) {
        double x[TTO_MAX_K];
        for (int i = 0; i < k; ++i) {
          double v = (i == c) ? 1.0 : 0.0;
          for (int q = 0; q < i; ++q) v -= L[i][q] * x[q];
          x[i] = v;
        }
        for (int i = 0; i < k; ++i) x[i] /= D[i];
        for (int i = k - 1; i >= 0; --i) {
          double v = x[i];
          for (int q = i + 1; q < k; ++q) v -= L[q][i] * x[q];
          x[i] = v;
        }
        for (int i = 0; i < k; ++i) {
          s_Ki[i][c] = x[i];
          s_Kif[i][c] = (float)x[i];
        }
      }
      for (int j = 0; j < k; ++j)  // off-diagonal pair sums for the outage rows' W^T K^-1 W
        for (int i = j + 1; i < k; ++i) s_Ki2[j][i] = s_Ki[j][i] + s_Ki[i][j];
    }
  }
  __syncthreads();
  const bool dead = s_island != 0;
  if (!dead && tid < k * nt) {
    int j = tid / nt, t = tid % nt;
    double v = 0.0;
    for (int q = 0; q < k; ++q) v += s_Ki[j][q] * s_rhs[t][q];
    s_psi[t][j] = v;
    s_psi32[t][j] = (float)v;
  }
  __syncthreads();

  const int TT = a.TT;
  const float qnan = __int_as_float(0x7fc00000);
  int c0cnt = 0;
  float umax = 0.f, vmax = 0.f;
  // monitored rows: f', U
  // The FP32 loops over the k split slots are unrolled to TTO_MAX_K
  // (predicated on k, which is uniform over the CTA) so that the per-slot
  // arrays stay in registers; timesteps are stored as they are computed.
  for (int l = tid; l < a.E_mon_pad; l += blockDim.x) {
    const int lr = min(l, a.E_mon - 1);
    const int e = a.mon[lr];
    float* fpr = a.fp + (size_t)b * TT * a.E_mon_pad + l;  // f' of row l, timestep t at t E_mon_pad
    float u[TTO_MAX_K];
    if (dead) {
#pragma unroll
      for (int j = 0; j < TTO_MAX_K; ++j) u[j] = 0.f;
      store_row_factors(a, b, l, u);
      for (int t = 0; t < TT; ++t) fpr[(size_t)t * a.E_mon_pad] = 0.f;
      continue;
    }
    // FP32 first (B300's FP64 pipe is narrow): W from the FP32 copy of the N
    // columns, U = W K^-1, f' = f0 + W psi, with an a-priori bound on the
    // rounding error of f': each FP32 sum of n terms errs by at most n u times
    // the sum of the absolute terms (u = 2^-24), and W's own sums and the FP32
    // N values add the same for W's terms, so |err f'| <= 32 u (|f0| + sum_j
    // |W|_j |psi_j|) with |W|_j the sum of the absolute W terms.  A row whose
    // bound exceeds 1e-5 of its limit is recomputed in FP64.
    float Wf[TTO_MAX_K], Wa[TTO_MAX_K];
#pragma unroll
    for (int j = 0; j < TTO_MAX_K; ++j) {
      float w = 0.f, wa = 0.f;
      if (j < k)
        for (int q = s_slot[j]; q < s_slot[j + 1]; ++q) {
          const float n = s_col32[q][e];
          w = fmaf(s_coef32[q], n, w);
          wa = fmaf(fabsf(s_coef32[q]), fabsf(n), wa);
        }
      Wf[j] = w;
      Wa[j] = wa;
    }
    // U of a monitored row only enters the TF32-split contraction: FP32 is
    // exact enough
#pragma unroll
    for (int jj = 0; jj < TTO_MAX_K; ++jj) {
      float uu = 0.f;
#pragma unroll
      for (int j = 0; j < TTO_MAX_K; ++j)
        if (jj < k && j < k) uu = fmaf(Wf[j], s_Kif[j][jj], uu);
      u[jj] = uu;
      umax = fmaxf(umax, fabsf(uu));
    }
    store_row_factors(a, b, l, u);
    const float lim = a.lim[lr];
    bool fp32_ok = true;
    int c0row = 0;
    for (int t = 0; t < TT; ++t) {
      float fv = 0.f;
      if (t < nt) {
        const float f0 = (float)a.f0[(size_t)a.tsel[t] * a.E + e];
        float f = f0, bound = fabsf(f0);
#pragma unroll
        for (int j = 0; j < TTO_MAX_K; ++j)
          if (j < k) {
            f = fmaf(Wf[j], s_psi32[t][j], f);
            bound = fmaf(Wa[j], fabsf(s_psi32[t][j]), bound);
          }
        fv = f;
        fp32_ok = fp32_ok && bound * (32.f / 16777216.f) <= 1e-5f * lim;
        if (l < a.E_mon && fabsf(f) > lim) ++c0row;
      }
      fpr[(size_t)t * a.E_mon_pad] = fv;
    }
    if (!fp32_ok) {  // the FP64 values replace the FP32 ones just written
      double W[TTO_MAX_K];
      for (int j = 0; j < k; ++j) {
        double w = 0.0;
        for (int q = s_slot[j]; q < s_slot[j + 1]; ++q) w += s_coef[q] * s_col[q][e];
        W[j] = w;
      }
      c0row = 0;
      for (int t = 0; t < nt; ++t) {
        double f = a.f0[(size_t)a.tsel[t] * a.E + e];
        for (int j = 0; j < k; ++j) f += W[j] * s_psi[t][j];
        const float fv = (float)f;
        fpr[(size_t)t * a.E_mon_pad] = fv;
        if (l < a.E_mon && fabsf(fv) > lim) ++c0row;
      }
    }
    c0cnt += c0row;
  }
  // outage rows: V, g, islanding of each outage
  int islcnt = 0;
  for (int c = tid; c < a.O_pad; c += blockDim.x) {
    const int cr = min(c, a.O - 1);
    const int e = a.out[cr];
    float v[TTO_MAX_K];
    if (dead) {
#pragma unroll
      for (int j = 0; j < TTO_MAX_K; ++j) v[j] = 0.f;
      store_col_v(a, b, c, v);
      for (int t = 0, ci = 0, tt = 0; t < TT; ++t) {
        store_col_g(a, b, c, t, ci, tt, t < nt ? qnan : 0.f);
        if (++tt == a.TC) tt = 0, ++ci;
      }
      continue;
    }
    // (the FP64 loops run to k: unrolled to TTO_MAX_K with predicates they
    // measured slower, the FP64 pipe being narrow)
    double W[TTO_MAX_K];
    for (int j = 0; j < k; ++j) {
      double w = 0.0;
      for (int q = s_slot[j]; q < s_slot[j + 1]; ++q) w += s_coef[q] * s_col[q][e];
      W[j] = w;
    }
    // N'_cc = N_cc - U_c . V_c = N_cc - (W^T K^-1 W) / b_c.  FP64 division is
    // a long instruction sequence on this part: 1 / b_c comes from the grid's
    // table, each row divides once (1 / N'_cc) and multiplies elsewhere.
    // W^T K^-1 W = sum_j W_j (Ki_jj W_j + sum_{i>j} (Ki_ji + Ki_ij) W_i).
    const double inv_be = a.invb[e];
    double q = 0.0;
    for (int j = 0; j < k; ++j) {
      double uu = s_Ki[j][j] * W[j];
      for (int i = j + 1; i < k; ++i) uu += s_Ki2[j][i] * W[i];
      q += uu * W[j];
    }
    const double npcc = a.Ncc[cr] - q * inv_be;
    for (int jj = 0; jj < TTO_MAX_K; ++jj) {
      v[jj] = jj < k ? (float)(W[jj] * inv_be) : 0.f;
      vmax = fmaxf(vmax, fabsf(v[jj]));
    }
    bool opened = false;  // an outage of an open branch is no contingency
    for (int q = 0; q < s_nd; ++q) opened = opened || s_dis[q] == e;
    const bool isl = opened || !(npcc > kIslandTol);
    if (isl && !opened && c < a.O) ++islcnt;
    const double inv_np = isl ? 0.0 : 1.0 / npcc;
    store_col_v(a, b, c, v);
    for (int t = 0, ci = 0, tt = 0; t < TT; ++t) {
      float g = 0.f;
      if (t < nt) {
        if (isl) {
          g = qnan;
        } else {
          double f = a.f0[(size_t)a.tsel[t] * a.E + e];
          for (int j = 0; j < k; ++j) f += W[j] * s_psi[t][j];
          g = (float)(f * inv_np);
        }
      }
      store_col_g(a, b, c, t, ci, tt, g);
      if (++tt == a.TC) tt = 0, ++ci;
    }
  }
  if (c0cnt) atomicAdd(&s_cnt_c0, c0cnt);
  if (islcnt) atomicAdd(&s_cnt_isl, islcnt);
  // magnitudes are >= 0, so the float bit patterns order like the values
  if (umax > 0.f) atomicMax(reinterpret_cast<int*>(&s_umax), __float_as_int(umax));
  if (vmax > 0.f) atomicMax(reinterpret_cast<int*>(&s_vmax), __float_as_int(vmax));
  if constexpr (BB) {
    // the split state the busbar setup needs (busbar_setup_kernel, one thread
    // per busbar node, runs after this kernel)
    SplitState& ss = a.bbstate[b];
    if (dead) {
      if (tid == 0) ss.k = -1;
    } else {
      const int ne = s_slot[k];
      if (tid == 0) {
        ss.k = k;
        ss.ns = s_ns;
        ss.nd = s_nd;
      }
      for (int i = tid; i <= k; i += blockDim.x) ss.slot[i] = s_slot[i];
      for (int i = tid; i < TTO_MAX_K; i += blockDim.x) {
        ss.st[i] = s_st[i];
        ss.mask[i] = s_mk[i];
        ss.dis[i] = s_dis[i];
      }
      for (int i = tid; i < ne; i += blockDim.x) {
        ss.e[i] = s_e[i];
        ss.col[i] = a.swcol[s_e[i]];
        ss.sign[i] = s_sign[i];
        ss.coef[i] = s_coef[i];
      }
      for (int i = tid; i < TTO_MAX_K * TTO_MAX_K; i += blockDim.x) (&ss.Ki[0][0])[i] = (&s_Ki[0][0])[i];
      for (int i = tid; i < a.TT * TTO_MAX_K; i += blockDim.x) (&ss.psi[0][0])[i] = (&s_psi[0][0])[i];
    }
  }
  __syncthreads();
  if (tid == 0) {
    TopoInfo inf;
    inf.island_base = s_island;
    inf.n_islanded = dead ? 0 : s_cnt_isl;
    inf.ns = s_ns;
    inf.nm = s_nm;
    inf.lambda_c0 = dead ? 0.f : (float)s_cnt_c0;
    inf.umax = s_umax;
    inf.vmax = s_vmax;
    inf.nd = s_nd;
    inf.nbisl = 0;  // busbar_setup_kernel counts the islanding busbar outages
    a.info[b] = inf;
  }
}

// Two instantiations: the busbar-outage setup needs many more registers and a
// large stack, which the plain split update should not pay for.
__global__ void __launch_bounds__(256) split_update_kernel(EvalArgs a) { split_update_body<false>(a, blockIdx.x); }
__global__ void __launch_bounds__(256) split_update_bb_kernel(EvalArgs a) { split_update_body<true>(a, blockIdx.x); }

// Job of topology i counted over all jobs of a mixed batch.
__device__ __forceinline__ int multi_job(const MultiArgs& m, int i) {
  int j = 0;
  for (int q = 1; q < m.n; ++q)
    if (i >= m.blk_start[q]) j = q;
  return j;
}

// The split update of every job of a mixed batch, one CTA per topology.
__global__ void __launch_bounds__(256) split_update_multi_kernel(const __grid_constant__ MultiArgs m) {
  const int j = multi_job(m, blockIdx.x);
  split_update_body<false>(m.job[j], blockIdx.x - m.blk_start[j]);
}

// ---------------------------------------------------------------- fitness
__device__ __forceinline__ void fitness_one(const EvalArgs& a, int b) {
  const TopoInfo inf = a.info[b];
  double lo = 0.0;
  float lc = 0.f, ml = 0.f;
  const float* pp = a.part + (size_t)b * a.n_parts * 4;
  for (int r = 0; r < a.n_parts; ++r) {
    lo += (double)pp[r * 4 + 0];
    lc += pp[r * 4 + 1];
    ml = fmaxf(ml, pp[r * 4 + 2]);
  }
  float fit;
  if (inf.island_base) {
    fit = -INFINITY;
  } else if (a.fitness_kind == TTO_FIT_F1) {
    fit = (float)(-(lo + 200.0 * inf.lambda_c0 + 50.0 * lc));
  } else if (a.fitness_kind == TTO_FIT_F2) {
    double lb = 0.0;
    for (int r = 0; r < a.n_rowtiles; ++r) lb += (double)a.bbpart[(size_t)b * a.n_rowtiles + r];
    fit = (float)(-(lo + 200.0 * inf.lambda_c0 + 50.0 * lc + fmax(lb - (double)*a.lbpre, 0.0)));
  } else {
    fit = (float)(-(lo + (double)ml));
  }
  a.fitness[b] = fit;
  const int cs = min(inf.ns, a.d_split - 1), cm = min(inf.nm, a.d_moved - 1), cd = min(inf.nd, a.d_disc - 1);
  if (a.desc) {
    a.desc[2 * b] = inf.ns;
    a.desc[2 * b + 1] = inf.nm;
  }
  if (a.cell) a.cell[b] = (cs * a.d_moved + cm) * a.d_disc + cd;
  if (a.island) a.island[b] = (uint8_t)((inf.island_base ? 1 : 0) | (inf.n_islanded > 0 ? 2 : 0));
  if (a.metrics) {
    float* m = a.metrics + (size_t)b * 4;
    m[0] = inf.island_base ? 0.f : (float)lo;
    m[1] = inf.island_base ? 0.f : ml;
    m[2] = inf.island_base ? 0.f : lc;
    m[3] = inf.lambda_c0;
  }
}

__global__ void fitness_kernel(EvalArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < a.B) fitness_one(a, b);
}

__global__ void fitness_multi_kernel(const __grid_constant__ MultiArgs m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.blk_start[m.n]) return;
  const int j = multi_job(m, i);
  fitness_one(m.job[j], i - m.blk_start[j]);
}

int launch_split_update_multi(const MultiArgs& m, cudaStream_t s) {
  if (m.blk_start[m.n] == 0) return TTO_OK;
  split_update_multi_kernel<<<m.blk_start[m.n], 256, 0, s>>>(m);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

int launch_fitness_multi(const MultiArgs& m, cudaStream_t s) {
  const int n = m.blk_start[m.n];
  if (n == 0) return TTO_OK;
  fitness_multi_kernel<<<(n + 127) / 128, 128, 0, s>>>(m);
  TTO_CUDA_TRY(cudaGetLastError());
  return TTO_OK;
}

// ---------------------------------------------------------------- workspace
void free_workspace(tto_grid* g) {
  Workspace& w = g->ws;
  void* ptrs[] = {w.U, w.V, w.Ua, w.Vb, w.gq, w.fp, w.gg, w.info, w.part, w.fit, w.cell, w.desc, w.island, w.topo};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  w = Workspace();
}

int ensure_workspace(tto_grid* g, int B, int T) {
  Workspace& w = g->ws;
  if (B <= w.cap_B && T <= w.cap_T) return TTO_OK;
  int nB = B > w.cap_B ? B : w.cap_B;
  int nT = T > w.cap_T ? T : w.cap_T;
  forget_grid_graphs(g);  // recorded graphs hold the old workspace addresses
  free_workspace(g);
  ++g->ws_epoch;
  const size_t Ep = g->E_mon_pad, Op = g->O_pad;
  TTO_CUDA_TRY(cudaMalloc(&w.U, (size_t)nB * Ep * 8 * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&w.V, (size_t)nB * Op * 8 * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&w.Ua, (size_t)nB * Ep * 16 * sizeof(uint32_t)));
  TTO_CUDA_TRY(cudaMalloc(&w.Vb, (size_t)nB * Op * 16 * sizeof(uint32_t)));
  TTO_CUDA_TRY(cudaMalloc(&w.gq, (size_t)nB * Op * nT * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&w.fp, (size_t)nB * nT * Ep * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&w.gg, (size_t)nB * Op * nT * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&w.info, (size_t)nB * sizeof(TopoInfo)));
  TTO_CUDA_TRY(cudaMalloc(&w.part, (size_t)nB * max_parts(g) * 4 * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&w.fit, (size_t)nB * sizeof(float)));
  TTO_CUDA_TRY(cudaMalloc(&w.cell, (size_t)nB * sizeof(int32_t)));
  TTO_CUDA_TRY(cudaMalloc(&w.desc, (size_t)nB * 2 * sizeof(int32_t)));
  TTO_CUDA_TRY(cudaMalloc(&w.island, (size_t)nB * sizeof(uint8_t)));
  TTO_CUDA_TRY(cudaMalloc(&w.topo, (size_t)nB * g->gw * sizeof(int32_t)));
  w.cap_B = nB;
  w.cap_T = nT;
  return TTO_OK;
}

int padded_T(int n_t) {
  const int opts[] = {1, 2, 4, 8, 16, 24, 32};
  for (int v : opts)
    if (n_t <= v) return v;
  return -1;
}

static int padded_K(int k) { return k <= 2 ? 2 : (k <= 4 ? 4 : 8); }

int evaluate_impl(tto_grid* g, const int32_t* topo, int B, const int32_t* tsel, int n_t,
                  const tto_eval_opts* o, float* fitness, int32_t* desc, int32_t* cell,
                  uint8_t* island, float* metrics, float* fmax, cudaStream_t s, EvalArgs* split_only,
                  bool busbar_setup, bool prepare_only) {
  if (!g || !o) return set_error(TTO_E_ARG, "null argument");
  if (B < 0) return set_error(TTO_E_ARG, "negative batch");
  if (B > 0 && (!topo || !fitness)) return set_error(TTO_E_ARG, "null topology or fitness buffer");
  if (o->d_split < 1 || o->d_moved < 1 || o->d_disc < 0) return set_error(TTO_E_ARG, "archive extents must be >= 1");
  if (o->precision < TTO_PREC_FP32 || o->precision > TTO_PREC_FP16X3) return set_error(TTO_E_ARG, "unknown precision");
  if (o->fitness_kind != TTO_FIT_WORKLOAD && o->fitness_kind != TTO_FIT_F1 && o->fitness_kind != TTO_FIT_F2)
    return set_error(TTO_E_ARG, "unknown fitness kind");
  if (n_t < 0 || n_t > TTO_MAX_T || (tsel == nullptr && g->T > TTO_MAX_T))
    return set_error(TTO_E_ARG, "n_t must be in [1, %d]", TTO_MAX_T);
  EvalArgs a;
  memset(&a, 0, sizeof(a));
  if (tsel == nullptr) {
    n_t = g->T;
    for (int t = 0; t < n_t; ++t) a.tsel[t] = t;
  } else {
    if (n_t < 1) return set_error(TTO_E_ARG, "n_t must be >= 1");
    for (int t = 0; t < n_t; ++t) {
      if (tsel[t] < 0 || tsel[t] >= g->T) return set_error(TTO_E_ARG, "timestep %d out of range", tsel[t]);
      a.tsel[t] = tsel[t];
    }
  }
  if (B == 0) return TTO_OK;
  const int TT = padded_T(n_t);
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  const bool bb = busbar_setup || o->fitness_kind == TTO_FIT_F2;
  if (o->fitness_kind == TTO_FIT_F2 && !busbar_setup) {
    bool same = g->d_lbpre && g->lbpre_nt == n_t;
    for (int t = 0; same && t < n_t; ++t) same = g->lbpre_tsel[t] == a.tsel[t];
    if (!same)
      return set_error(TTO_E_ARG, "lambda_f2 needs tto_grid_busbar_reference for these timesteps and limits first");
  }
  int rc = ensure_workspace(g, B, TT);
  if (rc) return rc;
  if (bb) {
    if (g->S < 1) return set_error(TTO_E_ARG, "the grid has no stations, so no busbar outages");
    rc = ensure_busbar(g, B, TT, s);
    if (rc) return rc;
  }
  Workspace& w = g->ws;
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
  a.KP = padded_K(g->gw);
  a.d_split = o->d_split;
  a.d_moved = o->d_moved;
  a.d_disc = o->d_disc > 1 ? o->d_disc : 1;
  a.topo = topo;
  a.B = B;
  a.U = w.U;
  a.V = w.V;
  a.fp = w.fp;
  a.gg = w.gg;
  a.Ua = w.Ua;
  a.Vb = w.Vb;
  a.gq = w.gq;
  a.info = w.info;
  a.part = w.part;
  a.fitness = fitness;
  a.desc = desc;
  a.cell = cell;
  a.island = island;
  a.metrics = metrics;
  a.fmax = fmax;
  a.fitness_kind = o->fitness_kind;
  a.n_rowtiles = g->n_rowtiles;
  a.n_parts = g->n_rowtiles;
  a.precision = o->precision;
  a.shape = g->tuned_shape[o->precision] >= 0 ? g->tuned_shape[o->precision] : 0;
  // the tcgen05 sweep follows: the split update writes its operand layouts
  // directly (no plain V, g; plain U only for the busbar sweep), with its
  // timestep passes of at most 4
  a.umma_packed = (!split_only && a.precision == TTO_PREC_TF32X3 && a.shape == kUmmaShape) ? 1 : 0;
  if (a.umma_packed) {
    a.TC = TT < 4 ? TT : 4;
    a.n_tch = TT / a.TC;
  }
  a.from = g->d_from;
  if (bb) fill_busbar_args(g, a);
  if (prepare_only) {  // arguments only: the caller launches (mixed-grid batches)
    *split_only = a;
    return TTO_OK;
  }
  cudaEvent_t* ev = nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TTO_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (g->prof_on && !split_only && g->prof_n < kProfileCalls && cap == cudaStreamCaptureStatusNone)
    ev = &g->prof_ev[kProfileEvents * g->prof_n++];
  if (ev) TTO_CUDA_TRY(cudaEventRecord(ev[0], s));
  if (bb) {
    split_update_bb_kernel<<<B, 256, 0, s>>>(a);
    TTO_CUDA_TRY(cudaGetLastError());
    const size_t n = (size_t)B * a.NB;
    busbar_setup_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
  } else {
    split_update_kernel<<<B, 256, 0, s>>>(a);
  }
  TTO_CUDA_TRY(cudaGetLastError());
  if (split_only) {
    *split_only = a;
    return TTO_OK;
  }
  if (ev) TTO_CUDA_TRY(cudaEventRecord(ev[1], s));
  if (a.precision != TTO_PREC_FP32) {
    rc = ensure_fragment_N(g, s);
    if (rc) return rc;
    a.Nf = g->d_Nf;
  }
  rc = launch_sweep(a, s);
  if (rc) return rc;
  if (ev) TTO_CUDA_TRY(cudaEventRecord(ev[2], s));
  if (bb) {
    rc = launch_busbar_sweep(a, s);
    if (rc) return rc;
  }
  if (ev) TTO_CUDA_TRY(cudaEventRecord(ev[3], s));
  fitness_kernel<<<(B + 127) / 128, 128, 0, s>>>(a);
  TTO_CUDA_TRY(cudaGetLastError());
  if (ev) TTO_CUDA_TRY(cudaEventRecord(ev[4], s));
  return TTO_OK;
}

}  // namespace tto

extern "C" {

int tto_grid_reserve(tto_grid* g, int32_t max_batch, int32_t n_t) {
  if (!g || max_batch < 1 || n_t < 1 || n_t > TTO_MAX_T) return tto::set_error(TTO_E_ARG, "bad reserve arguments");
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  return tto::ensure_workspace(g, max_batch, tto::padded_T(n_t));
}

int tto_evaluate_batch(tto_grid* g, const int32_t* topo, int32_t B, const int32_t* timesteps,
                       int32_t n_t, const tto_eval_opts* opts, float* fitness, int32_t* desc,
                       int32_t* cell, uint8_t* island, float* metrics, float* fmax, void* stream) {
  return tto::evaluate_impl(g, topo, B, timesteps, n_t, opts, fitness, desc, cell, island, metrics,
                            fmax, (cudaStream_t)stream);
}

int tto_grid_profile(tto_grid* g, int32_t enable) {
  if (!g) return tto::set_error(TTO_E_ARG, "null grid");
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  if (enable && g->prof_ev.empty()) {
    g->prof_ev.resize(tto::kProfileEvents * tto::kProfileCalls);
    for (auto& e : g->prof_ev) TTO_CUDA_TRY(cudaEventCreate(&e));
  }
  g->prof_on = enable ? 1 : 0;
  if (enable) g->prof_n = 0;
  return TTO_OK;
}

int tto_grid_profile_read(tto_grid* g, float* ms_stage, int32_t* n_calls) {
  if (!g || !ms_stage) return tto::set_error(TTO_E_ARG, "null argument");
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  // events per call: start, split update done, N-1 sweep done, busbar sweep
  // done (no busbar sweep: right after the previous one), reduction done
  static const int kFrom[4] = {0, 1, 3, 2}, kTo[4] = {1, 2, 4, 3};
  for (int q = 0; q < 4; ++q) ms_stage[q] = 0.f;
  for (int c = 0; c < g->prof_n; ++c) {
    const cudaEvent_t* ev = &g->prof_ev[tto::kProfileEvents * c];
    TTO_CUDA_TRY(cudaEventSynchronize(ev[tto::kProfileEvents - 1]));
    for (int q = 0; q < 4; ++q) {
      float ms = 0.f;
      TTO_CUDA_TRY(cudaEventElapsedTime(&ms, ev[kFrom[q]], ev[kTo[q]]));
      ms_stage[q] += ms;
    }
  }
  if (n_calls) *n_calls = g->prof_n;
  return TTO_OK;
}

int tto_debug_bounded_wait(tto_grid* g, int64_t cycles, void* stream) {
  if (!g || cycles < 1 || cycles > (int64_t)1 << 32) return tto::set_error(TTO_E_ARG, "cycles must be in [1, 2^32]");
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  return tto::bounded_wait_probe(g->d_status, (long long)cycles, (cudaStream_t)stream);
}

int tto_grid_sync_status(tto_grid* g, void* stream) {
  if (!g) return tto::set_error(TTO_E_ARG, "null grid");
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  TTO_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int st = 0;
  TTO_CUDA_TRY(cudaMemcpy(&st, g->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  int zero = 0;
  TTO_CUDA_TRY(cudaMemcpy(g->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice));
  if (st == TTO_E_TOPOLOGY) return tto::set_error(TTO_E_TOPOLOGY, "a genome named an unknown action or split a station twice");
  if (st == TTO_E_TIMEOUT) return tto::set_error(TTO_E_TIMEOUT, "a bounded device wait gave up");
  return st;
}

}  // extern "C"
