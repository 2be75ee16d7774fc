// Grid creation: input checks, one-time FP64 precompute and device upload.
//
// The reduced susceptance matrix B_r = A_r^T D A_r (slack row/column removed)
// is factorised once as L D L^T with a minimum-degree elimination order.  Each
// needed flow-response column is then one pair of sparse triangular solves:
//   M[:, c] = D A X (e_from(c) - e_to(c)),   N[:, c] = e_c - M[:, c],
// i.e. the PTDF of the pre-optimisation topology applied to a unit transfer
// across branch c (Sec. "Importer": PTDF precompute; Sec. "DC-Optimizer":
// low-rank updates built on it).  Columns are needed for every outage (the N-1
// sweep reads N[monitored][outage] in FP32 and N_cc in FP64) and for every
// branch a split can move (the split update reads those columns in FP64).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <set>
#include <thread>
#include <utility>

#include "tto_internal.h"

namespace tto {

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  return set_error(e == cudaErrorMemoryAllocation ? TTO_E_NOMEM : TTO_E_CUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

namespace {

// Symmetric sparse matrix factorised by Gaussian elimination on its graph,
// always eliminating a node of minimum current degree.
struct SparseLDL {
  int n = 0;
  std::vector<int> order;      // order[k] = node eliminated at step k
  std::vector<double> piv;     // pivot of step k
  std::vector<int> colptr;     // L column k: entries [colptr[k], colptr[k+1])
  std::vector<int> rowidx;     // node index of each entry
  std::vector<double> val;     // multiplier l_uv

  bool factor(int nn, std::vector<std::vector<std::pair<int, double>>> adj,
              std::vector<double> dg) {
    n = nn;
    order.clear();
    piv.clear();
    colptr.assign(1, 0);
    rowidx.clear();
    val.clear();
    std::vector<int> pos(n, -1);
    std::set<std::pair<int, int>> pq;
    for (int v = 0; v < n; ++v) pq.insert({(int)adj[v].size(), v});
    std::vector<double> scale(dg);
    for (int k = 0; k < n; ++k) {
      int v = pq.begin()->second;
      pq.erase(pq.begin());
      double dv = dg[v];
      if (!(dv > 1e-13 * scale[v])) return false;
      std::vector<std::pair<int, double>> nb;
      nb.swap(adj[v]);
      order.push_back(v);
      piv.push_back(dv);
      for (auto& e : nb) {
        rowidx.push_back(e.first);
        val.push_back(e.second / dv);
      }
      colptr.push_back((int)rowidx.size());
      for (auto& eu : nb) {
        int u = eu.first;
        double auv = eu.second;
        auto& au = adj[u];
        pq.erase({(int)au.size(), u});
        for (size_t i = 0; i < au.size(); ++i) {
          if (au[i].first == v) {
            au[i] = au.back();
            au.pop_back();
            break;
          }
        }
        for (size_t i = 0; i < au.size(); ++i) pos[au[i].first] = (int)i;
        for (auto& ew : nb) {
          int w = ew.first;
          if (w == u) continue;
          double delta = -auv * ew.second / dv;
          if (pos[w] >= 0) {
            au[pos[w]].second += delta;
          } else {
            pos[w] = (int)au.size();
            au.push_back({w, delta});
          }
        }
        for (size_t i = 0; i < au.size(); ++i) pos[au[i].first] = -1;
        dg[u] -= auv * auv / dv;
        pq.insert({(int)au.size(), u});
      }
    }
    return true;
  }

  // x <- (L D L^T)^{-1} x, x indexed by node.
  void solve(double* x) const {
    for (int k = 0; k < n; ++k) {
      double xv = x[order[k]];
      if (xv == 0.0) continue;
      for (int q = colptr[k]; q < colptr[k + 1]; ++q) x[rowidx[q]] -= val[q] * xv;
    }
    for (int k = 0; k < n; ++k) x[order[k]] /= piv[k];
    for (int k = n - 1; k >= 0; --k) {
      double s = x[order[k]];
      for (int q = colptr[k]; q < colptr[k + 1]; ++q) s -= val[q] * x[rowidx[q]];
      x[order[k]] = s;
    }
  }
};

int find_root(std::vector<int>& p, int x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

template <class T>
int upload(T** dst, const T* src, size_t n) {
  if (n == 0) n = 1;
  TTO_CUDA_TRY(cudaMalloc((void**)dst, n * sizeof(T)));
  if (src) TTO_CUDA_TRY(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return TTO_OK;
}

int validate(const tto_grid_desc* d) {
  if (!d) return set_error(TTO_E_ARG, "null descriptor");
  if (d->n_bus < 2 || d->n_branch < 1) return set_error(TTO_E_ARG, "need >= 2 buses and >= 1 branch");
  if (!d->from || !d->to || !d->b || !d->p || !d->limit)
    return set_error(TTO_E_ARG, "null branch/injection/limit array");
  if (d->slack < 0 || d->slack >= d->n_bus) return set_error(TTO_E_ARG, "slack out of range");
  if (d->n_time < 1) return set_error(TTO_E_ARG, "n_time must be >= 1");
  if (d->k_max < 1 || d->k_max > TTO_MAX_K) return set_error(TTO_E_ARG, "k_max must be in [1, %d]", TTO_MAX_K);
  if (d->n_dslot < 0 || d->k_max + d->n_dslot > TTO_MAX_K)
    return set_error(TTO_E_ARG, "k_max + n_dslot must be <= %d (n_dslot >= 0)", TTO_MAX_K);
  if (d->n_disc < 0 || (d->n_disc > 0 && !d->disc_branch)) return set_error(TTO_E_ARG, "bad disconnection set");
  for (int l = 0; l < d->n_branch; ++l) {
    int f = d->from[l], t = d->to[l];
    if (f < 0 || f >= d->n_bus || t < 0 || t >= d->n_bus || f == t)
      return set_error(TTO_E_ARG, "branch %d has invalid ends (%d, %d)", l, f, t);
    if (!(d->b[l] > 0.0) || !isfinite(d->b[l])) return set_error(TTO_E_ARG, "branch %d susceptance must be > 0", l);
    if (!(d->limit[l] > 0.0) || !isfinite(d->limit[l])) return set_error(TTO_E_ARG, "branch %d limit must be > 0", l);
  }
  for (size_t i = 0; i < (size_t)d->n_time * d->n_bus; ++i)
    if (!isfinite(d->p[i])) return set_error(TTO_E_ARG, "non-finite injection");
  if (d->n_monitored < 1 || !d->monitored) return set_error(TTO_E_ARG, "need monitored branches");
  if (d->n_outage < 1 || !d->outage) return set_error(TTO_E_ARG, "need outages");
  std::vector<char> seen(d->n_branch, 0);
  for (int i = 0; i < d->n_monitored; ++i) {
    int l = d->monitored[i];
    if (l < 0 || l >= d->n_branch || seen[l]) return set_error(TTO_E_ARG, "monitored id %d invalid or repeated", l);
    seen[l] = 1;
  }
  std::fill(seen.begin(), seen.end(), 0);
  for (int i = 0; i < d->n_disc; ++i) {
    int l = d->disc_branch[i];
    if (l < 0 || l >= d->n_branch || seen[l]) return set_error(TTO_E_ARG, "disconnection id %d invalid or repeated", l);
    seen[l] = 1;
  }
  std::fill(seen.begin(), seen.end(), 0);
  for (int i = 0; i < d->n_outage; ++i) {
    int l = d->outage[i];
    if (l < 0 || l >= d->n_branch || seen[l]) return set_error(TTO_E_ARG, "outage id %d invalid or repeated", l);
    seen[l] = 1;
  }
  if (d->n_station < 0) return set_error(TTO_E_ARG, "negative station count");
  if (d->n_station > 0 && (!d->station_bus || !d->asset_offset || !d->asset_branch))
    return set_error(TTO_E_ARG, "null station arrays");
  std::vector<char> busseen(d->n_bus, 0);
  if (d->n_station > 0 && d->asset_offset[0] != 0) return set_error(TTO_E_ARG, "asset_offset[0] must be 0");
  for (int s = 0; s < d->n_station; ++s) {
    int bus = d->station_bus[s];
    if (bus < 0 || bus >= d->n_bus || busseen[bus]) return set_error(TTO_E_ARG, "station %d bus invalid or repeated", s);
    if (bus == d->slack) return set_error(TTO_E_ARG, "station %d sits at the slack bus", s);
    busseen[bus] = 1;
    int a0 = d->asset_offset[s], a1 = d->asset_offset[s + 1];
    if (a1 - a0 < 2 || a1 - a0 > TTO_MAX_ASSETS) return set_error(TTO_E_ARG, "station %d needs 2..%d assets", s, TTO_MAX_ASSETS);
    int ninj = 0;
    for (int i = a0; i < a1; ++i) {
      int e = d->asset_branch[i];
      if (e == -1) {
        ++ninj;
        continue;
      }
      if (e < 0 || e >= d->n_branch || (d->from[e] != bus && d->to[e] != bus))
        return set_error(TTO_E_ARG, "station %d asset %d is not a branch at its bus", s, e);
      for (int j = a0; j < i; ++j)
        if (d->asset_branch[j] == e) return set_error(TTO_E_ARG, "station %d repeats asset %d", s, e);
    }
    if (ninj > 1) return set_error(TTO_E_ARG, "station %d has more than one injection asset", s);
  }
  if (d->n_action < 0 || (d->n_action > 0 && (!d->action_station || !d->action_mask)))
    return set_error(TTO_E_ARG, "bad action arrays");
  for (int a = 0; a < d->n_action; ++a) {
    int s = d->action_station[a];
    if (s < 0 || s >= d->n_station) return set_error(TTO_E_ARG, "action %d names station %d", a, s);
    if (a > 0 && s < d->action_station[a - 1]) return set_error(TTO_E_ARG, "actions must be grouped by ascending station");
    int a0 = d->asset_offset[s], m = d->asset_offset[s + 1] - a0;
    uint32_t mask = d->action_mask[a];
    if ((mask & 1u) || (mask >> m) != 0 || mask == 0)
      return set_error(TTO_E_ARG, "action %d mask 0x%x invalid for %d assets", a, mask, m);
    bool bb = false, ab = false;
    for (int i = 0; i < m; ++i) {
      bool on_b = (mask >> i) & 1u;
      if (d->asset_branch[a0 + i] >= 0) (on_b ? bb : ab) = true;
    }
    if (!bb || !ab) return set_error(TTO_E_ARG, "action %d leaves a busbar without a branch", a);
  }
  return TTO_OK;
}

}  // namespace

static int build_grid(const tto_grid_desc* d, tto_grid* g) {
  g->device = d->device;
  g->n_bus = d->n_bus;
  g->E = d->n_branch;
  g->slack = d->slack;
  g->T = d->n_time;
  g->E_mon = d->n_monitored;
  g->O = d->n_outage;
  g->S = d->n_station;
  g->A = d->n_action;
  g->k_max = d->k_max;
  g->n_disc = d->n_disc;
  g->n_dslot = d->n_dslot;
  g->gw = d->k_max + d->n_dslot;
  if (g->n_disc > 0) g->disc.assign(d->disc_branch, d->disc_branch + g->n_disc);
  g->E_mon_pad = (g->E_mon + kRowTile - 1) / kRowTile * kRowTile;
  g->O_pad = (g->O + kColPad - 1) / kColPad * kColPad;
  g->n_rowtiles = g->E_mon_pad / kRowTile;
  const int E = g->E, n = g->n_bus, T = g->T;
  g->from.assign(d->from, d->from + E);
  g->to.assign(d->to, d->to + E);
  g->b.assign(d->b, d->b + E);
  g->p.assign(d->p, d->p + (size_t)T * n);
  g->limit.assign(d->limit, d->limit + E);
  g->mon.assign(d->monitored, d->monitored + g->E_mon);
  g->out.assign(d->outage, d->outage + g->O);
  if (g->S > 0) {
    g->station_bus.assign(d->station_bus, d->station_bus + g->S);
    g->asset_off.assign(d->asset_offset, d->asset_offset + g->S + 1);
    g->asset_br.assign(d->asset_branch, d->asset_branch + g->asset_off[g->S]);
  } else {
    g->asset_off.assign(1, 0);
  }
  g->act_st.assign(d->action_station, d->action_station + g->A);
  g->act_mask.assign(d->action_mask, d->action_mask + g->A);
  g->act_off.assign(g->S + 1, 0);
  for (int a = 0; a < g->A; ++a) g->act_off[g->act_st[a] + 1]++;
  for (int s = 0; s < g->S; ++s) g->act_off[s + 1] += g->act_off[s];

  // connectivity of the unsplit grid
  {
    std::vector<int> par(n);
    for (int i = 0; i < n; ++i) par[i] = i;
    int comps = n;
    for (int l = 0; l < E; ++l) {
      int a = find_root(par, g->from[l]), c = find_root(par, g->to[l]);
      if (a != c) {
        par[c] = a;
        --comps;
      }
    }
    if (comps != 1) return set_error(TTO_E_DISCONNECTED, "the unsplit grid has %d components", comps);
  }

  // reduced susceptance matrix in graph form (slack removed)
  auto red = [&](int bus) { return bus < g->slack ? bus : bus - 1; };
  const int nr = n - 1;
  std::vector<std::vector<std::pair<int, double>>> adj(nr);
  std::vector<double> dg(nr, 0.0);
  for (int l = 0; l < E; ++l) {
    int f = g->from[l], t = g->to[l];
    double bl = g->b[l];
    if (f != g->slack) dg[red(f)] += bl;
    if (t != g->slack) dg[red(t)] += bl;
    if (f != g->slack && t != g->slack) {
      int rf = red(f), rt = red(t);
      bool merged = false;
      for (auto& e : adj[rf])
        if (e.first == rt) {
          e.second -= bl;
          merged = true;
        }
      if (merged) {
        for (auto& e : adj[rt])
          if (e.first == rf) e.second -= bl;
      } else {
        adj[rf].push_back({rt, -bl});
        adj[rt].push_back({rf, -bl});
      }
    }
  }
  SparseLDL ldl;
  if (!ldl.factor(nr, adj, dg)) return set_error(TTO_E_DISCONNECTED, "reduced susceptance matrix is singular");

  // columns needed: outages and the branches a split can move or a genome open
  std::vector<int> swcol(E, -1);
  std::vector<int> swlist;
  for (int s = 0; s < g->S; ++s)
    for (int i = g->asset_off[s]; i < g->asset_off[s + 1]; ++i) {
      int e = g->asset_br[i];
      if (e >= 0 && swcol[e] < 0) {
        swcol[e] = (int)swlist.size();
        swlist.push_back(e);
      }
    }
  for (int e : g->disc)
    if (swcol[e] < 0) {
      swcol[e] = (int)swlist.size();
      swlist.push_back(e);
    }
  g->n_sw = (int)swlist.size();
  std::vector<int> outpos(E, -1);
  for (int c = 0; c < g->O; ++c) outpos[g->out[c]] = c;
  std::vector<int> need;
  for (int e = 0; e < E; ++e)
    if (outpos[e] >= 0 || swcol[e] >= 0) need.push_back(e);

  const int Ep = g->E_mon_pad, Op = g->O_pad;
  std::vector<float> Nmo((size_t)Ep * Op);
  std::vector<double> Nsw((size_t)std::max(g->n_sw, 1) * E);
  std::vector<double> Ncc(g->O);
  g->f0.assign((size_t)T * E, 0.0);
  // injection responses of the station buses (busbar outages): flows for +1
  // at the station bus, withdrawn at the slack
  std::vector<double> Pst((size_t)std::max(g->S, 1) * E, 0.0);

  unsigned nthreads = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::atomic<int> next(0);
  const int njobs = (int)need.size() + T + g->S;
  auto worker = [&]() {
    std::vector<double> x(nr), col(E);
    for (;;) {
      int job = next.fetch_add(1);
      if (job >= njobs) break;
      std::fill(x.begin(), x.end(), 0.0);
      int c = -1;
      if (job < (int)need.size()) {
        c = need[job];
        if (g->from[c] != g->slack) x[red(g->from[c])] += 1.0;
        if (g->to[c] != g->slack) x[red(g->to[c])] -= 1.0;
      } else if (job < (int)need.size() + T) {
        int t = job - (int)need.size();
        for (int i = 0; i < n; ++i)
          if (i != g->slack) x[red(i)] = g->p[(size_t)t * n + i];
      } else {
        x[red(g->station_bus[job - (int)need.size() - T])] = 1.0;  // stations never sit at the slack
      }
      ldl.solve(x.data());
      for (int l = 0; l < E; ++l) {
        int f = g->from[l], t = g->to[l];
        double tf = f == g->slack ? 0.0 : x[red(f)];
        double tt = t == g->slack ? 0.0 : x[red(t)];
        col[l] = g->b[l] * (tf - tt);
      }
      if (c < 0) {
        int t = job - (int)need.size();
        if (t < T) std::copy(col.begin(), col.end(), g->f0.begin() + (size_t)t * E);
        else std::copy(col.begin(), col.end(), Pst.begin() + (size_t)(t - T) * E);
        continue;
      }
      // col = M[:, c]; N[:, c] = e_c - M[:, c]
      for (int l = 0; l < E; ++l) col[l] = (l == c ? 1.0 : 0.0) - col[l];
      if (swcol[c] >= 0) std::copy(col.begin(), col.end(), Nsw.begin() + (size_t)swcol[c] * E);
      int oc = outpos[c];
      if (oc >= 0) {
        Ncc[oc] = col[c];
        int cend = (oc == g->O - 1) ? Op : oc + 1;  // last outage fills the padded columns
        for (int cc = oc; cc < cend; ++cc) {
          for (int l = 0; l < g->E_mon; ++l) Nmo[(size_t)l * Op + cc] = (float)col[g->mon[l]];
          for (int l = g->E_mon; l < Ep; ++l) Nmo[(size_t)l * Op + cc] = (float)col[g->mon[g->E_mon - 1]];
        }
      }
    }
  };
  std::vector<std::thread> pool;
  for (unsigned i = 0; i < nthreads; ++i) pool.emplace_back(worker);
  for (auto& th : pool) th.join();

  // device copies
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  int rc;
  if ((rc = upload(&g->d_Nmo, Nmo.data(), Nmo.size()))) return rc;
  if ((rc = upload(&g->d_Nsw, Nsw.data(), Nsw.size()))) return rc;
  {
    std::vector<float> Nsw32(Nsw.size());
    for (size_t i = 0; i < Nsw.size(); ++i) Nsw32[i] = (float)Nsw[i];
    if ((rc = upload(&g->d_Nsw32, Nsw32.data(), Nsw32.size()))) return rc;
  }
  if ((rc = upload(&g->d_swcol, swcol.data(), swcol.size()))) return rc;
  if ((rc = upload(&g->d_Pst, Pst.data(), Pst.size()))) return rc;
  {
    std::vector<float> Pm((size_t)std::max(g->S, 1) * g->E_mon_pad, 0.f);
    for (int s = 0; s < g->S; ++s)
      for (int l = 0; l < g->E_mon; ++l) Pm[(size_t)s * g->E_mon_pad + l] = (float)Pst[(size_t)s * E + g->mon[l]];
    if ((rc = upload(&g->d_Pm, Pm.data(), Pm.size()))) return rc;
  }
  g->swlist = swlist;
  if ((rc = upload(&g->d_f0, g->f0.data(), g->f0.size()))) return rc;
  if ((rc = upload(&g->d_p, g->p.data(), g->p.size()))) return rc;
  if ((rc = upload(&g->d_b, g->b.data(), g->b.size()))) return rc;
  {
    std::vector<double> invb(g->b.size());
    for (size_t e = 0; e < invb.size(); ++e) invb[e] = 1.0 / g->b[e];
    if ((rc = upload(&g->d_invb, invb.data(), invb.size()))) return rc;
  }
  std::vector<float> lim(g->E_mon);
  for (int l = 0; l < g->E_mon; ++l) lim[l] = (float)g->limit[g->mon[l]];
  if ((rc = upload(&g->d_lim, lim.data(), lim.size()))) return rc;
  if ((rc = upload(&g->d_mon, g->mon.data(), g->mon.size()))) return rc;
  if ((rc = upload(&g->d_out, g->out.data(), g->out.size()))) return rc;
  if ((rc = upload(&g->d_Ncc, Ncc.data(), Ncc.size()))) return rc;
  if ((rc = upload(&g->d_from, g->from.data(), g->from.size()))) return rc;
  if ((rc = upload(&g->d_station_bus, g->station_bus.data(), g->station_bus.size()))) return rc;
  if ((rc = upload(&g->d_asset_off, g->asset_off.data(), g->asset_off.size()))) return rc;
  if ((rc = upload(&g->d_asset_br, g->asset_br.data(), g->asset_br.size()))) return rc;
  if ((rc = upload(&g->d_act_st, g->act_st.data(), g->act_st.size()))) return rc;
  if ((rc = upload(&g->d_act_off, g->act_off.data(), g->act_off.size()))) return rc;
  if ((rc = upload(&g->d_act_mask, g->act_mask.data(), g->act_mask.size()))) return rc;
  if ((rc = upload(&g->d_disc, g->disc.empty() ? nullptr : g->disc.data(), g->disc.size()))) return rc;
  int zero = 0;
  if ((rc = upload(&g->d_status, &zero, 1))) return rc;
  return TTO_OK;
}

static void release(tto_grid* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  forget_grid_graphs(g);
  free_workspace(g);
  void* ptrs[] = {g->d_from, g->d_Nf, g->d_Nmo, g->d_Nsw, g->d_Nsw32, g->d_swcol, g->d_Pst, g->d_Pm, g->d_Nswm,
                  g->d_lbpre, g->d_empty, g->d_bbrec, g->d_bbpart, g->d_bbstate, g->d_f0, g->d_p, g->d_b, g->d_invb, g->d_lim,
                  g->d_mon, g->d_out, g->d_Ncc, g->d_station_bus, g->d_asset_off,
                  g->d_asset_br, g->d_act_st, g->d_act_off, g->d_act_mask, g->d_disc, g->d_status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& e : g->prof_ev) cudaEventDestroy(e);
  delete g;
}

}  // namespace tto

extern "C" {

const char* tto_last_error(void) { return tto::g_err.c_str(); }

int tto_grid_create(const tto_grid_desc* d, tto_grid** out) {
  if (!out) return tto::set_error(TTO_E_ARG, "null output pointer");
  *out = nullptr;
  int rc = tto::validate(d);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0)
    return tto::set_error(TTO_E_CUDA, "no CUDA device");
  if (d->device < 0 || d->device >= ndev) return tto::set_error(TTO_E_ARG, "device %d out of range", d->device);
  tto_grid* g = new (std::nothrow) tto_grid();
  if (!g) return tto::set_error(TTO_E_NOMEM, "host allocation failed");
  static std::atomic<uint64_t> next_uid(1);
  g->uid = next_uid.fetch_add(1);
  try {
    rc = tto::build_grid(d, g);
  } catch (const std::bad_alloc&) {
    rc = tto::set_error(TTO_E_NOMEM, "host allocation failed");
  }
  if (rc) {
    tto::release(g);
    return rc;
  }
  *out = g;
  return TTO_OK;
}

int tto_grid_destroy(tto_grid* g) {
  tto::release(g);
  return TTO_OK;
}

int tto_grid_info(const tto_grid* g, int32_t* n_branch, int32_t* n_monitored, int32_t* n_outage,
                  int32_t* n_time, int32_t* k_max, int32_t* n_action) {
  if (!g) return tto::set_error(TTO_E_ARG, "null grid");
  if (n_branch) *n_branch = g->E;
  if (n_monitored) *n_monitored = g->E_mon;
  if (n_outage) *n_outage = g->O;
  if (n_time) *n_time = g->T;
  if (k_max) *k_max = g->k_max;
  if (n_action) *n_action = g->A;
  return TTO_OK;
}

int tto_grid_disc_info(const tto_grid* g, int32_t* n_disc, int32_t* n_dslot) {
  if (!g) return tto::set_error(TTO_E_ARG, "null grid");
  if (n_disc) *n_disc = g->n_disc;
  if (n_dslot) *n_dslot = g->n_dslot;
  return TTO_OK;
}

int tto_grid_base_flows(const tto_grid* g, double* f0_host) {
  if (!g || !f0_host) return tto::set_error(TTO_E_ARG, "null argument");
  memcpy(f0_host, g->f0.data(), g->f0.size() * sizeof(double));
  return TTO_OK;
}

int tto_grid_set_limits(tto_grid* g, const double* limit_host) {
  if (!g || !limit_host) return tto::set_error(TTO_E_ARG, "null argument");
  for (int l = 0; l < g->E; ++l)
    if (!(limit_host[l] > 0.0) || !isfinite(limit_host[l])) return tto::set_error(TTO_E_ARG, "limit %d must be > 0", l);
  g->limit.assign(limit_host, limit_host + g->E);
  std::vector<float> lim(g->E_mon);
  for (int l = 0; l < g->E_mon; ++l) lim[l] = (float)g->limit[g->mon[l]];
  TTO_CUDA_TRY(cudaSetDevice(g->device));
  TTO_CUDA_TRY(cudaMemcpy(g->d_lim, lim.data(), lim.size() * sizeof(float), cudaMemcpyHostToDevice));
  g->lbpre_nt = 0;  // lambda_b of the unsplit topology depends on the limits: recompute it
  return TTO_OK;
}

}  // extern "C"
