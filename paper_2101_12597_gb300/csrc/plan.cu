// Work plans of the mixed path's grid stages: per-system argument blocks in
// device memory and, per CTA, the list of jobs it runs (host code).
#include <algorithm>
#include <numeric>
#include <queue>
#include <vector>

#include "host.h"
#include "internal.h"

namespace etdm {

namespace {

// density jobs of one tile: its orbital chunks of 128, consecutive
void push_tile(std::vector<TcJob> &out, const etdm_handle *h, int s, int t, int nmc) {
  const int k0 = h->h_xr_off[t], nk = h->h_xr_off[t + 1] - k0;
  const int muo = h->h_mu_off[t], nu = h->h_mu_off[t + 1] - muo;
  for (int mc = 0; mc < nmc; ++mc)
    out.push_back(TcJob{make_int4(s, t, mc, nmc), make_int4(k0, nk, nu, muo)});
}

int chunks(const etdm_handle *h) { return (h->N + tc_max_list() - 1) / tc_max_list(); }

}  // namespace

void build_mixed_plan(etdm_handle *owner, const std::vector<etdm_handle *> &subs,
                      const int *d_active, int *d_flags, bool batch,
                      unsigned long long *vfix, size_t vfix_bytes, MixedPlan *P) {
  const int ns = (int)subs.size();
  const int sms = owner->num_sms;
  P->n_sys = ns;
  P->active = d_active;

  // per-system arguments
  std::vector<TcArgs> tc(ns);
  std::vector<DfArgs> df(ns);
  std::vector<OsArgs> os(ns);
  std::vector<VfArgs> vf(ns);
  long maxMM = 1, sumN = 0;
  for (auto *h : subs) sumN += h->N;
  P->omax = dalloc<unsigned long long>(owner, std::max<long>(sumN, 1));
  P->omax_bytes = (size_t)std::max<long>(sumN, 1) * sizeof(unsigned long long);
  for (int i = 0, off = 0; i < ns; ++i) {
    tc[i] = tc_args(subs[i]);
    df[i] = df_args(subs[i]);
    os[i] = os_args(subs[i]);
    os[i].omax = P->omax + off;
    off += subs[i]->N;
    vf[i] = vf_args(subs[i]);
    P->os_maxN = std::max(P->os_maxN, subs[i]->N);
    P->os_maxMN = std::max(P->os_maxMN, (long)subs[i]->M * subs[i]->N);
    maxMM = std::max(maxMM, (long)subs[i]->M * subs[i]->M);
  }
  const TcArgs *d_tc = dupload(owner, tc.data(), ns);
  P->df = dupload(owner, df.data(), ns);
  P->dfl = df_launch_plan(df);
  P->os = dupload(owner, os.data(), ns);
  P->vf = dupload(owner, vf.data(), ns);

  // density: per CTA a list of (system, tile, chunk, chunks)
  {
    long total_tiles = 0;
    for (auto *h : subs) total_tiles += h->n_tiles_tc;
    const int grid = (int)std::max<long>(1, std::min<long>(total_tiles, sms));
    std::vector<std::vector<TcJob>> per(grid);
    int max_nmc = 1;
    if (!batch) {  // tile t on CTA t mod grid, in order
      const etdm_handle *h = subs[0];
      const int nmc = chunks(h);
      for (int t = 0; t < h->n_tiles_tc; ++t) push_tile(per[t % grid], h, 0, t, nmc);
      max_nmc = nmc;
    } else {
      // longest processing time first: a job's cost is its K steps (plus the
      // read-out, about two K steps' worth) times its orbital chunks
      struct Item { long cost; int s, t; };
      std::vector<Item> items;
      items.reserve(total_tiles);
      for (int s = 0; s < ns; ++s) {
        const etdm_handle *h = subs[s];
        const int nmc = chunks(h);
        max_nmc = std::max(max_nmc, nmc);
        for (int t = 0; t < h->n_tiles_tc; ++t) {
          // a tile no function reaches keeps the zero density it was allocated with
          if (h->h_mu_off[t + 1] == h->h_mu_off[t]) continue;
          const long nk = h->h_xr_off[t + 1] - h->h_xr_off[t];
          items.push_back(Item{(nk + 2) * nmc, s, t});
        }
      }
      std::stable_sort(items.begin(), items.end(),
                       [](const Item &a, const Item &b) { return a.cost > b.cost; });
      using Load = std::pair<long, int>;  // (work so far, CTA)
      std::priority_queue<Load, std::vector<Load>, std::greater<Load>> q;
      for (int b = 0; b < grid; ++b) q.push(Load{0, b});
      for (const Item &it : items) {
        Load l = q.top();
        q.pop();
        push_tile(per[l.second], subs[it.s], it.s, it.t, chunks(subs[it.s]));
        q.push(Load{l.first + it.cost, l.second});
      }
    }
    std::vector<TcJob> jobs;
    std::vector<int> ptr(grid + 1, 0);
    for (int b = 0; b < grid; ++b) {
      jobs.insert(jobs.end(), per[b].begin(), per[b].end());
      ptr[b + 1] = (int)jobs.size();
    }
    P->rho = TcBatch{d_tc, dupload(owner, jobs.data(), jobs.size()),
                     dupload(owner, ptr.data(), ptr.size()), d_active, d_flags, grid, max_nmc};
  }

  // V: per CTA a contiguous run of (system, group)
  {
    std::vector<TcJob> jobs;
    std::vector<long> cost;
    for (int s = 0; s < ns; ++s) {
      const etdm_handle *h = subs[s];
      for (int g = 0; g < h->n_vg; ++g) {
        const int t0 = h->h_vg_t0[g], nt = h->h_vg_t0[g + 1] - t0;
        const int e0 = h->h_vg_eoff[g], np = h->h_vg_eoff[g + 1] - e0;
        if (batch && h->h_vg_nu[g] == 0) continue;  // an empty group adds nothing to V
        jobs.push_back(TcJob{make_int4(s, g, t0, nt),
                             make_int4(e0, np, h->h_vg_nu[g], h->h_vg_xoff[g])});
        cost.push_back((long)nt * (np + 32));
      }
    }
    const long nj = (long)jobs.size();
    const int grid = (int)std::max<long>(1, std::min<long>(nj, sms));
    std::vector<int> ptr(grid + 1, 0);
    if (!batch) {  // equal numbers of groups
      for (int b = 0; b <= grid; ++b) ptr[b] = (int)(nj * b / grid);
    } else {  // cut the run where the cumulative cost passes b / grid of the total
      const long tot = std::accumulate(cost.begin(), cost.end(), 0L);
      long acc = 0;
      int b = 1;
      for (long j = 0; j < nj && b < grid; ++j) {
        acc += cost[j];
        while (b < grid && acc * grid >= tot * b) ptr[b++] = (int)(j + 1);
      }
      while (b < grid) ptr[b++] = (int)nj;
      ptr[grid] = (int)nj;
    }
    P->v = TcBatch{d_tc, dupload(owner, jobs.data(), jobs.size()),
                   dupload(owner, ptr.data(), ptr.size()), d_active, d_flags, grid, 1};
  }
  P->vf_blocks = (int)std::min<long>(1024, (maxMM + 255) / 256);
  P->vfix = vfix;
  P->vfix_bytes = vfix_bytes;
}

}  // namespace etdm
