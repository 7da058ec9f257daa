// Batches of systems: many molecules of uneven size evaluated together.
//
// Each member system keeps its own set-up (lists, slices, S, T, C0, the Eq. 33
// orbital energies, the L-BFGS memory); the batch owns the packed vectors of
// all members' variables and the launch tables of the batched kernels:
//  - dense chains (Eq. 7, 12, 37 and the reverse pass): one block per system,
//    largest systems first, the block barrier in place of the grid barrier;
//  - density and V passes on the tensor cores: one launch over per-CTA job
//    lists of (system, tile) and (system, group), balanced over the SMs;
//  - potential passes: blockIdx.y picks the system;
//  - L-BFGS two-loop (Sec. 3.1): one block per system.
// A whole evaluation is one captured CUDA graph.  Minimization advances every
// system by one trial point per round: the round is one graph (commit of the
// accepted points, directions, trial points, evaluation, slopes, readback),
// and the host runs one line search (Eq. 25-29) per system between rounds;
// systems that are done are masked out in device memory.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "device.cuh"
#include "host.h"
#include "internal.h"
#include "linesearch.h"

namespace etdm {

namespace {

constexpr int kCtlFlags = 4;  // accept, dir, reset, eval
enum { CTL_ACCEPT = 0, CTL_DIR = 1, CTL_RESET = 2, CTL_EVAL = 3 };

// a <- a_e and g <- g_e for the systems whose accept flag is set
__global__ void commit_kernel(const long long *off, const int *accept, double *a,
                              const double *ae, double *g, const double *ge) {
  const int i = blockIdx.y;
  if (!accept[i]) return;
  for (long long e = off[i] + (long long)blockIdx.x * blockDim.x + threadIdx.x; e < off[i + 1];
       e += (long long)gridDim.x * blockDim.x) {
    a[e] = ae[e];
    g[e] = ge[e];
  }
}

// a_e = a + alpha_i p for the systems whose eval flag is set (alpha = 0: a)
__global__ void axpy_batch_kernel(const long long *off, const int *eval, const double *alpha,
                                  const double *a, const double *p, double *ae) {
  const int i = blockIdx.y;
  if (!eval[i]) return;
  const double al = alpha[i];
  for (long long e = off[i] + (long long)blockIdx.x * blockDim.x + threadIdx.x; e < off[i + 1];
       e += (long long)gridDim.x * blockDim.x)
    ae[e] = al == 0.0 ? a[e] : a[e] + al * p[e];
}

// out[i] = x_i . y_i for the systems whose flag is set; one block of 1024
// threads per system with the single-system dot product's order of additions
__global__ void __launch_bounds__(1024) dot_batch_kernel(const long long *off, const int *flag,
                                                         int n, const double *x, const double *y,
                                                         double *out) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    if (!flag[i]) continue;
    const double *xi = x + off[i], *yi = y + off[i];
    const long len = (long)(off[i + 1] - off[i]);
    double s = 0.0;
    for (long e = threadIdx.x; e < len; e += blockDim.x) s += xi[e] * yi[e];
    s = block_sum(s);
    if (threadIdx.x == 0) out[i] = s;
  }
}

// dst <- src (packed variables and energies) for the active systems only
__global__ void copy_active_kernel(const long long *off, const int *active, const double *g_src,
                                   double *g_dst, const double *E_src, double *E_dst) {
  const int i = blockIdx.y;
  if (!active[i]) return;
  if (g_dst)
    for (long long e = off[i] + (long long)blockIdx.x * blockDim.x + threadIdx.x; e < off[i + 1];
         e += (long long)gridDim.x * blockDim.x)
      g_dst[e] = g_src[e];
  if (E_dst && blockIdx.x == 0 && threadIdx.x == 0) E_dst[i] = E_src[i];
}

int *ctl_flags(etdm_handle *h, int k) { return (int *)h->d_ctlbuf + (long)k * h->members.size(); }
double *ctl_alpha(etdm_handle *h) {
  return (double *)(h->d_ctlbuf + (long)kCtlFlags * h->members.size() * sizeof(int));
}
size_t ctl_bytes(const etdm_handle *h) {
  const size_t n = h->members.size();
  return kCtlFlags * n * sizeof(int) + n * sizeof(double);
}
int stat_count(const etdm_handle *h) { return FLAG_NFLAGS * ((int)h->members.size() + 1); }

// The evaluation of every system on `s` (mixed path), the systems masked by
// `active` (the plan's mask is the same array).  With `timed`, CUDA events
// around each stage (outside a capture only).
void eval_body(etdm_handle *h, const MixedPlan &P, const int *active, cudaStream_t s,
               bool timed = false) {
  const int n = (int)h->members.size();
  auto stage = [&](int id, auto fn) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
      CUDA_TRY(cudaEventCreate(&e0));
      CUDA_TRY(cudaEventRecord(e0, s));
    }
    fn();
    if (timed) {
      CUDA_TRY(cudaEventCreate(&e1));
      CUDA_TRY(cudaEventRecord(e1, s));
      h->prof_events.push_back({id, {e0, e1}});
    }
  };
  stage(ETDM_STAGE_DENSE_FWD, [&] {
    CUDA_TRY(launch_dense_batch(h->d_dargs, h->d_order, n, active, h->dense_grid, true, false, s));
  });
  stage(ETDM_STAGE_RHO, [&] { CUDA_TRY(launch_mixed_rho(P, s)); });
  stage(ETDM_STAGE_POTENTIAL, [&] { CUDA_TRY(launch_mixed_potential(P, s)); });
  stage(ETDM_STAGE_VMAT, [&] { CUDA_TRY(launch_mixed_vmat(P, s)); });
  stage(ETDM_STAGE_DENSE_REV, [&] {
    CUDA_TRY(launch_dense_batch(h->d_dargs, h->d_order, n, active, h->dense_grid, true, true, s));
  });
}

// One minimization round (see the file comment); ctl and alpha come from the
// pinned mirror, the results and status words go back to it.
void round_body(etdm_handle *h, cudaStream_t s) {
  const int n = (int)h->members.size();
  const int vb = (int)std::min<long>(64, (h->nvar_tot / n + 255) / 256 + 1);
  CUDA_TRY(cudaMemcpyAsync(h->d_ctlbuf, h->h_ctl, ctl_bytes(h), cudaMemcpyHostToDevice, s));
  commit_kernel<<<dim3(vb, n), 256, 0, s>>>(h->d_off, ctl_flags(h, CTL_ACCEPT), h->d_a, h->d_ae,
                                             h->d_g, h->d_ge);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(launch_lbfgs_batch(h->d_largs, ctl_flags(h, CTL_DIR), ctl_flags(h, CTL_RESET), n,
                              h->lb_grid, s));
  dot_batch_kernel<<<std::min(n, 4 * h->num_sms), 1024, 0, s>>>(h->d_off, ctl_flags(h, CTL_DIR), n,
                                                               h->d_g, h->d_p, h->d_res + 2 * n);
  axpy_batch_kernel<<<dim3(vb, n), 256, 0, s>>>(h->d_off, ctl_flags(h, CTL_EVAL), ctl_alpha(h),
                                                 h->d_a, h->d_p, h->d_ae);
  CUDA_TRY(cudaGetLastError());
  eval_body(h, h->bplan_eval, ctl_flags(h, CTL_EVAL), s);
  dot_batch_kernel<<<std::min(n, 4 * h->num_sms), 1024, 0, s>>>(h->d_off, ctl_flags(h, CTL_EVAL), n,
                                                               h->d_ge, h->d_p, h->d_res + n);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(h->h_res, h->d_res, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(h->h_res + 3 * n, h->d_bflags, stat_count(h) * sizeof(int),
                           cudaMemcpyDeviceToHost, s));
}

// Capture `body` on the batch's stream into an executable graph; returns the
// number of kernel nodes.
template <class F>
long long capture(etdm_handle *h, cudaGraphExec_t *exec, F body) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed));
  try {
    body(h->cap);
  } catch (...) {
    cudaStreamEndCapture(h->cap, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  CUDA_TRY(cudaStreamEndCapture(h->cap, &g));
  size_t nn = 0;
  CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
  long long kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CUDA_TRY(cudaGraphNodeGetType(nd, &t));
    kernels += t == cudaGraphNodeTypeKernel;
  }
  cudaError_t e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  CUDA_TRY(e);
  return kernels;
}

// Raise on a device-side failure recorded in the status words read back with
// the last round (and clear them, so the handle stays usable).
void check_words(etdm_handle *h, const int *words) {
  const int n = (int)h->members.size();
  int code = 0, sys = -1;
  for (int i = 0; i <= n && !code; ++i)
    if (words[FLAG_NFLAGS * i + FLAG_ERR] != 0) {
      code = words[FLAG_NFLAGS * i + FLAG_ERR];
      sys = i;
    }
  if (!code) return;
  std::vector<int> zero(stat_count(h), 0);
  for (int i = 0; i <= n; ++i) zero[FLAG_NFLAGS * i + FLAG_J] = words[FLAG_NFLAGS * i + FLAG_J];
  CUDA_TRY(cudaMemcpy(h->d_bflags, zero.data(), zero.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (code == ETDM_ERR_TIMEOUT)
    throw Fail{code, "a bounded device-side wait of a batched grid pass gave up"};
  throw Fail{code, "numerical failure on the device in system " + std::to_string(sys) +
                       " (NaN/Inf, or |A_ov A_ov^T|_F > 4^8)"};
}

}  // namespace

// Autotuner of the batch's V pass: the number of 4x4x8 tiles whose V the
// tensor memory accumulates between two read-outs (a V group; the union of
// the group's functions stays within 128).  Small molecules have few
// functions, so long groups cut the read-outs and hand-overs per point; the
// exact order-0 accumulator allows up to 8 tiles.  Each candidate rebuilds the
// members' group tables and X^T slices and the batch's job lists, and the
// evaluation (dense chains, density, potential, V) is timed with CUDA events
// (two warm-up evaluations, then the mean of three); the fastest is kept and
// the members' own plans are rebuilt for it.
template <class F>
void autotune_vgroups(etdm_handle *h, F make_plan) {
  const int n = (int)h->members.size();
  const int cand[3] = {2, 4, 8};
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  double best_ms = 1e300;
  int best = cand[0], built = h->members[0]->vg_max;
  h->tune_ms.clear();
  for (int c : cand) {
    if (c != built) {
      for (etdm_handle *m : h->members) build_vgroups(m, c, h->cap);
      make_plan(&h->bplan_act);
      built = c;
    }
    for (int r = 0; r < 2; ++r) eval_body(h, h->bplan_act, h->d_act, h->cap);
    CUDA_TRY(cudaEventRecord(e0, h->cap));
    for (int r = 0; r < 3; ++r) eval_body(h, h->bplan_act, h->d_act, h->cap);
    CUDA_TRY(cudaEventRecord(e1, h->cap));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    h->tune_ms.push_back(c);
    h->tune_ms.push_back(ms / 3.0);
    if (ms / 3.0 < best_ms) {
      best_ms = ms / 3.0;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best != built) {
    for (etdm_handle *m : h->members) build_vgroups(m, best, h->cap);
    make_plan(&h->bplan_act);
  }
  for (etdm_handle *m : h->members)  // the members' own evaluations use the new groups
    build_mixed_plan(m, {m}, m->d_active1, m->d_flags, false, m->d_Vfix,
                     ((size_t)m->M * m->M + 1) * sizeof(unsigned long long), &m->plan);
  CUDA_TRY(cudaMemset(h->d_bflags, 0, stat_count(h) * sizeof(int)));
  CUDA_TRY(cudaStreamSynchronize(h->cap));
  h->tune_choice = best;
  (void)n;
}

void init_batch(etdm_handle *h, const etdm_system *sys, int n_sys, const etdm_options *opt) {
  if (!sys || n_sys < 1) throw Fail{ETDM_ERR_INVALID_ARG, "need n_sys >= 1 systems"};
  etdm_options o;
  etdm_default_options(&o);
  if (opt) o = *opt;
  h->device = o.device;
  h->precision = o.precision;
  h->lbfgs_m = o.lbfgs_m;
  h->gamma = o.gamma;
  h->beta0 = o.beta0;
  for (int i = 0; i < n_sys; ++i) {
    etdm_handle *m = new etdm_handle();
    h->members.push_back(m);
    try {
      init_system(m, &sys[i], &o);
    } catch (Fail &f) {
      f.msg = "system " + std::to_string(i) + ": " + f.msg;
      throw;
    }
  }
  CUDA_TRY(cudaSetDevice(h->device));
  CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  const int n = n_sys;
  h->var_off.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const etdm_handle *m = h->members[i];
    h->var_off[i + 1] = h->var_off[i] + (long)m->N * m->V;
    h->M = std::max(h->M, m->M);
    h->N = std::max(h->N, m->N);
    h->V = std::max(h->V, m->V);
  }
  h->nvar_tot = h->var_off[n];
  const long nv = std::max(h->nvar_tot, 1L);
  h->d_a = dalloc<double>(h, nv);
  h->d_g = dalloc<double>(h, nv);
  h->d_p = dalloc<double>(h, nv);
  h->d_ae = dalloc<double>(h, nv);
  h->d_ge = dalloc<double>(h, nv);
  h->d_res = dalloc<double>(h, 3 * n);
  h->d_ctlbuf = dalloc<unsigned char>(h, ctl_bytes(h));
  std::vector<int> ones(n, 1);
  h->d_act = dupload(h, ones.data(), n);
  h->act_host = ones;
  h->d_bflags = dalloc<int>(h, stat_count(h));
  std::vector<long long> off(h->var_off.begin(), h->var_off.end());
  h->d_off = dupload(h, off.data(), off.size());
  CUDA_TRY(cudaMallocHost(&h->h_ctl, ctl_bytes(h)));
  memset(h->h_ctl, 0, ctl_bytes(h));
  CUDA_TRY(cudaMallocHost(&h->h_res, 3 * n * sizeof(double) + stat_count(h) * sizeof(int)));
  if (h->precision != ETDM_PREC_MIXED) return;  // FP64: one launch sequence per system

  // the members' status words move into one array (one read-back per round);
  // each member's own evaluations use the same words
  for (int i = 0; i < n; ++i) {
    etdm_handle *m = h->members[i];
    m->d_flags = h->d_bflags + FLAG_NFLAGS * i;
    m->plan.rho.flags = m->plan.v.flags = m->d_flags;
  }
  int *bflag = h->d_bflags + FLAG_NFLAGS * n;

  // dense chains and L-BFGS of each member at its slice of the packed vectors
  std::vector<DenseArgs> da(n);
  std::vector<LbfgsArgs> la(n);
  for (int i = 0; i < n; ++i) {
    etdm_handle *m = h->members[i];
    const long o0 = h->var_off[i];
    m->n_gridpart = df_pot_blocks(m);
    m->pairs_last = true;  // the member's accessors read float pairs from now on
    da[i] = dense_args(m, h->d_ae + o0);
    da[i].g = h->d_ge + o0;
    da[i].E = h->d_res + i;
    da[i].flags = m->d_flags;
    la[i] = lbfgs_args(m, h->d_a + o0, h->d_g + o0, h->d_p + o0);
  }
  h->d_dargs = dupload(h, da.data(), n);
  h->d_largs = dupload(h, la.data(), n);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const etdm_handle *a = h->members[x], *b = h->members[y];
    return (long)a->M * a->M * a->N > (long)b->M * b->M * b->N;
  });
  h->d_order = dupload(h, order.data(), n);
  int bps = 1;
  if (occupancy_dense(&bps) != 0 || bps < 1) bps = 1;
  h->dense_grid = std::min(n, h->num_sms * bps);
  h->lb_grid = std::min(n, 4 * h->num_sms);

  // grid stages: the members' fixed-point V sums lie in one array (one reset per
  // evaluation); the members' own d_Vfix stay theirs for their own evaluations
  std::vector<size_t> vo(n + 1, 0);
  for (int i = 0; i < n; ++i) vo[i + 1] = vo[i] + (size_t)h->members[i]->M * h->members[i]->M + 1;
  unsigned long long *arena = dalloc<unsigned long long>(h, vo[n]);
  std::vector<unsigned long long *> own(n);
  for (int i = 0; i < n; ++i) {
    own[i] = h->members[i]->d_Vfix;
    h->members[i]->d_Vfix = arena + vo[i];
  }
  auto make_plan = [&](MixedPlan *P) {
    for (int i = 0; i < n; ++i) h->members[i]->d_Vfix = arena + vo[i];
    try {
      build_mixed_plan(h, h->members, h->d_act, bflag, true, arena,
                       vo[n] * sizeof(unsigned long long), P);
    } catch (...) {
      for (int i = 0; i < n; ++i) h->members[i]->d_Vfix = own[i];
      throw;
    }
    for (int i = 0; i < n; ++i) h->members[i]->d_Vfix = own[i];
  };
  CUDA_TRY(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  make_plan(&h->bplan_act);
  if (o.vgroup == 0 && n > 1) autotune_vgroups(h, make_plan);
  // the same tables masked by the round's eval flags instead
  h->bplan_eval = h->bplan_act;
  const int *ev = ctl_flags(h, CTL_EVAL);
  h->bplan_eval.active = h->bplan_eval.rho.active = h->bplan_eval.v.active = ev;

  // graphs (the launches once outside a capture first: kernel attributes are set)
  eval_body(h, h->bplan_act, h->d_act, h->cap);
  CUDA_TRY(cudaStreamSynchronize(h->cap));
  h->graph_kernels_eval =
      capture(h, &h->g_eval, [&](cudaStream_t s) { eval_body(h, h->bplan_act, h->d_act, s); });
  h->graph_kernels_round = capture(h, &h->g_round, [&](cudaStream_t s) { round_body(h, s); });
  CUDA_TRY(cudaMemset(h->d_bflags, 0, stat_count(h) * sizeof(int)));
  CUDA_TRY(cudaDeviceSynchronize());
}

void batch_release(etdm_handle *h) {
  if (h->g_eval) cudaGraphExecDestroy(h->g_eval);
  if (h->g_round) cudaGraphExecDestroy(h->g_round);
  h->g_eval = h->g_round = nullptr;
  if (h->cap) cudaStreamDestroy(h->cap);
  h->cap = nullptr;
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  if (h->h_res) cudaFreeHost(h->h_res);
  h->h_ctl = nullptr;
  h->h_res = nullptr;
  for (etdm_handle *m : h->members) {
    release_handle(m);
    delete m;
  }
  h->members.clear();
}

void batch_energy_grad(etdm_handle *h, const double *a, double *E, double *g, cudaStream_t s) {
  const int n = (int)h->members.size();
  if (a != h->d_ae)
    CUDA_TRY(cudaMemcpyAsync(h->d_ae, a, h->nvar_tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (h->precision == ETDM_PREC_MIXED && h->profiling) {  // the same kernels, timed per stage
    eval_body(h, h->bplan_act, h->d_act, s, true);
    h->launches += h->graph_kernels_eval;
  } else if (h->precision == ETDM_PREC_MIXED) {
    CUDA_TRY(cudaGraphLaunch(h->g_eval, s));
    h->launches += h->graph_kernels_eval;
  } else {  // the plain path: one launch sequence per (active) system
    for (int i = 0; i < n; ++i) {
      if (!h->act_host[i]) continue;
      eval_system(h->members[i], h->d_ae + h->var_off[i], h->d_res + i, h->d_ge + h->var_off[i], s);
      h->launches += h->members[i]->launches;
      h->members[i]->launches = 0;
    }
  }
  // the results of the active systems (inactive entries of E and g untouched)
  const bool gout = g && g != h->d_ge, Eout = E && E != h->d_res;
  if (gout || Eout) {
    const int vb = (int)std::min<long>(64, (h->nvar_tot / n + 255) / 256 + 1);
    copy_active_kernel<<<dim3(vb, n), 256, 0, s>>>(h->d_off, h->d_act, h->d_ge, gout ? g : nullptr,
                                                   h->d_res, Eout ? E : nullptr);
    CUDA_TRY(cudaGetLastError());
  }
}

void batch_check(etdm_handle *h, cudaStream_t s) {
  int *w = (int *)(h->h_res + 3 * h->members.size());
  CUDA_TRY(cudaMemcpyAsync(w, h->d_bflags, stat_count(h) * sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (h->precision == ETDM_PREC_MIXED) {
    check_words(h, w);
    return;
  }
  for (etdm_handle *m : h->members) {  // FP64 members keep their own status words
    const int rc = etdm_check(m, s);
    if (rc != ETDM_OK) throw Fail{rc, etdm_last_error(m)};
  }
}

void batch_energy_grad_host(etdm_handle *h, const double *a, double *E, double *g) {
  cudaStream_t s = 0;
  const int n = (int)h->members.size();
  CUDA_TRY(cudaMemcpyAsync(h->d_ae, a, h->nvar_tot * sizeof(double), cudaMemcpyHostToDevice, s));
  batch_energy_grad(h, h->d_ae, h->d_res, h->d_ge, s);
  const bool all = std::all_of(h->act_host.begin(), h->act_host.end(), [](int v) { return v != 0; });
  if (all) {
    CUDA_TRY(cudaMemcpyAsync(E, h->d_res, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (g) CUDA_TRY(cudaMemcpyAsync(g, h->d_ge, h->nvar_tot * sizeof(double), cudaMemcpyDeviceToHost, s));
    batch_check(h, s);
    return;
  }
  // a mask is set: copy back the active systems' entries only
  std::vector<double> Et(n), gt(g ? h->nvar_tot : 0);
  CUDA_TRY(cudaMemcpyAsync(Et.data(), h->d_res, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (g) CUDA_TRY(cudaMemcpyAsync(gt.data(), h->d_ge, h->nvar_tot * sizeof(double), cudaMemcpyDeviceToHost, s));
  batch_check(h, s);
  for (int i = 0; i < n; ++i) {
    if (!h->act_host[i]) continue;
    E[i] = Et[i];
    if (g) std::copy(gt.begin() + h->var_off[i], gt.begin() + h->var_off[i + 1], g + h->var_off[i]);
  }
}

void batch_minimize(etdm_handle *h, double *a_dev, int n_steps, double *E_hist, double *alpha_hist,
                    int32_t *trials_hist, cudaStream_t s) {
  const int n = (int)h->members.size();
  const int K = n_steps + 1;
  if (h->precision != ETDM_PREC_MIXED) {  // the plain path: each system minimized on its own
    for (int i = 0; i < n; ++i) {
      const int rc = etdm_minimize(h->members[i], a_dev + h->var_off[i], n_steps,
                                   E_hist ? E_hist + (long)i * K : nullptr,
                                   alpha_hist ? alpha_hist + (long)i * K : nullptr,
                                   trials_hist ? trials_hist + (long)i * K : nullptr, s);
      if (rc != ETDM_OK)
        throw Fail{rc, "system " + std::to_string(i) + ": " + etdm_last_error(h->members[i])};
      h->launches += h->members[i]->launches;
      h->members[i]->launches = 0;
    }
    return;
  }
  CUDA_TRY(cudaMemcpyAsync(h->d_a, a_dev, h->nvar_tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  struct Sys {
    LineSearch ls;
    double E = 0.0;     // energy at the current point
    int step = 0;       // steps finished
    bool done = false;  // all steps finished
    bool dir = true;    // the next round computes a direction (and its first trial)
    bool reset = false; // ... after erasing the memory
    bool commit = true; // the next round takes the last trial as the current point
  };
  std::vector<Sys> st(n);
  int *f = (int *)h->h_ctl;
  double *alpha = (double *)(h->h_ctl + kCtlFlags * n * sizeof(int));
  const double *res = h->h_res;
  auto run_round = [&]() {
    CUDA_TRY(cudaGraphLaunch(h->g_round, s));
    h->launches += h->graph_kernels_round;
    CUDA_TRY(cudaStreamSynchronize(s));
    check_words(h, (const int *)(h->h_res + 3 * n));
  };
  // round 0: every system at its start point (alpha = 0), committed next round
  for (int i = 0; i < n; ++i) {
    f[CTL_ACCEPT * n + i] = 0;
    f[CTL_DIR * n + i] = 0;
    f[CTL_RESET * n + i] = 0;
    f[CTL_EVAL * n + i] = 1;
    alpha[i] = 0.0;
  }
  run_round();
  for (int i = 0; i < n; ++i) {
    st[i].E = res[i];
    st[i].done = n_steps == 0;
    if (E_hist) E_hist[(long)i * K] = st[i].E;
    if (alpha_hist) alpha_hist[(long)i * K] = 0.0;
    if (trials_hist) trials_hist[(long)i * K] = 1;
  }
  for (;;) {
    bool any = false;
    for (int i = 0; i < n; ++i) {
      Sys &y = st[i];
      f[CTL_ACCEPT * n + i] = y.commit;
      f[CTL_DIR * n + i] = !y.done && y.dir;
      f[CTL_RESET * n + i] = !y.done && y.dir && y.reset;
      f[CTL_EVAL * n + i] = !y.done;
      alpha[i] = y.done ? 0.0 : (y.dir ? 1.0 : y.ls.alpha());
      any = any || y.commit || !y.done;
      y.commit = false;
    }
    if (!any) break;
    run_round();
    for (int i = 0; i < n; ++i) {
      Sys &y = st[i];
      if (y.done) continue;
      const double Et = res[i], d = res[n + i];
      if (y.dir) {
        const double d0 = res[2 * n + i];
        if (!(d0 < 0.0) && !y.reset) {  // not a descent direction: erase the memory,
          y.reset = true;               // precondition only, and try again
          continue;
        }
        y.dir = false;
        y.reset = false;
        y.ls.start(y.E, d0);
      }
      y.ls.feed(Et, d);
      if (!y.ls.done()) continue;
      // the accepted point is the last trial evaluated: committed next round
      if (y.ls.accepted()) {
        y.commit = true;
        y.E = y.ls.result().E;
      }
      ++y.step;
      const long k = (long)i * K + y.step;
      if (E_hist) E_hist[k] = y.E;
      if (alpha_hist) alpha_hist[k] = y.ls.accepted() ? y.ls.result().a : 0.0;
      if (trials_hist) trials_hist[k] = y.ls.trials();
      if (y.step == n_steps) y.done = true;
      else y.dir = true;
    }
  }
  CUDA_TRY(cudaMemcpyAsync(a_dev, h->d_a, h->nvar_tot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
}

}  // namespace etdm
