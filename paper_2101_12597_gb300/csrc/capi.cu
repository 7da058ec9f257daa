// C ABI of libetdm (include/etdm.h): handle set-up, the evaluation sequence,
// the L-BFGS / preconditioner entry points and the host line search.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <iterator>
#include <numeric>
#include <string>
#include <vector>

#include "host.h"
#include "internal.h"
#include "kpoint.h"
#include "linesearch.h"

using namespace etdm;

namespace {

// message of the last failure without a handle, per host thread (handles
// initialized from several threads at once do not race on it)
thread_local std::string g_init_err;

void release(etdm_handle *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  batch_release(h);
  for (auto &pe : h->prof_events) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  h->prof_events.clear();
  for (void *p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  h->h_pinned = nullptr;
}

int set_err(etdm_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg; else g_init_err = msg;
  return code;
}

// deferred device-side status (copied with the stream's other results: one
// synchronization)
int check_flags(etdm_handle *h, cudaStream_t s) {
  int *f = (int *)(h->h_pinned + 8);
  CUDA_TRY(cudaMemcpyAsync(f, h->d_flags, FLAG_NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (f[FLAG_ERR] != 0) {
    int code = f[FLAG_ERR];
    int zero = 0;
    CUDA_TRY(cudaMemcpy(h->d_flags + FLAG_ERR, &zero, sizeof(int), cudaMemcpyHostToDevice));
    if (code == ETDM_ERR_TIMEOUT) {
      CUDA_TRY(cudaMemset(h->d_bar, 0, 4 * sizeof(unsigned)));
      throw Fail{code, "a bounded device-side grid barrier gave up (blocks not co-resident?)"};
    }
    throw Fail{code, "numerical failure on the device (NaN/Inf, or |A_ov A_ov^T|_F > 4^8)"};
  }
  return ETDM_OK;
}

// One energy (+ gradient) evaluation, all on `s`.
void evaluate(etdm_handle *h, const double *a, double *E, double *g, cudaStream_t s) {
  if (h->kpath) {
    evaluate_k(h, a, E, g, s);
    return;
  }
  {
    StageTimer t(h, s, ETDM_STAGE_DENSE_FWD);
    CUDA_TRY(launch_dense_forward(h, a, s));
    t.done();
  }
  const bool mixed = h->precision == ETDM_PREC_MIXED && !h->in_setup;
  {
    StageTimer t(h, s, ETDM_STAGE_RHO);
    if (mixed) {
      CUDA_TRY(launch_mixed_rho(h->plan, s));
    } else {
      CUDA_TRY(launch_rho_fp64(h, h->d_D, h->d_rho, s));
    }
    t.done();
  }
  {
    StageTimer t(h, s, ETDM_STAGE_POTENTIAL);
    if (mixed) {  // float-pair half-spectrum pipeline; also resets V's fixed-point sums
      CUDA_TRY(launch_mixed_potential(h->plan, s));
      h->n_gridpart = df_pot_blocks(h);
    } else {
      CUDA_TRY(launch_pack_real(h, h->d_rho, h->d_fft, s));
      CUDA_TRY(fft3d(h, h->d_fft, -1, s));
      CUDA_TRY(launch_poisson_scale(h, h->d_fft, s));
      CUDA_TRY(fft3d(h, h->d_fft, +1, s));
      CUDA_TRY(launch_potential(h, s));
      h->n_gridpart = kPotBlocks;
    }
    t.done();
  }
  // kernels: dense forward and reverse; mixed: O slices (column maxima, then
  // the slices), density, 5 potential passes, V and its fixed-point
  // conversion; FP64: density, pack, 2 x 3 FFT passes, scale, potential (+ V
  // with the gradient)
  h->launches += 12;
  if (mixed) {  // also needed for the energy: first-order correction of D's quantization
    StageTimer t(h, s, ETDM_STAGE_VMAT);
    CUDA_TRY(launch_mixed_vmat(h->plan, s));
    t.done();
  } else if (g) {
    StageTimer t(h, s, ETDM_STAGE_VMAT);
    CUDA_TRY(launch_vmat_fp64(h, h->d_vtot, h->d_H, s));
    t.done();
    h->launches += 1;
  }
  {
    StageTimer t(h, s, ETDM_STAGE_DENSE_REV);
    CUDA_TRY(launch_dense_reverse(h, a, g, E, s));
    t.done();
  }
}

void lbfgs(etdm_handle *h, const double *a, const double *g, double *p, cudaStream_t s) {
  StageTimer t(h, s, ETDM_STAGE_LBFGS);
  CUDA_TRY(launch_lbfgs(h, a, g, p, s));
  t.done();
  h->launches += 1;
}

int factor_ok(int n) {
  int m = n;
  const int pr[] = {2, 3, 5, 7, 11, 13};
  for (int p : pr)
    while (m % p == 0) m /= p;
  return m == 1;
}

void validate(const etdm_system *sys, const etdm_options *opt) {
  auto bad = [](const std::string &m) { throw Fail{ETDM_ERR_INVALID_ARG, m}; };
  if (!sys) bad("sys is NULL");
  if (sys->n_atoms < 1 || !sys->pos || !sys->Z) bad("need n_atoms >= 1 with pos and Z");
  if (sys->n_basis < 2 || !sys->bf_atom || !sys->bf_exp || !sys->bf_rcut)
    bad("need n_basis >= 2 with bf_atom, bf_exp, bf_rcut");
  if (sys->n_electrons < 2 || sys->n_electrons % 2 || sys->n_electrons / 2 > sys->n_basis)
    bad("n_electrons must be even with 2 <= n_electrons <= 2 n_basis");
  if (sys->n_basis > (1 << 22)) bad("n_basis too large");
  double Lmin = 1e300;
  for (int a = 0; a < 3; ++a) {
    if (!(sys->box[a] > 0.0)) bad("box edges must be positive");
    Lmin = std::min(Lmin, sys->box[a]);
    if (sys->grid[a] < 2 || sys->grid[a] > kMaxFFT || !factor_ok(sys->grid[a]))
      bad("grid sizes must be in [2, 256] with prime factors <= 13");
  }
  for (int i = 0; i < sys->n_atoms; ++i)
    for (int a = 0; a < 3; ++a) {
      double x = sys->pos[3 * i + a];
      if (!(x >= 0.0 && x < sys->box[a])) bad("positions must lie in [0, box)");
    }
  for (int m = 0; m < sys->n_basis; ++m) {
    if (sys->bf_atom[m] < 0 || sys->bf_atom[m] >= sys->n_atoms) bad("bf_atom out of range");
    if (!(sys->bf_exp[m] > 0.0)) bad("bf_exp must be positive");
    if (!(sys->bf_rcut[m] > 0.0 && sys->bf_rcut[m] < 2.0 * Lmin))
      bad("bf_rcut must be in (0, 2 * min(box))");
  }
  if (!(sys->ion_sigma > 0.0)) bad("ion_sigma must be positive");
  const bool full = sys->n_k >= 1 || (opt && opt->param == ETDM_PARAM_FULL);
  if (sys->n_k < 0) bad("n_k must be >= 0");
  if (sys->n_k >= 1) {
    if (!sys->k_frac || !sys->k_w) bad("n_k >= 1 needs k_frac and k_w");
    double wsum = 0.0;
    for (int k = 0; k < sys->n_k; ++k) {
      if (!(sys->k_w[k] > 0.0)) bad("k-point weights must be positive");
      wsum += sys->k_w[k];
      for (int a = 0; a < 3; ++a)
        if (!std::isfinite(sys->k_frac[3 * k + a])) bad("k-points must be finite");
    }
    if (fabs(wsum - 1.0) > 1e-12) bad("k-point weights must sum to 1");
  }
  if (full) {
    if (!(sys->kT >= 0.0) || !std::isfinite(sys->kT)) bad("kT must be finite and >= 0");
    if (sys->kT == 0.0 && sys->n_k > 1) bad("kT = 0 (integer occupation) needs n_k <= 1");
    if (sys->n_basis > 1024) bad("the full-A path takes n_basis <= 1024");
    if (opt && opt->precision != ETDM_PREC_FP64) bad("the full-A path runs in FP64 only");
    if (opt && opt->param != ETDM_PARAM_FULL && opt->param != ETDM_PARAM_OCCVIRT)
      bad("unknown param");
  } else if (opt && opt->param != ETDM_PARAM_OCCVIRT) {
    bad("unknown param");
  }
  if (!full && sys->n_electrons / 2 >= sys->n_basis)
    bad("the occupied-virtual path needs a virtual orbital (n_electrons < 2 n_basis): "
        "with none, A_ov is empty and E does not depend on it");
  if (opt) {
    if (opt->expm != ETDM_EXPM_EIG && opt->expm != ETDM_EXPM_SS) bad("unknown expm");
    if (opt->expm == ETDM_EXPM_SS && !full) bad("expm = ETDM_EXPM_SS needs the full-A path");
    if (opt->ref_update < -1) bad("ref_update must be >= -1");
    if (opt->ref_update != 0 && opt->expm != ETDM_EXPM_SS)
      bad("ref_update needs expm = ETDM_EXPM_SS");
  }
  if (opt) {
    if (opt->precision != ETDM_PREC_FP64 && opt->precision != ETDM_PREC_MIXED)
      bad("unknown precision");
    if (opt->lbfgs_m < 1 || opt->lbfgs_m > 16) bad("lbfgs_m must be in [1, 16]");
    if (!(opt->gamma >= 0.0 && opt->gamma <= 1.0)) bad("gamma must be in [0, 1]");
    if (!(opt->beta0 > 0.0)) bad("beta0 must be positive");
    if (opt->dense_blocks < 0) bad("dense_blocks must be >= 0");
    if (opt->dense_tc < -1 || opt->dense_tc > 1) bad("dense_tc must be -1, 0 or 1");
    if (opt->vgroup < 0 || opt->vgroup > 8) bad("vgroup must be in [0, 8]");
    if (opt->functional != ETDM_FUNC_KS && opt->functional != ETDM_FUNC_PZSIC)
      bad("unknown functional");
    if (opt->functional == ETDM_FUNC_PZSIC) {
      if (!full) bad("PZ-SIC needs the full-A path (ETDM_PARAM_FULL)");
      if (sys->n_k > 1 || sys->kT != 0.0) bad("PZ-SIC runs at one k-point with kT = 0");
      if (sys->n_k == 1)
        for (int a = 0; a < 3; ++a)
          if (sys->k_frac[a] != 0.0) bad("PZ-SIC runs at the Gamma point");
    }
  }
}

// S^(-1/2) by the coupled Newton-Schulz iteration on S / c (c >= lambda_max).
void inverse_sqrt(etdm_handle *h, cudaStream_t s) {
  const int M = h->M;
  const long MM = (long)M * M;
  double *Y = dalloc<double>(h, MM), *Zm = dalloc<double>(h, MM), *Tm = dalloc<double>(h, MM),
         *Y2 = dalloc<double>(h, MM), *Z2 = dalloc<double>(h, MM), *sc = dalloc<double>(h, 2);
  CUDA_TRY(launch_max_rowsum(h->d_S, sc, M, s));
  double c = 0.0;
  CUDA_TRY(cudaMemcpyAsync(&c, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (!(c > 0.0) || !std::isfinite(c)) throw Fail{ETDM_ERR_NUMERIC, "overlap matrix is not finite"};
  CUDA_TRY(launch_ns_prep(h->d_S, Y, Zm, c, M, s));
  bool done = false;
  int extra = 0;
  for (int it = 0; it < 200; ++it) {
    Phase ph{};
    ph.m = M; ph.n = M; ph.k = M; ph.np = 1;
    ph.p[0] = Prod{Zm, Y, M, M, 0, 0, -0.5, 0};
    ph.diag = 1.5; ph.out = Tm; ph.ldo = M;
    CUDA_TRY(launch_gemm(ph, s));
    CUDA_TRY(launch_resid(Tm, sc + 1, M, s));
    Phase py{};
    py.m = M; py.n = M; py.k = M; py.np = 1;
    py.p[0] = Prod{Y, Tm, M, M, 0, 0, 1.0, 0};
    py.out = Y2; py.ldo = M;
    CUDA_TRY(launch_gemm(py, s));
    Phase pz = py;
    pz.p[0] = Prod{Tm, Zm, M, M, 0, 0, 1.0, 0};
    pz.out = Z2;
    CUDA_TRY(launch_gemm(pz, s));
    std::swap(Y, Y2);
    std::swap(Zm, Z2);
    double r = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&r, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (!std::isfinite(r)) throw Fail{ETDM_ERR_NUMERIC, "S^(-1/2) iteration diverged"};
    if (done && ++extra >= 2) break;
    if (2.0 * r < 1e-13) done = true;
  }
  if (!done)
    throw Fail{ETDM_ERR_NOT_CONVERGED,
               "S^(-1/2) Newton-Schulz iteration did not converge (S ill-conditioned?)"};
  // Z converged to (S / c)^(-1/2), so S^(-1/2) = Z / sqrt(c); the columns are
  // put in reference order later (S stays in d_S, readable through etdm_get_array)
  CUDA_TRY(launch_scale_copy(Zm, h->d_C0, 1.0 / sqrt(c), MM, s));
}

__global__ void extract_ptr_kernel(const long long *off, long long total, int M, int n_tiles,
                                   int *ptr) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t <= n_tiles;
       t += (long)gridDim.x * blockDim.x)
    ptr[t] = (t == n_tiles) ? (int)total : (int)off[t * (long)M];
}

__global__ void symmetrize_upper_kernel(double *H, int M) {
  long MM = (long)M * M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MM;
       e += (long)gridDim.x * blockDim.x) {
    int i = (int)(e / M), c = (int)(e % M);
    if (i > c) H[e] = H[(long)c * M + i];
  }
}

GridGeom make_geom(etdm_handle *h, int tx, int ty, int tz, int *n_tiles) {
  GridGeom g{};
  g.nx = h->n[0]; g.ny = h->n[1]; g.nz = h->n[2];
  g.tx = tx; g.ty = ty; g.tz = tz;
  g.nbx = (g.nx + tx - 1) / tx;
  g.nby = (g.ny + ty - 1) / ty;
  g.nbz = (g.nz + tz - 1) / tz;
  g.M = h->M;
  g.dV = h->dV;
  *n_tiles = g.nbx * g.nby * g.nbz;
  return g;
}

// Truncation lists of one tile geometry: count per (tile, mu), exclusive scan,
// fill in (tile, mu, image) order (sorted keys within a tile).
void build_lists(etdm_handle *h, const GridGeom &g, int n_tiles, int **d_ptr, int **d_keys,
                 long *n_entries, int *max_list, int limit, cudaStream_t s) {
  const int M = h->M;
  const long ncnt = (long)n_tiles * M;
  int *d_count = dalloc<int>(h, ncnt);
  long long *d_off = dalloc<long long>(h, ncnt);
  long long *d_tmp = dalloc<long long>(h, ncnt / 1024 + 4);
  CUDA_TRY(launch_list_count(h, g, n_tiles, d_count, s));
  CUDA_TRY(launch_scan(d_count, d_off, ncnt, d_tmp, s));
  long nb = (ncnt + 1023) / 1024;
  if (nb < 1) nb = 1;
  long long total = 0;
  CUDA_TRY(cudaMemcpy(&total, d_tmp + nb, sizeof(long long), cudaMemcpyDeviceToHost));
  if (total > 2000000000LL) throw Fail{ETDM_ERR_INVALID_ARG, "truncation lists too long"};
  *n_entries = (long)total;
  *d_keys = dalloc<int>(h, total);
  *d_ptr = dalloc<int>(h, n_tiles + 1);
  CUDA_TRY(launch_list_fill(h, g, n_tiles, d_off, *d_keys, s));
  extract_ptr_kernel<<<(n_tiles + 256) / 256, 256, 0, s>>>(d_off, total, M, n_tiles, *d_ptr);
  CUDA_TRY(cudaGetLastError());
  std::vector<int> ptr(n_tiles + 1);
  CUDA_TRY(cudaMemcpy(ptr.data(), *d_ptr, (n_tiles + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  *max_list = 0;
  for (int t = 0; t < n_tiles; ++t) *max_list = std::max(*max_list, ptr[t + 1] - ptr[t]);
  if (*max_list > limit)
    throw Fail{ETDM_ERR_INVALID_ARG,
               "a " + std::to_string(g.tx) + "x" + std::to_string(g.ty) + "x" +
                   std::to_string(g.tz) + " grid tile touches " + std::to_string(*max_list) +
                   " function images (limit " + std::to_string(limit) +
                   "): use a finer grid or shorter truncation radii"};
}

}  // namespace

// V groups of a mixed-precision handle: greedy runs of at most vg_max
// consecutive 4x4x8 tiles whose function lists have a union of at most 128
// functions, their tables and X^T slices (built on the device).  A rebuild
// frees the previous group arrays.
void etdm::build_vgroups(etdm_handle *h, int vg_max, cudaStream_t s) {
  const int T = h->n_tiles_tc;
  const std::vector<int> &tmu = h->h_tmu, &mu_off = h->h_mu_off;
  for (void *p : {(void *)h->d_vg_t0, (void *)h->d_vg_nu, (void *)h->d_vg_eoff,
                  (void *)h->d_vg_xoff, (void *)h->d_vg_mu, (void *)h->d_xv, (void *)h->d_vent})
    dfree(h, p);
  std::vector<int> vg_t0, vg_nu, vg_eoff(1, 0), vg_xoff(1, 0), vg_mu;
  std::vector<int> un, tmp;
  long xkb = 0;
  for (int t = 0; t < T;) {
    un.assign(tmu.begin() + mu_off[t], tmu.begin() + mu_off[t + 1]);
    int nt = 1;
    while (nt < std::min(vg_max, tc_group_max()) && t + nt < T) {
      tmp.clear();
      std::set_union(un.begin(), un.end(), tmu.begin() + mu_off[t + nt],
                     tmu.begin() + mu_off[t + nt + 1], std::back_inserter(tmp));
      if ((int)tmp.size() > tc_max_list()) break;
      un.swap(tmp);
      ++nt;
    }
    const int np = tc_v_entries((int)un.size());
    vg_t0.push_back(t);
    vg_nu.push_back((int)un.size());
    vg_mu.insert(vg_mu.end(), un.begin(), un.end());
    vg_mu.resize(vg_mu.size() + (np - un.size()), 0);
    vg_eoff.push_back((int)vg_mu.size());
    xkb += (long)np * nt * tc_v_slices();  // 256-byte units: 8 K steps x 32 B per slice
    if (xkb > INT32_MAX) throw Fail{ETDM_ERR_INVALID_ARG, "grid too large for the mixed path"};
    vg_xoff.push_back((int)xkb);
    t += nt;
  }
  vg_t0.push_back(T);
  h->vg_max = vg_max;
  h->n_vg = (int)vg_nu.size();
  h->xv_entries = vg_eoff.back();
  h->h_vg_t0 = vg_t0;
  h->h_vg_eoff = vg_eoff;
  h->h_vg_nu = vg_nu;
  h->h_vg_xoff = vg_xoff;
  h->d_vg_t0 = dupload(h, vg_t0.data(), vg_t0.size());
  h->d_vg_nu = dupload(h, vg_nu.data(), std::max<size_t>(vg_nu.size(), 1));
  h->d_vg_eoff = dupload(h, vg_eoff.data(), vg_eoff.size());
  h->d_vg_xoff = dupload(h, vg_xoff.data(), vg_xoff.size());
  h->d_vg_mu = dupload(h, vg_mu.data(), std::max<size_t>(vg_mu.size(), 1));
  h->d_xv = dalloc<uint8_t>(h, (size_t)vg_xoff.back() * 256);
  h->d_vent = dalloc<float4>(h, std::max<size_t>(vg_mu.size(), 1));
  CUDA_TRY(launch_xv_build(h, s));
}

// L-BFGS memory, line-search buffers and reduction scratch for h->nvar
// variables (both parametrizations).
void etdm::alloc_opt_buffers(etdm_handle *h) {
  int bpl = 0;
  if (occupancy_lbfgs(&bpl) != 0 || bpl < 1)
    throw Fail{ETDM_ERR_CUDA, "cannot size the cooperative L-BFGS kernel"};
  const long nvar = h->nvar;
  // L-BFGS: one block for small n (the grid barrier is then a block barrier);
  // else every SM, so the FP64 work per SM stays small (FP64 is the scarce
  // pipe), at most two elements per thread up to water32
  h->lb_blocks = nvar <= 512 ? 1
                             : (int)std::min<long>((long)h->num_sms * std::min(bpl, 2),
                                                   std::max<long>(h->num_sms, (nvar + 511) / 512));
  h->d_red = dalloc<double>(h, 4 * std::max(h->coop_blocks, h->lb_blocks) + 8);
  h->d_s = dalloc<double>(h, (long)h->lbfgs_m * nvar);
  h->d_y = dalloc<double>(h, (long)h->lbfgs_m * nvar);
  h->d_aprev = dalloc<double>(h, nvar);
  h->d_gprev = dalloc<double>(h, nvar);
  h->d_q = dalloc<double>(h, nvar);
  h->d_lbstate = dalloc<double>(h, 4 + 2 * 16);
  h->d_a = dalloc<double>(h, nvar);
  h->d_g = dalloc<double>(h, nvar);
  h->d_at = dalloc<double>(h, nvar);
  h->d_gt = dalloc<double>(h, nvar);
  h->d_p = dalloc<double>(h, nvar);
  h->d_dot = dalloc<double>(h, 4);
  h->d_dotpart = dalloc<double>(h, kDotBlocks);
  CUDA_TRY(cudaMallocHost(&h->h_pinned, 16 * sizeof(double)));  // [0, 8) values, [8, 16) status words
}

namespace {

void init_impl(etdm_handle *h, const etdm_system *sys, const etdm_options *opt) {
  validate(sys, opt);
  etdm_options o;
  etdm_default_options(&o);
  if (opt) o = *opt;
  h->device = o.device;
  h->precision = o.precision;
  h->lbfgs_m = o.lbfgs_m;
  h->gamma = o.gamma;
  h->beta0 = o.beta0;
  h->kpath = sys->n_k >= 1 || o.param == ETDM_PARAM_FULL;
  if (h->kpath) {
    h->nk = sys->n_k >= 1 ? sys->n_k : 1;
    h->h_kfrac.assign(3 * h->nk, 0.0);
    h->h_kw.assign(h->nk, 1.0);
    if (sys->n_k >= 1) {
      h->h_kfrac.assign(sys->k_frac, sys->k_frac + 3 * h->nk);
      h->h_kw.assign(sys->k_w, sys->k_w + h->nk);
    }
    h->kT = sys->kT;
    h->n_elec = sys->n_electrons;
    h->kexpm = o.expm;
    h->ref_every = o.ref_update;
    h->sic = o.functional == ETDM_FUNC_PZSIC;
  }
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (o.device < 0 || o.device >= ndev) throw Fail{ETDM_ERR_INVALID_ARG, "no such CUDA device"};
  CUDA_TRY(cudaSetDevice(o.device));
  CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, o.device));
  int coop = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, o.device));
  if (!coop) throw Fail{ETDM_ERR_CUDA, "device does not support cooperative launch"};

  const int M = sys->n_basis;
  h->M = M;
  h->N = sys->n_electrons / 2;
  h->V = M - h->N;
  h->n_atoms = sys->n_atoms;
  for (int a = 0; a < 3; ++a) {
    h->n[a] = sys->grid[a];
    h->L[a] = sys->box[a];
    h->h[a] = sys->box[a] / sys->grid[a];
  }
  h->G = (long)h->n[0] * h->n[1] * h->n[2];
  h->dV = h->h[0] * h->h[1] * h->h[2];
  h->omega = h->L[0] * h->L[1] * h->L[2];
  h->sigma = sys->ion_sigma;
  cudaStream_t s = 0;

  // system arrays
  std::vector<double> center(3 * M), alpha(M), norm(M), rcut(M), rc2(M);
  for (int m = 0; m < M; ++m) {
    int at = sys->bf_atom[m];
    for (int a = 0; a < 3; ++a) center[3 * m + a] = sys->pos[3 * at + a];
    alpha[m] = sys->bf_exp[m];
    norm[m] = pow(2.0 * alpha[m] / M_PI, 0.75);
    rcut[m] = sys->bf_rcut[m];
    rc2[m] = rcut[m] * rcut[m];
  }
  h->d_center = dalloc<double>(h, 3 * M);
  h->d_alpha = dalloc<double>(h, M);
  h->d_norm = dalloc<double>(h, M);
  h->d_rcut = dalloc<double>(h, M);
  h->d_rc2 = dalloc<double>(h, M);
  h->d_pos = dalloc<double>(h, 3 * sys->n_atoms);
  h->d_Z = dalloc<double>(h, sys->n_atoms);
  CUDA_TRY(cudaMemcpy(h->d_center, center.data(), 3 * M * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(h->d_alpha, alpha.data(), M * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(h->d_norm, norm.data(), M * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(h->d_rcut, rcut.data(), M * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(h->d_rc2, rc2.data(), M * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(h->d_pos, sys->pos, 3 * sys->n_atoms * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(h->d_Z, sys->Z, sys->n_atoms * 8, cudaMemcpyHostToDevice));

  // basis tables
  long tab = 0;
  for (int a = 0; a < 3; ++a) {
    h->tab_off[a] = tab;
    tab += (long)M * kImgN * h->n[a];
  }
  h->d_sq = dalloc<double>(h, tab);
  h->d_ex = dalloc<double>(h, tab);
  CUDA_TRY(launch_tables(h, s));

  // tiles and truncation lists (4^3 tiles for the FP64 passes)
  h->geom = make_geom(h, 4, 4, 4, &h->n_tiles);
  build_lists(h, h->geom, h->n_tiles, &h->d_tile_ptr, &h->d_keys, &h->n_entries, &h->max_list,
              kMaxList, s);
  if (h->precision == ETDM_PREC_MIXED) {  // 4 x 4 x 8 tiles for the tensor-core passes
    h->geom_tc = make_geom(h, 4, 4, 8, &h->n_tiles_tc);
    build_lists(h, h->geom_tc, h->n_tiles_tc, &h->d_tile_ptr_tc, &h->d_keys_tc,
                &h->n_entries_tc, &h->max_list_tc, tc_max_list(), s);
    h->d_tabf = dalloc<float4>(h, tab);
    CUDA_TRY(launch_tables_f32(h, s));
    std::vector<float> rc2f(M);
    for (int m = 0; m < M; ++m) rc2f[m] = (float)rc2[m];
    h->d_rc2f = dalloc<float>(h, M);
    CUDA_TRY(cudaMemcpy(h->d_rc2f, rc2f.data(), M * sizeof(float), cudaMemcpyHostToDevice));
    h->d_rowexp = dalloc<signed char>(h, h->G);
    // functions per tile (ascending: the image lists are sorted by key), the
    // density's K steps per tile, and the V groups: greedy runs of consecutive
    // tiles whose function lists have a union of at most tc_max_list() functions
    const int T = h->n_tiles_tc;
    h->d_nu_tc = dalloc<int>(h, std::max(T, 1));
    CUDA_TRY(launch_count_unique(h, h->d_nu_tc, s));
    std::vector<int> tptr(T + 1), keys(h->n_entries_tc);
    CUDA_TRY(cudaMemcpy(tptr.data(), h->d_tile_ptr_tc, (T + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    if (h->n_entries_tc > 0)
      CUDA_TRY(cudaMemcpy(keys.data(), h->d_keys_tc, h->n_entries_tc * sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<int> mu_off(T + 1, 0), tmu, xr_off(T + 1, 0);
    long xr = 0;
    for (int t = 0; t < T; ++t) {
      mu_off[t] = (int)tmu.size();
      for (int e = tptr[t]; e < tptr[t + 1]; ++e) {
        const int mu = keys[e] >> 9;
        if (e == tptr[t] || mu != tmu.back()) tmu.push_back(mu);
      }
      xr_off[t] = (int)xr;
      xr += tc_rho_steps((int)tmu.size() - mu_off[t]);
      if (xr > INT32_MAX) throw Fail{ETDM_ERR_INVALID_ARG, "grid too large for the mixed path"};
    }
    mu_off[T] = (int)tmu.size();
    xr_off[T] = (int)xr;
    h->xr_steps = xr;
    h->h_xr_off = xr_off;
    h->h_mu_off = mu_off;
    h->h_tmu = tmu;
    h->d_xr_off = dupload(h, xr_off.data(), xr_off.size());
    h->d_mu_off = dupload(h, mu_off.data(), mu_off.size());
    h->d_tmu = dupload(h, tmu.data(), std::max<size_t>(tmu.size(), 1));
    h->d_xr = dalloc<uint8_t>(h, (size_t)xr * 16384);              // 4 slices x 4 KB per K step
    h->d_vt = dalloc<float2>(h, (size_t)T * 128);
    CUDA_TRY(launch_xr_build(h, s));
    h->vg_max = (o.vgroup > 0) ? o.vgroup : 2;
    etdm::build_vgroups(h, h->vg_max, s);
    h->d_Osl = dalloc<uint2>(h, osl_elems(M, h->N));  // [chunk][M][osl_width(N)]
    const long ch = tc_max_list();  // orbitals per chunk of the density pass
    const long nsc = (h->N + ch - 1) / ch * ch;  // whole chunks, zero beyond N
    h->d_oscale = dalloc<float>(h, nsc);
    CUDA_TRY(cudaMemset(h->d_oscale, 0, nsc * sizeof(float)));
    h->d_dO = dalloc<double>(h, (long)M * h->N);
    h->d_TO = dalloc<double>(h, (long)M * h->N);
    h->d_Vfix = dalloc<unsigned long long>(h, (long)M * M + 1);
    h->d_Vfin = dalloc<float2>(h, (long)M * M);
    const long half = (long)h->n[0] * h->n[1] * (h->n[2] / 2 + 1);
    h->d_twf = dalloc<float4>(h, h->n[0] + h->n[1] + h->n[2]);
    h->d_half = dalloc<float4>(h, half);
    h->d_rhof = dalloc<float2>(h, h->G);
    h->d_vextf = dalloc<float2>(h, h->G);
    h->d_kpois = dalloc<float2>(h, half);
  }
  {
    unsigned long long *d_sum = dalloc<unsigned long long>(h, 1);
    CUDA_TRY(launch_npt2(h, d_sum, s));
    unsigned long long v = 0;
    CUDA_TRY(cudaMemcpy(&v, d_sum, 8, cudaMemcpyDeviceToHost));
    h->sum_npt2 = (long long)v;
  }

  // analytic S, T
  const long MM = (long)M * M;
  h->d_S = dalloc<double>(h, MM);
  h->d_T = dalloc<double>(h, MM);
  h->d_C0 = dalloc<double>(h, MM);
  CUDA_TRY(launch_overlap_kinetic(h, s));

  // grid buffers and v_ext
  h->d_vext = dalloc<double>(h, h->G);
  h->d_rho = dalloc<double>(h, h->G);
  h->d_vtot = dalloc<double>(h, h->G);
  h->d_fft = dalloc<double2>(h, h->G);
  h->d_tw = dalloc<double2>(h, h->n[0] + h->n[1] + h->n[2]);
  h->n_gridpart = kPotBlocks;
  h->d_gridpart = dalloc<double>(h, 3 * std::max(kPotBlocks, df_pot_blocks(h)));
  CUDA_TRY(launch_twiddles(h, s));
  CUDA_TRY(launch_vext_recip(h, s));
  CUDA_TRY(fft3d(h, h->d_fft, +1, s));
  CUDA_TRY(launch_real_part(h, h->d_fft, h->d_vext, s));
  if (h->precision == ETDM_PREC_MIXED) CUDA_TRY(launch_df_setup(h, s));  // twiddles, v_ext, Poisson kernel
  if (h->kpath) {  // full A over k-points: its own matrices and reference
    h->d_E = dalloc<double>(h, 2);
    h->d_eterms = dalloc<double>(h, 4);
    h->d_flags = dalloc<int>(h, FLAG_NFLAGS);
    h->d_bar = dalloc<unsigned>(h, 4);
    h->coop_blocks = 1;
    init_kpoints(h, sys);
    return;
  }

  // dense workspaces
  const int N = h->N, V = h->V;
  const long NN = (long)N * N;
  h->d_D = dalloc<double>(h, MM);
  h->d_H = dalloc<double>(h, MM);
  h->d_Uocc = dalloc<double>(h, (long)M * N);
  h->d_O = dalloc<double>(h, (long)M * N);
  h->d_P = dalloc<double>(h, NN);
  h->d_Qk = dalloc<double>(h, NN * 12);  // series workspace (Paterson-Stockmeyer)
  h->d_Wr = dalloc<double>(h, NN * 11);  // its reverse workspace
  h->d_Kt = dalloc<double>(h, NN * (kJmax + 1));
  h->d_St = dalloc<double>(h, NN * (kJmax + 1));
  h->d_Gbar = dalloc<double>(h, (long)M * N);
  h->d_Ubar = dalloc<double>(h, (long)M * N);
  for (int i = 0; i < 4; ++i) h->d_bar2[i] = dalloc<double>(h, NN);
  h->d_Abar = dalloc<double>(h, (long)N * V);
  h->d_E = dalloc<double>(h, 2);
  h->d_eterms = dalloc<double>(h, 4);
  h->d_scal = dalloc<double>(h, 4);
  h->d_flags = dalloc<int>(h, FLAG_NFLAGS);
  h->d_bar = dalloc<unsigned>(h, 4);
  h->d_eps = dalloc<double>(h, M);
  int bps = 0;
  if (occupancy_dense(&bps) != 0 || bps < 1)
    throw Fail{ETDM_ERR_CUDA, "cannot size the cooperative dense kernels"};
  // the dense chains' grid: as many blocks as the largest product has 8 x 16
  // output tiles (every SM at water32); one block for small systems, where a
  // grid barrier is then a block barrier
  {
    auto tiles = [](long m, long n) { return ((m + 7) / 8) * ((n + 15) / 16); };
    const long mt = std::max({tiles(N, N), tiles(N, V), tiles(V, N), tiles(M, N), tiles(M, M)});
    h->coop_blocks = mt <= 8 ? 1 : (int)std::min<long>(h->num_sms, mt);
    if (o.dense_blocks > 0) {
      if (o.dense_blocks > bps * h->num_sms)
        throw Fail{ETDM_ERR_INVALID_ARG, "dense_blocks exceeds the co-resident limit (" +
                                             std::to_string(bps * h->num_sms) + ")"};
      h->coop_blocks = o.dense_blocks;
    }
  }
  // tensor-core products of the float-pair chains: every product (dense_tc 1),
  // or those of at least 2^26 multiply-adds (0) when the system has one
  if (h->precision == ETDM_PREC_MIXED && o.dense_tc >= 0) {
    const long long big = std::max<long long>((long long)M * M * N, (long long)N * N * std::max(N, V));
    const long long min_work = o.dense_tc == 1 ? 1 : (1LL << 26);
    if (big >= min_work) {
      int bt = 0;
      if (occupancy_dense_tc(&bt) != 0 || bt < 1)
        throw Fail{ETDM_ERR_CUDA, "cannot size the tensor-core dense kernels"};
      h->dense_tc = true;
      h->tc_min_work = min_work;
      h->coop_blocks = std::min(h->coop_blocks, bt * h->num_sms);
      h->d_tc_asl = dalloc<uint8_t>(h, dense_tc_asl_bytes(M));
      h->d_tc_bsl = dalloc<uint8_t>(h, dense_tc_bsl_bytes(M));
      h->d_tc_rexp = dalloc<int>(h, (size_t)M + 128);
      h->d_tc_cexp = dalloc<int>(h, (size_t)M + 128);
    }
  }
  h->nvar = (long)N * V;
  etdm::alloc_opt_buffers(h);

  // reference orbitals: Loewdin S^(-1/2), columns by ascending diag of C0^T h_core C0
  inverse_sqrt(h, s);
  CUDA_TRY(cudaMemcpyAsync(h->d_H, h->d_T, MM * 8, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(launch_vmat_fp64(h, h->d_vext, h->d_H, s));
  symmetrize_upper_kernel<<<256, 256, 0, s>>>(h->d_H, M);
  CUDA_TRY(cudaGetLastError());
  double *d_diag = dalloc<double>(h, M);
  CUDA_TRY(launch_diag_quad(h->d_C0, h->d_H, d_diag, M, s));
  std::vector<double> diag(M);
  CUDA_TRY(cudaMemcpy(diag.data(), d_diag, M * 8, cudaMemcpyDeviceToHost));
  for (double v : diag)
    if (!std::isfinite(v)) throw Fail{ETDM_ERR_NUMERIC, "h_core diagonal is not finite"};
  h->order.resize(M);
  std::iota(h->order.begin(), h->order.end(), 0);
  std::stable_sort(h->order.begin(), h->order.end(),
                   [&](int x, int y) { return diag[x] < diag[y]; });
  int *d_perm = dalloc<int>(h, M);
  CUDA_TRY(cudaMemcpy(d_perm, h->order.data(), M * sizeof(int), cudaMemcpyHostToDevice));
  double *d_tmpC = dalloc<double>(h, MM);
  CUDA_TRY(cudaMemcpyAsync(d_tmpC, h->d_C0, MM * 8, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(launch_permute_cols(d_tmpC, d_perm, h->d_C0, M, s));
  if (h->precision == ETDM_PREC_MIXED) {  // the mixed path's dense chains run on float pairs
    h->d_C0p = dalloc<float2>(h, MM);
    h->d_Tp = dalloc<float2>(h, MM);
    h->d_Af = dalloc<float2>(h, h->nvar);
    CUDA_TRY(launch_to_pairs(h->d_C0, h->d_C0p, MM, s));
    CUDA_TRY(launch_to_pairs(h->d_T, h->d_Tp, MM, s));
  }

  if (h->precision == ETDM_PREC_MIXED) {  // device tables of the grid stages
    const int one = 1;
    h->d_active1 = dupload(h, &one, 1);
    build_mixed_plan(h, {h}, h->d_active1, h->d_flags, false, h->d_Vfix,
                     ((size_t)M * M + 1) * sizeof(unsigned long long), &h->plan);
  }

  // orbital energies of Eq. 33 at A = 0
  CUDA_TRY(cudaMemsetAsync(h->d_a, 0, h->nvar * 8, s));
  h->in_setup = true;
  evaluate(h, h->d_a, h->d_E, h->d_g, s);
  h->in_setup = false;
  check_flags(h, s);
  CUDA_TRY(launch_diag_quad(h->d_C0, h->d_H, h->d_eps, M, s));
  std::vector<double> st(4 + 32, 0.0);
  st[3] = h->beta0;
  CUDA_TRY(cudaMemcpy(h->d_lbstate, st.data(), st.size() * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaDeviceSynchronize());
}

}  // namespace

void etdm::init_system(etdm_handle *h, const etdm_system *sys, const etdm_options *opt) {
  init_impl(h, sys, opt);
}
void etdm::eval_system(etdm_handle *h, const double *a, double *E, double *g, cudaStream_t s) {
  evaluate(h, a, E, g, s);
}
void etdm::release_handle(etdm_handle *h) { release(h); }

void etdm::set_unbound_error(const std::string &msg) { g_init_err = msg; }

// ============================== C ABI =========================================
extern "C" {

void etdm_default_options(etdm_options *opt) {
  if (!opt) return;
  opt->precision = ETDM_PREC_FP64;
  opt->lbfgs_m = 3;
  opt->gamma = 0.25;
  opt->beta0 = 1.0;
  opt->device = 0;
  opt->dense_blocks = 0;
  opt->dense_tc = 0;
  opt->param = ETDM_PARAM_OCCVIRT;
  opt->expm = ETDM_EXPM_EIG;
  opt->ref_update = 0;
  opt->vgroup = 0;
  opt->functional = ETDM_FUNC_KS;
}

int etdm_init_basis(const etdm_system *sys, const etdm_options *opt, etdm_handle **out) {
  if (!out) return set_err(nullptr, ETDM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  etdm_handle *h = new etdm_handle();
  try {
    init_impl(h, sys, opt);
  } catch (const Fail &f) {
    release(h);
    delete h;
    return set_err(nullptr, f.code, f.msg);
  }
  *out = h;
  return ETDM_OK;
}

int etdm_energy_grad(etdm_handle *h, const double *a_dev, double *E_dev, double *g_dev,
                     void *stream) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  if (!a_dev || !E_dev) return set_err(h, ETDM_ERR_INVALID_ARG, "a_dev and E_dev are required");
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    if (!h->members.empty()) batch_energy_grad(h, a_dev, E_dev, g_dev, (cudaStream_t)stream);
    else evaluate(h, a_dev, E_dev, g_dev, (cudaStream_t)stream);
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

int etdm_energy_grad_host(etdm_handle *h, const double *a_host, double *E_host,
                          double *g_host) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  if (!a_host || !E_host) return set_err(h, ETDM_ERR_INVALID_ARG, "a_host and E_host are required");
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    if (!h->members.empty()) {
      batch_energy_grad_host(h, a_host, E_host, g_host);
      return ETDM_OK;
    }
    cudaStream_t s = 0;
    const long nvar = h->nvar;
    CUDA_TRY(cudaMemcpyAsync(h->d_a, a_host, nvar * 8, cudaMemcpyHostToDevice, s));
    evaluate(h, h->d_a, h->d_E, g_host ? h->d_g : nullptr, s);
    CUDA_TRY(cudaMemcpyAsync(E_host, h->d_E, 8, cudaMemcpyDeviceToHost, s));
    if (g_host) CUDA_TRY(cudaMemcpyAsync(g_host, h->d_g, nvar * 8, cudaMemcpyDeviceToHost, s));
    check_flags(h, s);
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

int etdm_precondition(etdm_handle *h, const double *g_dev, double *pg_dev, void *stream) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  if (!g_dev || !pg_dev) return set_err(h, ETDM_ERR_INVALID_ARG, "g_dev and pg_dev are required");
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    if (!h->members.empty()) {  // per system, at its slice of the packed vectors
      for (size_t i = 0; i < h->members.size(); ++i)
        CUDA_TRY(launch_precond(h->members[i], g_dev + h->var_off[i], pg_dev + h->var_off[i],
                                (cudaStream_t)stream));
      return ETDM_OK;
    }
    CUDA_TRY(launch_precond(h, g_dev, pg_dev, (cudaStream_t)stream));
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

int etdm_lbfgs_step(etdm_handle *h, const double *a_dev, const double *g_dev, double *p_dev,
                    void *stream) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  if (!a_dev || !g_dev || !p_dev)
    return set_err(h, ETDM_ERR_INVALID_ARG, "a_dev, g_dev and p_dev are required");
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    if (!h->members.empty()) {  // per system, at its slice of the packed vectors
      for (size_t i = 0; i < h->members.size(); ++i)
        lbfgs(h->members[i], a_dev + h->var_off[i], g_dev + h->var_off[i], p_dev + h->var_off[i],
              (cudaStream_t)stream);
      return ETDM_OK;
    }
    lbfgs(h, a_dev, g_dev, p_dev, (cudaStream_t)stream);
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

int etdm_lbfgs_reset(etdm_handle *h) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  for (etdm_handle *m : h->members) {
    const int rc = etdm_lbfgs_reset(m);
    if (rc != ETDM_OK) return set_err(h, rc, m->err);
  }
  if (!h->members.empty()) return ETDM_OK;
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaDeviceSynchronize());
    double st[4];
    CUDA_TRY(cudaMemcpy(st, h->d_lbstate, sizeof(st), cudaMemcpyDeviceToHost));
    st[0] = 0.0; st[1] = 0.0; st[2] = 0.0; st[3] = h->beta0;
    CUDA_TRY(cudaMemcpy(h->d_lbstate, st, sizeof(st), cudaMemcpyHostToDevice));
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

int etdm_set_reference(etdm_handle *h, int32_t sys, const double *C0_host, const double *occ_host) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  if (!h->members.empty()) {
    if (sys < 0 || sys >= (int32_t)h->members.size())
      return set_err(h, ETDM_ERR_INVALID_ARG, "no such system");
    const int rc = etdm_set_reference(h->members[sys], 0, C0_host, occ_host);
    return rc == ETDM_OK ? rc : set_err(h, rc, h->members[sys]->err);
  }
  if (sys != 0) return set_err(h, ETDM_ERR_INVALID_ARG, "a single-system handle has system 0 only");
  if (!C0_host) return set_err(h, ETDM_ERR_INVALID_ARG, "C0 is NULL");
  if (occ_host && !h->kpath)
    return set_err(h, ETDM_ERR_INVALID_ARG, "occupations are fixed (f = 2 / 0) on the occupied-virtual path");
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaDeviceSynchronize());
    cudaStream_t s = 0;
    const long MM = (long)h->M * h->M;
    if (h->kpath) {
      const long nf = (long)h->nk * h->M;
      if (occ_host) {
        double tot = 0.0;
        for (long q = 0; q < nf; ++q) {
          if (!std::isfinite(occ_host[q]) || occ_host[q] < 0.0)
            throw Fail{ETDM_ERR_INVALID_ARG, "occupations must be finite and >= 0"};
          tot += occ_host[q];
        }
        if (fabs(tot - h->n_elec) > 1e-9 * std::max(1.0, h->n_elec))
          throw Fail{ETDM_ERR_INVALID_ARG, "occupations must sum to n_electrons"};
        CUDA_TRY(cudaMemcpy(h->d_kf, occ_host, nf * 8, cudaMemcpyHostToDevice));
      }
      CUDA_TRY(cudaMemcpy(h->d_kC0, C0_host, (size_t)h->nk * MM * 16, cudaMemcpyHostToDevice));
      refresh_reference_k(h, s);
      check_flags(h, s);
    } else {
      for (long q = 0; q < MM; ++q)
        if (!std::isfinite(C0_host[q])) throw Fail{ETDM_ERR_INVALID_ARG, "C0 must be finite"};
      CUDA_TRY(cudaMemcpy(h->d_C0, C0_host, MM * 8, cudaMemcpyHostToDevice));
      if (h->d_C0p) CUDA_TRY(launch_to_pairs(h->d_C0, h->d_C0p, MM, s));
      CUDA_TRY(cudaMemsetAsync(h->d_a, 0, h->nvar * 8, s));
      h->in_setup = true;
      evaluate(h, h->d_a, h->d_E, h->d_g, s);
      h->in_setup = false;
      check_flags(h, s);
      CUDA_TRY(launch_diag_quad(h->d_C0, h->d_H, h->d_eps, h->M, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
  } catch (const Fail &f) {
    h->in_setup = false;
    return set_err(h, f.code, f.msg);
  }
  return etdm_lbfgs_reset(h);
}

int etdm_check(etdm_handle *h, void *stream) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    if (!h->members.empty()) batch_check(h, (cudaStream_t)stream);
    else check_flags(h, (cudaStream_t)stream);
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

// n_steps ETDM iterations (tol < 0), or iterations until the Eq. 45 residual
// of the current point is at most tol (at most n_steps of them); resid_hist
// and *steps_done are then filled too.
static int minimize_impl(etdm_handle *h, double *a_dev, int32_t n_steps, double *E_hist,
                         double *alpha_hist, int32_t *trials_hist, double tol,
                         double *resid_hist, int32_t *steps_done, void *stream) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  if (!a_dev || n_steps < 0) return set_err(h, ETDM_ERR_INVALID_ARG, "bad a_dev or n_steps");
  cudaStream_t s = (cudaStream_t)stream;
  const bool conv = tol >= 0.0;
  const long nvar = h->nvar;
  double *hp = h->h_pinned;
  if (!h->members.empty()) {
    if (conv) return set_err(h, ETDM_ERR_INVALID_ARG, "the convergence test runs on one system");
    try {
      CUDA_TRY(cudaSetDevice(h->device));
      batch_minimize(h, a_dev, n_steps, E_hist, alpha_hist, trials_hist, s);
    } catch (const Fail &f) {
      return set_err(h, f.code, f.msg);
    }
    return ETDM_OK;
  }
  struct WantResid {  // the evaluations of this call compute Eq. 45 (reset on exit)
    etdm_handle *h;
    WantResid(etdm_handle *hh, bool on) : h(hh) { h->want_resid = on; }
    ~WantResid() { h->want_resid = false; }
  } want(h, conv);
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    // E and g at the start point (values read back: E, g.p, g0.p, residual)
    evaluate(h, a_dev, h->d_dot, h->d_g, s);
    CUDA_TRY(cudaMemcpyAsync(hp, h->d_dot, 4 * 8, cudaMemcpyDeviceToHost, s));
    check_flags(h, s);
    double E = hp[0], resid = hp[3];
    if (E_hist) E_hist[0] = E;
    if (alpha_hist) alpha_hist[0] = 0.0;
    if (trials_hist) trials_hist[0] = 1;
    if (resid_hist) resid_hist[0] = resid;
    int done_steps = 0;
    // phi(alpha): E(a + alpha p) and grad . p, into hp[0], hp[1]
    struct Pt { double a, E, d; };
    double last_resid = resid;  // Eq. 45 at the last point evaluated
    auto phi = [&](double alpha) -> Pt {
      CUDA_TRY(launch_axpy(a_dev, alpha, h->d_p, h->d_at, nvar, s));
      evaluate(h, h->d_at, h->d_dot, h->d_gt, s);
      CUDA_TRY(launch_dot(h->d_gt, h->d_p, nvar, h->d_dot + 1, h->d_dotpart, s));
      h->launches += 3;
      CUDA_TRY(cudaMemcpyAsync(hp, h->d_dot, 4 * 8, cudaMemcpyDeviceToHost, s));
      check_flags(h, s);
      last_resid = hp[3];
      return Pt{alpha, hp[0], hp[1]};
    };
    LineSearch ls;
    int since_update = 0;
    for (int it = 1; it <= n_steps; ++it) {
      if (conv && resid <= tol) break;
      if (h->kpath && h->kexpm == ETDM_EXPM_SS && h->ref_every != 0) {
        // reference update of Sec. 3.5 before the step: C0 <- C0 exp(A), A <- 0,
        // the L-BFGS pairs erased (beta kept), orbital energies afresh
        bool upd = false;
        if (h->ref_every > 0) {
          upd = since_update >= h->ref_every;
        } else {
          double nL = 0.0, nC = 0.0;
          commutator_norms_k(h, a_dev, h->d_g, &nL, &nC, s);
          upd = nL < 3.0 * nC;
        }
        if (upd) {
          reference_update_k(h, a_dev, s);
          CUDA_TRY(cudaMemcpyAsync(hp, h->d_E, 8, cudaMemcpyDeviceToHost, s));
          check_flags(h, s);
          E = hp[0];
          double st[3] = {0.0, 0.0, 0.0};
          CUDA_TRY(cudaMemcpy(h->d_lbstate, st, sizeof(st), cudaMemcpyHostToDevice));
          since_update = 0;
          ++h->ref_updates;
        }
      }
      ++since_update;
      lbfgs(h, a_dev, h->d_g, h->d_p, s);
      CUDA_TRY(launch_dot(h->d_g, h->d_p, nvar, h->d_dot + 2, h->d_dotpart, s));
      h->launches += 2;
      // the first trial (alpha = 1) is queued before the direction is checked:
      // one synchronization for both; discarded if p is not a descent direction
      CUDA_TRY(launch_axpy(a_dev, 1.0, h->d_p, h->d_at, nvar, s));
      evaluate(h, h->d_at, h->d_dot, h->d_gt, s);
      CUDA_TRY(launch_dot(h->d_gt, h->d_p, nvar, h->d_dot + 1, h->d_dotpart, s));
      h->launches += 3;
      CUDA_TRY(cudaMemcpyAsync(hp, h->d_dot, 4 * 8, cudaMemcpyDeviceToHost, s));
      check_flags(h, s);
      last_resid = hp[3];
      double d0 = hp[2];
      const Pt first{1.0, hp[0], hp[1]};
      const bool have_first = d0 < 0.0;
      if (!(d0 < 0.0)) {  // not a descent direction: erase memory, precondition only
        CUDA_TRY(cudaStreamSynchronize(s));
        double st[3] = {0.0, 0.0, 0.0};
        CUDA_TRY(cudaMemcpy(h->d_lbstate, st, sizeof(st), cudaMemcpyHostToDevice));
        lbfgs(h, a_dev, h->d_g, h->d_p, s);
        CUDA_TRY(launch_dot(h->d_g, h->d_p, nvar, h->d_dot + 2, h->d_dotpart, s));
        h->launches += 2;
        CUDA_TRY(cudaMemcpyAsync(hp + 2, h->d_dot + 2, 8, cudaMemcpyDeviceToHost, s));
        check_flags(h, s);
        d0 = hp[2];
      }
      ls.start(E, d0);
      if (have_first) ls.feed(first.E, first.d);
      while (!ls.done()) {  // each trial leaves its point and gradient in d_at, d_gt
        const Pt cur = phi(ls.alpha());
        ls.feed(cur.E, cur.d);
      }
      if (ls.accepted()) {  // the accepted point is the last one evaluated
        CUDA_TRY(cudaMemcpyAsync(a_dev, h->d_at, nvar * 8, cudaMemcpyDeviceToDevice, s));
        std::swap(h->d_g, h->d_gt);
        E = ls.result().E;
        resid = last_resid;
      }
      if (E_hist) E_hist[it] = E;
      if (alpha_hist) alpha_hist[it] = ls.accepted() ? ls.result().a : 0.0;
      if (trials_hist) trials_hist[it] = ls.trials();
      if (resid_hist) resid_hist[it] = resid;
      done_steps = it;
    }
    if (steps_done) *steps_done = done_steps;
    CUDA_TRY(cudaStreamSynchronize(s));
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

int etdm_minimize(etdm_handle *h, double *a_dev, int32_t n_steps, double *E_hist,
                  double *alpha_hist, int32_t *trials_hist, void *stream) {
  return minimize_impl(h, a_dev, n_steps, E_hist, alpha_hist, trials_hist, -1.0, nullptr, nullptr,
                       stream);
}

int etdm_minimize_converge(etdm_handle *h, double *a_dev, int32_t max_steps, double tol,
                           double *E_hist, double *alpha_hist, int32_t *trials_hist,
                           double *resid_hist, int32_t *steps_done, void *stream) {
  if (!(tol >= 0.0)) return set_err(h, ETDM_ERR_INVALID_ARG, "tol must be >= 0");
  if (h && h->kpath)
    return set_err(h, ETDM_ERR_INVALID_ARG, "the Eq. 45 residual is built for the occupied-virtual path");
  return minimize_impl(h, a_dev, max_steps, E_hist, alpha_hist, trials_hist, tol, resid_hist,
                       steps_done, stream);
}

int etdm_layout(const etdm_handle *h, int64_t *dims) {
  if (!h || !dims) return ETDM_ERR_INVALID_ARG;
  if (!h->members.empty()) {  // a batch: totals over the systems (maxima for M, N, V, lists)
    for (int k = 0; k < ETDM_NDIMS; ++k) dims[k] = 0;
    for (const etdm_handle *m : h->members) {
      int64_t d[ETDM_NDIMS];
      etdm_layout(m, d);
      for (int k : {0, 1, 2, 6}) dims[k] = std::max(dims[k], d[k]);
      for (int k : {3, 4, 5, 10}) dims[k] += d[k];
      for (int k : {7, 8, 9}) dims[k] = d[k];
    }
    dims[11] = h->precision;
    return ETDM_OK;
  }
  dims[0] = h->M; dims[1] = h->N; dims[2] = h->V; dims[3] = h->G;
  dims[4] = h->n_tiles; dims[5] = h->n_entries; dims[6] = h->max_list;
  dims[7] = h->geom.tx; dims[8] = h->geom.ty; dims[9] = h->geom.tz;
  dims[10] = h->sum_npt2; dims[11] = h->precision;
  return ETDM_OK;
}

int64_t etdm_array_bytes(const etdm_handle *h, int32_t which) {
  if (h && which == ETDM_ARR_TUNE) return 64;
  if (!h || !h->members.empty()) return -1;  // a batch: ask its systems (etdm_system_handle)
  const int64_t M = h->M, N = h->N;
  if (h->kpath) {  // complex [n_k][M][M] matrices, [n_k][M] vectors
    const int64_t KM = (int64_t)h->nk * M * M, KV = (int64_t)h->nk * M;
    switch (which) {
      case ETDM_ARR_S: case ETDM_ARR_T: case ETDM_ARR_C0: case ETDM_ARR_H: case ETDM_ARR_D:
        return KM * 16;
      case ETDM_ARR_EPS: case ETDM_ARR_OCC: case ETDM_ARR_EPS_REF: case ETDM_ARR_OMEGA:
        return KV * 8;
      case ETDM_ARR_ORDER: case ETDM_ARR_UOCC: case ETDM_ARR_DOUBLINGS:
        return -1;
      default: break;
    }
  } else if (which == ETDM_ARR_OCC || which == ETDM_ARR_EPS_REF || which == ETDM_ARR_OMEGA) {
    return -1;
  }
  switch (which) {
    case ETDM_ARR_S: case ETDM_ARR_T: case ETDM_ARR_C0: case ETDM_ARR_H: case ETDM_ARR_D:
      return M * M * 8;
    case ETDM_ARR_ORDER: return M * 4;
    case ETDM_ARR_VEXT: case ETDM_ARR_RHO: case ETDM_ARR_VTOT: return (int64_t)h->G * 8;
    case ETDM_ARR_UOCC: return M * N * 8;
    case ETDM_ARR_TILE_PTR: return ((int64_t)h->n_tiles + 1) * 4;
    case ETDM_ARR_TILE_KEYS: return (int64_t)h->n_entries * 4;
    case ETDM_ARR_EPS: return M * 8;
    case ETDM_ARR_ETERMS: return 32;
    case ETDM_ARR_BETA: return 8;
    case ETDM_ARR_TILE_PTR_TC: return h->d_tile_ptr_tc ? ((int64_t)h->n_tiles_tc + 1) * 4 : 0;
    case ETDM_ARR_TILE_KEYS_TC: return h->d_keys_tc ? (int64_t)h->n_entries_tc * 4 : 0;
    case ETDM_ARR_TILE_NU_TC: return h->d_nu_tc ? (int64_t)h->n_tiles_tc * 4 : 0;
    case ETDM_ARR_VGROUP_T0: return h->d_vg_t0 ? ((int64_t)h->n_vg + 1) * 4 : 0;
    case ETDM_ARR_VGROUP_NU: return h->d_vg_nu ? (int64_t)h->n_vg * 4 : 0;
    case ETDM_ARR_DOUBLINGS: return 4;
    case ETDM_ARR_STATUS: return 4 * FLAG_NFLAGS;
    default: return -1;
  }
}

int etdm_get_array(etdm_handle *h, int32_t which, void *dst, int64_t n_bytes) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  int64_t want = etdm_array_bytes(h, which);
  if (want < 0 || !dst || n_bytes != want)
    return set_err(h, ETDM_ERR_INVALID_ARG, "unknown array or wrong byte count");
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaDeviceSynchronize());
    const void *src = nullptr;
    if (which == ETDM_ARR_TUNE) {
      double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      t[0] = h->members.empty() ? h->vg_max
                                : (h->tune_choice ? h->tune_choice : h->members[0]->vg_max);
      for (size_t i = 0; i < h->tune_ms.size() && i < 6; ++i) t[1 + i] = h->tune_ms[i];
      memcpy(dst, t, sizeof(t));
      return ETDM_OK;
    }
    if (h->kpath) {
      switch (which) {
        case ETDM_ARR_S: src = h->d_kS; break;
        case ETDM_ARR_T: src = h->d_kT; break;
        case ETDM_ARR_C0: src = h->d_kC0; break;
        case ETDM_ARR_H: src = h->d_kH; break;
        case ETDM_ARR_D: src = h->d_kD; break;
        case ETDM_ARR_EPS: src = h->d_eps; break;
        case ETDM_ARR_OCC: src = h->d_kf; break;
        case ETDM_ARR_EPS_REF: src = h->d_keps0; break;
        case ETDM_ARR_OMEGA: src = h->d_komega; break;
        default: break;
      }
      if (src) {
        CUDA_TRY(cudaMemcpy(dst, src, want, cudaMemcpyDeviceToHost));
        return ETDM_OK;
      }
    }
    switch (which) {
      case ETDM_ARR_S: src = h->d_S; break;
      case ETDM_ARR_T: src = h->d_T; break;
      case ETDM_ARR_C0: src = h->d_C0; break;
      case ETDM_ARR_ORDER: memcpy(dst, h->order.data(), want); return ETDM_OK;
      case ETDM_ARR_VEXT: src = h->d_vext; break;
      case ETDM_ARR_RHO: src = h->d_rho; break;
      case ETDM_ARR_VTOT: src = h->d_vtot; break;
      case ETDM_ARR_H: case ETDM_ARR_UOCC:
        src = which == ETDM_ARR_H ? h->d_H : h->d_Uocc;
        if (h->pairs_last) {  // the mixed path's dense chains hold float pairs
          // (its H is V, kept as the upper triangle of the fixed-point read-out)
          const bool hv = which == ETDM_ARR_H;
          double *tmp = nullptr;
          CUDA_TRY(cudaMalloc(&tmp, want));
          cudaError_t e = launch_from_pairs(hv ? h->d_Vfin : static_cast<const float2 *>(src), tmp,
                                            want / 8, 0);
          if (e == cudaSuccess) e = cudaMemcpy(dst, tmp, want, cudaMemcpyDeviceToHost);
          cudaFree(tmp);
          CUDA_TRY(e);
          if (hv) {
            double *d = static_cast<double *>(dst);
            const int64_t M = h->M;
            for (int64_t i = 1; i < M; ++i)
              for (int64_t c = 0; c < i; ++c) d[i * M + c] = d[c * M + i];
          }
          return ETDM_OK;
        }
        break;
      case ETDM_ARR_D: src = h->d_D; break;
      case ETDM_ARR_TILE_PTR: src = h->d_tile_ptr; break;
      case ETDM_ARR_TILE_KEYS: src = h->d_keys; break;
      case ETDM_ARR_EPS: src = h->d_eps; break;
      case ETDM_ARR_ETERMS: src = h->d_eterms; break;
      case ETDM_ARR_BETA: src = h->d_lbstate + 3; break;
      case ETDM_ARR_TILE_PTR_TC: src = h->d_tile_ptr_tc; break;
      case ETDM_ARR_TILE_KEYS_TC: src = h->d_keys_tc; break;
      case ETDM_ARR_TILE_NU_TC: src = h->d_nu_tc; break;
      case ETDM_ARR_VGROUP_T0: src = h->d_vg_t0; break;
      case ETDM_ARR_VGROUP_NU: src = h->d_vg_nu; break;
      case ETDM_ARR_DOUBLINGS: src = h->d_flags + FLAG_J; break;
      case ETDM_ARR_STATUS: src = h->d_flags; break;
    }
    if (want > 0) CUDA_TRY(cudaMemcpy(dst, src, want, cudaMemcpyDeviceToHost));
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

int etdm_set_profiling(etdm_handle *h, int on) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  h->profiling = on != 0;
  return ETDM_OK;
}

int etdm_stage_times(etdm_handle *h, double *ms, int64_t *counts) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaDeviceSynchronize());
    for (auto &pe : h->prof_events) {
      float t = 0.0f;
      CUDA_TRY(cudaEventElapsedTime(&t, pe.second.first, pe.second.second));
      h->stage_ms[pe.first] += t;
      h->stage_n[pe.first] += 1;
      cudaEventDestroy(pe.second.first);
      cudaEventDestroy(pe.second.second);
    }
    h->prof_events.clear();
    for (int i = 0; i < ETDM_NSTAGES; ++i) {
      if (ms) ms[i] = h->stage_ms[i];
      if (counts) counts[i] = h->stage_n[i];
      h->stage_ms[i] = 0.0;
      h->stage_n[i] = 0;
    }
    if (counts) counts[ETDM_NSTAGES - 1] = h->launches;
    h->launches = 0;
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

int etdm_pair_gemm(const double *A_dev, const double *B_dev, double *C_dev, int32_t m,
                   int32_t n, int32_t k, int32_t ta, int32_t tb, void *stream) {
  if (!A_dev || !B_dev || !C_dev || m < 1 || n < 1 || k < 1 || m > (1 << 16) || n > (1 << 16) ||
      k > (1 << 16))
    return set_err(nullptr, ETDM_ERR_INVALID_ARG, "need A, B, C and 1 <= m, n, k <= 65536");
  cudaStream_t s = (cudaStream_t)stream;
  etdm_handle scratch;  // owns the workspace of this call
  try {
    int dev = 0, sms = 0, bps = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (occupancy_dense_tc(&bps) != 0 || bps < 1)
      throw Fail{ETDM_ERR_CUDA, "cannot size the tensor-core product kernel"};
    const long big = std::max({(long)m, (long)n, (long)k});
    uint8_t *asl = dalloc<uint8_t>(&scratch, dense_tc_asl_bytes(big));
    uint8_t *bsl = dalloc<uint8_t>(&scratch, dense_tc_bsl_bytes(big));
    int *rexp = dalloc<int>(&scratch, big + 128), *cexp = dalloc<int>(&scratch, big + 128);
    unsigned *bar = dalloc<unsigned>(&scratch, 4);
    int *flags = dalloc<int>(&scratch, FLAG_NFLAGS);
    const long tiles = ((m + 127) / 128) * (long)((n + 63) / 64);
    const int blocks = (int)std::max<long>(1, std::min<long>(tiles, (long)sms * bps));
    CUDA_TRY(launch_pair_gemm(A_dev, B_dev, C_dev, m, n, k, ta, tb, asl, bsl, rexp, cexp, bar, flags,
                              blocks, s));
    int w[FLAG_NFLAGS];
    CUDA_TRY(cudaMemcpyAsync(w, flags, sizeof(w), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (w[FLAG_ERR] != 0)
      throw Fail{w[FLAG_ERR], "tensor-core product: device status " + std::to_string(w[FLAG_ERR]) +
                                  ", wait " + std::to_string(w[2]) + " gave up at count " +
                                  std::to_string(w[3])};
  } catch (const Fail &f) {
    release(&scratch);
    return set_err(nullptr, f.code, f.msg);
  }
  release(&scratch);
  return ETDM_OK;
}

int etdm_init_batch(const etdm_system *sys, int32_t n_sys, const etdm_options *opt,
                    etdm_handle **out) {
  if (!out) return set_err(nullptr, ETDM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!sys || n_sys < 1) return set_err(nullptr, ETDM_ERR_INVALID_ARG, "need n_sys >= 1 systems");
  etdm_handle *h = new etdm_handle();
  try {
    if (opt) validate(sys, opt);
    if (opt && opt->param != ETDM_PARAM_OCCVIRT)
      throw Fail{ETDM_ERR_INVALID_ARG, "batches take occupied-virtual Gamma-point systems"};
    for (int i = 0; sys && i < n_sys; ++i)
      if (sys[i].n_k != 0)
        throw Fail{ETDM_ERR_INVALID_ARG, "batches take Gamma-point systems (n_k = 0)"};
    init_batch(h, sys, n_sys, opt);
  } catch (const Fail &f) {
    release(h);
    delete h;
    return set_err(nullptr, f.code, f.msg);
  }
  *out = h;
  return ETDM_OK;
}

int32_t etdm_num_systems(const etdm_handle *h) {
  if (!h) return 0;
  return h->members.empty() ? 1 : (int32_t)h->members.size();
}

int etdm_system_layout(const etdm_handle *h, int32_t sys, int64_t *offset, int64_t *len) {
  if (!h || !offset || !len) return ETDM_ERR_INVALID_ARG;
  if (h->members.empty()) {
    if (sys != 0) return ETDM_ERR_INVALID_ARG;
    *offset = 0;
    *len = (int64_t)h->nvar;
    return ETDM_OK;
  }
  if (sys < 0 || sys >= (int32_t)h->members.size()) return ETDM_ERR_INVALID_ARG;
  *offset = h->var_off[sys];
  *len = h->var_off[sys + 1] - h->var_off[sys];
  return ETDM_OK;
}

etdm_handle *etdm_system_handle(etdm_handle *h, int32_t sys) {
  if (!h) return nullptr;
  if (h->members.empty()) return sys == 0 ? h : nullptr;
  if (sys < 0 || sys >= (int32_t)h->members.size()) return nullptr;
  return h->members[sys];
}

int etdm_set_active(etdm_handle *h, const int32_t *active_host) {
  if (!h) return set_err(nullptr, ETDM_ERR_STATE, "handle is NULL");
  if (h->members.empty() || !active_host)
    return set_err(h, ETDM_ERR_INVALID_ARG, "a batch handle and a mask are required");
  try {
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaDeviceSynchronize());
    std::vector<int> m(h->members.size());
    for (size_t i = 0; i < m.size(); ++i) m[i] = active_host[i] != 0;
    CUDA_TRY(cudaMemcpy(h->d_act, m.data(), m.size() * sizeof(int), cudaMemcpyHostToDevice));
    h->act_host = m;
  } catch (const Fail &f) {
    return set_err(h, f.code, f.msg);
  }
  return ETDM_OK;
}

const char *etdm_last_error(const etdm_handle *h) {
  return h ? h->err.c_str() : g_init_err.c_str();
}

void etdm_free(etdm_handle *h) {
  if (!h) return;
  release(h);
  delete h;
}

}  // extern "C"
