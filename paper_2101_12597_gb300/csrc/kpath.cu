// Set-up and one energy + gradient evaluation of the full-A path over
// k-points (Sec. 2-3 with fractional occupation), all on the device, FP64.
//
// Evaluation (per k-point, the k-points batched in every launch):
//   iA(k) from the variables (Eq. 22-24)      -> eigendecomposition iA = W Omega W^dagger
//   U = W exp(-i Omega) W^dagger (Eq. 35)     -> O = C0 U (Eq. 7) -> D = O f O^dagger (Eq. 12)
//   DR[R] = Re sum_k exp(2 pi i k.R) D(k)     -> rho on the grid (Eq. 2), potential and energy (Eq. 1)
//   VR[R] from v on the grid                   -> H(k) = T(k) + sum_R exp(-2 pi i k.R) VR[R] (Eq. 11)
//   L = [F, O^dagger H O] (Eq. 13)             -> G^T = W ((W^dagger L W) o Dt) W^dagger (Eq. 39-40)
//   dE/da = (2 - d_ij)/2 G (Eq. 41), real variables by Eq. 20.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "host.h"
#include "kpoint.h"

namespace etdm {

namespace {

void check_device_status(etdm_handle *h, cudaStream_t s, const char *where) {
  int f[FLAG_NFLAGS];
  CUDA_TRY(cudaStreamSynchronize(s));
  CUDA_TRY(cudaMemcpy(f, h->d_flags, sizeof(f), cudaMemcpyDeviceToHost));
  if (f[FLAG_ERR] == 0) return;
  const int code = f[FLAG_ERR];
  const int zero = 0;
  CUDA_TRY(cudaMemcpy(h->d_flags + FLAG_ERR, &zero, sizeof(int), cudaMemcpyHostToDevice));
  if (code == ETDM_ERR_NOT_CONVERGED)
    throw Fail{code, std::string(where) + ": the Hermitian eigensolver did not converge"};
  throw Fail{code, std::string(where) + ": S(k) not positive definite or a non-finite value"};
}

}  // namespace

void init_kpoints(etdm_handle *h, const etdm_system *sys) {
  cudaStream_t s = 0;
  const int M = h->M, nk = h->nk;
  const long MM = (long)M * M, KM = (long)nk * MM;
  double rmax = 0.0;
  for (int m = 0; m < M; ++m) rmax = std::max(rmax, sys->bf_rcut[m]);
  KGeom &G = h->kg;
  G.nk = nk;
  G.M = M;
  G.nR = 1;
  for (int a = 0; a < 3; ++a) {
    G.Rm[a] = std::min(2 * kImgMax, (int)floor(2.0 * rmax / h->L[a]) + 1);
    G.nR *= 2 * G.Rm[a] + 1;
  }
  h->d_kfrac = dupload(h, h->h_kfrac.data(), 3 * (size_t)nk);
  h->d_kw = dupload(h, h->h_kw.data(), (size_t)nk);
  G.kfrac = h->d_kfrac;
  h->N = sys->n_electrons / 2;
  h->V = M - h->N;
  h->nvar = KM;
  for (double2 **p : {&h->d_kS, &h->d_kT, &h->d_kC0, &h->d_kW, &h->d_kO, &h->d_kD, &h->d_kH,
                      &h->d_kX1, &h->d_kX2})
    *p = dalloc<double2>(h, KM);
  h->d_kf = dalloc<double>(h, nk * (size_t)M);
  h->d_keps0 = dalloc<double>(h, nk * (size_t)M);
  h->d_komega = dalloc<double>(h, nk * (size_t)M);
  h->d_eps = dalloc<double>(h, nk * (size_t)M);
  h->d_kDR = dalloc<double>(h, (size_t)G.nR * MM);
  h->d_kVR = dalloc<double>(h, (size_t)G.nR * MM);
  h->d_kwork = dalloc<unsigned char>(h, heev_work_bytes(M, nk));
  h->d_kpart = dalloc<double>(h, k_kinetic_parts());
  h->d_scal = dalloc<double>(h, 4);
  alloc_opt_buffers(h);
  h->d_kpden = dalloc<double>(h, h->nvar);
  h->d_kpw = dalloc<double>(h, h->nvar);
  if (h->sic) {
    for (double2 **p : {&h->d_sicD, &h->d_sicV, &h->d_sicS}) *p = dalloc<double2>(h, MM);
    h->d_sicX = dalloc<double2>(h, M);
    h->d_sicn = dalloc<double>(h, h->G);
    h->d_sicv = dalloc<double>(h, h->G);
    h->d_sicpart = dalloc<double>(h, (size_t)std::max(h->N, 1) * k_sic_parts());
  }
  if (h->kexpm == ETDM_EXPM_SS) {
    for (double2 **p : {&h->d_kB, &h->d_kB2, &h->d_kB3}) *p = dalloc<double2>(h, KM);
    h->d_knorm = dalloc<unsigned long long>(h, 1);
    h->d_kfro = dalloc<double>(h, 2 * k_fro2_parts());
  }

  // S(k), T(k); h_core(k) = T(k) + V_ext(k)
  CUDA_TRY(k_overlap_kinetic(h, s));
  CUDA_TRY(cudaMemsetAsync(h->d_kVR, 0, (size_t)G.nR * MM * 8, s));
  CUDA_TRY(launch_vmat_k(h, h->d_vext, h->d_kVR, s));
  CUDA_TRY(k_hamiltonian(G, h->d_kT, h->d_kVR, h->d_kH, s));
  CUDA_TRY(k_hermitize(h->d_kH, nk, M, s));
  // S^(-1/2) = Q w^(-1/2) Q^dagger from the eigendecomposition of S(k)
  CUDA_TRY(cudaMemcpyAsync(h->d_kX1, h->d_kS, KM * 16, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(k_hermitize(h->d_kX1, nk, M, s));
  CUDA_TRY(launch_heev(h->d_kX1, h->d_keps0, h->d_kW, M, nk, h->d_kwork, h->d_flags, s));
  CUDA_TRY(k_colscale(h->d_kW, h->d_keps0, h->d_kX1, nk, M, 1, h->d_flags, s));
  CUDA_TRY(zgemm_sq(h->d_kX1, 0, h->d_kW, 1, h->d_kX2, M, nk, s));  // X2 = S^(-1/2)
  check_device_status(h, s, "S(k)^(-1/2)");
  // generalized eigenvectors of h_core with S: C0 = S^(-1/2) Y, Y the
  // eigenvectors of S^(-1/2) h_core S^(-1/2) (ascending eigenvalues)
  CUDA_TRY(zgemm_sq(h->d_kH, 0, h->d_kX2, 0, h->d_kX1, M, nk, s));
  CUDA_TRY(zgemm_sq(h->d_kX2, 0, h->d_kX1, 0, h->d_kO, M, nk, s));
  CUDA_TRY(k_hermitize(h->d_kO, nk, M, s));
  CUDA_TRY(launch_heev(h->d_kO, h->d_keps0, h->d_kW, M, nk, h->d_kwork, h->d_flags, s));
  CUDA_TRY(zgemm_sq(h->d_kX2, 0, h->d_kW, 0, h->d_kC0, M, nk, s));
  CUDA_TRY(k_occupation(h->d_keps0, h->d_kw, nk, M, h->n_elec, h->kT, h->d_kf, h->d_scal, s));
  check_device_status(h, s, "reference orbitals");
  CUDA_TRY(cudaMemcpy(&h->mu, h->d_scal, sizeof(double), cudaMemcpyDeviceToHost));

  // orbital energies of Eq. 33 at A = 0: diag C0^dagger H C0
  refresh_reference_k(h, s);
  check_device_status(h, s, "orbital energies");
  std::vector<double> st(4 + 32, 0.0);
  st[3] = h->beta0;
  CUDA_TRY(cudaMemcpy(h->d_lbstate, st.data(), st.size() * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaDeviceSynchronize());
}

namespace {

// U = exp(A(a)) by scaling and squaring (Eq. 38): B = A / 2^s with
// |B|_1 <= 1, the degree-18 Taylor polynomial of B (truncation below
// 1 / 19! of |B|^19, under 1e-17) in Horner form in B^3 with coefficients
// c_3i I + c_3i+1 B + c_3i+2 B^2, then s squarings; only products (no solve),
// the form that keeps the work on the matrix-product engine.  The 1-norm is
// read back to size s (one synchronization).
void expm_ss_k(etdm_handle *h, const double *a, double2 *U, cudaStream_t s) {
  const int M = h->M, nk = h->nk;
  CUDA_TRY(k_build_iA(a, nk, M, h->d_kB, s, 0, 1.0));
  CUDA_TRY(k_norm1(h->d_kB, nk, M, h->d_knorm, s));
  unsigned long long bits = 0;
  CUDA_TRY(cudaMemcpyAsync(&bits, h->d_knorm, 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  double nrm;
  memcpy(&nrm, &bits, 8);
  if (!std::isfinite(nrm) || nrm > 1e9) throw Fail{ETDM_ERR_NUMERIC, "|A|_1 is not finite or too large"};
  int sq = 0;
  while (ldexp(1.0, sq) < nrm) ++sq;
  if (sq > 0) CUDA_TRY(k_build_iA(a, nk, M, h->d_kB, s, 0, ldexp(1.0, -sq)));
  CUDA_TRY(zgemm_sq(h->d_kB, 0, h->d_kB, 0, h->d_kB2, M, nk, s));   // B^2
  CUDA_TRY(zgemm_sq(h->d_kB2, 0, h->d_kB, 0, h->d_kB3, M, nk, s));  // B^3
  double c[19];
  c[0] = 1.0;
  for (int j = 1; j <= 18; ++j) c[j] = c[j - 1] / j;
  double2 *Y = h->d_kX1, *Yn = h->d_kX2;
  CUDA_TRY(k_poly(Y, h->d_kB, h->d_kB2, c[18], 0.0, 0.0, nk, M, s));  // c18 I
  for (int i = 5; i >= 0; --i) {  // Y <- q_i + B^3 Y
    CUDA_TRY(k_poly(Yn, h->d_kB, h->d_kB2, c[3 * i], c[3 * i + 1], c[3 * i + 2], nk, M, s));
    CUDA_TRY(zgemm_sq(h->d_kB3, 0, Y, 0, Yn, M, nk, s, 1.0, 1.0));
    std::swap(Y, Yn);
  }
  for (int j = 0; j < sq; ++j) {  // square s times
    CUDA_TRY(zgemm_sq(Y, 0, Y, 0, Yn, M, nk, s));
    std::swap(Y, Yn);
  }
  CUDA_TRY(cudaMemcpyAsync(U, Y, (size_t)nk * M * M * 16, cudaMemcpyDeviceToDevice, s));
  h->launches += 17 + (sq > 0 ? 1 : 0) + sq;
}

}  // namespace

// PZ-SIC (Gamma point, integer occupations): for each occupied orbital k the
// unit density n_k = |phi_k|^2 (the density pass with D = O_k O_k^dagger), its
// Hartree potential (the spectral Poisson solve) and spin-polarized exchange,
// the energy partials of -f_k (E_H[n_k] + E_x^pol[n_k]), the orbital potential
// matrix V^k (the V pass) and the column S[:, k] = O^dagger V^k O_k.
void sic_orbitals_k(etdm_handle *h, cudaStream_t s) {
  const int M = h->M;
  const KGeom &G = h->kg;
  const double fk = 2.0 * h->h_kw[0];
  for (int k = 0; k < h->N; ++k) {
    CUDA_TRY(k_rank1(h->d_kO, k, M, h->d_sicD, s));
    CUDA_TRY(k_dr(G, h->d_sicD, h->d_kDR, s));
    CUDA_TRY(launch_rho_k(h, h->d_kDR, h->d_sicn, s));
    CUDA_TRY(launch_pack_real(h, h->d_sicn, h->d_fft, s));
    CUDA_TRY(fft3d(h, h->d_fft, -1, s));
    CUDA_TRY(launch_poisson_scale(h, h->d_fft, s));
    CUDA_TRY(fft3d(h, h->d_fft, +1, s));
    CUDA_TRY(k_sic_potential(h->d_sicn, h->d_fft, h->d_sicv, h->G, h->dV, fk,
                             h->d_sicpart + (size_t)k * k_sic_parts(), s));
    CUDA_TRY(cudaMemsetAsync(h->d_kVR, 0, (size_t)G.nR * M * M * 8, s));
    CUDA_TRY(launch_vmat_k(h, h->d_sicv, h->d_kVR, s));
    CUDA_TRY(k_hamiltonian(G, nullptr, h->d_kVR, h->d_sicV, s));
    ZgemmArgs x{};  // X = V^k O_k
    x.A = h->d_sicV; x.B = h->d_kO + k; x.C = h->d_sicX;
    x.m = M; x.n = 1; x.k = M; x.lda = M; x.ldb = M; x.ldc = 1;
    x.opa = 0; x.opb = 0; x.alpha = make_double2(1.0, 0.0); x.beta = make_double2(0.0, 0.0);
    CUDA_TRY(launch_zgemm(x, 1, s));
    ZgemmArgs y{};  // S[:, k] = O^dagger X
    y.A = h->d_kO; y.B = h->d_sicX; y.C = h->d_sicS + k;
    y.m = M; y.n = 1; y.k = M; y.lda = M; y.ldb = 1; y.ldc = M;
    y.opa = 1; y.opb = 0; y.alpha = make_double2(1.0, 0.0); y.beta = make_double2(0.0, 0.0);
    CUDA_TRY(launch_zgemm(y, 1, s));
  }
  h->launches += 16L * h->N;
}

void refresh_reference_k(etdm_handle *h, cudaStream_t s) {
  const int M = h->M, nk = h->nk;
  CUDA_TRY(cudaMemsetAsync(h->d_a, 0, h->nvar * 8, s));
  evaluate_k(h, h->d_a, h->d_E, h->d_g, s);
  CUDA_TRY(zgemm_sq(h->d_kH, 0, h->d_kC0, 0, h->d_kX1, M, nk, s));
  CUDA_TRY(k_diag(h->d_kC0, h->d_kX1, h->d_eps, nk, M, s));
  CUDA_TRY(k_precond_parts(h->d_eps, h->d_kf, h->d_kw, nk, M, h->gamma, h->d_kpden, h->d_kpw, s));
}

void reference_update_k(etdm_handle *h, double *a, cudaStream_t s) {
  const int M = h->M, nk = h->nk;
  expm_ss_k(h, a, h->d_kW, s);
  CUDA_TRY(zgemm_sq(h->d_kC0, 0, h->d_kW, 0, h->d_kX1, M, nk, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_kC0, h->d_kX1, (size_t)nk * M * M * 16, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemsetAsync(a, 0, h->nvar * 8, s));
  refresh_reference_k(h, s);
}

void commutator_norms_k(etdm_handle *h, const double *a, const double *g, double *nL, double *nC,
                        cudaStream_t s) {
  const int M = h->M, nk = h->nk;
  const long KM = (long)nk * M * M;
  CUDA_TRY(k_build_iA(a, nk, M, h->d_kB, s, 0, 1.0));   // A
  CUDA_TRY(k_from_grad(g, h->d_kB2, nk, M, s));         // L
  CUDA_TRY(zgemm_sq(h->d_kB, 0, h->d_kB2, 0, h->d_kB3, M, nk, s));                  // A L
  CUDA_TRY(zgemm_sq(h->d_kB2, 0, h->d_kB, 0, h->d_kB3, M, nk, s, -1.0, 1.0));       // - L A
  CUDA_TRY(k_fro2(h->d_kB2, KM, h->d_kfro, s));
  CUDA_TRY(k_fro2(h->d_kB3, KM, h->d_kfro + k_fro2_parts(), s));
  std::vector<double> part(2 * k_fro2_parts());
  CUDA_TRY(cudaMemcpyAsync(part.data(), h->d_kfro, part.size() * 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  double l2 = 0.0, c2 = 0.0;
  for (int i = 0; i < k_fro2_parts(); ++i) {
    l2 += part[i];
    c2 += part[k_fro2_parts() + i];
  }
  *nL = sqrt(l2);
  *nC = sqrt(c2);
  h->launches += 6;
}

void evaluate_k(etdm_handle *h, const double *a, double *E, double *g, cudaStream_t s) {
  const int M = h->M, nk = h->nk;
  const long KM = (long)nk * M * M;
  const KGeom &G = h->kg;
  const bool ss = h->kexpm == ETDM_EXPM_SS;
  if (ss) {  // U = exp(A) by scaling and squaring (Eq. 38)
    StageTimer te(h, s, ETDM_STAGE_EIG);
    expm_ss_k(h, a, h->d_kW, s);
    te.done();
  } else {  // U = exp(A) through the eigendecomposition of iA (Eq. 35)
    StageTimer te(h, s, ETDM_STAGE_EIG);
    CUDA_TRY(k_build_iA(a, nk, M, h->d_kX1, s));
    CUDA_TRY(launch_heev(h->d_kX1, h->d_komega, h->d_kW, M, nk, h->d_kwork, h->d_flags, s,
                         h->tri_method));
    te.done();
  }
  StageTimer tf(h, s, ETDM_STAGE_DENSE_FWD);
  if (ss) {
    CUDA_TRY(zgemm_sq(h->d_kC0, 0, h->d_kW, 0, h->d_kO, M, nk, s));    // O = C0 U
  } else {
    CUDA_TRY(k_colscale(h->d_kW, h->d_komega, h->d_kX1, nk, M, 2, h->d_flags, s));
    CUDA_TRY(zgemm_sq(h->d_kX1, 0, h->d_kW, 1, h->d_kX2, M, nk, s));    // U
    CUDA_TRY(zgemm_sq(h->d_kC0, 0, h->d_kX2, 0, h->d_kO, M, nk, s));    // O = C0 U
  }
  CUDA_TRY(k_colscale(h->d_kO, h->d_kf, h->d_kX1, nk, M, 0, h->d_flags, s));
  CUDA_TRY(zgemm_sq(h->d_kX1, 0, h->d_kO, 1, h->d_kD, M, nk, s));     // D = O f O^dagger
  CUDA_TRY(k_dr(G, h->d_kD, h->d_kDR, s));
  tf.done();
  // density, potential, energy
  StageTimer tr(h, s, ETDM_STAGE_RHO);
  CUDA_TRY(launch_rho_k(h, h->d_kDR, h->d_rho, s));
  tr.done();
  StageTimer tp(h, s, ETDM_STAGE_POTENTIAL);
  CUDA_TRY(launch_pack_real(h, h->d_rho, h->d_fft, s));
  CUDA_TRY(fft3d(h, h->d_fft, -1, s));
  CUDA_TRY(launch_poisson_scale(h, h->d_fft, s));
  CUDA_TRY(fft3d(h, h->d_fft, +1, s));
  CUDA_TRY(launch_potential(h, s));
  h->n_gridpart = kPotBlocks;
  if (h->sic) sic_orbitals_k(h, s);
  tp.done();
  StageTimer tk(h, s, ETDM_STAGE_DENSE_REV);
  CUDA_TRY(k_energy(h->d_kD, h->d_kT, KM, h->d_kpart, h->d_gridpart, h->n_gridpart, h->d_eterms,
                    E, h->d_flags, s, h->sic ? h->d_sicpart : nullptr,
                    h->sic ? h->N * k_sic_parts() : 0));
  h->launches += 25;
  if (!g) {
    tk.done();
    return;
  }
  tk.done();
  // H(k), L = [F, O^dagger H O], and the Eq. 39 adjoint
  StageTimer tv(h, s, ETDM_STAGE_VMAT);
  CUDA_TRY(cudaMemsetAsync(h->d_kVR, 0, (size_t)G.nR * M * M * 8, s));
  CUDA_TRY(launch_vmat_k(h, h->d_vtot, h->d_kVR, s));
  tv.done();
  StageTimer tg(h, s, ETDM_STAGE_DENSE_REV);
  CUDA_TRY(k_hamiltonian(G, h->d_kT, h->d_kVR, h->d_kH, s));
  CUDA_TRY(zgemm_sq(h->d_kH, 0, h->d_kO, 0, h->d_kX1, M, nk, s));     // H O
  CUDA_TRY(zgemm_sq(h->d_kO, 1, h->d_kX1, 0, h->d_kX2, M, nk, s));    // O^dagger H O
  CUDA_TRY(k_commutator(h->d_kX2, h->d_kf, nk, M, s));                // L
  if (h->sic) CUDA_TRY(k_sic_L(h->d_kX2, h->d_sicS, h->d_kf, M, s));   // orbital potentials
  if (ss) {  // Eq. 42: G ~ L^T
    CUDA_TRY(k_grad_vars(h->d_kX2, g, nk, M, s));
    tg.done();
    h->launches += 5;
    return;
  }
  CUDA_TRY(zgemm_sq(h->d_kX2, 0, h->d_kW, 0, h->d_kX1, M, nk, s));    // L W
  CUDA_TRY(zgemm_sq(h->d_kW, 1, h->d_kX1, 0, h->d_kX2, M, nk, s));    // W^dagger L W
  CUDA_TRY(k_dtilde(h->d_kX2, h->d_komega, nk, M, s));
  CUDA_TRY(zgemm_sq(h->d_kW, 0, h->d_kX2, 0, h->d_kX1, M, nk, s));
  CUDA_TRY(zgemm_sq(h->d_kX1, 0, h->d_kW, 1, h->d_kX2, M, nk, s));    // G^T
  CUDA_TRY(k_grad_vars(h->d_kX2, g, nk, M, s));
  tg.done();
  h->launches += 11;
}

}  // namespace etdm
