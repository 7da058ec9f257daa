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
  CUDA_TRY(cudaMemsetAsync(h->d_a, 0, h->nvar * 8, s));
  evaluate_k(h, h->d_a, h->d_E, h->d_g, s);
  CUDA_TRY(zgemm_sq(h->d_kH, 0, h->d_kC0, 0, h->d_kX1, M, nk, s));
  CUDA_TRY(k_diag(h->d_kC0, h->d_kX1, h->d_eps, nk, M, s));
  CUDA_TRY(k_precond_parts(h->d_eps, h->d_kf, h->d_kw, nk, M, h->gamma, h->d_kpden, h->d_kpw, s));
  check_device_status(h, s, "orbital energies");
  std::vector<double> st(4 + 32, 0.0);
  st[3] = h->beta0;
  CUDA_TRY(cudaMemcpy(h->d_lbstate, st.data(), st.size() * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaDeviceSynchronize());
}

void evaluate_k(etdm_handle *h, const double *a, double *E, double *g, cudaStream_t s) {
  const int M = h->M, nk = h->nk;
  const long KM = (long)nk * M * M;
  const KGeom &G = h->kg;
  // U = exp(A) through the eigendecomposition of iA (Eq. 35)
  CUDA_TRY(k_build_iA(a, nk, M, h->d_kX1, s));
  CUDA_TRY(launch_heev(h->d_kX1, h->d_komega, h->d_kW, M, nk, h->d_kwork, h->d_flags, s));
  CUDA_TRY(k_colscale(h->d_kW, h->d_komega, h->d_kX1, nk, M, 2, h->d_flags, s));
  CUDA_TRY(zgemm_sq(h->d_kX1, 0, h->d_kW, 1, h->d_kX2, M, nk, s));    // U
  CUDA_TRY(zgemm_sq(h->d_kC0, 0, h->d_kX2, 0, h->d_kO, M, nk, s));    // O = C0 U
  CUDA_TRY(k_colscale(h->d_kO, h->d_kf, h->d_kX1, nk, M, 0, h->d_flags, s));
  CUDA_TRY(zgemm_sq(h->d_kX1, 0, h->d_kO, 1, h->d_kD, M, nk, s));     // D = O f O^dagger
  CUDA_TRY(k_dr(G, h->d_kD, h->d_kDR, s));
  // density, potential, energy
  CUDA_TRY(launch_rho_k(h, h->d_kDR, h->d_rho, s));
  CUDA_TRY(launch_pack_real(h, h->d_rho, h->d_fft, s));
  CUDA_TRY(fft3d(h, h->d_fft, -1, s));
  CUDA_TRY(launch_poisson_scale(h, h->d_fft, s));
  CUDA_TRY(fft3d(h, h->d_fft, +1, s));
  CUDA_TRY(launch_potential(h, s));
  h->n_gridpart = kPotBlocks;
  CUDA_TRY(k_energy(h->d_kD, h->d_kT, KM, h->d_kpart, h->d_gridpart, h->n_gridpart, h->d_eterms,
                    E, h->d_flags, s));
  h->launches += 25;
  if (!g) return;
  // H(k), L = [F, O^dagger H O], and the Eq. 39 adjoint
  CUDA_TRY(cudaMemsetAsync(h->d_kVR, 0, (size_t)G.nR * M * M * 8, s));
  CUDA_TRY(launch_vmat_k(h, h->d_vtot, h->d_kVR, s));
  CUDA_TRY(k_hamiltonian(G, h->d_kT, h->d_kVR, h->d_kH, s));
  CUDA_TRY(zgemm_sq(h->d_kH, 0, h->d_kO, 0, h->d_kX1, M, nk, s));     // H O
  CUDA_TRY(zgemm_sq(h->d_kO, 1, h->d_kX1, 0, h->d_kX2, M, nk, s));    // O^dagger H O
  CUDA_TRY(k_commutator(h->d_kX2, h->d_kf, nk, M, s));                // L
  CUDA_TRY(zgemm_sq(h->d_kX2, 0, h->d_kW, 0, h->d_kX1, M, nk, s));    // L W
  CUDA_TRY(zgemm_sq(h->d_kW, 1, h->d_kX1, 0, h->d_kX2, M, nk, s));    // W^dagger L W
  CUDA_TRY(k_dtilde(h->d_kX2, h->d_komega, nk, M, s));
  CUDA_TRY(zgemm_sq(h->d_kW, 0, h->d_kX2, 0, h->d_kX1, M, nk, s));
  CUDA_TRY(zgemm_sq(h->d_kX1, 0, h->d_kW, 1, h->d_kX2, M, nk, s));    // G^T
  CUDA_TRY(k_grad_vars(h->d_kX2, g, nk, M, s));
  h->launches += 11;
}

}  // namespace etdm
