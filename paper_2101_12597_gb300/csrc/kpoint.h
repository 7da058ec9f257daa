// Internal declarations of the full-A / k-point path (kpoint.cu, grid.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace etdm {

constexpr int kEigMax = 1024;  // largest matrix of the Hermitian eigensolver

// C[b] = alpha op(A[b]) op(B[b]) + beta C[b] over a batch (strides sA, sB, sC
// elements); op 0: X, op 1: X^dagger; row-major.
struct ZgemmArgs {
  const double2 *A, *B;
  double2 *C;
  int m, n, k;
  int lda, ldb, ldc;
  long sA, sB, sC;
  int opa, opb;
  double2 alpha, beta;
};
cudaError_t launch_zgemm(const ZgemmArgs &g, int batch, cudaStream_t s);
cudaError_t zgemm_sq(const double2 *A, int opa, const double2 *B, int opb, double2 *C, int n,
                     int batch, cudaStream_t s, double alpha = 1.0, double beta = 0.0);

// Hermitian eigensolver: A (destroyed) = V diag(w) V^dagger, w ascending.
size_t heev_work_bytes(int n, int batch);
// method 0: implicit QL on the tridiagonal (robust for any spectrum; used at
// set-up); 1: bisection and inverse iteration (parallel over the eigenvalues;
// used for iA(k) in every evaluation)
cudaError_t launch_heev(double2 *A, double *w, double2 *V, int n, int batch, void *work,
                        int *flags, cudaStream_t s, int method = 0);


}  // namespace etdm
namespace etdm {
// element-wise steps (kpoint.cu)
// scale * iA(k) (times_i = 1) or scale * A(k) (times_i = 0) from the variables
cudaError_t k_build_iA(const double *a, int nk, int M, double2 *iA, cudaStream_t s,
                       int times_i = 1, double scale = 1.0);
// scaling and squaring / approximate gradient helpers
cudaError_t k_norm1(const double2 *X, int nk, int M, unsigned long long *out, cudaStream_t s);
cudaError_t k_poly(double2 *Q, const double2 *B, const double2 *B2, double c0, double c1,
                   double c2, int nk, int M, cudaStream_t s);
cudaError_t k_from_grad(const double *g, double2 *L, int nk, int M, cudaStream_t s);
int k_fro2_parts();
cudaError_t k_fro2(const double2 *X, long n, double *part, cudaStream_t s);
// X = Y diag(s): mode 0 s = x, mode 1 s = x^(-1/2), mode 2 s = exp(-i x)
cudaError_t k_colscale(const double2 *Y, const double *x, double2 *X, int nk, int M, int mode,
                       int *flags, cudaStream_t s);
cudaError_t k_hermitize(double2 *X, int nk, int M, cudaStream_t s);
cudaError_t k_dr(const KGeom &G, const double2 *D, double *DR, cudaStream_t s);
cudaError_t k_hamiltonian(const KGeom &G, const double2 *T, const double *VR, double2 *H,
                          cudaStream_t s);
cudaError_t k_commutator(double2 *X, const double *f, int nk, int M, cudaStream_t s);
cudaError_t k_dtilde(double2 *X, const double *w, int nk, int M, cudaStream_t s);
cudaError_t k_grad_vars(const double2 *GT, double *g, int nk, int M, cudaStream_t s);
int k_kinetic_parts();
cudaError_t k_energy(const double2 *D, const double2 *T, long n, double *part,
                     const double *gridpart, int ngp, double *eterms, double *E, int *flags,
                     cudaStream_t s, const double *sicpart = nullptr, int nsp = 0);
// PZ-SIC (Gamma point): orbital density matrix, orbital potential and energy
// partials, the L correction
cudaError_t k_rank1(const double2 *O, int k, int M, double2 *D, cudaStream_t s);
int k_sic_parts();
cudaError_t k_sic_potential(const double *n, const double2 *vh, double *v, long G, double dV,
                            double fk, double *part, cudaStream_t s);
cudaError_t k_sic_L(double2 *L, const double2 *S, const double *f, int M, cudaStream_t s);
cudaError_t k_occupation(const double *eps, const double *kw, int nk, int M, double ne, double kT,
                         double *f, double *mu, cudaStream_t s);
cudaError_t k_diag(const double2 *C, const double2 *X, double *out, int nk, int M, cudaStream_t s);
cudaError_t k_precond_parts(const double *eps, const double *f, const double *kw, int nk, int M,
                            double gamma, double *den, double *wk, cudaStream_t s);
cudaError_t k_overlap_kinetic(etdm_handle *h, cudaStream_t s);
// grid passes resolved by lattice offset (grid.cu)
cudaError_t launch_rho_k(etdm_handle *h, const double *DR, double *rho, cudaStream_t s);
cudaError_t launch_vmat_k(etdm_handle *h, const double *v, double *VR, cudaStream_t s);
// set-up and one evaluation of the full-A path (kpath.cu)
void init_kpoints(etdm_handle *h, const etdm_system *sys);
void evaluate_k(etdm_handle *h, const double *a, double *E, double *g, cudaStream_t s);
// Eq. 33 orbital energies and preconditioner parts at the current reference
// (one evaluation at A = 0, E into h->d_E and the gradient into h->d_g)
void refresh_reference_k(etdm_handle *h, cudaStream_t s);
// PZ-SIC terms of the current orbitals (Gamma point): energy partials and S
void sic_orbitals_k(etdm_handle *h, cudaStream_t s);
// reference update of Sec. 3.5: C0 <- C0 exp(A(a)), a <- 0, then the refresh
void reference_update_k(etdm_handle *h, double *a, cudaStream_t s);
// |L| and |[A, L]| (Frobenius, all k-points) with L rebuilt from an
// approximate gradient g (Eq. 42) and A from a; synchronizes s
void commutator_norms_k(etdm_handle *h, const double *a, const double *g, double *nL,
                        double *nC, cudaStream_t s);
}  // namespace etdm
