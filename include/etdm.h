/*
 * etdm.h -- C ABI of the ETDM energy + gradient library (sm_103a).
 *
 * Exponential-transformation direct minimization (ETDM) of a Kohn-Sham
 * energy in a localized Gaussian basis, after Ivanov, Jonsson, Vegge and
 * Jonsson, arXiv:2101.12597.  The orbitals are O = C0 exp(A) (Eq. 7) with the
 * occupied-virtual parametrization A = [[0, A_ov], [-A_ov^T, 0]] (Eq. 36);
 * the library evaluates E(A_ov) (Eq. 1) and dE/dA_ov (Eq. 14, 20), applies
 * the diagonal preconditioner (Eq. 33-34) and the L-BFGS two-loop update
 * (Sec. 3.1), and runs the line search of Eq. 25-29 on the host.  With
 * k-points (or ETDM_PARAM_FULL) the variables are instead the full
 * skew-Hermitian A(k) of every k-point (Eq. 8, 22-24) over Bloch functions
 * (Eq. 5), with exp(A(k)) by Eq. 35 or Eq. 38 and the gradient of Eq. 39-42.
 *
 * The model Hamiltonian is: normalized s-type Gaussians truncated at a hard
 * radius, Gaussian ion charges, a spectral (FFT) Poisson solve and Slater
 * exchange, all on a periodic real-space grid.
 *
 * Conventions (every entry point):
 *  - Return value: ETDM_OK (0) or a negative ETDM_ERR_* status; nothing
 *    throws across the ABI.  etdm_last_error() gives a one-line message.
 *  - Pointers named *_dev are device pointers on the handle's device; *_host
 *    are host pointers.  All are caller-owned and borrowed only for the
 *    duration of the call (device work is ordered on the given stream; the
 *    caller keeps buffers alive until that stream reaches the call's end).
 *  - `stream` is a cudaStream_t passed as void* (NULL: the legacy default
 *    stream).  One handle must not be used from two streams at once.
 *  - Matrices are row-major FP64.  A_ov, g and p are N x V row-major
 *    (N occupied, V = M - N virtual orbitals), so g[i*V + j] = dE/dA_ov[i][j];
 *    on the full-A path they hold n_k M^2 reals per the layout under
 *    ETDM_PARAM_FULL.
 *  - Units: bohr, hartree.
 */
#ifndef ETDM_H
#define ETDM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct etdm_handle etdm_handle; /* opaque; owns all device memory */

enum {
  ETDM_OK = 0,
  ETDM_ERR_INVALID_ARG = -1, /* bad size, pointer or option */
  ETDM_ERR_CUDA = -2,        /* a CUDA call failed (message has the name) */
  ETDM_ERR_OOM = -3,         /* device allocation failed */
  ETDM_ERR_NOT_CONVERGED = -4, /* iterative init step did not converge */
  ETDM_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  ETDM_ERR_STATE = -6,       /* call order (e.g. precondition before init) */
  ETDM_ERR_NUMERIC = -7      /* NaN/Inf, S not positive definite, |P| too large */
};

enum {
  ETDM_PREC_FP64 = 0,  /* every step in FP64 */
  ETDM_PREC_MIXED = 1  /* density and V on tensor cores (exact BF16 slices
                          of split operands); potential, exp(A), O and the
                          adjoint on float pairs (about 47 bits); kinetic
                          energy, energy total, gradient and L-BFGS in FP64 */
};

enum {
  ETDM_PARAM_OCCVIRT = 0, /* A = [[0, A_ov], [-A_ov^T, 0]] (Eq. 36) at the Gamma
                             point, N = n_electrons / 2 doubly occupied orbitals;
                             variables: A_ov, N x V row-major */
  ETDM_PARAM_FULL = 1     /* the full skew-Hermitian A(k) of every k-point
                             (Eq. 8, 22-24), occupations fixed at the reference
                             (Fermi-Dirac at kT, or integer at kT = 0); variables
                             per k-point: Re a_ij (i < j), then Im a_ij (i <= j),
                             row-major over the upper triangle, M^2 per k-point,
                             the k-points one after another */
};

enum {
  ETDM_EXPM_EIG = 0, /* full A: exp(A(k)) = W exp(-i Omega) W^dagger from the FP64
                        eigendecomposition iA(k) = W Omega W^dagger (Eq. 35) and
                        the exact gradient of Eq. 39-41 */
  ETDM_EXPM_SS = 1   /* full A: exp(A(k)) by scaling and squaring (Eq. 38), with
                        the approximate gradient G ~ L^T (Eq. 42; exact at A = 0)
                        and, in etdm_minimize, the reference updates of Sec. 3.5
                        chosen by etdm_options.ref_update */
};

enum {
  ETDM_FUNC_KS = 0,    /* the Kohn-Sham functional of Eq. 1 (unitary invariant) */
  ETDM_FUNC_PZSIC = 1  /* Kohn-Sham plus the Perdew-Zunger self-interaction
                          correction (Sec. 2, Eq. 16-18): E - sum_k f_k (E_H[n_k] +
                          E_x[n_k, 0]) with the unit orbital densities n_k =
                          |phi_k|^2 and spin-polarized Slater exchange; the
                          gradient takes L_mk = [F, H]_mk + f_k <m|V^k|k> -
                          f_m <m|V^m|k>, V^k = v_H[n_k] + v_x[n_k, 0].  Full-A
                          path at the Gamma point with integer occupation
                          (n_k <= 1 at k = 0, kT = 0), FP64 */
};

/* One periodic system (Eq. 3-5).  All host pointers, read during
 * etdm_init_basis only.  n_k = 0 is the Gamma point alone; n_k >= 1 selects
 * the full-A path over the given k-points (Bloch functions of Eq. 5 without
 * the 1/sqrt(N) factor, so that S(k) is the overlap over one cell). */
typedef struct {
  int32_t n_atoms;
  const double *pos;      /* [n_atoms*3] positions, bohr, inside [0, box) */
  const double *Z;        /* [n_atoms] ion charges */
  int32_t n_basis;        /* M */
  const int32_t *bf_atom; /* [M] atom carrying each s-Gaussian */
  const double *bf_exp;   /* [M] exponents alpha, bohr^-2 */
  const double *bf_rcut;  /* [M] truncation radii, bohr (0 < r_c < 2 min box) */
  double box[3];          /* orthorhombic cell edges, bohr */
  int32_t grid[3];        /* grid points per axis; prime factors <= 13 */
  double ion_sigma;       /* Gaussian ion-charge width, bohr */
  int32_t n_electrons;    /* even, 2 <= n_electrons <= 2M; N = n_electrons/2;
                             the occupied-virtual path needs N < M */
  int32_t n_k;            /* k-points (0: Gamma point, occupied-virtual A) */
  const double *k_frac;   /* [n_k*3] k-points in fractional reciprocal coordinates */
  const double *k_w;      /* [n_k] positive weights summing to 1 */
  double kT;              /* Fermi-Dirac temperature of the reference occupations,
                             Hartree; 0: integer occupation (n_k <= 1 only) */
} etdm_system;

typedef struct {
  int32_t precision; /* ETDM_PREC_FP64 or ETDM_PREC_MIXED */
  int32_t lbfgs_m;   /* L-BFGS memory (Sec. 3.1: 3), 1..16 */
  double gamma;      /* Eq. 33 mixing (0.25) */
  double beta0;      /* beta before any step exists (1.0) */
  int32_t device;    /* CUDA device ordinal */
  int32_t dense_blocks; /* grid of the cooperative dense kernels: 0 picks it
                           from the largest product (every SM for large
                           systems); n > 0 fixes it (at most the co-resident
                           limit), which moves products onto 64 x 64 output
                           tiles once they have four per block */
  int32_t dense_tc;     /* mixed precision: 0 puts the products of the dense
                           chains with at least 2^26 multiply-adds on the tensor
                           cores (exact BF16 slices, about 2^-39 relative per
                           product), 1 every product, -1 none (float pairs on
                           the FP32 pipes) */
  int32_t param;        /* ETDM_PARAM_OCCVIRT (default; needs n_k = 0) or
                           ETDM_PARAM_FULL (needs ETDM_PREC_FP64; n_k = 0 then
                           means the Gamma point with weight 1); n_k >= 1
                           implies ETDM_PARAM_FULL */
  int32_t expm;         /* full A: ETDM_EXPM_EIG (default) or ETDM_EXPM_SS */
  int32_t ref_update;   /* ETDM_EXPM_SS: reference updates C0 <- C0 exp(A), A <- 0
                           in etdm_minimize (Sec. 3.5), each followed by erasing
                           the L-BFGS pairs and taking the Eq. 33 orbital
                           energies afresh at A = 0: 0 never (default), n > 0
                           after every n steps, -1 when |L| < 3 |[A, L]|
                           (Frobenius norms over all k-points, checked before
                           each step) */
  int32_t vgroup;       /* mixed precision: tiles (4 x 4 x 8) whose V the tensor
                           memory accumulates between two read-outs, 1..8; 0
                           (default) picks it: 2 for one system, and for a batch
                           the fastest of 2, 4 and 8 in timed evaluations at
                           set-up (the choice: ETDM_ARR_TUNE) */
  int32_t functional;   /* ETDM_FUNC_KS (default) or ETDM_FUNC_PZSIC */
} etdm_options;

/* Fill *opt with the defaults above (FP64, m = 3, gamma 0.25, beta0 1,
 * automatic dense grid, automatic tensor-core products). */
void etdm_default_options(etdm_options *opt);

/* Build everything that does not depend on A (Sec. 2, Eq. 4-6): grid basis
 * tables, truncation lists per grid tile, analytic S and T, v_ext, the
 * reference C0 = S^(-1/2) (columns ordered by ascending diagonal of
 * C0^T (T + V_ext) C0, the first N occupied) and the orbital energies of
 * Eq. 33 (diagonal of C0^T H C0 at A = 0).  The full-A path (n_k >= 1 or
 * ETDM_PARAM_FULL) instead builds S(k), T(k), h_core(k) = T(k) + V_ext(k),
 * takes C0(k) as the generalized eigenvectors of h_core(k) with S(k)
 * (ascending eigenvalues; FP64 Householder + QL eigensolver on the device),
 * sets the occupations f_m(k) = 2 w_k / (1 + exp((e_m(k) - mu) / kT)) with mu
 * by bisection to sum f = n_electrons (or f = 2 on the N lowest at kT = 0) and
 * keeps them fixed, and takes the Eq. 33 orbital energies as the diagonal of
 * C0(k)^dagger H(k) C0(k) at A = 0.  On success *out owns device
 * memory until etdm_free().  Errors: INVALID_ARG (sizes, radii, grid
 * factors, list lengths over the tile limit, k-point arrays, M > 1024 or mixed
 * precision on the full-A path), OOM, CUDA, NUMERIC (S not positive
 * definite), NOT_CONVERGED (S^(-1/2) iteration, or the eigensolver). */
int etdm_init_basis(const etdm_system *sys, const etdm_options *opt,
                    etdm_handle **out);

/* A batch of n_sys independent systems in one handle (molecules of uneven
 * size, each in its own cell; Sec. 4.1 evaluates such a set one molecule at a
 * time).  Every system is set up as by etdm_init_basis (same options); their
 * variables are packed one after another (etdm_system_layout gives each
 * system's offset and length), E_dev has n_sys entries, and the entry points
 * below take the packed vectors.  In mixed precision one evaluation of all
 * systems is one captured CUDA graph (batched dense chains, density, potential
 * and V passes), and etdm_minimize advances every system with its own line
 * search, one trial point per system per round; with ETDM_PREC_FP64 every
 * system runs its own launch sequence (the plain path).  Errors: those of
 * etdm_init_basis, with the failing system's index in the message. */
int etdm_init_batch(const etdm_system *sys, int32_t n_sys, const etdm_options *opt,
                    etdm_handle **out);

/* Systems in a handle (1 for etdm_init_basis handles, 0 for NULL). */
int32_t etdm_num_systems(const etdm_handle *h);

/* Offset and length (N_i V_i) of system `sys`'s variables in the packed a, g
 * and p vectors of a batch (system 0 of a single handle: 0 and N V). */
int etdm_system_layout(const etdm_handle *h, int32_t sys, int64_t *offset, int64_t *len);

/* The handle of system `sys` of a batch (the handle itself for system 0 of a
 * single handle), for etdm_layout and etdm_get_array; borrowed: it lives until
 * the batch is freed and must not be passed to etdm_free.  NULL if out of
 * range.  Its arrays reflect the batch's last evaluation. */
etdm_handle *etdm_system_handle(etdm_handle *h, int32_t sys);

/* Systems that the next etdm_energy_grad on a batch evaluates: active_host
 * [n_sys], nonzero = evaluate (all are active after set-up).  The inactive
 * systems' E and g entries are left as they are.  Synchronizes the device. */
int etdm_set_active(etdm_handle *h, const int32_t *active_host);

/* One energy + gradient evaluation (Eq. 1, 7, 12, 11, 14 / 39-41):
 * a_dev [N*V] (A_ov) -> E_dev [1] and g_dev [N*V] = dE/dA_ov (Eq. 20);
 * on the full-A path a_dev and g_dev hold n_k M^2 reals (ETDM_PARAM_FULL),
 * and with ETDM_EXPM_SS g_dev is the approximate gradient of Eq. 42.
 * On a batch: a_dev, g_dev packed per etdm_system_layout, E_dev [n_sys].
 * g_dev may be NULL (energy only).  Asynchronous on `stream`; numerical
 * failures (NaN/Inf, |P| beyond the exp range) are reported by the next
 * synchronizing call (etdm_check or a *_host call) as ETDM_ERR_NUMERIC. */
int etdm_energy_grad(etdm_handle *h, const double *a_dev, double *E_dev,
                     double *g_dev, void *stream);

/* Same with host buffers: copies a in, evaluates, copies E and g out and
 * synchronizes.  g_host may be NULL. */
int etdm_energy_grad_host(etdm_handle *h, const double *a_host,
                          double *E_host, double *g_host);

/* pg = P^(k) o g (Eq. 33) with the current beta^(k) (Eq. 34).  On a batch:
 * per system on the packed vectors (as is etdm_lbfgs_step). */
int etdm_precondition(etdm_handle *h, const double *g_dev, double *pg_dev,
                      void *stream);

/* L-BFGS direction (Sec. 3.1): if a previous point exists, push
 * (s, y) = (a - a_prev, g - g_prev) when s.y > 1e-30 and set beta = y.y/s.y
 * (Eq. 34); then the two-loop recursion with H0 = P^(k) gives p = -H g.
 * a and g become the previous point. */
int etdm_lbfgs_step(etdm_handle *h, const double *a_dev, const double *g_dev,
                    double *p_dev, void *stream);

/* Erase the L-BFGS memory (Sec. 3.4: after a reference update): no stored
 * pairs, no previous point, beta back to beta0. */
int etdm_lbfgs_reset(etdm_handle *h);

/* Run n_steps ETDM iterations from a_dev (updated in place): L-BFGS
 * direction, then the line search (alpha = 1 first; strong Wolfe Eq. 25-26,
 * or approximate Wolfe Eq. 27 with Eq. 28; cubic interpolation; at most 20
 * trials).  Per step i (0 = the start point) the host arrays, each of
 * n_steps+1 entries and each optional, receive E, the accepted alpha and the
 * number of evaluations.  Synchronizes `stream` once per trial.  On a batch
 * every system takes n_steps steps with its own line search and L-BFGS
 * memory (the same rules, so each system's trajectory is the one it would
 * take alone); the arrays are [n_sys][n_steps+1]; a mixed-precision batch
 * synchronizes once per round of trials. */
int etdm_minimize(etdm_handle *h, double *a_dev, int32_t n_steps,
                  double *E_hist, double *alpha_hist, int32_t *trials_hist,
                  void *stream);

/* Minimize to convergence (Sec. 3.5): the iterations of etdm_minimize until
 * the Eq. 45 residual of the current point, (1/N_e) sum_i f_i |H psi_i -
 * sum_j lambda_ij psi_j|^2 with H psi_i represented in the span of the basis
 * (lambda = O^T H O), is at most tol (Hartree^2; the paper's 1e-10 eV^2 is
 * 1.3505e-13), or max_steps iterations (the paper stops at 333).  The
 * residual is computed with every evaluation of the call, in the orthonormal
 * basis of C0: R = Ubar - U_occ U_occ^T Ubar with Ubar = C0^T (4 H O), value
 * |R|^2 / (16 N).  History arrays as etdm_minimize (max_steps + 1 entries,
 * optional), resid_hist receives the residual per step; *steps_done the
 * iterations taken (0 when the start point already meets tol).  One system
 * only: a batch returns ETDM_ERR_INVALID_ARG. */
int etdm_minimize_converge(etdm_handle *h, double *a_dev, int32_t max_steps, double tol,
                           double *E_hist, double *alpha_hist, int32_t *trials_hist,
                           double *resid_hist, int32_t *steps_done, void *stream);

/* Wait for `stream` and report any deferred device-side error. */
int etdm_check(etdm_handle *h, void *stream);

/* Sizes: dims[0..ETDM_NDIMS-1] = M, N, V, G (grid points), n_tiles,
 * list entries (sum over tiles), max list length, tile edge x, y, z,
 * sum over points of n_pt^2 (pairs of functions within r_c of a point),
 * precision. */
#define ETDM_NDIMS 12
int etdm_layout(const etdm_handle *h, int64_t *dims);

/* Copy an internal array to host memory (for inspection and tests).
 * `which` is one of ETDM_ARR_*; n_bytes must equal the array's size
 * (etdm_array_bytes).  Synchronizes the handle's work. */
enum {
  ETDM_ARR_S = 0,        /* [M*M] f64 overlap */
  ETDM_ARR_T = 1,        /* [M*M] f64 kinetic */
  ETDM_ARR_C0 = 2,       /* [M*M] f64 reference orbitals (columns) */
  ETDM_ARR_ORDER = 3,    /* [M] i32 Loewdin column of each C0 column */
  ETDM_ARR_VEXT = 4,     /* [G] f64 external potential on the grid */
  ETDM_ARR_RHO = 5,      /* [G] f64 density of the last evaluation */
  ETDM_ARR_VTOT = 6,     /* [G] f64 v_ext + v_H + v_x of the last evaluation */
  ETDM_ARR_H = 7,        /* [M*M] f64 Hamiltonian matrix, last evaluation (mixed
                            precision: its grid part V only) */
  ETDM_ARR_D = 8,        /* [M*M] f64 density matrix, last FP64-path evaluation
                            (the mixed path forms the density from O instead) */
  ETDM_ARR_UOCC = 9,     /* [M*N] f64 occupied columns of exp(A) */
  ETDM_ARR_TILE_PTR = 10,/* [n_tiles+1] i32 list offsets */
  ETDM_ARR_TILE_KEYS = 11,/* [entries] i32 keys mu*512 + (nx+4)*64 + (ny+4)*8 + (nz+4) */
  ETDM_ARR_EPS = 12,     /* [M] f64 orbital energies of Eq. 33 */
  ETDM_ARR_ETERMS = 13,  /* [4] f64 kinetic, external, Hartree, exchange */
  ETDM_ARR_BETA = 14,    /* [1] f64 current beta^(k) */
  ETDM_ARR_TILE_PTR_TC = 15,  /* mixed precision: 4x4x8-tile list offsets (i32) */
  ETDM_ARR_TILE_KEYS_TC = 16, /* mixed precision: 4x4x8-tile list keys (i32) */
  ETDM_ARR_TILE_NU_TC = 17,   /* mixed precision: functions per 4x4x8 tile, periodic
                                 images merged (i32, n_tiles entries) */
  ETDM_ARR_VGROUP_T0 = 18,    /* mixed precision: first 4x4x8 tile of each group of
                                 consecutive tiles the V pass accumulates in one pass
                                 (i32, groups + 1 entries, the last = n_tiles) */
  ETDM_ARR_VGROUP_NU = 19,    /* mixed precision: functions in each V group's union
                                 list (i32, one per group) */
  ETDM_ARR_DOUBLINGS = 20,    /* [1] i32 doubling steps j of the last evaluation's
                                 exp: the least j with b / 4^j <= 1, where
                                 b = min(|P|_F, |P^2|_F^(1/2), |P^4|_F^(1/4))
                                 bounds the spectral radius of P = A_ov A_ov^T */
  ETDM_ARR_STATUS = 21,       /* [4] i32 device status words: error code, doublings,
                                 then where a bounded wait of the tensor-core
                                 products gave up and at which count (0: none) */
  ETDM_ARR_OCC = 22,          /* full A: [n_k*M] f64 occupations f_m(k) (k-point
                                 weight and spin included) */
  ETDM_ARR_EPS_REF = 23,      /* full A: [n_k*M] f64 eigenvalues of h_core(k) with
                                 S(k) (ascending; the reference's) */
  ETDM_ARR_OMEGA = 24,        /* full A: [n_k*M] f64 eigenvalues of iA(k) at the
                                 last evaluation (Eq. 35) */
  ETDM_ARR_TUNE = 25,         /* [8] f64: tiles per V group in use, then up to three
                                 (tiles per group, ms per evaluation) pairs the
                                 set-up timed (zeros where none); batches too */
  ETDM_NARR = 26              /* number of array ids */
};
/* On the full-A path S, T, C0, H and D are complex128 (re, im interleaved)
 * [n_k][M][M] row-major per k-point, EPS is [n_k*M]; ORDER, UOCC and
 * DOUBLINGS do not exist there (etdm_array_bytes returns -1). */
int64_t etdm_array_bytes(const etdm_handle *h, int32_t which);
int etdm_get_array(etdm_handle *h, int32_t which, void *host_dst,
                   int64_t n_bytes);

/* Per-stage timing with CUDA events recorded on the calling stream around
 * each stage (off by default).  etdm_stage_times synchronizes, adds the
 * elapsed milliseconds since the last call into ms[ETDM_NSTAGES] and the
 * number of timed launches of each stage into counts[ETDM_NSTAGES]; the last
 * entry of counts is the number of kernel launches issued since the last
 * call. */
enum {
  ETDM_STAGE_DENSE_FWD = 0, /* exp(A), O = C0 U, D (cooperative kernel) */
  ETDM_STAGE_RHO = 1,       /* basis -> grid density */
  ETDM_STAGE_POTENTIAL = 2, /* FFT Poisson, exchange, energy partials */
  ETDM_STAGE_VMAT = 3,      /* grid -> basis Hamiltonian */
  ETDM_STAGE_DENSE_REV = 4, /* energy sum and analytic gradient */
  ETDM_STAGE_LBFGS = 5,     /* two-loop update */
  ETDM_STAGE_EIG = 6,       /* full A: exp(A(k)) itself, by the eigendecomposition
                               of iA(k) (Eq. 35) or by scaling and squaring
                               (Eq. 38); the rest of the dense forward work is
                               DENSE_FWD */
  ETDM_NSTAGES = 8
};
int etdm_set_profiling(etdm_handle *h, int on);
int etdm_stage_times(etdm_handle *h, double *ms, int64_t *counts);

/* Message of the last failed call on h (or, when h is NULL, of the calling
 * thread's last failed call without a handle: init, the allocation-free
 * direction, the tensor-core product).  Valid until the next call on the same
 * handle (or, for NULL, the next failing such call on the same thread). */
const char *etdm_last_error(const etdm_handle *h);

/* Allocation-free L-BFGS direction.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory where they need
 * a direction (inside a stream capture with a frozen memory pool, frameworks
 * that only hand out pre-registered buffers, drivers that forbid cudaMalloc
 * after start-up).  It computes p = -H g with the same two-loop recursion as
 * etdm_lbfgs_step, from a pair history the caller keeps, and allocates
 * nothing: its reduction scratch is a fixed 2.3 KB file-scope device array.
 *   g_dev  [n]      gradient
 *   s_dev  [m*n]    steps s_i = a_(i+1) - a_i, oldest (i = 0) to newest
 *   y_dev  [m*n]    gradient changes y_i; every pair needs y_i . s_i > 0
 *   h0_dev [n]      diagonal initial inverse Hessian (any positive diagonal)
 *   p_dev  [n]      output direction (may not alias the inputs)
 * Limits: 0 <= m <= 16 and 0 <= n <= 2^40; larger m returns
 * ETDM_ERR_INVALID_ARG with a message for etdm_last_error(NULL).  n = 0
 * returns ETDM_OK at once without touching the device (the status word then
 * keeps the previous call's value).  The first
 * call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call clears the array's barrier and
 * status words and shares the array, so calls that overlap on the GPU (two
 * streams or host threads at once) race.  Asynchronous on `stream`: a failure
 * on the device (a grid barrier that gave up, a pair with y . s <= 0) leaves
 * p_dev incomplete and is reported by etdm_lbfgs_direction_noalloc_status. */
int etdm_lbfgs_direction_noalloc(const double *g_dev, const double *s_dev,
                                 const double *y_dev, int32_t m, int64_t n,
                                 const double *h0_dev, double *p_dev, void *stream);

/* Status of the last etdm_lbfgs_direction_noalloc call on the current device:
 * waits for `stream` (the stream that call ran on), reads the scratch array's
 * status word into host memory without allocating, and returns ETDM_OK,
 * ETDM_ERR_TIMEOUT (a bounded grid barrier gave up) or ETDM_ERR_NUMERIC (a
 * pair without positive finite curvature), with a message for
 * etdm_last_error(NULL).  The word keeps its value until the next direction
 * call clears it. */
int etdm_lbfgs_direction_noalloc_status(void *stream);

/* C = op(A) op(B) for FP64 device matrices (row-major; op(X) = X, or X^T
 * when ta / tb is nonzero; A is m x k after op, B k x n, C m x n) on the
 * tensor-core path of the mixed-precision dense chains (Eq. 7, 37 and their
 * reverse pass): rows of op(A) and columns of op(B) cut into five exact BF16
 * slices each after a power-of-two scaling, the slice products of orders <= 4
 * accumulated in tensor memory (orders 0, 1 and 2 exactly, one sum each over
 * 336-element K chunks; orders 3 and 4 together in one FP32 sum), the chunks
 * summed in float pairs.  Relative error about
 * 2^-39 of |A||B| per entry.  Allocates its workspace, synchronizes `stream`;
 * a bounded wait that gave up returns ETDM_ERR_TIMEOUT.  1 <= m, n, k <= 65536. */
int etdm_pair_gemm(const double *A_dev, const double *B_dev, double *C_dev, int32_t m,
                   int32_t n, int32_t k, int32_t ta, int32_t tb, void *stream);

/* Replace the reference orbitals C0 of system `sys` (0 for a single-system
 * handle) that O = C0 exp(A) rotates (Eq. 6-7), for example with C0 exp(A) of
 * an accepted point (the reference update of Sec. 3.5).  Then re-evaluates
 * at A = 0 for the Eq. 33 orbital energies (diagonal of C0^dagger H C0) and
 * erases the L-BFGS memory (beta back to beta0).
 *   C0_host   occupied-virtual path: [M*M] f64 row-major, columns are the
 *             orbitals, the first N occupied; full-A path: [n_k*M*M]
 *             complex128 (re, im interleaved), row-major per k-point.
 *   occ_host  full-A path only: [n_k*M] occupations f_m(k) (weight and spin
 *             included, finite, >= 0, summing to n_electrons), or NULL to keep
 *             the current ones; must be NULL on the occupied-virtual path.
 * The columns must be orthonormal in the S (S(k)) metric; that is not
 * checked.  Host pointers, read during the call; synchronizes the device.
 * Errors: INVALID_ARG, CUDA, NUMERIC. */
int etdm_set_reference(etdm_handle *h, int32_t sys, const double *C0_host,
                       const double *occ_host);

/* Release all device memory of h (NULL is a no-op). */
void etdm_free(etdm_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* ETDM_H */
