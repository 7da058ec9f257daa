// Internal declarations shared by the translation units of libetdm.
// Nothing here is part of the C ABI (include/etdm.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/etdm.h"

namespace etdm {

constexpr int kImgMax = 3;          // |n| <= 3 lattice images per axis
constexpr int kImgN = 2 * kImgMax + 1;
constexpr int kTaylor = 10;         // Taylor terms of cos sqrt(Q), sin sqrt(Q)/sqrt(Q)
constexpr int kJmax = 8;            // doublings: |P|_F <= 4^8
constexpr int kMaxList = 200;       // max truncation-list length per tile (FP64 path)
constexpr int kPotBlocks = 512;     // blocks (and energy partials) of the potential pass
constexpr int kMaxFFT = 256;        // max grid points per axis
constexpr long kSpinLimit = 2000000;   // bounded device waits (a few seconds at most)

// device-side status words
enum { FLAG_ERR = 0, FLAG_J = 1, FLAG_NFLAGS = 4 };

struct GridGeom {
  int nx, ny, nz;
  int tx, ty, tz;      // tile edges
  int nbx, nby, nbz;   // tiles per axis
  int M;
  double dV;
};

// Basis tables on the grid axes: for function mu, image n and axis point i,
//   sq[a][mu][n+3][i] = (x_i - (d_mu + n L))^2   (exact op order)
//   ex[a][mu][n+3][i] = exp(-alpha_mu * sq)
struct Tables {
  const double *sq[3];
  const double *ex[3];
  const double *norm;  // (2 alpha / pi)^(3/4)
  const double *rc2;   // r_c * r_c
};

// One dense product term for the cooperative dense kernels.  The matrices hold
// the kernel's element type (FP64, or float pairs in the mixed path's chains);
// f64 marks operands held as FP64 whatever the element type (bit 0: A, bit 1: B);
// bit 2: A symmetric with its upper triangle stored
// and a symmetric A read from its upper triangle (bit 2).
struct Prod {
  const void *A;
  const void *B;
  int lda, ldb;
  int ta, tb;   // op(A)[i][k] = ta ? A[k*lda+i] : A[i*lda+k]; same for B
  double alpha;
  int f64;
};

// out[i][j] = sum_p alpha_p op(A_p) op(B_p) + sum_q beta_q C_q + diag * I
// (out written as FP64 when out64 is set, else in the element type)
struct Phase {
  int m, n, k;
  int np;
  Prod p[3];
  int nc;                  // terms C_q added in the epilogue (q < nc <= 4)
  const void *C[4]; int ldc[4]; double beta[4];
  double diag;
  void *out; int ldo;
  int out64;
};

// Arguments of the dense chains.  In the mixed path's float-pair instantiation
// the matrices marked (R) hold (hi, lo) float pairs in their 8-byte slots; A,
// g, dO, the reductions and the energies are FP64 in both.
struct DenseArgs {
  int M, N, V;
  const double *A;       // a, N x V (FP64)
  double *Af;            // (R) A as float pairs, N x V (mixed path only)
  double *P;             // (R) N x N
  double *Qk;            // (R) [12][N*N] series workspace: Q^1..Q^4, blocks, Horner terms
  double *Kt;            // (R) [kJmax+1][N*N] cos sqrt(Q_t) - I
  double *St;            // (R) [kJmax+1][N*N] sin sqrt(Q_t)/sqrt(Q_t)
  double *Uocc;          // (R) M x N
  double *O;             // (R) M x N
  double *D;             // M x M (FP64 path)
  double *H;             // (R) M x M
  double *TO;            // (R) M x N, T O (mixed path)
  const void *C0;        // (R) M x M
  const void *T;         // (R) M x M
  double *Gbar, *Ubar;   // (R) M x N
  double *Kbar[2], *Sbar[2];         // (R) cotangents of the doubling steps, ping-pong
  double *Abar;                      // (R) N x V
  double *Wr;            // (R) [11][N*N] reverse workspace of the series
  double *g;             // N x V output, FP64 (may be null)
  double *E;             // scalar output (may be null)
  double *resid;         // Eq. 45 residual output, Hartree^2 (null: not computed; needs g)
  // tensor-core products of the float-pair chains: slice workspace and the
  // size (m n k) from which a phase uses them
  uint8_t *tc_asl, *tc_bsl;
  int *tc_rexp, *tc_cexp;
  long long tc_min_work;
  double *eterms;        // [4] kinetic, external, hartree, exchange
  const double *gridpart;  // [n_gridpart][3] energy partials of the grid
  const void *Vacc;      // (R) mixed path: upper-triangle V from the grid pass, else null
  const double *dO;      // mixed path: O - Oq for the first-order energy correction
  int n_gridpart;
  double *red;           // reduction scratch [gridDim][2]
  int *flags;
  unsigned *bar;         // grid barrier {count, generation}
  double *scal;          // [0] = 4^-j
  double ck[kTaylor + 1], sk[kTaylor + 1];
};

// Orbitals per chunk row of the O slices: all of them (N rounded up to even)
// up to 128, else 128.  The slices are stored chunk by chunk, [chunk][M][ocw],
// so that the rows of consecutive functions of one chunk are consecutive in
// memory (the density pass gathers a run of them with one bulk copy).
__host__ __device__ inline int osl_width(int N) {
  const int np = N + (N & 1);
  return np <= 128 ? np : 128;
}
__host__ __device__ inline long osl_elems(int M, int N) {
  const int np = N + (N & 1), w = osl_width(N);
  return (long)((np + w - 1) / w) * w * M;
}

// Arguments of the tensor-core grid passes for one system (mixed path):
// 4 x 4 x 8 tiles, their lists and the resident operand slices.
struct TcArgs {
  GridGeom g;  // 4 x 4 x 8 tiles
  int n_tiles;
  const int *tile_ptr, *keys;   // image lists (set-up only)
  const float4 *tab[3];         // per axis [mu][img][i]: (sq, c hi, c lo, 0),
                                // c = norm^(1/3) exp(-alpha sq) as a float pair
  const float *rc2f;            // [M]
  const int *nu;                // [n_tiles] functions per tile (images merged)
  const int *xr_off;            // [n_tiles + 1] density K steps before each tile
  const int *mu_off;            // [n_tiles + 1] functions of the tiles before each tile
  const int *tmu;               // functions of each tile, ascending
  int n_vg;                     // V groups: runs of consecutive tiles, union <= kNmax functions
  const int *vg_t0;             // [n_vg + 1] first tile of each group
  const int *vg_nu;             // [n_vg] functions of the group's union
  const int *vg_eoff;           // [n_vg + 1] padded union entries before each group
  const int *vg_xoff;           // [n_vg + 1] 256-byte units of X^T slices before each group
  const int *vg_mu;             // union function lists, ascending, padded
  uint8_t *xr;                  // density X slices, 16 KB per K step
  uint8_t *xv;                  // V X^T slices, 1 KB per padded union entry and tile
  float4 *vent;                 // per padded union entry: (mu bits, 2^(e_a - 8), bound, 0)
  signed char *rowexp;          // [G] density row exponents e_p
  const uint2 *Osl;             // BF16 slices of column-scaled O (x = K0 | K1 << 16, y = K2) in
                                // chunks of ocw orbitals: [chunk][M][ocw] (see osl_width)
  const float *oscale;          // [chunks * 128] 2^g_m, zero beyond N
  int Nocc, NoccP;              // occupied orbitals; N rounded up to even
  int ocw;                      // orbitals per O-slice chunk row
  double *rho;                  // [G]
  float2 *rhof;                 // [G] rho as float pairs
  const double *v;              // [G]
  float2 *vt;                   // [n_tiles][128] v dV at the tile points (float pairs)
  unsigned long long *Vfix;     // [M][M] V (upper triangle) in fixed point, then [M*M] = max|v| bits
  double dV;
  int *flags;
};

// One job of a grid pass, with the table entries it needs (one 32-byte load):
//   density: a = (system, tile, orbital chunk, chunks of the tile),
//            b = (first K step, K steps, functions, first function entry);
//   V:       a = (system, group, first tile, tiles),
//            b = (first union entry, padded entries, functions, X^T offset).
struct TcJob {
  int4 a, b;
};

// One launch of a grid pass over one or several systems: the systems'
// arguments and, per CTA, a list of jobs in the order the CTA runs them (the
// chunks of a density tile consecutive in one CTA's list).  A system whose
// active flag is 0 is skipped by every role.
struct TcBatch {
  const TcArgs *sys;   // [n_sys] (device)
  const TcJob *jobs;   // (device)
  const int *cta_ptr;  // [grid + 1] (device): CTA b runs jobs[cta_ptr[b] .. cta_ptr[b + 1])
  const int *active;   // [n_sys] (device)
  int *flags;          // status words: a bounded wait that gave up sets the timeout
  int grid;            // CTAs of the launch
  int max_nmc;         // largest number of orbital chunks of a job (density)
};

// Float-pair potential pipeline of the mixed path (fftdf.cu): per system, the
// radix plans of the three axes and the buffers of the half-spectrum
// transforms.
struct DfPlan {
  int n, nst;
  int radix[12];
};

struct DfArgs {
  int nx, ny, nz, nzh;
  DfPlan px, py, pz;
  const float4 *twx, *twy, *twz;
  float4 *H;               // [nx][ny][nzh] half spectrum
  const float2 *rhof;      // [G] rho as float pairs
  const float2 *vextf;     // [G] v_ext as float pairs
  const float2 *kpois;     // [nx][ny][nzh] 4 pi / (|G|^2 Ng), 0 at G = 0
  double *vtot;            // [G] (FP64 copy of v for the array interface)
  float2 *vt;              // [n_tiles][128] v dV in tile order
  unsigned *vmax_bits;     // max |v| as float bits
  double *part;            // [3 * blocks] energy partial sums
  float2 dV;
  float2 cx;               // (3 / pi)^(1/3)
  GridGeom gtc;            // 4 x 4 x 8 tiles of the potential-matrix pass
};

// Sizes of one launch of the potential passes over one or several systems.
struct DfLaunch {
  int n_sys, zb, yb, xb;     // systems; z, y and x blocks of the largest
  size_t smz, smy, smx;      // dynamic shared memory of the passes
  bool big;                  // some axis has a radix 7, 11 or 13
};

// Column slices of one system's occupied orbitals (mixed path).
struct OsArgs {
  const float2 *O;  // [M][N] float pairs from the dense chain
  int M, N, NP;     // NP = N rounded up to even
  int ocw;          // orbitals per O-slice chunk row (osl_width)
  uint2 *Osl;       // [chunk][M][ocw]
  float *oscale;    // [whole chunks of 128] 2^g_m
  double *dO;       // [M][N] O - Oq
  unsigned long long *omax;  // [N] max |O| of each column as the bits of a double
};

// V of one system from its fixed-point sums (mixed path).
struct VfArgs {
  const unsigned long long *Vfix;  // [M*M + 1]
  int M;
  float2 *Vout;                    // [M][M], upper triangle written
};

// Device tables of the mixed path's grid stages (O slices, density,
// potential, V) for one system or a batch of systems.
struct MixedPlan {
  int n_sys = 0;
  const int *active = nullptr;  // [n_sys] (device)
  TcBatch rho{}, v{};
  const DfArgs *df = nullptr;   // [n_sys] (device)
  DfLaunch dfl{};
  const OsArgs *os = nullptr;   // [n_sys] (device)
  int os_maxN = 0;
  long os_maxMN = 0;
  unsigned long long *omax = nullptr;  // every system's column maxima, one array
  size_t omax_bytes = 0;               // zeroed before each evaluation's O slicing
  const VfArgs *vf = nullptr;   // [n_sys] (device)
  int vf_blocks = 1;
  unsigned long long *vfix = nullptr;  // every system's fixed-point V sums, one array
  size_t vfix_bytes = 0;               // zeroed before each evaluation's potential pass
};

struct LbfgsArgs {
  long n;
  int N, V, m;
  const double *a, *g;
  double *p;
  double *s, *y;         // [m][n]
  double *aprev, *gprev, *q;
  double *state;         // [0]=count [1]=head [2]=have_prev [3]=beta [4..4+m)=rho [..+m)=alpha
  const double *eps;     // [M]
  const double *pden;    // full A: [n] 2 (1 - gamma) |(e_i - e_j)(f_i - f_j)| (null: occupied-virtual)
  const double *pw;      // full A: [n] k-point weight of each variable
  double gamma;
  double *red;           // [4*gridDim]: two halves of two sums each
  unsigned *bar;
  int *flags;
};

// Lattice offsets R = n_a - n_b between two images that meet in a tile (the
// full-A path's real-space density and potential matrices): |R_x| <= Rm[0]
// etc., index ((Rx + Rm0)(2 Rm1 + 1) + Ry + Rm1)(2 Rm2 + 1) + Rz + Rm2.
struct KGeom {
  int nk, M;
  int Rm[3];
  int nR;
  const double *kfrac;  // [nk][3] k-points in fractional reciprocal coordinates (device)
};

}  // namespace etdm

struct etdm_handle {
  int device = 0;
  int precision = ETDM_PREC_FP64;
  bool in_setup = false;  // set-up evaluations use the FP64 passes
  int lbfgs_m = 3;
  double gamma = 0.25, beta0 = 1.0;
  int M = 0, N = 0, V = 0, n_atoms = 0;
  long nvar = 0;          // variables: N V (occupied-virtual) or n_k M^2 (full A)
  // full A over k-points (etdm_system.n_k >= 1 or ETDM_PARAM_FULL): complex
  // FP64 matrices [n_k][M][M], row-major
  bool kpath = false;
  int nk = 0;
  double kT = 0.0, mu = 0.0, n_elec = 0.0;
  etdm::KGeom kg{};
  std::vector<double> h_kfrac, h_kw;
  double *d_kfrac = nullptr, *d_kw = nullptr;
  double *d_kf = nullptr;       // [n_k][M] occupations (weight and spin included)
  double *d_keps0 = nullptr;    // [n_k][M] eigenvalues of h_core(k) (reference)
  double *d_komega = nullptr;   // [n_k][M] eigenvalues of iA(k), last evaluation
  double *d_kpden = nullptr, *d_kpw = nullptr;  // [nvar] preconditioner parts
  double *d_kpart = nullptr;    // kinetic-energy block partials
  double2 *d_kS = nullptr, *d_kT = nullptr, *d_kC0 = nullptr;
  double2 *d_kW = nullptr, *d_kO = nullptr, *d_kD = nullptr, *d_kH = nullptr;
  double2 *d_kX1 = nullptr, *d_kX2 = nullptr;
  double *d_kDR = nullptr, *d_kVR = nullptr;  // [nR][M][M]
  void *d_kwork = nullptr;      // eigensolver workspace
  bool kref_set = false;        // reference given by etdm_set_reference
  int kexpm = 0;                // ETDM_EXPM_EIG (Eq. 35, Eq. 39) or ETDM_EXPM_SS (Eq. 38, Eq. 42)
  int tri_method = 1;           // tridiagonal eigenpairs of iA(k): 1 bisection + inverse iteration, 0 QL
  int ref_every = 0;            // reference updates in etdm_minimize (ETDM_EXPM_SS)
  long long ref_updates = 0;    // reference updates made so far
  double2 *d_kB = nullptr, *d_kB2 = nullptr, *d_kB3 = nullptr;  // scaling and squaring
  unsigned long long *d_knorm = nullptr;  // 1-norm of A (double bits)
  double *d_kfro = nullptr;     // Frobenius partials
  // PZ-SIC (Gamma point, integer occupations)
  bool sic = false;
  double2 *d_sicD = nullptr, *d_sicV = nullptr, *d_sicS = nullptr, *d_sicX = nullptr;
  double *d_sicn = nullptr, *d_sicv = nullptr, *d_sicpart = nullptr;
  int n[3] = {0, 0, 0};
  long G = 0;
  double L[3], h[3], dV = 0, omega = 0, sigma = 0;
  etdm::GridGeom geom{};
  int n_tiles = 0;
  long n_entries = 0;
  int max_list = 0;
  long long sum_npt2 = 0;
  int num_sms = 0;
  int coop_blocks = 0;
  int lb_blocks = 0;
  std::string err;
  std::vector<int> order;

  // system
  double *d_center = nullptr, *d_alpha = nullptr, *d_norm = nullptr,
         *d_rc2 = nullptr, *d_rcut = nullptr, *d_pos = nullptr, *d_Z = nullptr;
  double *d_sq = nullptr, *d_ex = nullptr;
  long tab_off[3] = {0, 0, 0};
  int *d_tile_ptr = nullptr, *d_keys = nullptr;
  // mixed-precision grid passes: 4 x 4 x 8 tiles and their lists
  etdm::GridGeom geom_tc{};
  int n_tiles_tc = 0, max_list_tc = 0;
  long n_entries_tc = 0;
  int *d_tile_ptr_tc = nullptr, *d_keys_tc = nullptr;
  float4 *d_tabf = nullptr;
  float *d_rc2f = nullptr;
  signed char *d_rowexp = nullptr;
  // operand slices resident in HBM (built once at set-up; periodic images of a
  // function in one tile merged into one entry)
  int *d_nu_tc = nullptr;                // [n_tiles_tc] functions per tile
  int *d_xr_off = nullptr;               // [n_tiles_tc + 1] density K steps before a tile
  int *d_mu_off = nullptr;               // [n_tiles_tc + 1] functions of the tiles before a tile
  int *d_tmu = nullptr;                  // functions of each tile (ascending)
  // V groups: runs of consecutive 4x4x8 tiles whose function lists have a union
  // of at most 128 functions; the V pass accumulates a group in one pass
  int n_vg = 0;
  int vg_max = 2;                        // tiles per V group at most (this handle's choice)
  std::vector<int> h_tmu;                // host copy of d_tmu (V groups are rebuilt from it)
  int *d_vg_t0 = nullptr;                // [n_vg + 1] first tile of each group
  int *d_vg_nu = nullptr;                // [n_vg] functions in the group's union
  int *d_vg_eoff = nullptr;              // [n_vg + 1] padded union entries before a group
  int *d_vg_xoff = nullptr;              // [n_vg + 1] 256-byte units of X^T slices before a group
  int *d_vg_mu = nullptr;                // union function lists (ascending, padded)
  uint8_t *d_xr = nullptr, *d_xv = nullptr;
  float4 *d_vent = nullptr;              // per padded V group entry
  float2 *d_vt = nullptr;                // [n_tiles_tc][128] v dV in tile order
  long xr_steps = 0, xv_entries = 0;
  // host copies of the per-tile K steps and the V groups (job tables)
  std::vector<int> h_xr_off, h_vg_t0, h_vg_eoff, h_mu_off, h_vg_nu, h_vg_xoff;
  // device tables of the grid stages of this handle's evaluations
  etdm::MixedPlan plan{};
  int *d_active1 = nullptr;              // [1] = 1
  bool want_resid = false;               // evaluations also compute the Eq. 45 residual
  bool dense_tc = false;                 // the float-pair chains use the tensor cores
  long long tc_min_work = 0;
  uint8_t *d_tc_asl = nullptr, *d_tc_bsl = nullptr;
  int *d_tc_rexp = nullptr, *d_tc_cexp = nullptr;
  uint2 *d_Osl = nullptr;     // [M][N + N % 2] BF16 slices of O
  float *d_oscale = nullptr;  // [N]
  double *d_dO = nullptr;     // [M][N] O - Oq
  double *d_TO = nullptr;     // [M][N] T O
  unsigned long long *d_Vfix = nullptr;  // [M*M + 1] V in fixed point, then max|v| bits
  // float-pair potential pipeline of the mixed path
  float4 *d_twf = nullptr;    // twiddles of the three axes, float-pair complex
  float4 *d_half = nullptr;   // [nx][ny][nz/2+1] half spectrum
  float2 *d_rhof = nullptr;   // [G] rho as float pairs
  float2 *d_vextf = nullptr;  // [G] v_ext as float pairs
  float2 *d_kpois = nullptr;  // [nx][ny][nz/2+1] Poisson kernel
  float2 *d_Vfin = nullptr;   // [M][M] V (upper triangle), float pairs
  float2 *d_C0p = nullptr, *d_Tp = nullptr;  // C0 and T as float pairs
  float2 *d_Af = nullptr;     // [N][V] A as float pairs
  bool pairs_last = false;    // the last evaluation left float pairs in H, Uocc
  // matrices
  double *d_S = nullptr, *d_T = nullptr, *d_C0 = nullptr;
  double *d_D = nullptr, *d_H = nullptr, *d_Uocc = nullptr, *d_O = nullptr;
  double *d_P = nullptr, *d_Qk = nullptr, *d_Kt = nullptr, *d_St = nullptr;
  double *d_Gbar = nullptr, *d_Ubar = nullptr;
  double *d_bar2[4] = {nullptr};
  double *d_Wr = nullptr;
  double *d_Abar = nullptr;
  // grid
  double *d_vext = nullptr, *d_rho = nullptr, *d_vtot = nullptr;
  double2 *d_fft = nullptr;
  double2 *d_tw = nullptr;   // twiddles per axis (n[0]+n[1]+n[2])
  double *d_gridpart = nullptr;
  int n_gridpart = 0;
  // scalars / flags
  double *d_E = nullptr, *d_eterms = nullptr, *d_scal = nullptr;
  double *d_red = nullptr;
  int *d_flags = nullptr;
  unsigned *d_bar = nullptr;
  double *d_eps = nullptr;
  // L-BFGS
  double *d_s = nullptr, *d_y = nullptr, *d_aprev = nullptr, *d_gprev = nullptr,
         *d_q = nullptr, *d_lbstate = nullptr;
  // host-API staging and line search buffers
  double *d_a = nullptr, *d_g = nullptr, *d_at = nullptr, *d_gt = nullptr,
         *d_p = nullptr, *d_dot = nullptr;
  double *d_dotpart = nullptr;  // [kDotBlocks] partial sums of the line-search dots
  double *h_pinned = nullptr;
  std::vector<void *> allocs;
  // a batch of systems (etdm_init_batch): the members own every per-system
  // array; the batch owns the packed variable vectors, the batched launch
  // tables and the captured graphs
  std::vector<etdm_handle *> members;
  std::vector<long> var_off;          // [n_sys + 1] offsets of the systems' variables
  long nvar_tot = 0;
  double *d_ae = nullptr, *d_ge = nullptr;  // evaluation point and its gradient (packed)
  double *d_res = nullptr;            // [3 n_sys]: E | g.p at the trial | g.p at the start
  unsigned char *d_ctlbuf = nullptr;  // round control: [4 n_sys] int flags, then [n_sys] alpha
  int *d_act = nullptr;               // [n_sys] the active mask of etdm_energy_grad
  std::vector<int> act_host;          // its host copy
  int *d_bflags = nullptr;            // [FLAG_NFLAGS (n_sys + 1)]: members', then the batch's
  long long *d_off = nullptr;         // [n_sys + 1] var_off on the device
  etdm::DenseArgs *d_dargs = nullptr;
  etdm::LbfgsArgs *d_largs = nullptr;
  int *d_order = nullptr;             // systems by decreasing dense work
  int dense_grid = 0, lb_grid = 0;
  etdm::MixedPlan bplan_act{}, bplan_eval{};  // grid stages masked by d_act / by the eval flags
  cudaStream_t cap = nullptr;         // stream the graphs are captured on
  cudaGraphExec_t g_eval = nullptr, g_round = nullptr;
  long long graph_kernels_eval = 0, graph_kernels_round = 0;
  unsigned char *h_ctl = nullptr;     // pinned mirror of d_ctlbuf
  double *h_res = nullptr;            // pinned: [3 n_sys] results, then the status words
  int tune_choice = 0;                // tiles per V group the autotuner picked (0: not tuned)
  std::vector<double> tune_ms;        // (tiles per group, ms per batched evaluation) tried
  // optional per-stage CUDA-event timing (etdm_set_profiling)
  bool profiling = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_events;
  double stage_ms[16] = {0};
  long long stage_n[16] = {0};
  long long launches = 0;
};

namespace etdm {

// ---- launch wrappers (return cudaError_t of the launch) --------------------
// grid basis and lists (grid.cu)
cudaError_t launch_tables(etdm_handle *h, cudaStream_t s);
cudaError_t launch_list_count(etdm_handle *h, const GridGeom &g, int n_tiles, int *d_count,
                              cudaStream_t s);
cudaError_t launch_list_fill(etdm_handle *h, const GridGeom &g, int n_tiles, const long long *d_off,
                             int *d_keys, cudaStream_t s);
cudaError_t launch_scan(const int *d_in, long long *d_out, long n, long long *d_tmp,
                        cudaStream_t s);
cudaError_t launch_npt2(etdm_handle *h, unsigned long long *d_sum, cudaStream_t s);
cudaError_t launch_overlap_kinetic(etdm_handle *h, cudaStream_t s);
cudaError_t launch_rho_fp64(etdm_handle *h, const double *D, double *rho, cudaStream_t s);
cudaError_t launch_vmat_fp64(etdm_handle *h, const double *v, double *Hacc, cudaStream_t s);
// fft and potential (potential.cu)
cudaError_t launch_twiddles(etdm_handle *h, cudaStream_t s);
cudaError_t fft3d(etdm_handle *h, double2 *data, int sign, cudaStream_t s);
cudaError_t launch_vext_recip(etdm_handle *h, cudaStream_t s);
cudaError_t launch_real_part(etdm_handle *h, const double2 *src, double *dst, cudaStream_t s);
cudaError_t launch_pack_real(etdm_handle *h, const double *src, double2 *dst, cudaStream_t s);
cudaError_t launch_poisson_scale(etdm_handle *h, double2 *data, cudaStream_t s);
cudaError_t launch_potential(etdm_handle *h, cudaStream_t s);
// dense (dense.cu)
cudaError_t launch_gemm(const Phase &ph, cudaStream_t s);
cudaError_t launch_dense_forward(etdm_handle *h, const double *a, cudaStream_t s);
cudaError_t launch_dense_reverse(etdm_handle *h, const double *a, double *g, double *E,
                                 cudaStream_t s);
cudaError_t launch_lbfgs(etdm_handle *h, const double *a, const double *g, double *p,
                         cudaStream_t s);
cudaError_t launch_precond(etdm_handle *h, const double *g, double *pg, cudaStream_t s);
// out = x . y over n elements: kDotBlocks block partials into part, then one
// block sums them in index order (the same result on every call)
constexpr int kDotBlocks = 512;
cudaError_t launch_dot(const double *x, const double *y, long n, double *out, double *part,
                       cudaStream_t s);
cudaError_t launch_axpy(const double *x, double alpha, const double *p, double *out, long n,
                        cudaStream_t s);
cudaError_t launch_permute_cols(const double *src, const int *d_perm, double *dst, int M,
                                cudaStream_t s);
cudaError_t launch_diag_quad(const double *C, const double *Hm, double *out, int M,
                             cudaStream_t s);
cudaError_t launch_ns_prep(const double *S, double *Y, double *Zm, double c, int M,
                           cudaStream_t s);
cudaError_t launch_resid(const double *ZY, double *out, int M, cudaStream_t s);
cudaError_t launch_scale_copy(const double *src, double *dst, double c, long n, cudaStream_t s);
cudaError_t launch_max_rowsum(const double *S, double *out, int M, cudaStream_t s);
// mixed-precision grid passes (mixed.cu)
cudaError_t launch_tables_f32(etdm_handle *h, cudaStream_t s);
cudaError_t launch_count_unique(etdm_handle *h, int *d_nu, cudaStream_t s);
cudaError_t launch_df_setup(etdm_handle *h, cudaStream_t s);
DfArgs df_args(etdm_handle *h);
DfLaunch df_launch_plan(const std::vector<DfArgs> &args);
cudaError_t launch_df_potential(const DfLaunch &L, const DfArgs *av, const int *active,
                                cudaStream_t s);
int df_pot_blocks(etdm_handle *h);
cudaError_t launch_operand_build(etdm_handle *h, cudaStream_t s);  // both below
cudaError_t launch_xr_build(etdm_handle *h, cudaStream_t s);  // density X slices
cudaError_t launch_xv_build(etdm_handle *h, cudaStream_t s);  // V X^T slices of the groups
int tc_rho_steps(int nu);
int tc_v_entries(int nu);
int tc_group_max();
int tc_v_slices();
TcArgs tc_args(etdm_handle *h);
OsArgs os_args(etdm_handle *h);
VfArgs vf_args(etdm_handle *h);
// the grid stages of one evaluation over the systems of a plan
cudaError_t launch_mixed_rho(const MixedPlan &P, cudaStream_t s);        // O slices, density
cudaError_t launch_mixed_potential(const MixedPlan &P, cudaStream_t s);  // V sums reset, potential
cudaError_t launch_mixed_vmat(const MixedPlan &P, cudaStream_t s);       // V pass, fixed point -> pairs
int tc_max_list();
// message for etdm_last_error(NULL) from calls that take no handle
void set_unbound_error(const std::string &msg);
int occupancy_dense(int *blocks_per_sm);
int occupancy_dense_tc(int *blocks_per_sm);  // the tensor-core variants (with their shared memory)
cudaError_t launch_pair_gemm(const double *A, const double *B, double *C, int m, int n, int k,
                             int ta, int tb, uint8_t *asl, uint8_t *bsl, int *rexp, int *cexp,
                             unsigned *bar, int *flags, int blocks, cudaStream_t s);
size_t dense_tc_asl_bytes(long M);
size_t dense_tc_bsl_bytes(long M);
// arguments of one system's dense chains at the point a (g, E: set by the caller)
DenseArgs dense_args(etdm_handle *h, const double *a);
LbfgsArgs lbfgs_args(etdm_handle *h, const double *a, const double *g, double *p);
// batched dense chains: block b runs systems order[b], order[b + grid], ...
cudaError_t launch_dense_batch(const DenseArgs *av, const int *order, int n, const int *active,
                               int grid, bool pairs, bool reverse, cudaStream_t s);
cudaError_t launch_lbfgs_batch(const LbfgsArgs *av, const int *dir, const int *reset, int n,
                               int grid, cudaStream_t s);
cudaError_t launch_to_pairs(const double *src, float2 *dst, long n, cudaStream_t s);
cudaError_t launch_from_pairs(const float2 *src, double *dst, long n, cudaStream_t s);
int occupancy_lbfgs(int *blocks_per_sm);

}  // namespace etdm
