// Dense FP64 algebra of one ETDM evaluation: exp(A) for the occupied-virtual
// parametrization (Eq. 36-37), O = C0 U, D = O F O^T (Eq. 12), and the
// analytic gradient dE/dA_ov (Eq. 14) by reverse-mode differentiation of the
// same steps; plus the L-BFGS two-loop update (Sec. 3.1) and the diagonal
// preconditioner (Eq. 33-34).
//
// cos sqrt(P) and sin sqrt(P)/sqrt(P) (P = A_ov A_ov^T) are entire functions
// of P.  They are evaluated without an eigendecomposition: Taylor series of
// Q = P / 4^j with |Q|_F <= 1, then j doubling steps
//   cos 2x = 1 + 4k + 2k^2 (k = cos x - 1),  sin 2x / 2x = (sin x / x) cos x,
// which keep the small quantity k = cos x - 1 without cancellation.  The two
// degree-10 series are evaluated by Paterson-Stockmeyer blocking: Q^2, Q^3,
// Q^4, blocks B_i = sum_r c_{4i+r} Q^r (r < 4), and Horner in Q^4,
//   p(Q) = B_0 + Q^4 (B_1 + Q^4 B_2),
// four dependent product steps instead of nine; the reverse pass follows the
// same graph backwards.
//
// Each chain of small dependent products runs as ONE cooperative launch over
// all SMs with a bounded grid barrier between products (FP64 is the scarce
// resource on this GPU; spreading each product over every SM is what counts).
#include <cooperative_groups.h>
#include <math.h>

#include "device.cuh"
#include "internal.h"

namespace etdm {

constexpr int BM = 8, BN = 16, BK = 32, NT = 256;
constexpr int NG = 128;  // threads of one K group: a tile's K chunks alternate between two groups
static_assert(kTaylor >= 8 && kTaylor <= 11, "Paterson-Stockmeyer blocks assume degree 8..11");
// slots of the forward series workspace Qk
enum { kQ1 = 0, kQ2, kQ3, kQ4, kBc0, kBc1, kBc2, kBs0, kBs1, kBs2, kTc, kTs, kQslots };
// slots of the reverse workspace Wr
enum { kQ4b = 0, kTcb, kTsb, kBc2b, kBs2b, kQ1bB, kQ2bB, kQ3b, kQ2b, kQ1bt, kQ1b, kWslots };

__device__ __forceinline__ double opA(const Prod &P, int i, int k) {
  return P.ta ? P.A[(long)k * P.lda + i] : P.A[(long)i * P.lda + k];
}
__device__ __forceinline__ double opB(const Prod &P, int k, int j) {
  return P.tb ? P.B[(long)j * P.ldb + k] : P.B[(long)k * P.ldb + j];
}

// One output tile (BM x BN) of a phase.  The block's two groups of 128 threads
// (one output each) take alternate K chunks and add their partial sums at the
// end, which doubles the FP64 work in flight per SM.  Each group double-buffers
// its chunks in shared memory: the next chunk's global loads are in flight in
// registers while the current one is multiplied.
constexpr int kLa = BM * BK / NG, kLb = BK * BN / NG;  // elements per thread per chunk
__device__ void phase_tile(const Phase &ph, int tile, double (*As)[2][BM][BK + 1],
                           double (*Bs)[2][BK][BN + 1], double *part) {
  const int tilesN = (ph.n + BN - 1) / BN;
  const int r0 = (tile / tilesN) * BM, c0 = (tile % tilesN) * BN;
  const int tid = threadIdx.x % NG, grp = threadIdx.x / NG;
  const int ty = tid / BN, tx = tid % BN;
  const int i = r0 + ty, j = c0 + tx;
  const int nch = (ph.k + BK - 1) / BK, nit = (nch + 1) / 2;
  double acc = 0.0;
  for (int q = 0; q < ph.np; ++q) {
    const Prod P = ph.p[q];
    if (P.alpha == 0.0) continue;
    // this thread's load slots: (row, k) of A and (k, col) of B within a chunk
    int ai[kLa], ak[kLa], bk[kLb], bj[kLb];
#pragma unroll
    for (int u = 0; u < kLa; ++u) {
      const int e = tid + u * NG;
      if (P.ta) { ak[u] = e / BM; ai[u] = e % BM; } else { ai[u] = e / BK; ak[u] = e % BK; }
    }
#pragma unroll
    for (int u = 0; u < kLb; ++u) {
      const int e = tid + u * NG;
      if (P.tb) { bj[u] = e / BK; bk[u] = e % BK; } else { bk[u] = e / BN; bj[u] = e % BN; }
    }
    double ra[kLa], rb[kLb];
    auto load = [&](int c) {  // chunk c (zeros beyond K)
      const int k0 = c * BK;
#pragma unroll
      for (int u = 0; u < kLa; ++u) {
        const int gi = r0 + ai[u], gk = k0 + ak[u];
        ra[u] = (gi < ph.m && gk < ph.k) ? opA(P, gi, gk) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kLb; ++u) {
        const int gk = k0 + bk[u], gj = c0 + bj[u];
        rb[u] = (gk < ph.k && gj < ph.n) ? opB(P, gk, gj) : 0.0;
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int u = 0; u < kLa; ++u) As[grp][buf][ai[u]][ak[u]] = ra[u];
#pragma unroll
      for (int u = 0; u < kLb; ++u) Bs[grp][buf][bk[u]][bj[u]] = rb[u];
    };
    load(grp);
    store(0);
    __syncthreads();
    double ac[4] = {0.0, 0.0, 0.0, 0.0};  // four independent FMA chains
    for (int it = 0; it < nit; ++it) {  // this group's chunks grp, grp + 2, ...
      const int buf = it & 1;
      const bool more = it + 1 < nit;
      if (more) load(2 * (it + 1) + grp);
#pragma unroll
      for (int kk = 0; kk < BK; kk += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          ac[u] = fma(As[grp][buf][ty][kk + u], Bs[grp][buf][kk + u][tx], ac[u]);
      }
      if (more) store(buf ^ 1);
      __syncthreads();
    }
    acc += P.alpha * ((ac[0] + ac[1]) + (ac[2] + ac[3]));
  }
  if (grp == 1) part[tid] = acc;
  __syncthreads();
  if (grp == 0 && i < ph.m && j < ph.n) {
    double v = acc + part[tid];
    if (ph.C1) v += ph.beta1 * ph.C1[(long)i * ph.ldc1 + j];
    if (ph.C2) v += ph.beta2 * ph.C2[(long)i * ph.ldc2 + j];
    if (i == j) v += ph.diag;
    ph.out[(long)i * ph.ldo + j] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ int phase_tiles(const Phase &ph) {
  if (ph.m <= 0 || ph.n <= 0) return 0;
  return ((ph.m + BM - 1) / BM) * ((ph.n + BN - 1) / BN);
}

// Run independent phases over one shared tile index space (no barrier).
__device__ void run_phases(const Phase *ph, int count) {
  __shared__ double As[2][2][BM][BK + 1];
  __shared__ double Bs[2][2][BK][BN + 1];
  __shared__ double part[NG];
  int total = 0;
  for (int c = 0; c < count; ++c) total += phase_tiles(ph[c]);
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int c = 0, base = 0;
    while (t - base >= phase_tiles(ph[c])) { base += phase_tiles(ph[c]); ++c; }
    phase_tile(ph[c], t - base, As, Bs, part);
  }
}

__device__ __forceinline__ Prod mk(const double *A, int lda, int ta, const double *B, int ldb,
                                   int tb, double alpha) {
  Prod p;
  p.A = A; p.B = B; p.lda = lda; p.ldb = ldb; p.ta = ta; p.tb = tb; p.alpha = alpha;
  return p;
}

__device__ __forceinline__ Phase mkphase(int m, int n, int k, double *out, int ldo) {
  Phase ph;
  ph.m = m; ph.n = n; ph.k = k; ph.np = 0;
  ph.C1 = nullptr; ph.ldc1 = 0; ph.beta1 = 0.0;
  ph.C2 = nullptr; ph.ldc2 = 0; ph.beta2 = 0.0;
  ph.diag = 0.0; ph.out = out; ph.ldo = ldo;
  return ph;
}

#define BARRIER_OR_RETURN()                      \
  do {                                           \
    if (!grid_barrier(a.bar, a.flags)) return;   \
  } while (0)

// Forward: P, j, Q^k, Taylor series, doublings, U_occ = [cos sqrt P; -A^T s(P)],
// O = C0 U_occ, then D = 2 O O^T and H <- T (FP64 grid passes) or T O (mixed).
__global__ void __launch_bounds__(NT) dense_forward_kernel(DenseArgs a) {
  const int M = a.M, N = a.N, V = a.V;
  const long NN = (long)N * N;
  const long gtid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long gstride = (long)gridDim.x * blockDim.x;
  __shared__ int sh_j;
  __shared__ double sh_sc;

  {  // P = A_ov A_ov^T
    Phase ph = mkphase(N, N, V, a.P, N);
    ph.np = 1; ph.p[0] = mk(a.A, V, 0, a.A, V, 1, 1.0);
    run_phases(&ph, 1);
  }
  BARRIER_OR_RETURN();
  {
    double s = 0.0;
    for (long e = gtid; e < NN; e += gstride) s += a.P[e] * a.P[e];
    s = block_sum(s);
    if (threadIdx.x == 0) a.red[blockIdx.x] = s;
  }
  BARRIER_OR_RETURN();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += a.red[b];
    double nrm = sqrt(t);
    int j = 0;
    while (nrm > 1.0 && j <= kJmax) { nrm *= 0.25; ++j; }
    if (!(t == t) || isinf(t)) j = kJmax + 1;
    sh_j = j;
    sh_sc = ldexp(1.0, -2 * j);
  }
  __syncthreads();
  const int J = sh_j;
  const double sc = sh_sc;
  if (J > kJmax) {
    if (gtid == 0) atomicExch(a.flags + FLAG_ERR, ETDM_ERR_NUMERIC);
    return;
  }
  if (gtid == 0) { a.flags[FLAG_J] = J; a.scal[0] = sc; }
  double *const Qs = a.Qk;
  auto slot = [&](int k) { return Qs + (long)k * NN; };
  for (long e = gtid; e < NN; e += gstride) slot(kQ1)[e] = sc * a.P[e];
  BARRIER_OR_RETURN();
  {  // Q^2
    Phase ph = mkphase(N, N, N, slot(kQ2), N);
    ph.np = 1; ph.p[0] = mk(slot(kQ1), N, 0, slot(kQ1), N, 0, 1.0);
    run_phases(&ph, 1);
  }
  BARRIER_OR_RETURN();
  {  // Q^3 = Q Q^2, Q^4 = Q^2 Q^2
    Phase ph[2];
    ph[0] = mkphase(N, N, N, slot(kQ3), N);
    ph[0].np = 1; ph[0].p[0] = mk(slot(kQ1), N, 0, slot(kQ2), N, 0, 1.0);
    ph[1] = mkphase(N, N, N, slot(kQ4), N);
    ph[1].np = 1; ph[1].p[0] = mk(slot(kQ2), N, 0, slot(kQ2), N, 0, 1.0);
    run_phases(ph, 2);
  }
  BARRIER_OR_RETURN();
  for (long e = gtid; e < NN; e += gstride) {  // blocks B_i = sum_r c_{4i+r} Q^r
    const int i = (int)(e / N), c = (int)(e % N);
    const double q[4] = {i == c ? 1.0 : 0.0, slot(kQ1)[e], slot(kQ2)[e], slot(kQ3)[e]};
    for (int b = 0; b < 3; ++b) {
      double bc = 0.0, bs = 0.0;
      for (int r = 0; r < 4; ++r) {
        const int k = 4 * b + r;
        if (k <= kTaylor) { bc += a.ck[k] * q[r]; bs += a.sk[k] * q[r]; }
      }
      slot(kBc0 + b)[e] = bc;
      slot(kBs0 + b)[e] = bs;
    }
  }
  BARRIER_OR_RETURN();
  {  // T = B_1 + Q^4 B_2 for both series
    Phase ph[2];
    ph[0] = mkphase(N, N, N, slot(kTc), N);
    ph[0].np = 1; ph[0].p[0] = mk(slot(kQ4), N, 0, slot(kBc2), N, 0, 1.0);
    ph[0].C1 = slot(kBc1); ph[0].ldc1 = N; ph[0].beta1 = 1.0;
    ph[1] = mkphase(N, N, N, slot(kTs), N);
    ph[1].np = 1; ph[1].p[0] = mk(slot(kQ4), N, 0, slot(kBs2), N, 0, 1.0);
    ph[1].C1 = slot(kBs1); ph[1].ldc1 = N; ph[1].beta1 = 1.0;
    run_phases(ph, 2);
  }
  BARRIER_OR_RETURN();
  {  // k = cos sqrt(Q) - 1 = B_0 + Q^4 T_c, s = sin sqrt(Q) / sqrt(Q) = B_0 + Q^4 T_s
    Phase ph[2];
    ph[0] = mkphase(N, N, N, a.Kt, N);
    ph[0].np = 1; ph[0].p[0] = mk(slot(kQ4), N, 0, slot(kTc), N, 0, 1.0);
    ph[0].C1 = slot(kBc0); ph[0].ldc1 = N; ph[0].beta1 = 1.0;
    ph[1] = mkphase(N, N, N, a.St, N);
    ph[1].np = 1; ph[1].p[0] = mk(slot(kQ4), N, 0, slot(kTs), N, 0, 1.0);
    ph[1].C1 = slot(kBs0); ph[1].ldc1 = N; ph[1].beta1 = 1.0;
    run_phases(ph, 2);
  }
  BARRIER_OR_RETURN();
  for (int t = 0; t < J; ++t) {  // doubling: k' = 4k + 2k^2, s' = s + s k
    const double *Kc = a.Kt + (long)t * NN, *Sc = a.St + (long)t * NN;
    Phase ph[2];
    ph[0] = mkphase(N, N, N, a.Kt + (long)(t + 1) * NN, N);
    ph[0].np = 1; ph[0].p[0] = mk(Kc, N, 0, Kc, N, 0, 2.0);
    ph[0].C1 = Kc; ph[0].ldc1 = N; ph[0].beta1 = 4.0;
    ph[1] = mkphase(N, N, N, a.St + (long)(t + 1) * NN, N);
    ph[1].np = 1; ph[1].p[0] = mk(Sc, N, 0, Kc, N, 0, 1.0);
    ph[1].C1 = Sc; ph[1].ldc1 = N; ph[1].beta1 = 1.0;
    run_phases(ph, 2);
    BARRIER_OR_RETURN();
  }
  {
    const double *KJ = a.Kt + (long)J * NN, *SJ = a.St + (long)J * NN;
    for (long e = gtid; e < NN; e += gstride) {
      int i = (int)(e / N), c = (int)(e % N);
      a.Uocc[e] = KJ[e] + (i == c ? 1.0 : 0.0);
    }
    Phase ph = mkphase(V, N, N, a.Uocc + NN, N);  // -A^T s(P)
    ph.np = 1; ph.p[0] = mk(a.A, V, 1, SJ, N, 0, -1.0);
    run_phases(&ph, 1);
  }
  BARRIER_OR_RETURN();
  {
    Phase ph = mkphase(M, N, M, a.O, N);  // O = C0 U_occ
    ph.np = 1; ph.p[0] = mk(a.C0, M, 0, a.Uocc, N, 0, 1.0);
    run_phases(&ph, 1);
  }
  BARRIER_OR_RETURN();
  if (a.Vacc) {  // mixed path: the density comes from O on the grid; T O for the kinetic energy and dE/dO
    Phase ph = mkphase(M, N, M, a.TO, N);
    ph.np = 1; ph.p[0] = mk(a.T, M, 0, a.O, N, 0, 1.0);
    run_phases(&ph, 1);
  } else {
    Phase ph = mkphase(M, M, N, a.D, M);  // D = 2 O O^T (Eq. 12, f = 2)
    ph.np = 1; ph.p[0] = mk(a.O, N, 0, a.O, N, 1, 2.0);
    run_phases(&ph, 1);
    const long MM = (long)M * M;
    for (long e = gtid; e < MM; e += gstride) a.H[e] = a.T[e];
  }
}

// Reverse: E = Tr(D T) + grid terms; dE/dO = 4 H O; dE/dU = C0^T (4 H O);
// (mixed path: Tr(D T) = 2 sum O o (T O), 4 H O = 4 T O + 4 V O);
// back through U_occ, the doublings, the Taylor powers and P = A A^T.
__global__ void __launch_bounds__(NT) dense_reverse_kernel(DenseArgs a, int want_grad) {
  const int M = a.M, N = a.N, V = a.V;
  const long NN = (long)N * N, MM = (long)M * M;
  const long gtid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long gstride = (long)gridDim.x * blockDim.x;
  const bool mixed = a.Vacc != nullptr;
  const long MN = (long)M * N;
  {
    double s = 0.0;
    if (mixed) {  // Tr(D T) = 2 sum O o (T O); H <- V (symmetric, from the upper triangle)
      for (long e = gtid; e < MN; e += gstride) s += 2.0 * a.O[e] * a.TO[e];
      for (long e = gtid; e < MM; e += gstride) {
        int i = (int)(e / M), c = (int)(e % M);
        a.H[e] = i <= c ? a.Vacc[e] : a.Vacc[(long)c * M + i];
      }
    } else {
      for (long e = gtid; e < MM; e += gstride) s += a.D[e] * a.T[e];
      if (want_grad) {  // the grid pass accumulated the upper triangle of H
        for (long e = gtid; e < MM; e += gstride) {
          int i = (int)(e / M), c = (int)(e % M);
          if (i > c) a.H[e] = a.H[(long)c * M + i];
        }
      }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) a.red[blockIdx.x] = s;
  }
  BARRIER_OR_RETURN();
  if (mixed) {
    // dE_pot/dO = 4 V O into Ubar (scratch until Ubar is formed); the kinetic
    // energy is exact (FP64 O), only the grid energy saw Oq
    Phase ph = mkphase(M, N, M, a.Ubar, N);
    ph.np = 1; ph.p[0] = mk(a.H, M, 0, a.O, N, 0, 4.0);
    run_phases(&ph, 1);
    BARRIER_OR_RETURN();
    // Gbar = dE/dO = 4 T O + 4 V O; first-order correction of the density's O
    // quantization, sum (4 V O) o (O - Oq)
    double c = 0.0;
    for (long e = gtid; e < MN; e += gstride) {
      const double u = a.Ubar[e];
      a.Gbar[e] = 4.0 * a.TO[e] + u;
      c += u * a.dO[e];
    }
    c = block_sum(c);
    if (threadIdx.x == 0) a.red[gridDim.x + blockIdx.x] = c;
    BARRIER_OR_RETURN();
  } else if (want_grad) {
    Phase ph = mkphase(M, N, M, a.Gbar, N);  // Gbar = dE/dO = 4 H O
    ph.np = 1; ph.p[0] = mk(a.H, M, 0, a.O, N, 0, 4.0);
    run_phases(&ph, 1);
    BARRIER_OR_RETURN();
  }
  if (blockIdx.x == 0) {  // energy terms: tree sums over the block partials, all threads of block 0
    double kin = 0.0, corr = 0.0, t3[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      kin += a.red[b];
      if (mixed) corr += a.red[gridDim.x + b];
    }
    for (int b = threadIdx.x; b < a.n_gridpart; b += blockDim.x)
      for (int q = 0; q < 3; ++q) t3[q] += a.gridpart[3 * b + q];
    kin = block_sum(kin);
    corr = block_sum(corr);
    for (int q = 0; q < 3; ++q) t3[q] = block_sum(t3[q]);
    if (threadIdx.x == 0) {
      const double E = kin + t3[0] + t3[1] + t3[2] + corr;
      a.eterms[0] = kin; a.eterms[1] = t3[0]; a.eterms[2] = t3[1]; a.eterms[3] = t3[2] + corr;
      if (a.E) *a.E = E;
      if (!(E == E) || isinf(E)) atomicExch(a.flags + FLAG_ERR, ETDM_ERR_NUMERIC);
    }
  }
  if (!want_grad) return;
  {
    Phase ph = mkphase(M, N, M, a.Ubar, N);  // Ubar = C0^T Gbar
    ph.np = 1; ph.p[0] = mk(a.C0, M, 1, a.Gbar, N, 0, 1.0);
    run_phases(&ph, 1);
  }
  BARRIER_OR_RETURN();
  const int J = a.flags[FLAG_J];
  const double sc = a.scal[0];
  const double *Ubv = a.Ubar + NN;  // rows N..M-1 (V x N)
  {
    Phase ph[2];
    ph[0] = mkphase(N, N, V, a.Sbar[0], N);  // Sbar_J = -A Ubar_v
    ph[0].np = 1; ph[0].p[0] = mk(a.A, V, 0, Ubv, N, 0, -1.0);
    ph[1] = mkphase(N, V, N, a.Abar, V);     // Abar = -S_J Ubar_v^T
    ph[1].np = 1; ph[1].p[0] = mk(a.St + (long)J * NN, N, 0, Ubv, N, 1, -1.0);
    run_phases(ph, 2);
  }
  BARRIER_OR_RETURN();
  const double *kb = a.Ubar;  // Kbar_J = cotangent of cos sqrt(P) = Ubar_o
  const double *sb = a.Sbar[0];
  int pp = 0;
  for (int t = J - 1; t >= 0; --t) {
    const double *Kc = a.Kt + (long)t * NN, *Sc = a.St + (long)t * NN;
    double *kbo = a.Kbar[pp], *sbo = a.Sbar[1 - pp];
    Phase ph[2];
    ph[0] = mkphase(N, N, N, sbo, N);
    ph[0].np = 1; ph[0].p[0] = mk(sb, N, 0, Kc, N, 0, 1.0);
    ph[0].C1 = sb; ph[0].ldc1 = N; ph[0].beta1 = 1.0;
    ph[1] = mkphase(N, N, N, kbo, N);
    ph[1].np = 3;
    ph[1].p[0] = mk(kb, N, 0, Kc, N, 0, 2.0);
    ph[1].p[1] = mk(Kc, N, 0, kb, N, 0, 2.0);
    ph[1].p[2] = mk(Sc, N, 0, sb, N, 0, 1.0);
    ph[1].C1 = kb; ph[1].ldc1 = N; ph[1].beta1 = 4.0;
    run_phases(ph, 2);
    BARRIER_OR_RETURN();
    kb = kbo; sb = sbo; pp = 1 - pp;
  }
  // back through k = B_0 + Q^4 T_c, s = B_0 + Q^4 T_s (all forward matrices are
  // symmetric, so for C = X Y: Xbar += Cbar Y, Ybar += X Cbar)
  const double *const Qs = a.Qk;
  auto slot = [&](int k) { return Qs + (long)k * NN; };
  auto wr = [&](int k) { return a.Wr + (long)k * NN; };
  {
    Phase ph[3];
    ph[0] = mkphase(N, N, N, wr(kQ4b), N);  // Q4bar = kbar T_c + sbar T_s
    ph[0].np = 2;
    ph[0].p[0] = mk(kb, N, 0, slot(kTc), N, 0, 1.0);
    ph[0].p[1] = mk(sb, N, 0, slot(kTs), N, 0, 1.0);
    ph[1] = mkphase(N, N, N, wr(kTcb), N);  // T_c bar = Q^4 kbar
    ph[1].np = 1; ph[1].p[0] = mk(slot(kQ4), N, 0, kb, N, 0, 1.0);
    ph[2] = mkphase(N, N, N, wr(kTsb), N);  // T_s bar = Q^4 sbar
    ph[2].np = 1; ph[2].p[0] = mk(slot(kQ4), N, 0, sb, N, 0, 1.0);
    run_phases(ph, 3);
  }
  BARRIER_OR_RETURN();
  {  // back through T = B_1 + Q^4 B_2
    Phase ph[3];
    ph[0] = mkphase(N, N, N, wr(kQ4b), N);  // Q4bar += T_c bar B_c2 + T_s bar B_s2
    ph[0].np = 2;
    ph[0].p[0] = mk(wr(kTcb), N, 0, slot(kBc2), N, 0, 1.0);
    ph[0].p[1] = mk(wr(kTsb), N, 0, slot(kBs2), N, 0, 1.0);
    ph[0].C1 = wr(kQ4b); ph[0].ldc1 = N; ph[0].beta1 = 1.0;
    ph[1] = mkphase(N, N, N, wr(kBc2b), N);  // B_c2 bar = Q^4 T_c bar
    ph[1].np = 1; ph[1].p[0] = mk(slot(kQ4), N, 0, wr(kTcb), N, 0, 1.0);
    ph[2] = mkphase(N, N, N, wr(kBs2b), N);  // B_s2 bar = Q^4 T_s bar
    ph[2].np = 1; ph[2].p[0] = mk(slot(kQ4), N, 0, wr(kTsb), N, 0, 1.0);
    run_phases(ph, 3);
  }
  BARRIER_OR_RETURN();
  // the blocks' cotangents to the powers: Q^r bar = sum_i c_{4i+r} B_ci bar + s_{4i+r} B_si bar
  for (long e = gtid; e < NN; e += gstride) {
    const double bcb[3] = {kb[e], wr(kTcb)[e], wr(kBc2b)[e]};
    const double bsb[3] = {sb[e], wr(kTsb)[e], wr(kBs2b)[e]};
    double qb[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < 3; ++b)
      for (int r = 1; r < 4; ++r) {
        const int k = 4 * b + r;
        if (k <= kTaylor) qb[r] += a.ck[k] * bcb[b] + a.sk[k] * bsb[b];
      }
    wr(kQ1bB)[e] = qb[1];
    wr(kQ2bB)[e] = qb[2];
    wr(kQ3b)[e] = qb[3];
  }
  BARRIER_OR_RETURN();
  {  // back through Q^4 = Q^2 Q^2 and Q^3 = Q Q^2
    Phase ph[2];
    ph[0] = mkphase(N, N, N, wr(kQ2b), N);  // Q2bar = Q2bar_B + Q4bar Q^2 + Q^2 Q4bar + Q Q3bar
    ph[0].np = 3;
    ph[0].p[0] = mk(wr(kQ4b), N, 0, slot(kQ2), N, 0, 1.0);
    ph[0].p[1] = mk(slot(kQ2), N, 0, wr(kQ4b), N, 0, 1.0);
    ph[0].p[2] = mk(slot(kQ1), N, 0, wr(kQ3b), N, 0, 1.0);
    ph[0].C1 = wr(kQ2bB); ph[0].ldc1 = N; ph[0].beta1 = 1.0;
    ph[1] = mkphase(N, N, N, wr(kQ1bt), N);  // Qbar_t = Q1bar_B + Q3bar Q^2
    ph[1].np = 1; ph[1].p[0] = mk(wr(kQ3b), N, 0, slot(kQ2), N, 0, 1.0);
    ph[1].C1 = wr(kQ1bB); ph[1].ldc1 = N; ph[1].beta1 = 1.0;
    run_phases(ph, 2);
  }
  BARRIER_OR_RETURN();
  {  // back through Q^2 = Q Q: Qbar = Qbar_t + Q2bar Q + Q Q2bar
    Phase ph = mkphase(N, N, N, wr(kQ1b), N);
    ph.np = 2;
    ph.p[0] = mk(wr(kQ2b), N, 0, slot(kQ1), N, 0, 1.0);
    ph.p[1] = mk(slot(kQ1), N, 0, wr(kQ2b), N, 0, 1.0);
    ph.C1 = wr(kQ1bt); ph.ldc1 = N; ph.beta1 = 1.0;
    run_phases(&ph, 1);
  }
  BARRIER_OR_RETURN();
  {  // Q = sc P: Pbar + Pbar^T = sc (Qbar + Qbar^T)
    const double *Qb = wr(kQ1b);
    for (long e = gtid; e < NN; e += gstride) {
      int i = (int)(e / N), c = (int)(e % N);
      a.Psym[e] = sc * (Qb[e] + Qb[(long)c * N + i]);
    }
  }
  BARRIER_OR_RETURN();
  {
    Phase ph = mkphase(N, V, N, a.g, V);  // g = Abar + (Pbar + Pbar^T) A
    ph.np = 1; ph.p[0] = mk(a.Psym, N, 0, a.A, V, 0, 1.0);
    ph.C1 = a.Abar; ph.ldc1 = V; ph.beta1 = 1.0;
    run_phases(&ph, 1);
  }
}

// Plain (non-cooperative) product for set-up work.
__global__ void __launch_bounds__(NT) gemm_kernel(Phase ph) { run_phases(&ph, 1); }

// ---- L-BFGS two-loop (Sec. 3.1) with H0 = P^(k) (Eq. 33-34) ---------------
__device__ __forceinline__ double precond_elem(const double *eps, int N, int V, long e,
                                               double gamma, double beta) {
  int i = (int)(e / V), jv = (int)(e % V);
  double d = (eps[i] - eps[N + jv]) * 2.0;  // (e_i - e_j)(f_i - f_j), f = 2 / 0
  return 1.0 / (2.0 * (1.0 - gamma) * fabs(d) + gamma * beta);
}

// Dot product of the whole grid: every block gets the same value.
__device__ double grid_dot_finish(LbfgsArgs &a, double part, bool *ok) {
  part = block_sum(part);
  if (threadIdx.x == 0) a.red[blockIdx.x] = part;
  if (!grid_barrier(a.bar, a.flags)) { *ok = false; return 0.0; }
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += a.red[b];
    tot = t;
  }
  __syncthreads();
  double r = tot;
  // a second barrier keeps red[] from being overwritten before all blocks read it
  if (!grid_barrier(a.bar, a.flags)) { *ok = false; return 0.0; }
  return r;
}

__global__ void __launch_bounds__(256) lbfgs_kernel(LbfgsArgs a) {
  const long n = a.n;
  const int m = a.m;
  const long gtid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long gstride = (long)gridDim.x * blockDim.x;
  double *st = a.state;
  int count = (int)st[0], head = (int)st[1];
  const bool have_prev = st[2] != 0.0;
  double beta = st[3];
  bool ok = true;
  if (have_prev) {  // candidate pair into slot `head`
    double *sn = a.s + (long)head * n, *yn = a.y + (long)head * n;
    double p1 = 0.0, p2 = 0.0;
    for (long e = gtid; e < n; e += gstride) {
      double sv = a.a[e] - a.aprev[e], yv = a.g[e] - a.gprev[e];
      sn[e] = sv; yn[e] = yv;
      p1 += sv * yv; p2 += yv * yv;
    }
    double sy = grid_dot_finish(a, p1, &ok); if (!ok) return;
    double yy = grid_dot_finish(a, p2, &ok); if (!ok) return;
    if (sy > 1e-30) {
      beta = yy / sy;
      st[4 + head] = 1.0 / sy;  // rho of the slot (identical in every block)
      head = (head + 1) % m;
      count = count < m ? count + 1 : m;
    }
  }
  for (long e = gtid; e < n; e += gstride) {
    a.aprev[e] = a.a[e];
    a.gprev[e] = a.g[e];
    a.q[e] = a.g[e];
  }
  // first loop: newest to oldest
  double alph[16];
  for (int c = 0; c < count; ++c) {
    int slot = (head - 1 - c + 2 * m) % m;
    const double *sv = a.s + (long)slot * n, *yv = a.y + (long)slot * n;
    double part = 0.0;
    for (long e = gtid; e < n; e += gstride) part += sv[e] * a.q[e];
    double sq = grid_dot_finish(a, part, &ok); if (!ok) return;
    double al = st[4 + slot] * sq;
    alph[c] = al;
    for (long e = gtid; e < n; e += gstride) a.q[e] -= al * yv[e];
  }
  // r = H0 q
  for (long e = gtid; e < n; e += gstride)
    a.q[e] *= precond_elem(a.eps, a.N, a.V, e, a.gamma, beta);
  // second loop: oldest to newest
  for (int c = count - 1; c >= 0; --c) {
    int slot = (head - 1 - c + 2 * m) % m;
    const double *sv = a.s + (long)slot * n, *yv = a.y + (long)slot * n;
    double part = 0.0;
    for (long e = gtid; e < n; e += gstride) part += yv[e] * a.q[e];
    double yr = grid_dot_finish(a, part, &ok); if (!ok) return;
    double be = st[4 + slot] * yr;
    double coef = alph[c] - be;
    for (long e = gtid; e < n; e += gstride) a.q[e] += coef * sv[e];
  }
  for (long e = gtid; e < n; e += gstride) a.p[e] = -a.q[e];
  if (!grid_barrier(a.bar, a.flags)) return;
  if (gtid == 0) {
    st[0] = count; st[1] = head; st[2] = 1.0; st[3] = beta;
  }
}

__global__ void precond_kernel(const double *eps, int N, int V, double gamma,
                               const double *state, const double *g, double *pg) {
  long n = (long)N * V;
  double beta = state[3];
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    pg[e] = precond_elem(eps, N, V, e, gamma, beta) * g[e];
}

// Deterministic single-block dot product (line-search scalars).
__global__ void __launch_bounds__(1024) dot_kernel(const double *x, const double *y, long n,
                                                   double *out) {
  double s = 0.0;
  for (long e = threadIdx.x; e < n; e += blockDim.x) s += x[e] * y[e];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void axpy_kernel(const double *x, double alpha, const double *p, double *out,
                            long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    out[e] = x[e] + alpha * p[e];
}

__global__ void permute_cols_kernel(const double *src, const int *perm, double *dst, int M) {
  long MM = (long)M * M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MM;
       e += (long)gridDim.x * blockDim.x) {
    int r = (int)(e / M), c = (int)(e % M);
    dst[e] = src[(long)r * M + perm[c]];
  }
}

// out[j] = sum_{m,n} C[m][j] Hm[m][n] C[n][j]
__global__ void __launch_bounds__(256) diag_quad_kernel(const double *C, const double *Hm,
                                                        double *out, int M) {
  int j = blockIdx.x;
  double s = 0.0;
  for (long e = threadIdx.x; e < (long)M * M; e += blockDim.x) {
    int r = (int)(e / M), c = (int)(e % M);
    s += C[(long)r * M + j] * Hm[e] * C[(long)c * M + j];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) out[j] = s;
}

__global__ void ns_prep_kernel(const double *S, double *Y, double *Zm, double c, int M) {
  long MM = (long)M * M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MM;
       e += (long)gridDim.x * blockDim.x) {
    int r = (int)(e / M), q = (int)(e % M);
    Y[e] = S[e] / c;
    Zm[e] = (r == q) ? 1.0 : 0.0;
  }
}

__global__ void __launch_bounds__(1024) resid_kernel(const double *ZY, double *out, int M) {
  double mx = 0.0;
  for (long e = threadIdx.x; e < (long)M * M; e += blockDim.x) {
    int r = (int)(e / M), q = (int)(e % M);
    double d = fabs(ZY[e] - (r == q ? 1.0 : 0.0));
    if (!(d <= mx)) mx = d;  // NaN propagates
  }
  __shared__ double red[1024];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double o = red[threadIdx.x + s];
      if (!(o <= red[threadIdx.x])) red[threadIdx.x] = o;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void __launch_bounds__(1024) max_rowsum_kernel(const double *S, double *out, int M) {
  double mx = 0.0;
  for (int r = threadIdx.x; r < M; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < M; ++c) s += fabs(S[(long)r * M + c]);
    mx = fmax(mx, s);
  }
  __shared__ double red[1024];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void scale_copy_kernel(const double *src, double *dst, double c, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    dst[e] = c * src[e];
}

// ---- host wrappers ----------------------------------------------------------

static DenseArgs dense_args(etdm_handle *h, const double *a) {
  DenseArgs d{};
  d.M = h->M; d.N = h->N; d.V = h->V;
  d.A = a;
  d.P = h->d_P; d.Qk = h->d_Qk; d.Kt = h->d_Kt; d.St = h->d_St;
  d.Uocc = h->d_Uocc; d.O = h->d_O; d.D = h->d_D; d.H = h->d_H; d.TO = h->d_TO;
  d.C0 = h->d_C0; d.T = h->d_T;
  d.Gbar = h->d_Gbar; d.Ubar = h->d_Ubar;
  d.Kbar[0] = h->d_bar2[0]; d.Kbar[1] = h->d_bar2[1];
  d.Sbar[0] = h->d_bar2[2]; d.Sbar[1] = h->d_bar2[3];
  d.Z[0] = h->d_bar2[4]; d.Z[1] = h->d_bar2[5];
  d.Qbar = h->d_Qbar; d.Abar = h->d_Abar; d.Psym = h->d_Psym; d.Wr = h->d_Wr;
  d.eterms = h->d_eterms;
  d.gridpart = h->d_gridpart; d.n_gridpart = h->n_gridpart;
  if (h->precision == ETDM_PREC_MIXED && !h->in_setup) { d.Vacc = h->d_Vfin; d.dO = h->d_dO; }
  d.red = h->d_red; d.flags = h->d_flags; d.bar = h->d_bar; d.scal = h->d_scal;
  // c_k = (-1)^k/(2k)!, s_k = (-1)^k/(2k+1)!
  double f = 1.0;
  d.ck[0] = 0.0; d.sk[0] = 1.0;
  for (int k = 1; k <= kTaylor; ++k) {
    double f2k = f * (2 * k);                 // (2k)!  (f = (2k-1)!)
    double f2k1 = f2k * (2 * k + 1);          // (2k+1)!
    double sg = (k % 2) ? -1.0 : 1.0;
    d.ck[k] = sg / f2k;
    d.sk[k] = sg / f2k1;
    f = f2k1;
  }
  return d;
}

cudaError_t launch_dense_forward(etdm_handle *h, const double *a, cudaStream_t s) {
  DenseArgs d = dense_args(h, a);
  void *args[] = {&d};
  return cudaLaunchCooperativeKernel((void *)dense_forward_kernel, dim3(h->coop_blocks),
                                     dim3(NT), args, 0, s);
}

cudaError_t launch_dense_reverse(etdm_handle *h, const double *a, double *g, double *E,
                                 cudaStream_t s) {
  DenseArgs d = dense_args(h, a);
  d.g = g; d.E = E;
  int want = g != nullptr;
  void *args[] = {&d, &want};
  return cudaLaunchCooperativeKernel((void *)dense_reverse_kernel, dim3(h->coop_blocks),
                                     dim3(NT), args, 0, s);
}

cudaError_t launch_gemm(const Phase &ph, cudaStream_t s) {
  int tiles = ((ph.m + BM - 1) / BM) * ((ph.n + BN - 1) / BN);
  if (tiles <= 0) return cudaSuccess;
  gemm_kernel<<<tiles, NT, 0, s>>>(ph);
  return cudaGetLastError();
}

cudaError_t launch_lbfgs(etdm_handle *h, const double *a, const double *g, double *p,
                         cudaStream_t s) {
  LbfgsArgs d{};
  d.n = (long)h->N * h->V; d.N = h->N; d.V = h->V; d.m = h->lbfgs_m;
  d.a = a; d.g = g; d.p = p;
  d.s = h->d_s; d.y = h->d_y; d.aprev = h->d_aprev; d.gprev = h->d_gprev; d.q = h->d_q;
  d.state = h->d_lbstate; d.eps = h->d_eps; d.gamma = h->gamma;
  d.red = h->d_red; d.bar = h->d_bar; d.flags = h->d_flags;
  void *args[] = {&d};
  return cudaLaunchCooperativeKernel((void *)lbfgs_kernel, dim3(h->lb_blocks), dim3(256), args,
                                     0, s);
}

cudaError_t launch_precond(etdm_handle *h, const double *g, double *pg, cudaStream_t s) {
  long n = (long)h->N * h->V;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4 * h->num_sms) blocks = 4 * h->num_sms;
  if (blocks < 1) blocks = 1;
  precond_kernel<<<blocks, 256, 0, s>>>(h->d_eps, h->N, h->V, h->gamma, h->d_lbstate, g, pg);
  return cudaGetLastError();
}

cudaError_t launch_dot(const double *x, const double *y, long n, double *out, double *,
                       cudaStream_t s) {
  dot_kernel<<<1, 1024, 0, s>>>(x, y, n, out);
  return cudaGetLastError();
}

cudaError_t launch_axpy(const double *x, double alpha, const double *p, double *out, long n,
                        cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  axpy_kernel<<<blocks, 256, 0, s>>>(x, alpha, p, out, n);
  return cudaGetLastError();
}

cudaError_t launch_permute_cols(const double *src, const int *perm, double *dst, int M,
                                cudaStream_t s) {
  permute_cols_kernel<<<256, 256, 0, s>>>(src, perm, dst, M);
  return cudaGetLastError();
}

cudaError_t launch_diag_quad(const double *C, const double *Hm, double *out, int M,
                             cudaStream_t s) {
  diag_quad_kernel<<<M, 256, 0, s>>>(C, Hm, out, M);
  return cudaGetLastError();
}

cudaError_t launch_ns_prep(const double *S, double *Y, double *Zm, double c, int M,
                           cudaStream_t s) {
  ns_prep_kernel<<<256, 256, 0, s>>>(S, Y, Zm, c, M);
  return cudaGetLastError();
}

cudaError_t launch_resid(const double *ZY, double *out, int M, cudaStream_t s) {
  resid_kernel<<<1, 1024, 0, s>>>(ZY, out, M);
  return cudaGetLastError();
}

cudaError_t launch_max_rowsum(const double *S, double *out, int M, cudaStream_t s) {
  max_rowsum_kernel<<<1, 1024, 0, s>>>(S, out, M);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(const double *src, double *dst, double c, long n,
                              cudaStream_t s) {
  scale_copy_kernel<<<256, 256, 0, s>>>(src, dst, c, n);
  return cudaGetLastError();
}

int occupancy_dense(int *bps) {
  int a = 0, b = 0;
  cudaError_t e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, dense_forward_kernel, NT, 0);
  cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, dense_reverse_kernel, NT, 0);
  if (e1 != cudaSuccess || e2 != cudaSuccess) return -1;
  *bps = a < b ? a : b;
  return 0;
}

int occupancy_lbfgs(int *bps) {
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, lbfgs_kernel, 256, 0) != cudaSuccess)
    return -1;
  return 0;
}

}  // namespace etdm
