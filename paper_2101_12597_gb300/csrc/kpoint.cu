// The full-A path with k-point sampling (Sec. 2-3 with fractional occupation):
// complex FP64 dense kernels (batched over the k-points), the Hermitian
// eigensolver behind Eq. 35 and Eq. 39, and the element-wise steps between
// them.  The grid passes of this path are in grid.cu (density and V resolved
// by lattice offset), the sequencing in capi.cu.
//
// Layout: every complex matrix is row-major M x M (double2 = re, im), the
// k-points' matrices one after another.
#include <math.h>

#include <algorithm>
#include <vector>

#include "device.cuh"
#include "host.h"
#include "kpoint.h"

namespace etdm {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// acc += a * b
__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

// ---- batched complex GEMM ----------------------------------------------------
// C[b] = alpha op(A[b]) op(B[b]) + beta C[b], op(X) = X (0) or X^dagger (1).
// 64 x 64 output tiles, K steps of 16, 4 x 4 outputs per thread; FP64 FMA.
constexpr int kZB = 64, kZK = 16;

__global__ void __launch_bounds__(256) zgemm_kernel(ZgemmArgs g) {
  __shared__ double2 As[kZK][kZB];
  __shared__ double2 Bs[kZK][kZB];
  const int b = blockIdx.z;
  const double2 *A = g.A + (long)b * g.sA;
  const double2 *B = g.B + (long)b * g.sB;
  double2 *C = g.C + (long)b * g.sC;
  const int row0 = blockIdx.y * kZB, col0 = blockIdx.x * kZB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < g.k; k0 += kZK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = threadIdx.x + 256 * r;
      if (g.opa == 0) {  // op(A)[i][kk] = A[i][kk]: kk fastest
        const int i = e / kZK, kk = e % kZK;
        const int gi = row0 + i, gk = k0 + kk;
        As[kk][i] = (gi < g.m && gk < g.k) ? A[(long)gi * g.lda + gk] : make_double2(0.0, 0.0);
      } else {           // op(A)[i][kk] = conj(A[kk][i]): i fastest
        const int kk = e / kZB, i = e % kZB;
        const int gi = row0 + i, gk = k0 + kk;
        As[kk][i] = (gi < g.m && gk < g.k) ? cconj(A[(long)gk * g.lda + gi]) : make_double2(0.0, 0.0);
      }
      if (g.opb == 0) {  // op(B)[kk][j] = B[kk][j]: j fastest
        const int kk = e / kZB, j = e % kZB;
        const int gj = col0 + j, gk = k0 + kk;
        Bs[kk][j] = (gj < g.n && gk < g.k) ? B[(long)gk * g.ldb + gj] : make_double2(0.0, 0.0);
      } else {           // op(B)[kk][j] = conj(B[j][kk]): kk fastest
        const int j = e / kZK, kk = e % kZK;
        const int gj = col0 + j, gk = k0 + kk;
        Bs[kk][j] = (gj < g.n && gk < g.k) ? cconj(B[(long)gj * g.ldb + gk]) : make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kZK; ++kk) {
      double2 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = row0 + ty * 4 + i;
    if (gi >= g.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = col0 + tx * 4 + j;
      if (gj >= g.n) continue;
      double2 v = cmul(g.alpha, acc[i][j]);
      double2 *c = C + (long)gi * g.ldc + gj;
      if (g.beta.x != 0.0 || g.beta.y != 0.0) v = cadd(v, cmul(g.beta, *c));
      *c = v;
    }
  }
}

cudaError_t launch_zgemm(const ZgemmArgs &g, int batch, cudaStream_t s) {
  if (g.m <= 0 || g.n <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((g.n + kZB - 1) / kZB, (g.m + kZB - 1) / kZB, batch);
  zgemm_kernel<<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

// Square n x n batch: C = alpha op(A) op(B) + beta C with the k-point stride n^2.
cudaError_t zgemm_sq(const double2 *A, int opa, const double2 *B, int opb, double2 *C, int n,
                     int batch, cudaStream_t s, double alpha, double beta) {
  ZgemmArgs g;
  g.A = A; g.B = B; g.C = C;
  g.m = g.n = g.k = n;
  g.lda = g.ldb = g.ldc = n;
  g.sA = g.sB = g.sC = (long)n * n;
  g.opa = opa; g.opb = opb;
  g.alpha = make_double2(alpha, 0.0);
  g.beta = make_double2(beta, 0.0);
  return launch_zgemm(g, batch, s);
}

// ---- Hermitian eigensolver (FP64) ------------------------------------------------
// A = V diag(w) V^dagger for a batch of n x n Hermitian matrices, in three
// kernels: Householder reduction to a tridiagonal T = Q^dagger A Q (a group
// of blocks per matrix, the matrix held in L2), implicit QL iterations with
// Wilkinson shifts on the real tridiagonal Phi^dagger T Phi (Phi a diagonal of
// phases; the sweeps replicated in blocks of rows of Z), and the
// back-transformation V = Q Phi Z (blocks over slabs of columns).
// Eigenvalues ascending.

// Reflector j maps x = A[j+1 .., j] to alpha e_1: H_j = I - 2 u u^dagger with
// u = (x - alpha e_1) / |x - alpha e_1|, alpha = -(x_0/|x_0|) |x|; u is stored
// in hv[j][j+1 ..] (zero when the column is already reduced).  The trailing
// block becomes H A H = A - 2 u w^dagger - 2 w u^dagger, w = p - (u^dagger p) u,
// p = A u.  d[j] = Re A[j][j], e[j] = T[j+1][j].
// The reduction runs on a group of G blocks per matrix (a cooperative launch,
// gridDim = (G, batch)): row i of the trailing matrix belongs to block
// i mod G.  Step j: the owner of row j forms the reflector from that row (the
// column below the diagonal, conjugated) and publishes u; after a group
// barrier every block forms p_i = (A_t u)_i for its rows and a partial of
// K = u^dagger p; after a second barrier every block forms w = p - K u and
// applies the rank-2 update to its rows.  The group barrier is two words per
// matrix, its waits bounded (ETDM_ERR_TIMEOUT, then every block returns).
struct HtrdWork {
  double2 *u;      // [batch][n] reflector of the current step
  double2 *p;      // [batch][n] A_t u
  double *kpart;   // [batch][G] partials of u^dagger p
  int *skip;       // [batch] the current step needs no reflection
  unsigned *bar;   // [batch][2] group barrier: count, generation
};

__device__ __forceinline__ bool group_barrier(unsigned *bar, unsigned nb, int *flags) {
  __syncthreads();
  if (nb == 1) return true;
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = ld_acquire_gpu(bar + 1);
    const unsigned arrived = atom_add_acq_rel_gpu(bar, 1u);
    if (arrived == nb - 1) {
      st_relaxed_gpu(bar, 0u);
      st_release_gpu(bar + 1, g + 1);
    } else {
      long it = 0;
      while (ld_acquire_gpu(bar + 1) == g) {
        if (++it > kSpinLimit) {
          atomicExch(flags + FLAG_ERR, ETDM_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    if (*(volatile int *)(flags + FLAG_ERR) == ETDM_ERR_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(512) zhetrd_group_kernel(double2 *Ab, double2 *hvb, double *db,
                                                            double2 *eb, int n, HtrdWork W,
                                                            int *flags) {
  extern __shared__ double2 hsm[];
  double2 *u = hsm;       // [n]
  double2 *w = hsm + n;   // [n]
  __shared__ double2 alpha_s;
  __shared__ double inv_s, kr_s;
  __shared__ int skip_s;
  const int b = blockIdx.y, G = gridDim.x, r = blockIdx.x;
  double2 *A = Ab + (long)b * n * n;
  double2 *hv = hvb + (long)b * n * n;
  double2 *ug = W.u + (long)b * n, *pg = W.p + (long)b * n;
  double *kp = W.kpart + (long)b * G;
  unsigned *bar = W.bar + 2 * b;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int j = 0; j + 1 < n; ++j) {
    const int m = n - j - 1, o = j + 1;
    __syncthreads();  // this block's updates of its rows (row j among them) are done
    if (j % G == r) {  // the owner of row j: the reflector from conj(A[j][o..])
      const double2 *row = A + (long)j * n + o;
      double tail = 0.0;
      for (int l = 1 + tid; l < m; l += nt) tail += row[l].x * row[l].x + row[l].y * row[l].y;
      tail = block_sum(tail);
      if (tid == 0) {
        const double2 x0 = cconj(row[0]);
        const double ax0 = hypot(x0.x, x0.y);
        if (tail == 0.0) {
          skip_s = 1;
          alpha_s = x0;
        } else {
          const double xn = sqrt(ax0 * ax0 + tail);
          const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
          alpha_s = make_double2(-ph.x * xn, -ph.y * xn);
          const double v0 = ax0 + xn;
          const double inv = 1.0 / sqrt(v0 * v0 + tail);
          inv_s = inv;
          ug[0] = make_double2(ph.x * v0 * inv, ph.y * v0 * inv);
          skip_s = 0;
        }
        W.skip[b] = skip_s;
        eb[(long)b * n + j] = alpha_s;
      }
      __syncthreads();
      double2 *hrow = hv + (long)j * n;
      if (skip_s) {
        for (int i = tid; i < n; i += nt) hrow[i] = make_double2(0.0, 0.0);
      } else {
        for (int l = 1 + tid; l < m; l += nt) ug[l] = cscale(cconj(row[l]), inv_s);
        __syncthreads();
        for (int i = tid; i < n; i += nt) hrow[i] = i >= o ? ug[i - o] : make_double2(0.0, 0.0);
      }
    }
    if (!group_barrier(bar, G, flags)) return;
    if (*(volatile int *)(W.skip + b)) {
      if (!group_barrier(bar, G, flags)) return;  // (keeps the barrier count of the group)
      continue;
    }
    for (int l = tid; l < m; l += nt) u[l] = ug[l];
    __syncthreads();
    // p_i = (A_t u)_i for the rows of this block: a warp per row
    double kpart = 0.0;
    for (int q = warp; (long)q * G + ((r - o % G + G) % G) < m; q += nw) {
      const int i = q * G + ((r - o % G + G) % G);  // trailing row index with (o + i) % G == r
      const double2 *row = A + (long)(o + i) * n + o;
      double2 s4[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                       make_double2(0.0, 0.0)};
      int l = lane;
      for (; l + 96 < m; l += 128) {
        const double2 a0 = row[l], a1 = row[l + 32], a2 = row[l + 64], a3 = row[l + 96];
        cfma(s4[0], a0, u[l]);
        cfma(s4[1], a1, u[l + 32]);
        cfma(s4[2], a2, u[l + 64]);
        cfma(s4[3], a3, u[l + 96]);
      }
      for (; l < m; l += 32) cfma(s4[0], row[l], u[l]);
      double2 sv = cadd(cadd(s4[0], s4[1]), cadd(s4[2], s4[3]));
      for (int sh = 16; sh > 0; sh >>= 1) {
        sv.x += __shfl_xor_sync(0xffffffffu, sv.x, sh);
        sv.y += __shfl_xor_sync(0xffffffffu, sv.y, sh);
      }
      if (lane == 0) {
        pg[i] = sv;
        kpart += u[i].x * sv.x + u[i].y * sv.y;  // Re(conj(u_i) p_i)
      }
    }
    kpart = block_sum(kpart);
    if (tid == 0) kp[r] = kpart;
    if (!group_barrier(bar, G, flags)) return;
    if (tid == 0) {
      double k = 0.0;
      for (int q = 0; q < G; ++q) k += kp[q];
      kr_s = k;
    }
    __syncthreads();
    const double kr = kr_s;
    for (int l = tid; l < m; l += nt) w[l] = csub(pg[l], cscale(u[l], kr));
    __syncthreads();
    // A_t -= 2 (u w^dagger + w u^dagger) on this block's rows
    for (int q = warp; (long)q * G + ((r - o % G + G) % G) < m; q += nw) {
      const int i = q * G + ((r - o % G + G) % G);
      double2 *row = A + (long)(o + i) * n + o;
      const double2 ui = cscale(u[i], 2.0), wi = cscale(w[i], 2.0);
      int l = lane;
      for (; l + 96 < m; l += 128) {
        double2 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = row[l + 32 * k];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = l + 32 * k;
          double2 t = cmul(ui, cconj(w[c]));
          cfma(t, wi, cconj(u[c]));
          row[c] = csub(a[k], t);
        }
      }
      for (; l < m; l += 32) {
        double2 t = cmul(ui, cconj(w[l]));
        cfma(t, wi, cconj(u[l]));
        row[l] = csub(row[l], t);
      }
    }
  }
  if (!group_barrier(bar, G, flags)) return;
  for (int i = r * nt + tid; i < n; i += G * nt) db[(long)b * n + i] = A[(long)i * n + i].x;
  if (r == 0 && tid == 0) eb[(long)b * n + n - 1] = make_double2(0.0, 0.0);
  if (r == 0)
    for (int i = tid; i < n; i += nt) hv[(long)(n - 1) * n + i] = make_double2(0.0, 0.0);
}

// Implicit QL with Wilkinson shifts on the real tridiagonal (d, |e|).  The
// rows of Z are split over kQlRows-row blocks: every block of a matrix runs the
// same scalar sweeps (bit-identical: the same code on the same data) and
// applies them to its own rows, held in shared memory by columns (Zs[c][r]).
// Warp 0's lane 0 computes sweep t into one half of a double buffer while
// warp 1 applies sweep t - 1 from the other; a block barrier separates the
// sweeps.  More than 60 sweeps for one eigenvalue sets ETDM_ERR_NOT_CONVERGED.
// Block 0 of each matrix ranks the eigenvalues (ties by index) and writes the
// phases Phi with T = Phi T_r Phi^dagger.
constexpr int kQlRows = 32;

struct QlSweep {
  int hi, st, valid;
};

// sqrt(x^2 + y^2) for the magnitudes of a normalized eigenproblem (no overflow
// below 1e150)
__device__ __forceinline__ double ql_norm(double x, double y) { return sqrt(fma(x, x, y * y)); }

// 1 / sqrt(x) for x in [1e-30, 1e30]: a single-precision seed (relative error
// below 2^-21) refined by two Newton-Raphson steps y <- y (3 - x y^2) / 2, each
// of which squares the relative error (2^-42, then below the FP64 rounding):
// the QL sweep's only square root and division, in fewer dependent FP64
// operations than a correctly rounded sqrt and divide
__device__ __forceinline__ double ql_rsqrt(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  return y;
}

__global__ void __launch_bounds__(64) ztql_kernel(const double *db, const double2 *eb, double *wb,
                                                   double2 *phib, double *Ztb, int *permb,
                                                   int *flags, int n, int rows) {
  extern __shared__ double qsm[];
  double *d = qsm, *e = qsm + n;
  double *cs = qsm + 2 * n, *sn = qsm + 4 * n;  // [2][n] each
  double *Zs = qsm + 6 * n;                      // [n][rows]
  __shared__ QlSweep sw[2];
  __shared__ int finished;
  const int b = blockIdx.y, r0 = blockIdx.x * rows, tid = threadIdx.x;
  const int nr = min(rows, n - r0);
  for (int q = tid; q < n * rows; q += blockDim.x) {
    const int c = q / rows, r = q % rows;
    Zs[q] = (r0 + r == c) ? 1.0 : 0.0;
  }
  for (int i = tid; i < n; i += blockDim.x) {
    d[i] = db[(long)b * n + i];
    const double2 ei = eb[(long)b * n + i];
    e[i] = ql_norm(ei.x, ei.y);
  }
  if (tid == 0) {
    sw[0].valid = sw[1].valid = 0;
    finished = 0;
  }
  __syncthreads();
  if (blockIdx.x == 0 && tid == 0) {  // phases: T[j+1][j] = phi_(j+1) conj(phi_j) |e_j|
    double2 ph = make_double2(1.0, 0.0);
    phib[(long)b * n] = ph;
    for (int j = 0; j + 1 < n; ++j) {
      const double2 ej = eb[(long)b * n + j];
      const double a = e[j];
      if (a > 0.0) ph = cmul(ph, make_double2(ej.x / a, ej.y / a));
      phib[(long)b * n + j + 1] = ph;
    }
  }
  // scalar state of lane 0 of warp 0
  const double eps = 2.220446049250313e-16;
  double anorm = 0.0;
  int l = 0, iter = 0;
  if (tid == 0)
    for (int j = 0; j < n; ++j) anorm = fmax(anorm, fabs(d[j]) + e[j] + (j ? e[j - 1] : 0.0));
  for (int t = 0;; ++t) {
    const int cur = t & 1, prev = cur ^ 1;
    if (tid == 0) {  // the next sweep (or the end) into buffer cur
      QlSweep out{0, 0, 0};
      bool done = false;
      while (!done) {
        if (l >= n) {
          done = true;
          break;
        }
        int m = l;
        for (; m < n - 1; ++m) {
          const double dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= eps * dd || fabs(e[m]) <= eps * eps * anorm) break;
        }
        if (m == l) {  // eigenvalue l converged
          ++l;
          iter = 0;
          continue;
        }
        if (++iter > 60) {
          atomicExch(flags + FLAG_ERR, ETDM_ERR_NOT_CONVERGED);
          l = n;
          continue;
        }
        double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
        double r = ql_norm(g, 1.0);
        g = d[m] - d[l] + e[l] / (g + copysign(r, g));
        double s = 1.0, c = 1.0, pp = 0.0;
        double *csb = cs + cur * n, *snb = sn + cur * n;
        int i = m - 1;
        for (; i >= l; --i) {
          const double f = s * e[i], bb = c * e[i];
          const double x = fma(f, f, g * g);
          double inv;
          if (x >= 1e-30 && x <= 1e30) {
            inv = ql_rsqrt(x);
            r = x * inv;
          } else {
            r = sqrt(x);
            inv = 1.0 / r;
          }
          e[i + 1] = r;
          if (r == 0.0) {  // underflow: deflate here
            d[i + 1] -= pp;
            e[m] = 0.0;
            break;
          }
          s = f * inv;
          c = g * inv;
          g = d[i + 1] - pp;
          r = (d[i] - g) * s + 2.0 * c * bb;
          pp = s * r;
          d[i + 1] = g + pp;
          g = c * r - bb;
          csb[i] = c;
          snb[i] = s;
        }
        if (i < l) {
          d[l] -= pp;
          e[l] = g;
          e[m] = 0.0;
        }
        out = QlSweep{m, i + 1, 1};
        break;
      }
      sw[cur] = out;
      if (done) finished = 1;
    } else if (tid >= 32 && tid - 32 < nr && sw[prev].valid) {  // warp 1: sweep t - 1 on its row
      const int rr = tid - 32;
      const int hi = sw[prev].hi, st = sw[prev].st;
      const double *csb = cs + prev * n, *snb = sn + prev * n;
      double carry = Zs[hi * rows + rr];
      for (int i = hi - 1; i >= st; --i) {
        const double zi = Zs[i * rows + rr];
        Zs[(i + 1) * rows + rr] = snb[i] * zi + csb[i] * carry;
        carry = csb[i] * zi - snb[i] * carry;
      }
      Zs[st * rows + rr] = carry;
    }
    __syncthreads();
    // no sweep t: sweep t - 1 was applied in this step, so every rotation is in
    // (finished is written once, before the barrier, and read after it)
    if (finished) break;
  }
  __syncthreads();
  double *Zt = Ztb + (long)b * n * n;
  for (int q = tid; q < n * rows; q += blockDim.x) {
    const int c = q / rows, r = q % rows;
    if (r < nr) Zt[(long)c * n + r0 + r] = Zs[q];
  }
  if (blockIdx.x == 0)
    for (int i = tid; i < n; i += blockDim.x) {
      int rk = 0;
      const double di = d[i];
      for (int j = 0; j < n; ++j) rk += (d[j] < di) || (d[j] == di && j < i);
      wb[(long)b * n + rk] = di;
      permb[(long)b * n + rk] = i;
    }
}

// ---- tridiagonal eigenpairs by bisection and inverse iteration --------------------
// The parallel alternative to the QL sweeps for the real tridiagonal (d, |e|):
// the matrix splits where an off-diagonal is negligible; slot i (row i) is the
// (i - p)-th eigenpair of the block [p, q) containing row i.  Each thread finds
// its eigenvalue by bisection on the block's Sturm count (in parallel over the
// eigenvalues), then inverse iteration (tridiagonal LU with partial pivoting,
// three solves from a pseudo-random start) gives its vector, supported on the
// block.  Eigenvalues of a block closer than 1e-3 |T| form a cluster (a
// rank-deficient A gives one large cluster at zero): a block per cluster then
// orthonormalizes the cluster's vectors in order by classical Gram-Schmidt
// applied twice, which leaves an orthonormal basis of the cluster's invariant
// subspace.  Then the eigenvalues are ranked.
__device__ __forceinline__ bool tri_split(const double *d, const double *ae, int j) {
  // off-diagonal j (between rows j and j + 1) is negligible
  return ae[j] <= 2.2204460492503131e-16 * (fabs(d[j]) + fabs(d[j + 1])) || ae[j] <= 1e-300;
}

// the block [p, q) containing row i
__device__ void tri_block(const double *d, const double *ae, int n, int i, int *p, int *q) {
  int a = i, b = i + 1;
  while (a > 0 && !tri_split(d, ae, a - 1)) --a;
  while (b < n && !tri_split(d, ae, b - 1)) ++b;
  *p = a;
  *q = b;
}

// eigenvalues of block [p, q) below x (Sturm count; a pivot of magnitude below
// pivmin is replaced by -pivmin)
__device__ int tri_count(const double *d, const double *ae, int p, int q, double x, double pivmin) {
  int c = 0;
  double v = d[p] - x;
  if (fabs(v) < pivmin) v = -pivmin;
  c += v < 0.0;
  for (int j = p + 1; j < q; ++j) {
    v = (d[j] - x) - ae[j - 1] * ae[j - 1] / v;
    if (fabs(v) < pivmin) v = -pivmin;
    c += v < 0.0;
  }
  return c;
}

__global__ void __launch_bounds__(128) tri_bisect_kernel(const double *db, const double2 *eb,
                                                          double *lam, double *aeb, int n) {
  const int b = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  const double *d = db + (long)b * n;
  double *ae = aeb + (long)b * n;
  // |e| once per matrix (block 0 of the matrix writes, the others compute their own copy)
  __shared__ double sae[kEigMax], sd[kEigMax];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double2 ej = eb[(long)b * n + j];
    sae[j] = j < n - 1 ? hypot(ej.x, ej.y) : 0.0;
    sd[j] = d[j];
    if (blockIdx.x == 0) ae[j] = sae[j];
  }
  __syncthreads();
  if (i >= n) return;
  int p, q;
  tri_block(sd, sae, n, i, &p, &q);
  const int li = i - p;
  double lo = 1e300, hi = -1e300, emax = 0.0;  // Gershgorin bounds of the block
  for (int j = p; j < q; ++j) {
    const double r = (j > p ? sae[j - 1] : 0.0) + (j + 1 < q ? sae[j] : 0.0);
    lo = fmin(lo, sd[j] - r);
    hi = fmax(hi, sd[j] + r);
    if (j + 1 < q) emax = fmax(emax, sae[j]);
  }
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, emax * emax);
  const double tnorm = fmax(fabs(lo), fabs(hi));
  lo -= 2.2e-16 * tnorm + pivmin;
  hi += 2.2e-16 * tnorm + pivmin;
  for (int it = 0; it < 200; ++it) {  // invariant: count(lo) <= li < count(hi)
    const double mid = 0.5 * (lo + hi);
    if (!(hi - lo > 2.2e-16 * (fabs(lo) + fabs(hi)) + 2.0 * pivmin) || mid <= lo || mid >= hi) break;
    if (tri_count(sd, sae, p, q, mid, pivmin) <= li) lo = mid; else hi = mid;
  }
  lam[(long)b * n + i] = 0.5 * (lo + hi);
}

// inverse iteration for the eigenpairs of a cluster [c0, c1) of block [p, q):
// x <- (T_block - lambda I)^{-1} x, normalized, orthogonalized against the
// cluster's earlier vectors; three solves per vector
__global__ void __launch_bounds__(64) tri_invit_kernel(const double *db, const double *aeb,
                                                        const double *lamb, double *Ztb,
                                                        double *workb, int n) {
  const int b = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double *d = db + (long)b * n, *ae = aeb + (long)b * n, *lam = lamb + (long)b * n;
  double *Zt = Ztb + (long)b * n * n;
  int p, q;
  tri_block(d, ae, n, i, &p, &q);
  double tnorm = 0.0;
  for (int j = p; j < q; ++j)
    tnorm = fmax(tnorm, fabs(d[j]) + (j > p ? ae[j - 1] : 0.0) + (j + 1 < q ? ae[j] : 0.0));
  const int s = q - p;
  double *u0 = workb + ((long)b * n + i) * 5 * n;  // scratch of this thread: 5 s doubles
  double *u1 = u0 + s, *u2 = u1 + s, *lm = u2 + s, *x = lm + s;
  const double tiny = fmax(2.2e-16 * tnorm, 1e-150);  // a zero pivot's stand-in
  {
    const int c = i;
    const double lc = lam[c];
    // LU with partial pivoting of T_block - lc I (lm < 0 marks an interchange)
    double a = d[p] - lc, bsup = s > 1 ? ae[p] : 0.0;
    for (int k = 0; k + 1 < s; ++k) {
      const double cs = ae[p + k], dn = d[p + k + 1] - lc;
      const double un = k + 2 < s ? ae[p + k + 1] : 0.0;
      if (fabs(a) >= fabs(cs)) {
        if (a == 0.0) a = tiny;
        const double l = cs / a;
        u0[k] = a; u1[k] = bsup; u2[k] = 0.0; lm[k] = l;
        a = dn - l * bsup;
        bsup = un;
      } else {  // interchange rows k and k + 1; |l| < 1 is kept as -l - 2 (< -1)
        const double l = a / cs;
        u0[k] = cs; u1[k] = dn; u2[k] = un; lm[k] = -l - 2.0;
        a = bsup - l * dn;
        bsup = -l * un;
      }
    }
    if (a == 0.0) a = tiny;
    u0[s - 1] = a;
    // the start vector: a fixed pseudo-random vector (hash of the row)
    for (int k = 0; k < s; ++k) {
      unsigned h = (unsigned)(k + 1) * 2654435761u ^ (unsigned)(c - p + 7) * 40503u;
      h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
      x[k] = (double)(h & 0xFFFFFF) / 16777216.0 - 0.5;
    }
    for (int it = 0; it < 3; ++it) {
      // forward: the row operations of the factorization
      for (int k = 0; k + 1 < s; ++k) {
        if (lm[k] < -1.0) {  // interchange rows k, k + 1, then eliminate
          const double l = -(lm[k] + 2.0);
          const double t = x[k];
          x[k] = x[k + 1];
          x[k + 1] = t - l * x[k];
        } else {
          x[k + 1] -= lm[k] * x[k];
        }
      }
      // back substitution with U (three diagonals)
      x[s - 1] /= u0[s - 1];
      if (s > 1) x[s - 2] = (x[s - 2] - u1[s - 2] * x[s - 1]) / u0[s - 2];
      for (int k = s - 3; k >= 0; --k) x[k] = (x[k] - u1[k] * x[k + 1] - u2[k] * x[k + 2]) / u0[k];
      double mx = 0.0;  // scale by the largest entry first (the solve can grow x by 1/tiny)
      for (int k = 0; k < s; ++k) mx = fmax(mx, fabs(x[k]));
      if (mx > 0.0 && mx < 1e300) for (int k = 0; k < s; ++k) x[k] /= mx;
      double nrm = 0.0;
      for (int k = 0; k < s; ++k) nrm += x[k] * x[k];
      nrm = 1.0 / sqrt(nrm);
      for (int k = 0; k < s; ++k) x[k] *= nrm;
    }
    double *zc = Zt + (long)c * n;
    for (int r = 0; r < n; ++r) zc[r] = (r >= p && r < q) ? x[r - p] : 0.0;
  }
}

// Classical Gram-Schmidt, twice, over the vectors of each cluster of two or
// more (a block per possible cluster start; warps form the dot products along
// the rows, threads the updates)
__global__ void __launch_bounds__(256) tri_orth_kernel(const double *db, const double *aeb,
                                                        const double *lamb, double *Ztb, int n) {
  __shared__ double coef[kEigMax];
  __shared__ double red[8];
  const int b = blockIdx.y, c0 = blockIdx.x;
  const double *d = db + (long)b * n, *ae = aeb + (long)b * n, *lam = lamb + (long)b * n;
  double *Zt = Ztb + (long)b * n * n;
  int p, q;
  tri_block(d, ae, n, c0, &p, &q);
  double tnorm = 0.0;
  for (int j = p; j < q; ++j)
    tnorm = fmax(tnorm, fabs(d[j]) + (j > p ? ae[j - 1] : 0.0) + (j + 1 < q ? ae[j] : 0.0));
  const double ortol = 1e-3 * tnorm;
  if (c0 > p && lam[c0] - lam[c0 - 1] < ortol) return;  // not the start of a cluster
  int c1 = c0 + 1;
  while (c1 < q && lam[c1] - lam[c1 - 1] < ortol) ++c1;
  if (c1 - c0 < 2) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = c0 + 1; j < c1; ++j) {
    double *zj = Zt + (long)j * n;
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = c0 + warp; i < j; i += 8) {  // coef_i = z_i . z_j
        const double *zi = Zt + (long)i * n;
        double sdot = 0.0;
        for (int r = p + lane; r < q; r += 32) sdot += zi[r] * zj[r];
        for (int o = 16; o > 0; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
        if (lane == 0) coef[i - c0] = sdot;
      }
      __syncthreads();
      for (int r = p + tid; r < q; r += blockDim.x) {  // z_j -= sum_i coef_i z_i
        double v = zj[r];
        for (int i = c0; i < j; ++i) v -= coef[i - c0] * Zt[(long)i * n + r];
        zj[r] = v;
      }
      __syncthreads();
    }
    double sq = 0.0;
    for (int r = p + tid; r < q; r += blockDim.x) sq += zj[r] * zj[r];
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    double tot = 0.0;
    for (int w2 = 0; w2 < 8; ++w2) tot += red[w2];
    const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
    for (int r = p + tid; r < q; r += blockDim.x) zj[r] *= inv;
    __syncthreads();
  }
}

// rank the eigenvalues (ascending, ties by slot) and the phases Phi
__global__ void __launch_bounds__(256) tri_rank_kernel(const double *lamb, const double2 *eb,
                                                        double *wb, int *permb, double2 *phib,
                                                        int n) {
  const int b = blockIdx.x;
  const double *lam = lamb + (long)b * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int rk = 0;
    const double li = lam[i];
    for (int j = 0; j < n; ++j) rk += (lam[j] < li) || (lam[j] == li && j < i);
    wb[(long)b * n + rk] = li;
    permb[(long)b * n + rk] = i;
  }
  if (threadIdx.x == 0) {  // T[j+1][j] = phi_(j+1) conj(phi_j) |e_j|
    double2 ph = make_double2(1.0, 0.0);
    phib[(long)b * n] = ph;
    for (int j = 0; j + 1 < n; ++j) {
      const double2 ej = eb[(long)b * n + j];
      const double a = hypot(ej.x, ej.y);
      if (a > 0.0) ph = cmul(ph, make_double2(ej.x / a, ej.y / a));
      phib[(long)b * n + j + 1] = ph;
    }
  }
}

// V[:, c] = H_0 ... H_(n-3) Phi Z[:, perm[c]] for a slab of kBackW columns.
constexpr int kBackW = 8;
__global__ void __launch_bounds__(256) zback_kernel(const double2 *hvb, const double2 *phib,
                                                     const double *Ztb, const int *permb,
                                                     double2 *Vb, int n) {
  extern __shared__ double2 W[];  // [n][kBackW]
  __shared__ double2 sc[kBackW];
  const int b = blockIdx.y, c0 = blockIdx.x * kBackW;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const double2 *hv = hvb + (long)b * n * n;
  const double *Zt = Ztb + (long)b * n * n;
  const int nc = min(kBackW, n - c0);
  for (int q = tid; q < n * kBackW; q += nt) {
    const int c = q / n, r = q % n;
    double2 v = make_double2(0.0, 0.0);
    if (c < nc) v = cscale(phib[(long)b * n + r], Zt[(long)permb[(long)b * n + c0 + c] * n + r]);
    W[r * kBackW + c] = v;
  }
  __syncthreads();
  for (int j = n - 3; j >= 0; --j) {
    const int o = j + 1, m = n - o;
    const double2 *u = hv + (long)j * n + o;
    if (warp < kBackW) {  // s_c = u^dagger W[o.., c], a warp per column
      double2 s = make_double2(0.0, 0.0);
      for (int i = lane; i < m; i += 32) cfma(s, cconj(u[i]), W[(o + i) * kBackW + warp]);
      for (int q = 16; q > 0; q >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, q);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, q);
      }
      if (lane == 0) sc[warp] = cscale(s, 2.0);
    }
    __syncthreads();
    for (int q = tid; q < m * kBackW; q += nt) {
      const int i = q / kBackW, c = q % kBackW;
      W[(o + i) * kBackW + c] = csub(W[(o + i) * kBackW + c], cmul(u[i], sc[c]));
    }
    __syncthreads();
  }
  for (int q = tid; q < n * kBackW; q += nt) {
    const int r = q / kBackW, c = q % kBackW;
    if (c < nc) Vb[(long)b * n * n + (long)r * n + c0 + c] = W[r * kBackW + c];
  }
}

constexpr int kHtrdGroup = 16;  // blocks per matrix of the group reduction, at most

size_t heev_work_bytes(int n, int batch) {
  const size_t nn = (size_t)n * n * batch;
  return nn * 16 /* hv */ + nn * 8 /* Z */ + (size_t)n * batch * (8 + 16 + 16 + 4) +
         (size_t)batch * (2 * n * 16 + kHtrdGroup * 8 + 4 + 8) +
         (size_t)batch * n * (16 + 5 * (size_t)n * 8) /* bisection: lambda, |e|, scratch */ +
         256 * 16;
}

// A (destroyed) -> w ascending, V (columns); work from heev_work_bytes.
// method 0: QL sweeps; method 1: bisection and inverse iteration.
cudaError_t launch_heev(double2 *A, double *w, double2 *V, int n, int batch, void *work,
                        int *flags, cudaStream_t s, int method) {
  if (n < 1 || n > kEigMax || batch < 1) return cudaErrorInvalidValue;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char *p = (char *)work;
  const size_t nn = (size_t)n * n * batch;
  double2 *hv = (double2 *)p; p += al(nn * 16);
  double *Z = (double *)p; p += al(nn * 8);
  double *d = (double *)p; p += al((size_t)n * batch * 8);
  double2 *e = (double2 *)p; p += al((size_t)n * batch * 16);
  double2 *phi = (double2 *)p; p += al((size_t)n * batch * 16);
  int *perm = (int *)p; p += al((size_t)n * batch * 4);
  HtrdWork hw;
  hw.u = (double2 *)p; p += al((size_t)batch * n * 16);
  hw.p = (double2 *)p; p += al((size_t)batch * n * 16);
  hw.kpart = (double *)p; p += al((size_t)batch * kHtrdGroup * 8);
  hw.skip = (int *)p; p += al((size_t)batch * 4);
  hw.bar = (unsigned *)p; p += al((size_t)batch * 2 * sizeof(unsigned));
  double *lam = (double *)p; p += al((size_t)batch * n * 8);
  double *ae = (double *)p; p += al((size_t)batch * n * 8);
  double *tw = (double *)p;
  cudaError_t err;
  const int smt = 2 * n * (int)sizeof(double2);
  err = cudaFuncSetAttribute(zhetrd_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smt);
  if (err != cudaSuccess) return err;
  // blocks per matrix: up to kHtrdGroup, about 32 rows each, all co-resident
  int dev = 0, sms = 0, per_sm = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
  if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zhetrd_group_kernel, 512, smt)) !=
      cudaSuccess)
    return err;
  int G = std::min(kHtrdGroup, std::max(1, (n + 31) / 32));
  while (G > 1 && (long)G * batch > (long)sms * per_sm) --G;
  if ((long)G * batch > (long)sms * per_sm) return cudaErrorInvalidConfiguration;
  if ((err = cudaMemsetAsync(hw.bar, 0, (size_t)batch * 2 * sizeof(unsigned), s)) != cudaSuccess)
    return err;
  {
    void *args[] = {&A, &hv, &d, &e, &n, &hw, &flags};
    err = cudaLaunchCooperativeKernel((void *)zhetrd_group_kernel, dim3(G, batch), dim3(512), args,
                                      smt, s);
    if (err != cudaSuccess) return err;
  }
  if (method == 1) {
    tri_bisect_kernel<<<dim3((n + 127) / 128, batch), 128, 0, s>>>(d, e, lam, ae, n);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    tri_invit_kernel<<<dim3((n + 63) / 64, batch), 64, 0, s>>>(d, ae, lam, Z, tw, n);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    tri_orth_kernel<<<dim3(n, batch), 256, 0, s>>>(d, ae, lam, Z, n);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    tri_rank_kernel<<<batch, 256, 0, s>>>(lam, e, w, perm, phi, n);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  } else {
    // rows of Z per block: up to kQlRows, as many as 200 KB of shared memory holds
    const int rows = std::max(1, std::min(kQlRows, (200 * 1024 / 8 - 6 * n) / n));
    const int smq = (6 * n + n * rows) * (int)sizeof(double);
    err = cudaFuncSetAttribute(ztql_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smq);
    if (err != cudaSuccess) return err;
    ztql_kernel<<<dim3((n + rows - 1) / rows, batch), 64, smq, s>>>(d, e, w, phi, Z, perm, flags,
                                                                    n, rows);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const int smb = n * kBackW * (int)sizeof(double2);
  err = cudaFuncSetAttribute(zback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
  if (err != cudaSuccess) return err;
  zback_kernel<<<dim3((n + kBackW - 1) / kBackW, batch), 256, smb, s>>>(hv, phi, Z, perm, V, n);
  return cudaGetLastError();
}

// ---- element-wise steps of the k-point path ----------------------------------------
// Variables of one k-point (Eq. 22-24): Re a_ij for i < j, then Im a_ij for
// i <= j, both row-major over the upper triangle.
__host__ __device__ inline long k_re_idx(long i, long j, long M) { return i * M - i * (i + 1) / 2 + (j - i - 1); }
__host__ __device__ inline long k_im_idx(long i, long j, long M) { return i * M - i * (i - 1) / 2 + (j - i); }

// scale * iA(k) (times_i) or scale * A(k) from the variables: A_ij = a_ij
// (i < j), A_ji = -conj(a_ij), A_ii = i Im a_ii (skew-Hermitian, Eq. 8).
__global__ void k_build_iA_kernel(const double *a, int nk, int M, double2 *iA, int times_i,
                                  double scale) {
  const long MM = (long)M * M, nre = (long)M * (M - 1) / 2;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / MM, r = q % MM;
    const int i = (int)(r / M), j = (int)(r % M);
    const double *v = a + k * MM;
    double2 z;
    if (i < j) z = make_double2(-v[nre + k_im_idx(i, j, M)], v[k_re_idx(i, j, M)]);
    else if (i > j) z = make_double2(-v[nre + k_im_idx(j, i, M)], -v[k_re_idx(j, i, M)]);
    else z = make_double2(-v[nre + k_im_idx(i, i, M)], 0.0);
    if (!times_i) z = make_double2(z.y, -z.x);  // A = -i (iA)
    iA[q] = cscale(z, scale);
  }
}

// X[k][r][c] = Y[k][r][c] s[k][c]: mode 0 s = x (real), mode 1 s = x^(-1/2)
// (x <= 0 sets ETDM_ERR_NUMERIC), mode 2 s = exp(-i x) (Eq. 35).
__global__ void k_colscale_kernel(const double2 *Y, const double *x, double2 *X, int nk, int M,
                                  int mode, int *flags) {
  const long MM = (long)M * M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / MM;
    const int c = (int)(q % M);
    const double xv = x[k * M + c];
    double2 s;
    if (mode == 0) {
      s = make_double2(xv, 0.0);
    } else if (mode == 1) {
      if (!(xv > 0.0)) atomicExch(flags + FLAG_ERR, ETDM_ERR_NUMERIC);
      s = make_double2(xv > 0.0 ? 1.0 / sqrt(xv) : 0.0, 0.0);
    } else {
      double sn, cs;
      sincos(xv, &sn, &cs);
      s = make_double2(cs, -sn);
    }
    X[q] = cmul(Y[q], s);
  }
}

// X = (X + X^dagger) / 2, per k-point.
__global__ void k_hermitize_kernel(double2 *X, int nk, int M) {
  const long MM = (long)M * M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / MM, r = q % MM;
    const int i = (int)(r / M), j = (int)(r % M);
    if (i > j) continue;
    double2 *x = X + k * MM;
    const double2 a = x[(long)i * M + j], b = x[(long)j * M + i];
    const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    x[(long)i * M + j] = h;
    x[(long)j * M + i] = cconj(h);
  }
}

__device__ inline void k_offset(const KGeom &G, int ridx, int *R) {
  const int ny = 2 * G.Rm[1] + 1, nz = 2 * G.Rm[2] + 1;
  R[2] = ridx % nz - G.Rm[2];
  R[1] = (ridx / nz) % ny - G.Rm[1];
  R[0] = ridx / (nz * ny) - G.Rm[0];
}

// exp(2 pi i k.R) for fractional k
__device__ inline double2 k_phase(const double *kf, const int *R) {
  const double x = 2.0 * (kf[0] * R[0] + kf[1] * R[1] + kf[2] * R[2]);
  double sn, cs;
  sincospi(x, &sn, &cs);
  return make_double2(cs, sn);
}

// Real-space density matrix per lattice offset (Eq. 2 summed over k):
// DR[R][mu][nu] = Re sum_k exp(2 pi i k.R) D_k[mu][nu].
__global__ void k_dr_kernel(KGeom G, const double2 *D, double *DR) {
  const long MM = (long)G.M * G.M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < G.nR * MM;
       q += (long)gridDim.x * blockDim.x) {
    const int ridx = (int)(q / MM);
    const long r = q % MM;
    int R[3];
    k_offset(G, ridx, R);
    double s = 0.0;
    for (int k = 0; k < G.nk; ++k) {
      const double2 ph = k_phase(G.kfrac + 3 * k, R);
      const double2 d = D[k * MM + r];
      s += ph.x * d.x - ph.y * d.y;
    }
    DR[q] = s;
  }
}

// H_k = T_k + sum_R exp(-2 pi i k.R) VR[R] (Eq. 11 with Bloch functions).
__global__ void k_hamiltonian_kernel(KGeom G, const double2 *T, const double *VR, double2 *H) {
  const long MM = (long)G.M * G.M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < G.nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const int k = (int)(q / MM);
    const long r = q % MM;
    double2 h = T ? T[q] : make_double2(0.0, 0.0);
    for (int ridx = 0; ridx < G.nR; ++ridx) {
      int R[3];
      k_offset(G, ridx, R);
      const double2 ph = k_phase(G.kfrac + 3 * k, R);
      const double v = VR[ridx * MM + r];
      h.x += ph.x * v;
      h.y -= ph.y * v;
    }
    H[q] = h;
  }
}

// L_ij = (f_i - f_j) Hmo_ij (Eq. 13), in place.
__global__ void k_commutator_kernel(double2 *X, const double *f, int nk, int M) {
  const long MM = (long)M * M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / MM, r = q % MM;
    const int i = (int)(r / M), j = (int)(r % M);
    X[q] = cscale(X[q], f[k * M + i] - f[k * M + j]);
  }
}

// Lt_ab *= Dt_ab = int_0^1 exp(-i t (w_a - w_b)) dt = (1 - e^(-i d)) / (i d)
// (Eq. 40, sign as fixed by Eq. 42), series for |d| < 1e-3.
__global__ void k_dtilde_kernel(double2 *X, const double *w, int nk, int M) {
  const long MM = (long)M * M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / MM, r = q % MM;
    const int a = (int)(r / M), b = (int)(r % M);
    const double d = w[k * M + a] - w[k * M + b];
    double2 t;
    if (fabs(d) < 1e-3) {
      t = make_double2(1.0 - d * d / 6.0, -0.5 * d + d * d * d / 24.0);
    } else {
      double sn, cs;
      sincos(d, &sn, &cs);
      t = make_double2(sn / d, (cs - 1.0) / d);  // (1 - cos d + i sin d) / (i d)
    }
    X[q] = cmul(X[q], t);
  }
}

// Real-variable gradient from G^T (Eq. 39, 41, 20): dE/da_ij = (2 - d_ij)/2 G_ij,
// dE/dRe a_ij = 2 Re, dE/dIm a_ij = -2 Im.
__global__ void k_grad_vars_kernel(const double2 *GT, double *g, int nk, int M) {
  const long MM = (long)M * M, nre = (long)M * (M - 1) / 2;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / MM, r = q % MM;
    const int i = (int)(r / M), j = (int)(r % M);
    if (i > j) continue;
    const double2 G = GT[k * MM + (long)j * M + i];  // G_ij
    double *gk = g + k * MM;
    if (i < j) {
      gk[k_re_idx(i, j, M)] = 2.0 * G.x;
      gk[nre + k_im_idx(i, j, M)] = -2.0 * G.y;
    } else {
      gk[nre + k_im_idx(i, i, M)] = -G.y;
    }
  }
}

// Kinetic energy sum_k Re Tr(D_k T_k) = sum Re(D_mn conj(T_mn)) (T Hermitian):
// one partial per block.
__global__ void __launch_bounds__(256) k_kinetic_kernel(const double2 *D, const double2 *T, long n,
                                                        double *part) {
  double s = 0.0;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    s += D[q].x * T[q].x + D[q].y * T[q].y;
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// E = kinetic + external + Hartree + exchange (Eq. 1) from the partials.
__global__ void __launch_bounds__(1024) k_energy_kernel(const double *kpart, int nkp,
                                                        const double *gridpart, int ngp,
                                                        const double *sicpart, int nsp,
                                                        double *eterms, double *E, int *flags) {
  double kin = 0.0, t3[3] = {0.0, 0.0, 0.0}, sic = 0.0;
  for (int b = threadIdx.x; b < nkp; b += blockDim.x) kin += kpart[b];
  for (int b = threadIdx.x; b < nsp; b += blockDim.x) sic += sicpart[b];
  for (int b = threadIdx.x; b < ngp; b += blockDim.x)
    for (int q = 0; q < 3; ++q) t3[q] += gridpart[3 * b + q];
  kin = block_sum(kin);
  sic = block_sum(sic);
  for (int q = 0; q < 3; ++q) t3[q] = block_sum(t3[q]);
  if (threadIdx.x == 0) {
    const double e = kin + t3[0] + t3[1] + t3[2] + sic;
    eterms[0] = kin; eterms[1] = t3[0]; eterms[2] = t3[1]; eterms[3] = t3[2];
    if (E) *E = e;
    if (!(e == e) || isinf(e)) atomicExch(flags + FLAG_ERR, ETDM_ERR_NUMERIC);
  }
}

// 1 / (1 + exp(x)) without overflow
__device__ inline double k_fd(double x) {
  const double e = exp(-fabs(x));
  return x > 0.0 ? e / (1.0 + e) : 1.0 / (1.0 + e);
}

// Occupations of the reference (fixed afterwards): kT > 0: f_m(k) = 2 w_k
// FD((eps_m(k) - mu) / kT) with mu by bisection to sum f = n_e; kT = 0 (one
// k-point): f = 2 on the n_e / 2 lowest eigenvalues (eps ascending per k).
__global__ void __launch_bounds__(1024) k_occupation_kernel(const double *eps, const double *kw,
                                                            int nk, int M, double ne, double kT,
                                                            double *f, double *mu_out) {
  __shared__ double lo_s, hi_s;
  const long n = (long)nk * M;
  if (kT == 0.0) {
    const int N = (int)(ne / 2.0 + 0.5);
    for (long q = threadIdx.x; q < n; q += blockDim.x) f[q] = (q % M) < N ? 2.0 * kw[q / M] : 0.0;
    if (threadIdx.x == 0) *mu_out = 0.0;
    return;
  }
  {  // bracket: [min eps - 50 kT - 1, max eps + 50 kT + 1]
    __shared__ double red[2][32];
    double a = 1e300, b = -1e300;
    for (long q = threadIdx.x; q < n; q += blockDim.x) {
      a = fmin(a, eps[q]);
      b = fmax(b, eps[q]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    if (l == 0) { red[0][w] = a; red[1][w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double A = 1e300, B = -1e300;
      for (int i = 0; i < nw; ++i) { A = fmin(A, red[0][i]); B = fmax(B, red[1][i]); }
      lo_s = A - 50.0 * kT - 1.0;
      hi_s = B + 50.0 * kT + 1.0;
    }
    __syncthreads();
  }
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo_s + hi_s);
    double c = 0.0;
    for (long q = threadIdx.x; q < n; q += blockDim.x) c += 2.0 * kw[q / M] * k_fd((eps[q] - mid) / kT);
    c = block_sum(c);
    if (threadIdx.x == 0) {
      if (c < ne) lo_s = mid; else hi_s = mid;
    }
    __syncthreads();
    const double lo = lo_s, hi = hi_s;
    __syncthreads();
    if (hi - lo <= 1e-13 * fmax(1.0, fabs(0.5 * (lo + hi)))) break;
  }
  const double mu = 0.5 * (lo_s + hi_s);
  for (long q = threadIdx.x; q < n; q += blockDim.x) f[q] = 2.0 * kw[q / M] * k_fd((eps[q] - mu) / kT);
  if (threadIdx.x == 0) *mu_out = mu;
}

// eps_m(k) = Re (C^dagger X)_mm with X = H C (Eq. 33's orbital energies).
__global__ void k_diag_kernel(const double2 *C, const double2 *X, double *out, int nk, int M) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < (long)nk * M;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / M;
    const int m = (int)(q % M);
    const double2 *c = C + k * M * M, *x = X + k * M * M;
    double s = 0.0;
    for (int mu = 0; mu < M; ++mu) {
      const double2 a = c[(long)mu * M + m], b = x[(long)mu * M + m];
      s += a.x * b.x + a.y * b.y;
    }
    out[q] = s;
  }
}

// Preconditioner parts per variable (Eq. 33-34 with the k-point weight on
// beta): den = 2 (1 - gamma) |(e_i - e_j)(f_i - f_j)|, wk = w_k; the same for
// Re a_ij and Im a_ij.
__global__ void k_precond_parts_kernel(const double *eps, const double *f, const double *kw,
                                       int nk, int M, double gamma, double *den, double *wk) {
  const long MM = (long)M * M, nre = (long)M * (M - 1) / 2;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / MM, r = q % MM;
    const int i = (int)(r / M), j = (int)(r % M);
    if (i > j) continue;
    const double *e = eps + k * M, *fk = f + k * M;
    const double dv = 2.0 * (1.0 - gamma) * fabs((e[i] - e[j]) * (fk[i] - fk[j]));
    const long base = k * MM;
    if (i < j) {
      den[base + k_re_idx(i, j, M)] = dv;
      wk[base + k_re_idx(i, j, M)] = kw[k];
    }
    den[base + nre + k_im_idx(i, j, M)] = dv;
    wk[base + nre + k_im_idx(i, j, M)] = kw[k];
  }
}

// S(k), T(k) of normalized s-Gaussians (analytic; Eq. 4, 11 with Bloch
// functions): sum over images n with |d_mu - d_nu - n L| < r_c,mu + r_c,nu of
// exp(2 pi i k.n) s(R), the inclusion test in a fixed operation order.
__global__ void k_overlap_kinetic_kernel(const double *center, const double *alpha,
                                         const double *rcut, int M, double L0, double L1,
                                         double L2, int n0, int n1, int n2, const double *kfrac,
                                         int nk, double2 *S, double2 *T) {
  const long MM = (long)M * M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const int k = (int)(q / MM);
    const long e = q % MM;
    const int mu = (int)(e / M), nu = (int)(e % M);
    const double a = alpha[mu], b = alpha[nu];
    const double xi = a * b / (a + b);
    const double pre = pow(2.0 * sqrt(a * b) / (a + b), 1.5);
    const double cut = __dadd_rn(rcut[mu], rcut[nu]);
    const double cut2 = __dmul_rn(cut, cut);
    const double d0 = __dsub_rn(center[mu * 3], center[nu * 3]);
    const double d1 = __dsub_rn(center[mu * 3 + 1], center[nu * 3 + 1]);
    const double d2 = __dsub_rn(center[mu * 3 + 2], center[nu * 3 + 2]);
    const double *kf = kfrac + 3 * k;
    double2 s = make_double2(0.0, 0.0), t = make_double2(0.0, 0.0);
    for (int ix = -n0; ix <= n0; ++ix)
      for (int iy = -n1; iy <= n1; ++iy)
        for (int iz = -n2; iz <= n2; ++iz) {
          const double r0 = __dsub_rn(d0, __dmul_rn((double)ix, L0));
          const double r1 = __dsub_rn(d1, __dmul_rn((double)iy, L1));
          const double r2 = __dsub_rn(d2, __dmul_rn((double)iz, L2));
          const double R2 = __dadd_rn(__dadd_rn(__dmul_rn(r0, r0), __dmul_rn(r1, r1)),
                                      __dmul_rn(r2, r2));
          if (R2 < cut2) {
            const int n[3] = {ix, iy, iz};
            const double2 ph = k_phase(kf, n);
            const double v = pre * exp(-xi * R2);
            const double tv = xi * (3.0 - 2.0 * xi * R2) * v;
            s.x += ph.x * v; s.y += ph.y * v;
            t.x += ph.x * tv; t.y += ph.y * tv;
          }
        }
    S[q] = s;
    T[q] = t;
  }
}

static int k_blocks(long n);

// ---- Perdew-Zunger self-interaction correction (Gamma point) ------------------------
// D = O_k O_k^dagger for orbital column k (the unit orbital density's matrix)
__global__ void k_rank1_kernel(const double2 *O, int k, int M, double2 *D) {
  const long MM = (long)M * M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < MM; q += (long)gridDim.x * blockDim.x) {
    const int mu = (int)(q / M), nu = (int)(q % M);
    D[q] = cmul(O[(long)mu * M + k], cconj(O[(long)nu * M + k]));
  }
}

// v_k = v_H[n_k] + v_x^pol[n_k] with v_x^pol = -(6/pi)^(1/3) n^(1/3) (a fully
// polarized density), and the block partials of -f_k (E_H + E_x^pol):
// part[b] = -f_k dV (sum n v_H / 2 + sum e_x^pol), e_x^pol = 3/4 n v_x^pol
__global__ void __launch_bounds__(256) k_sic_potential_kernel(const double *n, const double2 *vh,
                                                              double *v, long G, double dV,
                                                              double fk, double *part) {
  const double cx = cbrt(6.0 / M_PI);
  double s = 0.0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < G; e += (long)gridDim.x * blockDim.x) {
    const double r = n[e];
    const double rp = r > 0.0 ? r : 0.0;
    const double vx = -cx * cbrt(rp);
    const double h = vh[e].x;
    v[e] = h + vx;
    s += 0.5 * r * h + 0.75 * rp * vx;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = -fk * dV * s;
}

// L += S diag(f) - (S diag(f))^dagger, S_mk = <phi_m|V^k|phi_k>
__global__ void k_sic_L_kernel(double2 *L, const double2 *S, const double *f, int M) {
  const long MM = (long)M * M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < MM; q += (long)gridDim.x * blockDim.x) {
    const int m = (int)(q / M), k = (int)(q % M);
    const double2 a = cscale(S[q], f[k]);
    const double2 b = cscale(cconj(S[(long)k * M + m]), f[m]);
    L[q] = cadd(L[q], csub(a, b));
  }
}

cudaError_t k_rank1(const double2 *O, int k, int M, double2 *D, cudaStream_t s) {
  k_rank1_kernel<<<k_blocks((long)M * M), 256, 0, s>>>(O, k, M, D);
  return cudaGetLastError();
}
int k_sic_parts() { return 256; }
cudaError_t k_sic_potential(const double *n, const double2 *vh, double *v, long G, double dV,
                            double fk, double *part, cudaStream_t s) {
  k_sic_potential_kernel<<<k_sic_parts(), 256, 0, s>>>(n, vh, v, G, dV, fk, part);
  return cudaGetLastError();
}
cudaError_t k_sic_L(double2 *L, const double2 *S, const double *f, int M, cudaStream_t s) {
  k_sic_L_kernel<<<k_blocks((long)M * M), 256, 0, s>>>(L, S, f, M);
  return cudaGetLastError();
}

// ---- launchers ------------------------------------------------------------------------
static int k_blocks(long n) {
  long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t k_build_iA(const double *a, int nk, int M, double2 *iA, cudaStream_t s,
                       int times_i, double scale) {
  k_build_iA_kernel<<<k_blocks((long)nk * M * M), 256, 0, s>>>(a, nk, M, iA, times_i, scale);
  return cudaGetLastError();
}

// ---- scaling and squaring (Eq. 38) and the approximate gradient (Eq. 42) ------
// max over k-points of the largest column sum of |X| (the 1-norm), as the
// bits of a non-negative double (their integer order is the value order)
__global__ void k_norm1_kernel(const double2 *X, int nk, int M, unsigned long long *out) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < (long)nk * M;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / M;
    const int c = (int)(q % M);
    const double2 *x = X + k * M * M;
    double sum = 0.0;
    for (int r = 0; r < M; ++r) sum += hypot(x[(long)r * M + c].x, x[(long)r * M + c].y);
    atomicMax(out, (unsigned long long)__double_as_longlong(sum));
  }
}

// Q = c0 I + c1 B + c2 B2 (a Horner coefficient of the Taylor polynomial in B^3)
__global__ void k_poly_kernel(double2 *Q, const double2 *B, const double2 *B2, double c0,
                              double c1, double c2, int nk, int M) {
  const long MM = (long)M * M;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const long r = q % MM;
    double2 v = make_double2(c1 * B[q].x + c2 * B2[q].x, c1 * B[q].y + c2 * B2[q].y);
    if (r / M == r % M) v.x += c0;
    Q[q] = v;
  }
}

// L(k) from approximate-gradient variables (Eq. 42: dE/da_ij = (2 - d_ij)/2 L_ji):
// L_ji = (g_re - i g_im) / 2 for i < j, L_ii = -i g_im, L_ij = -conj(L_ji).
__global__ void k_from_grad_kernel(const double *g, double2 *L, int nk, int M) {
  const long MM = (long)M * M, nre = (long)M * (M - 1) / 2;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nk * MM;
       q += (long)gridDim.x * blockDim.x) {
    const long k = q / MM, r = q % MM;
    const int row = (int)(r / M), col = (int)(r % M);
    const double *gk = g + k * MM;
    double2 v;
    if (row == col) {
      v = make_double2(0.0, -gk[nre + k_im_idx(row, row, M)]);
    } else if (row > col) {  // L_ji with j = row > i = col
      v = make_double2(0.5 * gk[k_re_idx(col, row, M)], -0.5 * gk[nre + k_im_idx(col, row, M)]);
    } else {                 // L_ij = -conj(L_ji)
      v = make_double2(-0.5 * gk[k_re_idx(row, col, M)], -0.5 * gk[nre + k_im_idx(row, col, M)]);
    }
    L[q] = v;
  }
}

// sum |X|^2 (Frobenius norm squared over all k-points): block partials
__global__ void __launch_bounds__(256) k_fro2_kernel(const double2 *X, long n, double *part) {
  double s = 0.0;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    s += X[q].x * X[q].x + X[q].y * X[q].y;
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

cudaError_t k_norm1(const double2 *X, int nk, int M, unsigned long long *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_norm1_kernel<<<k_blocks((long)nk * M), 256, 0, s>>>(X, nk, M, out);
  return cudaGetLastError();
}
cudaError_t k_poly(double2 *Q, const double2 *B, const double2 *B2, double c0, double c1,
                   double c2, int nk, int M, cudaStream_t s) {
  k_poly_kernel<<<k_blocks((long)nk * M * M), 256, 0, s>>>(Q, B, B2, c0, c1, c2, nk, M);
  return cudaGetLastError();
}
cudaError_t k_from_grad(const double *g, double2 *L, int nk, int M, cudaStream_t s) {
  k_from_grad_kernel<<<k_blocks((long)nk * M * M), 256, 0, s>>>(g, L, nk, M);
  return cudaGetLastError();
}
int k_fro2_parts() { return 256; }
cudaError_t k_fro2(const double2 *X, long n, double *part, cudaStream_t s) {
  k_fro2_kernel<<<k_fro2_parts(), 256, 0, s>>>(X, n, part);
  return cudaGetLastError();
}
cudaError_t k_colscale(const double2 *Y, const double *x, double2 *X, int nk, int M, int mode,
                       int *flags, cudaStream_t s) {
  k_colscale_kernel<<<k_blocks((long)nk * M * M), 256, 0, s>>>(Y, x, X, nk, M, mode, flags);
  return cudaGetLastError();
}
cudaError_t k_hermitize(double2 *X, int nk, int M, cudaStream_t s) {
  k_hermitize_kernel<<<k_blocks((long)nk * M * M), 256, 0, s>>>(X, nk, M);
  return cudaGetLastError();
}
cudaError_t k_dr(const KGeom &G, const double2 *D, double *DR, cudaStream_t s) {
  k_dr_kernel<<<k_blocks((long)G.nR * G.M * G.M), 256, 0, s>>>(G, D, DR);
  return cudaGetLastError();
}
cudaError_t k_hamiltonian(const KGeom &G, const double2 *T, const double *VR, double2 *H,
                          cudaStream_t s) {
  k_hamiltonian_kernel<<<k_blocks((long)G.nk * G.M * G.M), 256, 0, s>>>(G, T, VR, H);
  return cudaGetLastError();
}
cudaError_t k_commutator(double2 *X, const double *f, int nk, int M, cudaStream_t s) {
  k_commutator_kernel<<<k_blocks((long)nk * M * M), 256, 0, s>>>(X, f, nk, M);
  return cudaGetLastError();
}
cudaError_t k_dtilde(double2 *X, const double *w, int nk, int M, cudaStream_t s) {
  k_dtilde_kernel<<<k_blocks((long)nk * M * M), 256, 0, s>>>(X, w, nk, M);
  return cudaGetLastError();
}
cudaError_t k_grad_vars(const double2 *GT, double *g, int nk, int M, cudaStream_t s) {
  k_grad_vars_kernel<<<k_blocks((long)nk * M * M), 256, 0, s>>>(GT, g, nk, M);
  return cudaGetLastError();
}
int k_kinetic_parts() { return 512; }
cudaError_t k_energy(const double2 *D, const double2 *T, long n, double *part,
                     const double *gridpart, int ngp, double *eterms, double *E, int *flags,
                     cudaStream_t s, const double *sicpart, int nsp) {
  k_kinetic_kernel<<<k_kinetic_parts(), 256, 0, s>>>(D, T, n, part);
  k_energy_kernel<<<1, 1024, 0, s>>>(part, k_kinetic_parts(), gridpart, ngp, sicpart, nsp, eterms,
                                     E, flags);
  return cudaGetLastError();
}
cudaError_t k_occupation(const double *eps, const double *kw, int nk, int M, double ne, double kT,
                         double *f, double *mu, cudaStream_t s) {
  k_occupation_kernel<<<1, 1024, 0, s>>>(eps, kw, nk, M, ne, kT, f, mu);
  return cudaGetLastError();
}
cudaError_t k_diag(const double2 *C, const double2 *X, double *out, int nk, int M, cudaStream_t s) {
  k_diag_kernel<<<k_blocks((long)nk * M), 256, 0, s>>>(C, X, out, nk, M);
  return cudaGetLastError();
}
cudaError_t k_precond_parts(const double *eps, const double *f, const double *kw, int nk, int M,
                            double gamma, double *den, double *wk, cudaStream_t s) {
  k_precond_parts_kernel<<<k_blocks((long)nk * M * M), 256, 0, s>>>(eps, f, kw, nk, M, gamma, den, wk);
  return cudaGetLastError();
}
cudaError_t k_overlap_kinetic(etdm_handle *h, cudaStream_t s) {
  double rmax = 0.0;
  std::vector<double> rc(h->M);
  CUDA_TRY(cudaMemcpy(rc.data(), h->d_rcut, h->M * sizeof(double), cudaMemcpyDeviceToHost));
  for (double r : rc) rmax = std::max(rmax, r);
  int nimg[3];
  for (int a = 0; a < 3; ++a) nimg[a] = (int)floor(2.0 * rmax / h->L[a]) + 1;
  k_overlap_kinetic_kernel<<<k_blocks((long)h->nk * h->M * h->M), 256, 0, s>>>(
      h->d_center, h->d_alpha, h->d_rcut, h->M, h->L[0], h->L[1], h->L[2], nimg[0], nimg[1],
      nimg[2], h->d_kfrac, h->nk, h->d_kS, h->d_kT);
  return cudaGetLastError();
}

}  // namespace etdm
