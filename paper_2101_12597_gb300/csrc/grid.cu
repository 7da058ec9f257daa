// Real-space grid work of one ETDM evaluation (FP64 path) and its set-up:
//  - separable basis tables of the truncated, periodic s-Gaussians (Eq. 5 at
//    the Gamma point), with the hard cut r^2 < r_c^2 decided in FP64 with a
//    fixed operation order so the truncation lists are bit-exact;
//  - per-tile truncation lists (function images touching a grid tile);
//  - analytic overlap and kinetic matrices (Eq. 4 and the kinetic part of
//    Eq. 11) of normalized s-Gaussians summed over lattice images;
//  - basis -> grid density rho(r) = sum chi_mu D_mu,nu chi_nu (Eq. 2, 12);
//  - grid -> basis potential matrix V_mu,nu = dV sum chi_mu v chi_nu (Eq. 11).
#include <math.h>

#include "device.cuh"
#include "internal.h"
#include "kpoint.h"

namespace etdm {

// ---- tables -----------------------------------------------------------------
__global__ void tables_kernel(const double *center, const double *alpha, int M, int n_ax,
                              double h, double L, int ax, double *sq, double *ex) {
  long total = (long)M * kImgN * n_ax;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int i = (int)(e % n_ax);
    int img = (int)((e / n_ax) % kImgN);
    int mu = (int)(e / ((long)n_ax * kImgN));
    double x = __dmul_rn((double)i, h);
    double c = __dadd_rn(center[mu * 3 + ax], __dmul_rn((double)(img - kImgMax), L));
    double d = __dsub_rn(x, c);
    double s = __dmul_rn(d, d);
    sq[e] = s;
    ex[e] = exp(-alpha[mu] * s);
  }
}

cudaError_t launch_tables(etdm_handle *h, cudaStream_t s) {
  const int nn[3] = {h->n[0], h->n[1], h->n[2]};
  for (int ax = 0; ax < 3; ++ax) {
    long total = (long)h->M * kImgN * nn[ax];
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    tables_kernel<<<blocks, 256, 0, s>>>(h->d_center, h->d_alpha, h->M, nn[ax], h->h[ax],
                                         h->L[ax], ax, h->d_sq + h->tab_off[ax],
                                         h->d_ex + h->tab_off[ax]);
  }
  return cudaGetLastError();
}

struct TileRange {
  int i0, i1, j0, j1, k0, k1;
};

__device__ __forceinline__ TileRange tile_range(const GridGeom &g, int t) {
  int bz = t % g.nbz, by = (t / g.nbz) % g.nby, bx = t / (g.nbz * g.nby);
  TileRange r;
  r.i0 = bx * g.tx; r.i1 = min(r.i0 + g.tx, g.nx);
  r.j0 = by * g.ty; r.j1 = min(r.j0 + g.ty, g.ny);
  r.k0 = bz * g.tz; r.k1 = min(r.k0 + g.tz, g.nz);
  return r;
}

__device__ __forceinline__ int img_limit(double rc, double L) {
  int m = (int)floor(rc / L) + 1;
  return m < kImgMax ? m : kImgMax;
}

// Visit the images of mu that reach tile t, in (nx, ny, nz) lexicographic order.
// Inclusion: min over the tile of ((sqx + sqy) + sqz) < r_c^2; by monotonicity of
// rounded addition this equals "some point of the tile is inside".
template <typename F>
__device__ void for_tile_images(const GridGeom &g, const double *sqx, const double *sqy,
                                const double *sqz, const double *rcut, const double *rc2,
                                const double *Lb, int t, int mu, F f) {
  TileRange r = tile_range(g, t);
  int mx = img_limit(rcut[mu], Lb[0]), my = img_limit(rcut[mu], Lb[1]),
      mz = img_limit(rcut[mu], Lb[2]);
  for (int ix = -mx; ix <= mx; ++ix) {
    const double *px = sqx + ((long)mu * kImgN + ix + kImgMax) * g.nx;
    double a = INFINITY;
    for (int i = r.i0; i < r.i1; ++i) a = fmin(a, px[i]);
    if (!(a < rc2[mu])) continue;
    for (int iy = -my; iy <= my; ++iy) {
      const double *py = sqy + ((long)mu * kImgN + iy + kImgMax) * g.ny;
      double b = INFINITY;
      for (int j = r.j0; j < r.j1; ++j) b = fmin(b, py[j]);
      double ab = __dadd_rn(a, b);
      if (!(ab < rc2[mu])) continue;
      for (int iz = -mz; iz <= mz; ++iz) {
        const double *pz = sqz + ((long)mu * kImgN + iz + kImgMax) * g.nz;
        double c = INFINITY;
        for (int k = r.k0; k < r.k1; ++k) c = fmin(c, pz[k]);
        if (__dadd_rn(ab, c) < rc2[mu]) f(ix, iy, iz);
      }
    }
  }
}

__global__ void list_count_kernel(GridGeom g, const double *sqx, const double *sqy,
                                  const double *sqz, const double *rcut, const double *rc2,
                                  double L0, double L1, double L2, int n_tiles, int *count) {
  const double Lb[3] = {L0, L1, L2};
  long total = (long)n_tiles * g.M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int t = (int)(e / g.M), mu = (int)(e % g.M);
    int c = 0;
    for_tile_images(g, sqx, sqy, sqz, rcut, rc2, Lb, t, mu, [&](int, int, int) { ++c; });
    count[e] = c;
  }
}

__global__ void list_fill_kernel(GridGeom g, const double *sqx, const double *sqy,
                                 const double *sqz, const double *rcut, const double *rc2,
                                 double L0, double L1, double L2, int n_tiles,
                                 const long long *off, int *keys) {
  const double Lb[3] = {L0, L1, L2};
  long total = (long)n_tiles * g.M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int t = (int)(e / g.M), mu = (int)(e % g.M);
    long long o = off[e];
    for_tile_images(g, sqx, sqy, sqz, rcut, rc2, Lb, t, mu, [&](int ix, int iy, int iz) {
      keys[o++] = mu * 512 + (ix + 4) * 64 + (iy + 4) * 8 + (iz + 4);
    });
  }
}

cudaError_t launch_list_count(etdm_handle *h, const GridGeom &g, int n_tiles, int *d_count,
                              cudaStream_t s) {
  long total = (long)n_tiles * h->M;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  list_count_kernel<<<blocks, 256, 0, s>>>(
      g, h->d_sq + h->tab_off[0], h->d_sq + h->tab_off[1], h->d_sq + h->tab_off[2],
      h->d_rcut, h->d_rc2, h->L[0], h->L[1], h->L[2], n_tiles, d_count);
  return cudaGetLastError();
}

cudaError_t launch_list_fill(etdm_handle *h, const GridGeom &g, int n_tiles, const long long *d_off,
                             int *d_keys, cudaStream_t s) {
  long total = (long)n_tiles * h->M;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  list_fill_kernel<<<blocks, 256, 0, s>>>(
      g, h->d_sq + h->tab_off[0], h->d_sq + h->tab_off[1], h->d_sq + h->tab_off[2],
      h->d_rcut, h->d_rc2, h->L[0], h->L[1], h->L[2], n_tiles, d_off, d_keys);
  return cudaGetLastError();
}

// ---- exclusive scan (int -> int64), three passes ----------------------------
constexpr int kScanB = 1024;

__global__ void __launch_bounds__(kScanB) scan_block_kernel(const int *in, long long *out,
                                                            long n, long long *blocksum) {
  __shared__ long long sh[kScanB];
  long i = (long)blockIdx.x * kScanB + threadIdx.x;
  long long v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < kScanB; o <<= 1) {
    long long t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == kScanB - 1) blocksum[blockIdx.x] = sh[threadIdx.x];
}

__global__ void __launch_bounds__(1024) scan_sums_kernel(long long *blocksum, long nb,
                                                         long long *total) {
  // single block, sequential chunks of 1024
  __shared__ long long sh[1024];
  long long carry = 0;
  for (long base = 0; base < nb; base += 1024) {
    long i = base + threadIdx.x;
    long long v = i < nb ? blocksum[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      long long t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) blocksum[i] = carry + sh[threadIdx.x] - v;
    long long last = sh[1023];
    __syncthreads();
    carry += last;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_add_kernel(long long *out, long n, const long long *blocksum) {
  long i = (long)blockIdx.x * kScanB + threadIdx.x;
  if (i < n) out[i] += blocksum[blockIdx.x];
}

// d_tmp: [nblocks + 1] scratch; d_out[n] gets the exclusive scan and
// d_tmp[nblocks] the total.
cudaError_t launch_scan(const int *d_in, long long *d_out, long n, long long *d_tmp,
                        cudaStream_t s) {
  long nb = (n + kScanB - 1) / kScanB;
  if (nb < 1) nb = 1;
  scan_block_kernel<<<(unsigned)nb, kScanB, 0, s>>>(d_in, d_out, n, d_tmp);
  scan_sums_kernel<<<1, 1024, 0, s>>>(d_tmp, nb, d_tmp + nb);
  scan_add_kernel<<<(unsigned)nb, kScanB, 0, s>>>(d_out, n, d_tmp);
  return cudaGetLastError();
}

// ---- per-point function counts: sum_p n_pt(p)^2 ------------------------------
__device__ __forceinline__ void decode_key(int key, int &mu, int &ix, int &iy, int &iz) {
  mu = key >> 9;
  ix = ((key >> 6) & 7) - 4 + kImgMax;
  iy = ((key >> 3) & 7) - 4 + kImgMax;
  iz = (key & 7) - 4 + kImgMax;
}

__global__ void npt2_kernel(GridGeom g, const int *tile_ptr, const int *keys, Tables tb,
                            unsigned long long *sum) {
  int t = blockIdx.x;
  TileRange r = tile_range(g, t);
  int kb = tile_ptr[t], ke = tile_ptr[t + 1];
  unsigned long long acc = 0;
  int npts = g.tx * g.ty * g.tz;
  for (int p = threadIdx.x; p < npts; p += blockDim.x) {
    int pk = p % g.tz, pj = (p / g.tz) % g.ty, pi = p / (g.tz * g.ty);
    int i = r.i0 + pi, j = r.j0 + pj, k = r.k0 + pk;
    if (i >= r.i1 || j >= r.j1 || k >= r.k1) continue;
    int c = 0;
    for (int e = kb; e < ke; ++e) {
      int mu, ix, iy, iz;
      decode_key(keys[e], mu, ix, iy, iz);
      double r2 = __dadd_rn(__dadd_rn(tb.sq[0][((long)mu * kImgN + ix) * g.nx + i],
                                      tb.sq[1][((long)mu * kImgN + iy) * g.ny + j]),
                            tb.sq[2][((long)mu * kImgN + iz) * g.nz + k]);
      if (r2 < tb.rc2[mu]) ++c;
    }
    acc += (unsigned long long)c * c;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sum, acc);
}

static Tables tables_of(etdm_handle *h) {
  Tables tb;
  for (int a = 0; a < 3; ++a) {
    tb.sq[a] = h->d_sq + h->tab_off[a];
    tb.ex[a] = h->d_ex + h->tab_off[a];
  }
  tb.norm = h->d_norm;
  tb.rc2 = h->d_rc2;
  return tb;
}

cudaError_t launch_npt2(etdm_handle *h, unsigned long long *d_sum, cudaStream_t s) {
  npt2_kernel<<<h->n_tiles, 128, 0, s>>>(h->geom, h->d_tile_ptr, h->d_keys, tables_of(h),
                                         d_sum);
  return cudaGetLastError();
}

// ---- analytic S and T ---------------------------------------------------------
__global__ void overlap_kinetic_kernel(const double *center, const double *alpha,
                                       const double *rcut, int M, double L0, double L1,
                                       double L2, double *S, double *T) {
  long MM = (long)M * M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MM;
       e += (long)gridDim.x * blockDim.x) {
    int mu = (int)(e / M), nu = (int)(e % M);
    double a = alpha[mu], b = alpha[nu];
    double xi = a * b / (a + b);
    double pre = pow(2.0 * sqrt(a * b) / (a + b), 1.5);
    // pair images with |d_mu - d_nu - R| < r_c,mu + r_c,nu; the inclusion test
    // uses a fixed operation order without contraction (boundary pairs exist)
    double cut = __dadd_rn(rcut[mu], rcut[nu]);
    double cut2 = __dmul_rn(cut, cut);
    double d0 = __dsub_rn(center[mu * 3], center[nu * 3]);
    double d1 = __dsub_rn(center[mu * 3 + 1], center[nu * 3 + 1]);
    double d2 = __dsub_rn(center[mu * 3 + 2], center[nu * 3 + 2]);
    double s = 0.0, t = 0.0;
    for (int ix = -kImgMax; ix <= kImgMax; ++ix)
      for (int iy = -kImgMax; iy <= kImgMax; ++iy)
        for (int iz = -kImgMax; iz <= kImgMax; ++iz) {
          double r0 = __dsub_rn(d0, __dmul_rn((double)ix, L0));
          double r1 = __dsub_rn(d1, __dmul_rn((double)iy, L1));
          double r2 = __dsub_rn(d2, __dmul_rn((double)iz, L2));
          double R2 = __dadd_rn(__dadd_rn(__dmul_rn(r0, r0), __dmul_rn(r1, r1)),
                                __dmul_rn(r2, r2));
          if (R2 < cut2) {
            double v = pre * exp(-xi * R2);
            s += v;
            t += xi * (3.0 - 2.0 * xi * R2) * v;
          }
        }
    S[e] = s;
    T[e] = t;
  }
}

cudaError_t launch_overlap_kinetic(etdm_handle *h, cudaStream_t s) {
  long MM = (long)h->M * h->M;
  int blocks = (int)((MM + 127) / 128);
  if (blocks > 8192) blocks = 8192;
  overlap_kinetic_kernel<<<blocks, 128, 0, s>>>(h->d_center, h->d_alpha, h->d_rcut, h->M,
                                                h->L[0], h->L[1], h->L[2], h->d_S, h->d_T);
  return cudaGetLastError();
}

// ---- FP64 grid passes: one block per 4x4x4 tile ------------------------------
constexpr int kTP = 64;        // points per tile (4 x 4 x 4)
constexpr int kRhoThreads = 256;
constexpr int kChunk = 16;     // rows of D staged at once

// X[e][p] = chi of list entry e at tile point p (0 outside the grid or r_c).
__device__ void build_tile_basis(const GridGeom &g, const Tables &tb, const int *keys, int n,
                                 const TileRange &r, int *mu_s, double *X) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) mu_s[e] = keys[e] >> 9;
  for (int q = threadIdx.x; q < n * kTP; q += blockDim.x) {
    int e = q / kTP, p = q % kTP;
    int pk = p % g.tz, pj = (p / g.tz) % g.ty, pi = p / (g.tz * g.ty);
    int i = r.i0 + pi, j = r.j0 + pj, k = r.k0 + pk;
    double v = 0.0;
    if (i < r.i1 && j < r.j1 && k < r.k1) {
      int mu, ix, iy, iz;
      decode_key(keys[e], mu, ix, iy, iz);
      long bx = ((long)mu * kImgN + ix) * g.nx + i;
      long by = ((long)mu * kImgN + iy) * g.ny + j;
      long bz = ((long)mu * kImgN + iz) * g.nz + k;
      double r2 = __dadd_rn(__dadd_rn(tb.sq[0][bx], tb.sq[1][by]), tb.sq[2][bz]);
      if (r2 < tb.rc2[mu]) v = tb.norm[mu] * tb.ex[0][bx] * tb.ex[1][by] * tb.ex[2][bz];
    }
    X[e * kTP + p] = v;
  }
}

__global__ void __launch_bounds__(kRhoThreads) rho_fp64_kernel(GridGeom g, Tables tb,
                                                               const int *tile_ptr,
                                                               const int *keys,
                                                               const double *D, double *rho) {
  extern __shared__ double smem[];
  const int t = blockIdx.x;
  const int kb = tile_ptr[t], n = tile_ptr[t + 1] - kb;
  double *X = smem;                       // [n][64]
  double *Dc = X + (long)n * kTP;         // [kChunk][n]
  int *mu_s = (int *)(Dc + (long)kChunk * n);
  __shared__ double part[kRhoThreads];
  TileRange r = tile_range(g, t);
  build_tile_basis(g, tb, keys + kb, n, r, mu_s, X);
  __syncthreads();
  const int p = threadIdx.x % kTP, grp = threadIdx.x / kTP, ngrp = kRhoThreads / kTP;
  double acc = 0.0;
  for (int a0 = 0; a0 < n; a0 += kChunk) {
    int rows = min(kChunk, n - a0);
    for (int q = threadIdx.x; q < rows * n; q += blockDim.x) {
      int rr = q / n, b = q % n;
      Dc[rr * n + b] = D[(long)mu_s[a0 + rr] * g.M + mu_s[b]];
    }
    __syncthreads();
    for (int rr = grp; rr < rows; rr += ngrp) {
      const double *drow = Dc + rr * n;
      double y = 0.0;
      for (int b = 0; b < n; ++b) y = fma(drow[b], X[b * kTP + p], y);
      acc = fma(X[(a0 + rr) * kTP + p], y, acc);
    }
    __syncthreads();
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < kTP) {
    double s = 0.0;
    for (int q = 0; q < ngrp; ++q) s += part[q * kTP + threadIdx.x];
    int pk = p % g.tz, pj = (p / g.tz) % g.ty, pi = p / (g.tz * g.ty);
    int i = r.i0 + pi, j = r.j0 + pj, k = r.k0 + pk;
    if (i < r.i1 && j < r.j1 && k < r.k1) rho[((long)i * g.ny + j) * g.nz + k] = s;
  }
}

static size_t rho_smem(int n) {
  return (size_t)n * kTP * 8 + (size_t)kChunk * n * 8 + (size_t)n * 4 + 16;
}

cudaError_t launch_rho_fp64(etdm_handle *h, const double *D, double *rho, cudaStream_t s) {
  size_t sm = rho_smem(h->max_list);
  cudaError_t e = cudaFuncSetAttribute(rho_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  rho_fp64_kernel<<<h->n_tiles, kRhoThreads, sm, s>>>(h->geom, tables_of(h), h->d_tile_ptr,
                                                      h->d_keys, D, rho);
  return cudaGetLastError();
}

// V_ab = dV sum_p X_ap v_p X_bp for a <= b (keys sorted, so mu_a <= mu_b);
// accumulated into the upper triangle of Hacc.
__global__ void __launch_bounds__(kRhoThreads) vmat_fp64_kernel(GridGeom g, Tables tb,
                                                                const int *tile_ptr,
                                                                const int *keys,
                                                                const double *v,
                                                                double *Hacc) {
  extern __shared__ double smem[];
  const int t = blockIdx.x;
  const int kb = tile_ptr[t], n = tile_ptr[t + 1] - kb;
  double *X = smem;                          // [n][65] padded
  double *Xv = X + (long)n * (kTP + 1);      // [n][65]
  int *mu_s = (int *)(Xv + (long)n * (kTP + 1));
  __shared__ double vp[kTP];
  TileRange r = tile_range(g, t);
  // build padded X
  for (int e = threadIdx.x; e < n; e += blockDim.x) mu_s[e] = keys[kb + e] >> 9;
  if (threadIdx.x < kTP) {
    int p = threadIdx.x;
    int pk = p % g.tz, pj = (p / g.tz) % g.ty, pi = p / (g.tz * g.ty);
    int i = r.i0 + pi, j = r.j0 + pj, k = r.k0 + pk;
    vp[p] = (i < r.i1 && j < r.j1 && k < r.k1) ? v[((long)i * g.ny + j) * g.nz + k] * g.dV
                                                 : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n * kTP; q += blockDim.x) {
    int e = q / kTP, p = q % kTP;
    int pk = p % g.tz, pj = (p / g.tz) % g.ty, pi = p / (g.tz * g.ty);
    int i = r.i0 + pi, j = r.j0 + pj, k = r.k0 + pk;
    double val = 0.0;
    if (i < r.i1 && j < r.j1 && k < r.k1) {
      int mu, ix, iy, iz;
      decode_key(keys[kb + e], mu, ix, iy, iz);
      long bx = ((long)mu * kImgN + ix) * g.nx + i;
      long by = ((long)mu * kImgN + iy) * g.ny + j;
      long bz = ((long)mu * kImgN + iz) * g.nz + k;
      double r2 = __dadd_rn(__dadd_rn(tb.sq[0][bx], tb.sq[1][by]), tb.sq[2][bz]);
      if (r2 < tb.rc2[mu]) val = tb.norm[mu] * tb.ex[0][bx] * tb.ex[1][by] * tb.ex[2][bz];
    }
    X[e * (kTP + 1) + p] = val;
    Xv[e * (kTP + 1) + p] = val * vp[p];
  }
  __syncthreads();
  // pairs (a, b) with a <= b: warp per a, lanes over b
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int a = warp; a < n; a += nw) {
    const double *xa = Xv + a * (kTP + 1);
    for (int b = a + lane; b < n; b += 32) {
      const double *xb = X + b * (kTP + 1);
      double s = 0.0;
#pragma unroll 8
      for (int p = 0; p < kTP; ++p) s = fma(xa[p], xb[p], s);
      int ma = mu_s[a], mb = mu_s[b];
      if (ma == mb && a != b) s *= 2.0;
      if (s != 0.0) atomicAdd(Hacc + (long)ma * g.M + mb, s);
    }
  }
}

cudaError_t launch_vmat_fp64(etdm_handle *h, const double *v, double *Hacc, cudaStream_t s) {
  size_t sm = (size_t)h->max_list * (kTP + 1) * 16 + (size_t)h->max_list * 4 + 16;
  cudaError_t e = cudaFuncSetAttribute(vmat_fp64_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  vmat_fp64_kernel<<<h->n_tiles, kRhoThreads, sm, s>>>(h->geom, tables_of(h), h->d_tile_ptr,
                                                       h->d_keys, v, Hacc);
  return cudaGetLastError();
}


// ---- full A over k-points: the grid passes resolved by lattice offset --------
// With Bloch functions (Eq. 5) the density of Eq. 2 summed over k is
//   rho(r) = sum_(a, b) eta_a(r) eta_b(r) DR[n_a - n_b][mu_a][mu_b],
// a, b the (function, image) entries of the tile's list and
// DR[R] = Re sum_k exp(2 pi i k.R) D_k; the potential matrix of Eq. 11 is
//   V_k = sum_R exp(-2 pi i k.R) VR[R],  VR[R][mu][nu] = dV sum over the
// entries of mu and nu with n_a - n_b = R of sum_r eta_a v eta_b.  Both passes
// stay real; the phases are applied to the small dense matrices.  A pair whose
// offset lies outside the table has no grid point within r_c of both images
// (the table covers |R_x| < 2 r_c / L_x + 1), so it contributes nothing.
__device__ inline int k_ridx(const KGeom &G, int ka, int kb) {
  const int rx = ((ka >> 6) & 7) - ((kb >> 6) & 7);
  const int ry = ((ka >> 3) & 7) - ((kb >> 3) & 7);
  const int rz = (ka & 7) - (kb & 7);
  if (abs(rx) > G.Rm[0] || abs(ry) > G.Rm[1] || abs(rz) > G.Rm[2]) return -1;
  return ((rx + G.Rm[0]) * (2 * G.Rm[1] + 1) + ry + G.Rm[1]) * (2 * G.Rm[2] + 1) + rz + G.Rm[2];
}

__global__ void __launch_bounds__(kRhoThreads) rho_k_kernel(GridGeom g, Tables tb,
                                                            const int *tile_ptr,
                                                            const int *keys, KGeom G,
                                                            const double *DR, double *rho) {
  extern __shared__ double smem[];
  const int t = blockIdx.x;
  const int kb = tile_ptr[t], n = tile_ptr[t + 1] - kb;
  double *X = smem;                       // [n][64]
  double *Dc = X + (long)n * kTP;         // [kChunk][n]
  int *mu_s = (int *)(Dc + (long)kChunk * n);
  int *key_s = mu_s + n;
  __shared__ double part[kRhoThreads];
  TileRange r = tile_range(g, t);
  build_tile_basis(g, tb, keys + kb, n, r, mu_s, X);
  for (int e = threadIdx.x; e < n; e += blockDim.x) key_s[e] = keys[kb + e];
  __syncthreads();
  const long MM = (long)g.M * g.M;
  const int p = threadIdx.x % kTP, grp = threadIdx.x / kTP, ngrp = kRhoThreads / kTP;
  double acc = 0.0;
  for (int a0 = 0; a0 < n; a0 += kChunk) {
    int rows = min(kChunk, n - a0);
    for (int q = threadIdx.x; q < rows * n; q += blockDim.x) {
      int rr = q / n, b = q % n;
      const int ri = k_ridx(G, key_s[a0 + rr], key_s[b]);
      Dc[rr * n + b] = ri < 0 ? 0.0 : DR[ri * MM + (long)mu_s[a0 + rr] * g.M + mu_s[b]];
    }
    __syncthreads();
    for (int rr = grp; rr < rows; rr += ngrp) {
      const double *drow = Dc + rr * n;
      double y = 0.0;
      for (int b = 0; b < n; ++b) y = fma(drow[b], X[b * kTP + p], y);
      acc = fma(X[(a0 + rr) * kTP + p], y, acc);
    }
    __syncthreads();
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < kTP) {
    double s = 0.0;
    for (int q = 0; q < ngrp; ++q) s += part[q * kTP + threadIdx.x];
    int pk = p % g.tz, pj = (p / g.tz) % g.ty, pi = p / (g.tz * g.ty);
    int i = r.i0 + pi, j = r.j0 + pj, k = r.k0 + pk;
    if (i < r.i1 && j < r.j1 && k < r.k1) rho[((long)i * g.ny + j) * g.nz + k] = s;
  }
}

cudaError_t launch_rho_k(etdm_handle *h, const double *DR, double *rho, cudaStream_t s) {
  size_t sm = rho_smem(h->max_list) + (size_t)h->max_list * 4;
  cudaError_t e = cudaFuncSetAttribute(rho_k_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  rho_k_kernel<<<h->n_tiles, kRhoThreads, sm, s>>>(h->geom, tables_of(h), h->d_tile_ptr,
                                                   h->d_keys, h->kg, DR, rho);
  return cudaGetLastError();
}

// VR[R][mu_a][mu_b] += dV sum_p X_ap v_p X_bp for every ordered pair of list
// entries (computed once per unordered pair).
__global__ void __launch_bounds__(kRhoThreads) vmat_k_kernel(GridGeom g, Tables tb,
                                                             const int *tile_ptr,
                                                             const int *keys, KGeom G,
                                                             const double *v, double *VR) {
  extern __shared__ double smem[];
  const int t = blockIdx.x;
  const int kb = tile_ptr[t], n = tile_ptr[t + 1] - kb;
  double *X = smem;                          // [n][65] padded
  double *Xv = X + (long)n * (kTP + 1);      // [n][65]
  int *mu_s = (int *)(Xv + (long)n * (kTP + 1));
  int *key_s = mu_s + n;
  __shared__ double vp[kTP];
  TileRange r = tile_range(g, t);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    key_s[e] = keys[kb + e];
    mu_s[e] = keys[kb + e] >> 9;
  }
  if (threadIdx.x < kTP) {
    int p = threadIdx.x;
    int pk = p % g.tz, pj = (p / g.tz) % g.ty, pi = p / (g.tz * g.ty);
    int i = r.i0 + pi, j = r.j0 + pj, k = r.k0 + pk;
    vp[p] = (i < r.i1 && j < r.j1 && k < r.k1) ? v[((long)i * g.ny + j) * g.nz + k] * g.dV
                                                 : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n * kTP; q += blockDim.x) {
    int e = q / kTP, p = q % kTP;
    int pk = p % g.tz, pj = (p / g.tz) % g.ty, pi = p / (g.tz * g.ty);
    int i = r.i0 + pi, j = r.j0 + pj, k = r.k0 + pk;
    double val = 0.0;
    if (i < r.i1 && j < r.j1 && k < r.k1) {
      int mu, ix, iy, iz;
      decode_key(key_s[e], mu, ix, iy, iz);
      long bx = ((long)mu * kImgN + ix) * g.nx + i;
      long by = ((long)mu * kImgN + iy) * g.ny + j;
      long bz = ((long)mu * kImgN + iz) * g.nz + k;
      double r2 = __dadd_rn(__dadd_rn(tb.sq[0][bx], tb.sq[1][by]), tb.sq[2][bz]);
      if (r2 < tb.rc2[mu]) val = tb.norm[mu] * tb.ex[0][bx] * tb.ex[1][by] * tb.ex[2][bz];
    }
    X[e * (kTP + 1) + p] = val;
    Xv[e * (kTP + 1) + p] = val * vp[p];
  }
  __syncthreads();
  const long MM = (long)g.M * g.M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int a = warp; a < n; a += nw) {
    const double *xa = Xv + a * (kTP + 1);
    for (int b = a + lane; b < n; b += 32) {
      const int rab = k_ridx(G, key_s[a], key_s[b]);
      if (rab < 0) continue;
      const double *xb = X + b * (kTP + 1);
      double s = 0.0;
#pragma unroll 8
      for (int p = 0; p < kTP; ++p) s = fma(xa[p], xb[p], s);
      if (s == 0.0) continue;
      const int ma = mu_s[a], mb = mu_s[b];
      atomicAdd(VR + rab * MM + (long)ma * g.M + mb, s);
      if (a != b) atomicAdd(VR + k_ridx(G, key_s[b], key_s[a]) * MM + (long)mb * g.M + ma, s);
    }
  }
}

cudaError_t launch_vmat_k(etdm_handle *h, const double *v, double *VR, cudaStream_t s) {
  size_t sm = (size_t)h->max_list * (kTP + 1) * 16 + (size_t)h->max_list * 8 + 16;
  cudaError_t e = cudaFuncSetAttribute(vmat_k_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  vmat_k_kernel<<<h->n_tiles, kRhoThreads, sm, s>>>(h->geom, tables_of(h), h->d_tile_ptr,
                                                    h->d_keys, h->kg, v, VR);
  return cudaGetLastError();
}

}  // namespace etdm
