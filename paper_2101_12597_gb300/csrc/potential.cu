// Potential and energy terms on the grid (Eq. 1): the spectral Poisson solve
// v_H(G) = 4 pi rho(G) / G^2 (G != 0), the external potential of Gaussian ion
// charges, Slater exchange, and the grid sums of the energy.
//
// The 3-D FFT is three passes of batched 1-D mixed-radix Stockham transforms
// (radices 2..13), one pass per axis, each line held in shared memory in FP64.
#include <math.h>

#include "device.cuh"
#include "internal.h"

namespace etdm {

constexpr int kFftLines = 16;
constexpr int kFftThreads = 256;

struct FftPlan {
  int n;
  int nst;
  int radix[12];
};

static FftPlan make_plan(int n) {
  FftPlan p{};
  p.n = n;
  int m = n;
  const int order[] = {4, 2, 3, 5, 7, 11, 13};
  for (int r : order) {
    while (m % r == 0) { p.radix[p.nst++] = r; m /= r; }
  }
  return p;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// w(k) = exp(sign * 2 pi i k / n) from the forward table exp(-2 pi i k / n)
__device__ __forceinline__ double2 tw_at(const double2 *tw, int k, int sign) {
  double2 w = tw[k];
  if (sign > 0) w.y = -w.y;
  return w;
}

template <int R>
__device__ __forceinline__ void dft_small(double2 *v, const double2 *tw, int n, int sign) {
  double2 out[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    double2 acc = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      int idx = (int)(((long)r * q % R) * (n / R));
      double2 w = tw_at(tw, idx, sign);
      double2 t = cmul(v[r], w);
      acc.x += t.x; acc.y += t.y;
    }
    out[q] = acc;
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = out[q];
}

__device__ __forceinline__ void dft4(double2 *v, int sign) {
  double2 a = make_double2(v[0].x + v[2].x, v[0].y + v[2].y);
  double2 b = make_double2(v[0].x - v[2].x, v[0].y - v[2].y);
  double2 c = make_double2(v[1].x + v[3].x, v[1].y + v[3].y);
  double2 d = make_double2(v[1].x - v[3].x, v[1].y - v[3].y);
  // forward: multiply d by -i; inverse: by +i
  double2 dr = sign < 0 ? make_double2(d.y, -d.x) : make_double2(-d.y, d.x);
  v[0] = make_double2(a.x + c.x, a.y + c.y);
  v[2] = make_double2(a.x - c.x, a.y - c.y);
  v[1] = make_double2(b.x + dr.x, b.y + dr.y);
  v[3] = make_double2(b.x - dr.x, b.y - dr.y);
}

template <int R>
__device__ void stockham_stage(const double2 *in, double2 *out, int n, int Ns, int lines,
                               const double2 *tw, int sign) {
  const int nb = n / R;
  for (int q = threadIdx.x; q < lines * nb; q += blockDim.x) {
    int l = q / nb, j = q % nb;
    const double2 *src = in + (long)l * n;
    double2 v[R];
    int k = j % Ns;
    int step = n / (Ns * R);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      double2 x = src[j + r * nb];
      if (r > 0 && k > 0) x = cmul(x, tw_at(tw, (r * k * step) % n, sign));
      v[r] = x;
    }
    if (R == 4) dft4(v, sign);
    else if (R == 2) {
      double2 a = v[0], b = v[1];
      v[0] = make_double2(a.x + b.x, a.y + b.y);
      v[1] = make_double2(a.x - b.x, a.y - b.y);
    } else dft_small<R>(v, tw, n, sign);
    double2 *dst = out + (long)l * n;
    int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[base + r * Ns] = v[r];
  }
}

// Layout [A][n][Bdim]; transform along n.  Each block takes kFftLines lines.
__global__ void __launch_bounds__(kFftThreads) fft_axis_kernel(double2 *data, long A, long Bdim,
                                                               const double2 *tw, FftPlan plan,
                                                               int sign) {
  extern __shared__ double2 fsm[];
  const int n = plan.n;
  double2 *b0 = fsm, *b1 = fsm + kFftLines * n;
  long a0, bb0;
  int lines;
  if (Bdim == 1) {
    a0 = (long)blockIdx.x * kFftLines;
    bb0 = 0;
    lines = (int)min((long)kFftLines, A - a0);
  } else {
    long chunks = (Bdim + kFftLines - 1) / kFftLines;
    a0 = blockIdx.x / chunks;
    bb0 = (blockIdx.x % chunks) * kFftLines;
    lines = (int)min((long)kFftLines, Bdim - bb0);
  }
  // load
  if (Bdim == 1) {
    const double2 *src = data + a0 * n;
    for (int q = threadIdx.x; q < lines * n; q += blockDim.x) b0[q] = src[q];
  } else {
    for (int q = threadIdx.x; q < kFftLines * n; q += blockDim.x) {
      int i = q / kFftLines, l = q % kFftLines;
      if (l < lines) b0[l * n + i] = data[(a0 * n + i) * Bdim + bb0 + l];
    }
  }
  __syncthreads();
  int Ns = 1;
  double2 *in = b0, *out = b1;
  for (int s = 0; s < plan.nst; ++s) {
    int R = plan.radix[s];
    switch (R) {
      case 2: stockham_stage<2>(in, out, n, Ns, lines, tw, sign); break;
      case 3: stockham_stage<3>(in, out, n, Ns, lines, tw, sign); break;
      case 4: stockham_stage<4>(in, out, n, Ns, lines, tw, sign); break;
      case 5: stockham_stage<5>(in, out, n, Ns, lines, tw, sign); break;
      case 7: stockham_stage<7>(in, out, n, Ns, lines, tw, sign); break;
      case 11: stockham_stage<11>(in, out, n, Ns, lines, tw, sign); break;
      default: stockham_stage<13>(in, out, n, Ns, lines, tw, sign); break;
    }
    __syncthreads();
    Ns *= R;
    double2 *t = in; in = out; out = t;
  }
  if (Bdim == 1) {
    double2 *dst = data + a0 * n;
    for (int q = threadIdx.x; q < lines * n; q += blockDim.x) dst[q] = in[q];
  } else {
    for (int q = threadIdx.x; q < kFftLines * n; q += blockDim.x) {
      int i = q / kFftLines, l = q % kFftLines;
      if (l < lines) data[(a0 * n + i) * Bdim + bb0 + l] = in[l * n + i];
    }
  }
}

__global__ void twiddle_kernel(double2 *tw, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    tw[k] = make_double2(c, -s);
  }
}

cudaError_t launch_twiddles(etdm_handle *h, cudaStream_t s) {
  long off = 0;
  for (int a = 0; a < 3; ++a) {
    twiddle_kernel<<<(h->n[a] + 127) / 128, 128, 0, s>>>(h->d_tw + off, h->n[a]);
    off += h->n[a];
  }
  return cudaGetLastError();
}

// sign -1: F(k) = sum_j f(j) e^{-2 pi i jk/n}; sign +1: unnormalized inverse.
cudaError_t fft3d(etdm_handle *h, double2 *data, int sign, cudaStream_t s) {
  const int nx = h->n[0], ny = h->n[1], nz = h->n[2];
  const long dims_A[3] = {1, nx, (long)nx * ny};
  const long dims_B[3] = {(long)ny * nz, nz, 1};
  const long tw_off[3] = {0, nx, (long)nx + ny};
  for (int ax = 2; ax >= 0; --ax) {
    int n = h->n[ax];
    FftPlan plan = make_plan(n);
    long A = dims_A[ax], Bd = dims_B[ax];
    long blocks = (Bd == 1) ? (A + kFftLines - 1) / kFftLines
                            : A * ((Bd + kFftLines - 1) / kFftLines);
    size_t sm = (size_t)2 * kFftLines * n * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(fft_axis_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    fft_axis_kernel<<<(unsigned)blocks, kFftThreads, sm, s>>>(data, A, Bd, h->d_tw + tw_off[ax],
                                                              plan, sign);
  }
  return cudaGetLastError();
}

__device__ __forceinline__ double gcomp(int k, int n, double h) {
  int sk = (k < (n + 1) / 2) ? k : k - n;
  double val = 1.0 / ((double)n * h);
  return (2.0 * M_PI) * ((double)sk * val);
}

// v_ext(G) = -(4 pi / (Omega G^2)) exp(-G^2 sigma^2 / 2) sum_I Z_I exp(-i G.R_I)
__global__ void vext_recip_kernel(double2 *out, int nx, int ny, int nz, double hx, double hy,
                                  double hz, const double *pos, const double *Z, int n_atoms,
                                  double omega, double sigma) {
  long G = (long)nx * ny * nz;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < G;
       e += (long)gridDim.x * blockDim.x) {
    int k = (int)(e % nz), j = (int)((e / nz) % ny), i = (int)(e / ((long)ny * nz));
    double gx = gcomp(i, nx, hx), gy = gcomp(j, ny, hy), gz = gcomp(k, nz, hz);
    double g2 = gx * gx + gy * gy + gz * gz;
    double2 acc = make_double2(0.0, 0.0);
    if (e != 0) {
      for (int I = 0; I < n_atoms; ++I) {
        double ph = -(gx * pos[3 * I] + gy * pos[3 * I + 1] + gz * pos[3 * I + 2]);
        double sn, cs;
        sincos(ph, &sn, &cs);
        acc.x += Z[I] * cs;
        acc.y += Z[I] * sn;
      }
      double f = -4.0 * M_PI / (omega * g2) * exp(-g2 * sigma * sigma / 2.0);
      acc.x *= f;
      acc.y *= f;
    }
    out[e] = acc;
  }
}

cudaError_t launch_vext_recip(etdm_handle *h, cudaStream_t s) {
  vext_recip_kernel<<<2048, 256, 0, s>>>(h->d_fft, h->n[0], h->n[1], h->n[2], h->h[0], h->h[1],
                                         h->h[2], h->d_pos, h->d_Z, h->n_atoms, h->omega,
                                         h->sigma);
  return cudaGetLastError();
}

__global__ void real_part_kernel(const double2 *src, double *dst, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    dst[e] = src[e].x;
}

cudaError_t launch_real_part(etdm_handle *h, const double2 *src, double *dst, cudaStream_t s) {
  real_part_kernel<<<2048, 256, 0, s>>>(src, dst, h->G);
  return cudaGetLastError();
}

__global__ void pack_real_kernel(const double *src, double2 *dst, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    dst[e] = make_double2(src[e], 0.0);
}

cudaError_t launch_pack_real(etdm_handle *h, const double *src, double2 *dst, cudaStream_t s) {
  pack_real_kernel<<<2048, 256, 0, s>>>(src, dst, h->G);
  return cudaGetLastError();
}

// data(G) *= 4 pi / (G^2 * Ng) (G != 0), 0 at G = 0
__global__ void poisson_scale_kernel(double2 *data, int nx, int ny, int nz, double hx,
                                     double hy, double hz) {
  long G = (long)nx * ny * nz;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < G;
       e += (long)gridDim.x * blockDim.x) {
    int k = (int)(e % nz), j = (int)((e / nz) % ny), i = (int)(e / ((long)ny * nz));
    double gx = gcomp(i, nx, hx), gy = gcomp(j, ny, hy), gz = gcomp(k, nz, hz);
    double g2 = gx * gx + gy * gy + gz * gz;
    double f = (e == 0) ? 0.0 : 4.0 * M_PI / (g2 * (double)G);
    double2 v = data[e];
    data[e] = make_double2(v.x * f, v.y * f);
  }
}

cudaError_t launch_poisson_scale(etdm_handle *h, double2 *data, cudaStream_t s) {
  poisson_scale_kernel<<<2048, 256, 0, s>>>(data, h->n[0], h->n[1], h->n[2], h->h[0],
                                            h->h[1], h->h[2]);
  return cudaGetLastError();
}

// v = v_ext + v_H + v_x; partial sums of rho v_ext, rho v_H / 2, eps_x (times dV)
__global__ void __launch_bounds__(256) potential_kernel(const double *rho, const double2 *vh,
                                                        const double *vext, double *vtot,
                                                        long G, double dV, double *part) {
  const double cx = cbrt(3.0 / M_PI);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < G;
       e += (long)gridDim.x * blockDim.x) {
    double r = rho[e];
    double rp = r > 0.0 ? r : 0.0;
    double r13 = cbrt(rp);
    double vx = -cx * r13;
    double ex = -0.75 * cx * rp * r13;
    double h = vh[e].x;
    double ve = vext[e];
    vtot[e] = ve + h + vx;
    s0 += r * ve;
    s1 += r * h;
    s2 += ex;
  }
  s0 = block_sum(s0);
  s1 = block_sum(s1);
  s2 = block_sum(s2);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = dV * s0;
    part[3 * blockIdx.x + 1] = 0.5 * dV * s1;
    part[3 * blockIdx.x + 2] = dV * s2;
  }
}

cudaError_t launch_potential(etdm_handle *h, cudaStream_t s) {
  potential_kernel<<<kPotBlocks, 256, 0, s>>>(h->d_rho, h->d_fft, h->d_vext, h->d_vtot, h->G,
                                              h->dV, h->d_gridpart);
  return cudaGetLastError();
}

}  // namespace etdm
