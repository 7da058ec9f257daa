// Hartree potential, exchange and the grid energy terms of the mixed-precision
// path (Eq. 1, 4), in float-pair ("double-float", about 44 significant bits)
// arithmetic: FP32 runs far faster than FP64 on this GPU, and the Poisson solve
// needs about 1e-10 relative accuracy, not the full 53 bits.
//
// rho is real, so the 3-D transform runs on half a spectrum:
//   1. z lines, forward: two real lines as one complex transform, split by
//      conjugate symmetry into their half spectra (kz = 0 .. nz/2);
//   2. y lines, forward;
//   3. x lines: forward, times 4 pi / (|G|^2 Ng) (0 at G = 0), inverse;
//   4. y lines, inverse;
//   5. z lines, inverse: two half spectra rebuilt into one complex line whose
//      real and imaginary parts are the two real potentials; then, per point,
//      v = v_ext + v_H + v_x, the energy sums (Eq. 1 terms), v dV in the tile
//      order of the potential-matrix pass, and max |v|.
// Each pass holds 8 or 16 lines in shared memory and runs mixed-radix Stockham
// stages (radices 2, 3, 4, 5, 7, 11, 13) on float-pair complex numbers.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace etdm {

constexpr int kDfThreads = 256;
constexpr int kZPairs = 8;    // line pairs per block of the z passes
constexpr int kXYLines = 8;   // lines per block of the x and y passes (4 blocks per SM)

// ---- float-pair scalars (hi, lo) and complex numbers ---------------------------
struct dcx {
  float2 re, im;
};

// Every operation below is an explicit round-to-nearest intrinsic: the
// compiler may not contract a product and a sum into one fused operation,
// which would break the error-free transformations (for a b - c d, fusing the
// TwoSum's p - q into fma(a, b, -q) would leave the product at FP32 accuracy).
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 fdf_add(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  const float e = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s.x, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s.x)));
}
__device__ __forceinline__ float2 fdf_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 fdf_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}
// a b - c d, one renormalization
__device__ __forceinline__ float2 fdf_dot_sub(float2 a, float2 b, float2 c, float2 d) {
  const float p = __fmul_rn(a.x, b.x), q = __fmul_rn(c.x, d.x);
  const float ep = __fmaf_rn(a.x, b.x, -p), eq = __fmaf_rn(c.x, d.x, -q);
  const float2 s = two_sum(p, -q);
  float e = __fadd_rn(s.y, __fsub_rn(ep, eq));
  e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
  e = __fmaf_rn(-c.x, d.y, __fmaf_rn(-c.y, d.x, e));
  const float h = __fadd_rn(s.x, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s.x)));
}
// a b + c d, one renormalization
__device__ __forceinline__ float2 fdf_dot_add(float2 a, float2 b, float2 c, float2 d) {
  return fdf_dot_sub(a, b, fdf_neg(c), d);
}
__device__ __forceinline__ float2 fdf_scale2(float2 a, float s) {  // s a power of two
  return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s));
}

__device__ __forceinline__ dcx cx_ld(float4 v) {
  return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ float4 cx_st(dcx c) { return make_float4(c.re.x, c.re.y, c.im.x, c.im.y); }
__device__ __forceinline__ dcx cx_add(dcx a, dcx b) { return {fdf_add(a.re, b.re), fdf_add(a.im, b.im)}; }
__device__ __forceinline__ dcx cx_sub(dcx a, dcx b) {
  return {fdf_add(a.re, fdf_neg(b.re)), fdf_add(a.im, fdf_neg(b.im))};
}
__device__ __forceinline__ dcx cx_mul(dcx a, dcx w) {
  return {fdf_dot_sub(a.re, w.re, a.im, w.im), fdf_dot_add(a.re, w.im, a.im, w.re)};
}
__device__ __forceinline__ dcx cx_conj(dcx a) { return {a.re, fdf_neg(a.im)}; }
// times -i (sign < 0) or +i (sign > 0)
__device__ __forceinline__ dcx cx_rot(dcx a, int sign) {
  return sign < 0 ? dcx{a.im, fdf_neg(a.re)} : dcx{fdf_neg(a.im), a.re};
}

// w^m, w = exp(sign 2 pi i / n), from the forward table exp(-2 pi i m / n)
__device__ __forceinline__ dcx tw_get(const float4 *tw, int m, int sign) {
  dcx w = cx_ld(tw[m]);
  return sign > 0 ? cx_conj(w) : w;
}

// One Stockham stage of radix R over `lines` lines of length n (in -> out).
template <int R>
__device__ void df_stage(const float4 *in, float4 *out, int n, int Ns, int lines, const float4 *tw,
                         int sign) {
  const int nb = n / R;
  const int step = n / (Ns * R);
  for (int q = threadIdx.x; q < lines * nb; q += blockDim.x) {
    const int l = q / nb, j = q % nb;
    const int k = j % Ns;
    const float4 *src = in + (long)l * n;
    dcx v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      dcx x = cx_ld(src[j + r * nb]);
      if (r > 0 && k > 0) x = cx_mul(x, tw_get(tw, (r * k * step) % n, sign));
      v[r] = x;
    }
    if (R == 2) {
      const dcx a = v[0], b = v[1];
      v[0] = cx_add(a, b);
      v[1] = cx_sub(a, b);
    } else if (R == 4) {
      const dcx a = cx_add(v[0], v[2]), b = cx_sub(v[0], v[2]);
      const dcx c = cx_add(v[1], v[3]), d = cx_rot(cx_sub(v[1], v[3]), sign);
      v[0] = cx_add(a, c);
      v[2] = cx_sub(a, c);
      v[1] = cx_add(b, d);
      v[3] = cx_sub(b, d);
    } else {
      dcx o[R];
#pragma unroll
      for (int qq = 0; qq < R; ++qq) {
        dcx acc = v[0];
#pragma unroll
        for (int r = 1; r < R; ++r) acc = cx_add(acc, cx_mul(v[r], tw_get(tw, ((r * qq) % R) * nb, sign)));
        o[qq] = acc;
      }
#pragma unroll
      for (int qq = 0; qq < R; ++qq) v[qq] = o[qq];
    }
    float4 *dst = out + (long)l * n;
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[base + r * Ns] = cx_st(v[r]);
  }
}

// In-place (ping-pong) transform of `lines` lines held in b0; returns the buffer
// holding the result.  Ends with a block barrier.  BIG: radices 7, 11, 13 are
// compiled in (only grids with those factors need them; they cost registers).
template <bool BIG>
__device__ float4 *df_fft(float4 *b0, float4 *b1, const DfPlan &pl, int lines, const float4 *tw,
                          int sign) {
  int Ns = 1;
  float4 *in = b0, *out = b1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    switch (R) {
      case 2: df_stage<2>(in, out, pl.n, Ns, lines, tw, sign); break;
      case 3: df_stage<3>(in, out, pl.n, Ns, lines, tw, sign); break;
      case 4: df_stage<4>(in, out, pl.n, Ns, lines, tw, sign); break;
      case 5: df_stage<5>(in, out, pl.n, Ns, lines, tw, sign); break;
      default:
        if constexpr (BIG) {
          if (R == 7) df_stage<7>(in, out, pl.n, Ns, lines, tw, sign);
          else if (R == 11) df_stage<11>(in, out, pl.n, Ns, lines, tw, sign);
          else df_stage<13>(in, out, pl.n, Ns, lines, tw, sign);
        }
        break;
    }
    __syncthreads();
    Ns *= R;
    float4 *t = in;
    in = out;
    out = t;
  }
  return in;
}

__device__ void load_tw(float4 *dst, const float4 *src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ---- pass 1: z lines, forward, real pairs -> half spectra ----------------------
// Every pass runs over one or several systems: blockIdx.y picks the system
// (its arguments in av[], skipped when its active flag is 0), blockIdx.x the
// lines; blocks beyond the system's lines return at once.
template <bool BIG>
__global__ void __launch_bounds__(kDfThreads, 4) zfwd_kernel(const DfArgs *av, const int *active) {
  extern __shared__ __align__(16) float4 zsm[];
  if (!active[blockIdx.y]) return;
  const DfArgs &a = av[blockIdx.y];
  const long NL = (long)a.nx * a.ny;
  const long L0 = (long)blockIdx.x * kZPairs * 2;
  if (L0 >= NL) return;
  const int nz = a.nz, nzh = a.nzh;
  float4 *tw = zsm, *b0 = zsm + nz, *b1 = b0 + kZPairs * nz;
  load_tw(tw, a.twz, nz);
  for (int q = threadIdx.x; q < kZPairs * nz; q += blockDim.x) {
    const int p = q / nz, z = q % nz;
    const long La = L0 + 2 * p, Lb = La + 1;
    const float2 re = La < NL ? a.rhof[La * nz + z] : make_float2(0.f, 0.f);
    const float2 im = Lb < NL ? a.rhof[Lb * nz + z] : make_float2(0.f, 0.f);
    b0[q] = make_float4(re.x, re.y, im.x, im.y);
  }
  __syncthreads();
  const float4 *X = df_fft<BIG>(b0, b1, a.pz, kZPairs, tw, -1);
  // F_a(k) = (X(k) + conj X(-k)) / 2,  F_b(k) = (X(k) - conj X(-k)) / (2i)
  for (int q = threadIdx.x; q < kZPairs * nzh; q += blockDim.x) {
    const int p = q / nzh, k = q % nzh;
    const long La = L0 + 2 * p, Lb = La + 1;
    const dcx F = cx_ld(X[p * nz + k]), G = cx_conj(cx_ld(X[p * nz + (nz - k) % nz]));
    const dcx s = cx_add(F, G), d = cx_sub(F, G);
    if (La < NL)
      a.H[La * nzh + k] = cx_st({fdf_scale2(s.re, 0.5f), fdf_scale2(s.im, 0.5f)});
    if (Lb < NL)
      a.H[Lb * nzh + k] = cx_st({fdf_scale2(d.im, 0.5f), fdf_scale2(fdf_neg(d.re), 0.5f)});
  }
}

// ---- passes 2 and 4: y lines (fixed x, kz) --------------------------------------
template <bool BIG>
__global__ void __launch_bounds__(kDfThreads, 4) yfft_kernel(const DfArgs *av, const int *active,
                                                             int sign) {
  extern __shared__ __align__(16) float4 ysm[];
  if (!active[blockIdx.y]) return;
  const DfArgs &a = av[blockIdx.y];
  const int ny = a.ny, nzh = a.nzh;
  const long nlines = (long)a.nx * nzh;
  const long q0 = (long)blockIdx.x * kXYLines;
  if (q0 >= nlines) return;
  float4 *tw = ysm, *b0 = ysm + ny, *b1 = b0 + kXYLines * ny;
  load_tw(tw, a.twy, ny);
  const int lines = (int)min((long)kXYLines, nlines - q0);
  for (int q = threadIdx.x; q < kXYLines * ny; q += blockDim.x) {
    const int y = q / kXYLines, l = q % kXYLines;
    if (l < lines) {
      const long line = q0 + l, x = line / nzh, kz = line % nzh;
      b0[l * ny + y] = a.H[(x * ny + y) * nzh + kz];
    }
  }
  __syncthreads();
  const float4 *Y = df_fft<BIG>(b0, b1, a.py, lines, tw, sign);
  for (int q = threadIdx.x; q < kXYLines * ny; q += blockDim.x) {
    const int y = q / kXYLines, l = q % kXYLines;
    if (l < lines) {
      const long line = q0 + l, x = line / nzh, kz = line % nzh;
      a.H[(x * ny + y) * nzh + kz] = Y[l * ny + y];
    }
  }
}

// ---- pass 3: x lines, forward, Poisson kernel, inverse ---------------------------
template <bool BIG>
__global__ void __launch_bounds__(kDfThreads, 4) xpois_kernel(const DfArgs *av, const int *active) {
  extern __shared__ __align__(16) float4 xsm[];
  if (!active[blockIdx.y]) return;
  const DfArgs &a = av[blockIdx.y];
  const int nx = a.nx, ny = a.ny, nzh = a.nzh;
  const long nlines = (long)ny * nzh;
  const long q0 = (long)blockIdx.x * kXYLines;
  if (q0 >= nlines) return;
  float4 *tw = xsm, *b0 = xsm + nx, *b1 = b0 + kXYLines * nx;
  load_tw(tw, a.twx, nx);
  const int lines = (int)min((long)kXYLines, nlines - q0);
  const long stride = (long)ny * nzh;
  for (int q = threadIdx.x; q < kXYLines * nx; q += blockDim.x) {
    const int x = q / kXYLines, l = q % kXYLines;
    if (l < lines) b0[l * nx + x] = a.H[x * stride + q0 + l];
  }
  __syncthreads();
  float4 *Xf = df_fft<BIG>(b0, b1, a.px, lines, tw, -1);
  for (int q = threadIdx.x; q < kXYLines * nx; q += blockDim.x) {
    const int x = q / kXYLines, l = q % kXYLines;
    if (l < lines) {
      const float2 kp = a.kpois[x * stride + q0 + l];
      const dcx v = cx_ld(Xf[l * nx + x]);
      Xf[l * nx + x] = cx_st({fdf_mul(v.re, kp), fdf_mul(v.im, kp)});
    }
  }
  __syncthreads();
  float4 *other = Xf == b0 ? b1 : b0;
  const float4 *Xi = df_fft<BIG>(Xf, other, a.px, lines, tw, +1);
  for (int q = threadIdx.x; q < kXYLines * nx; q += blockDim.x) {
    const int x = q / kXYLines, l = q % kXYLines;
    if (l < lines) a.H[x * stride + q0 + l] = Xi[l * nx + x];
  }
}

// rho^(1/3) as a float pair: FP32 root, one Newton step in float-pair arithmetic
__device__ __forceinline__ float2 fdf_cbrt(float2 r) {
  if (!(r.x > 0.f)) return make_float2(0.f, 0.f);
  const float y = cbrtf(r.x);
  const float y2 = __fmul_rn(y, y);
  const float2 yy = make_float2(y2, __fmaf_rn(y, y, -y2));  // y^2 exactly
  const float2 y3 = fdf_mul(yy, make_float2(y, 0.f));
  const float2 res = fdf_add(y3, fdf_neg(r));       // y^3 - r
  const float corr = res.x / (3.f * y * y);          // Newton: y - (y^3 - r) / (3 y^2)
  return fdf_add(make_float2(y, 0.f), make_float2(-corr, 0.f));
}

__device__ __forceinline__ float2 warp_fdf_sum(float2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    const float2 w = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
    v = fdf_add(v, w);
  }
  return v;
}

// ---- pass 5: z lines, inverse, half spectra pairs -> real potentials; potential --
template <bool BIG>
__global__ void __launch_bounds__(kDfThreads, 4) zinv_pot_kernel(const DfArgs *av, const int *active) {
  extern __shared__ __align__(16) float4 zsm[];
  if (!active[blockIdx.y]) return;
  const DfArgs &a = av[blockIdx.y];
  const long NL = (long)a.nx * a.ny;
  const long L0 = (long)blockIdx.x * kZPairs * 2;
  if (L0 >= NL) return;
  const int nz = a.nz, nzh = a.nzh;
  float4 *tw = zsm, *b0 = zsm + nz, *b1 = b0 + kZPairs * nz;
  load_tw(tw, a.twz, nz);
  // Z(k) = Va(k) + i Vb(k), with V(k) = conj V(nz - k) for k > nz/2
  for (int q = threadIdx.x; q < kZPairs * nz; q += blockDim.x) {
    const int p = q / nz, k = q % nz;
    const long La = L0 + 2 * p, Lb = La + 1;
    const bool up = k >= nzh;
    const int kk = up ? nz - k : k;
    dcx va = La < NL ? cx_ld(a.H[La * nzh + kk]) : dcx{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    dcx vb = Lb < NL ? cx_ld(a.H[Lb * nzh + kk]) : dcx{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (up) { va = cx_conj(va); vb = cx_conj(vb); }
    b0[q] = cx_st(cx_add(va, cx_rot(vb, +1)));
  }
  __syncthreads();
  const float4 *Zr = df_fft<BIG>(b0, b1, a.pz, kZPairs, tw, +1);
  const float2 cxp = a.cx;  // (3 / pi)^(1/3)
  float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0;
  float vm = 0.f;
  for (int q = threadIdx.x; q < kZPairs * 2 * nz; q += blockDim.x) {
    const int pl = q / nz, z = q % nz;  // line La + pl, pl = 2 p + (0 | 1)
    const long L = L0 + pl;
    if (L >= NL) continue;
    const dcx zz = cx_ld(Zr[(pl >> 1) * nz + z]);
    const float2 vh = (pl & 1) ? zz.im : zz.re;
    const long gp = L * nz + z;
    const float2 r = a.rhof[gp], ve = a.vextf[gp];
    const float2 r13 = fdf_cbrt(r);
    const float2 vx = fdf_neg(fdf_mul(cxp, r13));                   // -(3 rho / pi)^(1/3)
    const float2 v = fdf_add(fdf_add(ve, vh), vx);
    s0 = fdf_add(s0, fdf_mul(r, ve));
    s1 = fdf_add(s1, fdf_mul(r, vh));
    s2 = fdf_add(s2, fdf_mul(r, vx));                                // eps_x = (3/4) rho v_x
    vm = fmaxf(vm, fabsf(v.x) * 1.0001f);
    a.vtot[gp] = (double)v.x + (double)v.y;
    // tile order of the potential-matrix pass
    const int i = (int)(L / a.ny), j = (int)(L % a.ny);
    const int t = ((i >> 2) * a.gtc.nby + (j >> 2)) * a.gtc.nbz + (z >> 3);
    const int p = ((i & 3) << 5) + ((j & 3) << 3) + (z & 7);
    a.vt[(long)t * 128 + p] = fdf_mul(v, a.dV);
  }
  s0 = warp_fdf_sum(s0);
  s1 = warp_fdf_sum(s1);
  s2 = warp_fdf_sum(s2);
  vm = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(vm)));
  __shared__ float2 red[3][kDfThreads / 32];
  __shared__ float redm[kDfThreads / 32];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][w] = s0; red[1][w] = s1; red[2][w] = s2; redm[w] = vm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t0 = red[0][0], t1 = red[1][0], t2 = red[2][0];
    float m = redm[0];
    for (int k = 1; k < kDfThreads / 32; ++k) {
      t0 = fdf_add(t0, red[0][k]);
      t1 = fdf_add(t1, red[1][k]);
      t2 = fdf_add(t2, red[2][k]);
      m = fmaxf(m, redm[k]);
    }
    const double dv = (double)a.dV.x + (double)a.dV.y;
    a.part[3 * blockIdx.x] = dv * ((double)t0.x + (double)t0.y);
    a.part[3 * blockIdx.x + 1] = 0.5 * dv * ((double)t1.x + (double)t1.y);
    a.part[3 * blockIdx.x + 2] = 0.75 * dv * ((double)t2.x + (double)t2.y);
    atomicMax(a.vmax_bits, __float_as_uint(m));
  }
}

// ---- set-up ------------------------------------------------------------------------
__global__ void df_split_kernel(const double *src, float2 *dst, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const double v = src[e];
    const float hi = (float)v;
    dst[e] = make_float2(hi, (float)(v - (double)hi));
  }
}

__global__ void df_twiddle_kernel(float4 *tw, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    const float ch = (float)c, sh = (float)(-s);
    tw[k] = make_float4(ch, (float)(c - (double)ch), sh, (float)(-s - (double)sh));
  }
}

__device__ __forceinline__ double gcomp_df(int k, int n, double h) {
  const int sk = (k < (n + 1) / 2) ? k : k - n;
  return (2.0 * M_PI) * ((double)sk / ((double)n * h));
}

__global__ void df_kpois_kernel(float2 *kp, int nx, int ny, int nz, int nzh, double hx, double hy,
                                double hz) {
  const long total = (long)nx * ny * nzh;
  const double Ng = (double)nx * ny * nz;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int k = (int)(e % nzh), j = (int)((e / nzh) % ny), i = (int)(e / ((long)ny * nzh));
    const double gx = gcomp_df(i, nx, hx), gy = gcomp_df(j, ny, hy), gz = gcomp_df(k, nz, hz);
    const double g2 = gx * gx + gy * gy + gz * gz;
    const double f = (e == 0) ? 0.0 : 4.0 * M_PI / (g2 * Ng);
    const float hi = (float)f;
    kp[e] = make_float2(hi, (float)(f - (double)hi));
  }
}

static DfPlan df_plan(int n) {
  DfPlan p{};
  p.n = n;
  int m = n;
  const int order[] = {4, 2, 3, 5, 7, 11, 13};
  for (int r : order)
    while (m % r == 0) { p.radix[p.nst++] = r; m /= r; }
  return p;
}

DfArgs df_args(etdm_handle *h) {
  DfArgs a{};
  a.nx = h->n[0]; a.ny = h->n[1]; a.nz = h->n[2];
  a.nzh = h->n[2] / 2 + 1;
  a.px = df_plan(a.nx); a.py = df_plan(a.ny); a.pz = df_plan(a.nz);
  a.twx = h->d_twf; a.twy = h->d_twf + a.nx; a.twz = h->d_twf + a.nx + a.ny;
  a.H = h->d_half;
  a.rhof = h->d_rhof;
  a.vextf = h->d_vextf;
  a.kpois = h->d_kpois;
  a.vtot = h->d_vtot;
  a.vt = h->d_vt;
  a.vmax_bits = (unsigned *)(h->d_Vfix + (long)h->M * h->M);
  a.part = h->d_gridpart;
  const float dh = (float)h->dV;
  a.dV = make_float2(dh, (float)(h->dV - (double)dh));
  const double cxd = cbrt(3.0 / M_PI);
  const float ch = (float)cxd;
  a.cx = make_float2(ch, (float)(cxd - (double)ch));
  a.gtc = h->geom_tc;
  return a;
}

int df_pot_blocks(etdm_handle *h) {
  const long NL = (long)h->n[0] * h->n[1];
  return (int)((NL + 2 * kZPairs - 1) / (2 * kZPairs));
}

cudaError_t launch_df_setup(etdm_handle *h, cudaStream_t s) {
  long off = 0;
  for (int ax = 0; ax < 3; ++ax) {
    df_twiddle_kernel<<<(h->n[ax] + 127) / 128, 128, 0, s>>>(h->d_twf + off, h->n[ax]);
    off += h->n[ax];
  }
  df_split_kernel<<<1024, 256, 0, s>>>(h->d_vext, h->d_vextf, h->G);
  const int nzh = h->n[2] / 2 + 1;
  df_kpois_kernel<<<1024, 256, 0, s>>>(h->d_kpois, h->n[0], h->n[1], h->n[2], nzh, h->h[0],
                                       h->h[1], h->h[2]);
  return cudaGetLastError();
}

// Sizes of a batched launch of the five passes over the systems' arguments
// (host copies): blocks per system (the largest), shared memory, radices.
DfLaunch df_launch_plan(const std::vector<DfArgs> &args) {
  DfLaunch L{};
  for (const DfArgs &a : args) {
    L.zb = std::max(L.zb, (int)(((long)a.nx * a.ny + 2 * kZPairs - 1) / (2 * kZPairs)));
    L.yb = std::max(L.yb, (int)(((long)a.nx * a.nzh + kXYLines - 1) / kXYLines));
    L.xb = std::max(L.xb, (int)(((long)a.ny * a.nzh + kXYLines - 1) / kXYLines));
    L.smz = std::max(L.smz, (size_t)(a.nz + 2 * kZPairs * a.nz) * sizeof(float4));
    L.smy = std::max(L.smy, (size_t)(a.ny + 2 * kXYLines * a.ny) * sizeof(float4));
    L.smx = std::max(L.smx, (size_t)(a.nx + 2 * kXYLines * a.nx) * sizeof(float4));
    for (const DfPlan *p : {&a.px, &a.py, &a.pz})
      for (int i = 0; i < p->nst; ++i) L.big = L.big || p->radix[i] > 5;
  }
  L.n_sys = (int)args.size();
  return L;
}

template <bool BIG>
static cudaError_t df_potential(const DfLaunch &L, const DfArgs *av, const int *active,
                                cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(zfwd_kernel<BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smz)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(zinv_pot_kernel<BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smz)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(yfft_kernel<BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smy)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(xpois_kernel<BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smx)) != cudaSuccess) return e;
  zfwd_kernel<BIG><<<dim3(L.zb, L.n_sys), kDfThreads, L.smz, s>>>(av, active);
  yfft_kernel<BIG><<<dim3(L.yb, L.n_sys), kDfThreads, L.smy, s>>>(av, active, -1);
  xpois_kernel<BIG><<<dim3(L.xb, L.n_sys), kDfThreads, L.smx, s>>>(av, active);
  yfft_kernel<BIG><<<dim3(L.yb, L.n_sys), kDfThreads, L.smy, s>>>(av, active, +1);
  zinv_pot_kernel<BIG><<<dim3(L.zb, L.n_sys), kDfThreads, L.smz, s>>>(av, active);
  return cudaGetLastError();
}

cudaError_t launch_df_potential(const DfLaunch &L, const DfArgs *av, const int *active,
                                cudaStream_t s) {
  return L.big ? df_potential<true>(L, av, active, s) : df_potential<false>(L, av, active, s);
}

}  // namespace etdm
