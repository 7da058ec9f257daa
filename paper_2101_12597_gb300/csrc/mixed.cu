// Mixed-precision grid passes on the 5th-generation tensor cores (tcgen05).
//
// basis -> grid density (Eq. 2, 3, 12) in orbital form: per 128-point tile
// (4 x 4 x 8) whose list holds n <= 128 basis functions (periodic images of a
// function that reach the tile are summed into one entry),
//     phi = X O_loc  (128 x n x N_occ),  rho_p = 2 sum_m phi_pm^2 ,
// a sum of positive terms (the same density as sum X D X, whose terms cancel
// heavily in a non-orthogonal basis).  X rows and O columns are cut into exact
// integer slices held in BF16 ("Ozaki" splitting), each slice carrying its
// power of two:
//     X_pa = 2^(e_p-8) (I0 + I1 + I2 + I3)   (X as a float pair),
//     O_am = 2^(g_m-8) (K0 + K1 + K2),       I_k, K_k in 2^-8k {-128 .. 128}.
// A product of slices of orders i and j is 2^-8(i+j) times an integer, and
// every accumulator (at most four products per K step, <= 128 entries of
// <= 2^14) stays below 2^24 units of its order, so the four FP32 accumulators of
// slice order 0..3 in tensor memory are exact whatever rounding the accumulator
// applies (the tensor-core accumulator truncates).  X is resolved to about 2^-31 of its row maximum, which the
// cancellation in X O needs; the 24-bit quantization of O is coherent and is
// removed to first order in the energy by sum (4 V O) o (O - Oq) (dense
// reverse kernel); the rest (order >= 4 terms, FP32 square sums) is unbiased
// and incoherent across grid points.
//
// grid -> basis potential matrix (Eq. 11): V_ab = dV sum_p X_pa v_p X_pb with
// X^T and (v X)^T rows cut into four exact integer slices each (exponent per
// entry from a separable bound over the tile) and slice orders 0..3 in four
// exact accumulators.  The gradient amplifies errors of V by the large
// Loewdin coefficients (O^T V O), so V is kept to about 2^-31 of its row
// scale.  Each tile's part is added into V as 64-bit fixed point (unit 2^-46 of
// the power of two above max|v|, which leaves 2^17 of headroom over the bound
// |V_ab| <= max|v| |X_a| |X_b|) with integer reductions in L2: exact and
// independent of the order of the additions, and free of FP64 arithmetic,
// which is slow on this part.
//
// The basis values never change during a minimization, so both X operands
// (per-point exponents for the density, per-entry exponents for V) are sliced
// once at set-up and kept in HBM in the exact shared-memory image of a K step
// (the canonical K-major no-swizzle layout: 8-row x 16-byte core matrices).  Per
// evaluation one thread streams them with bulk asynchronous copies (TMA) into a
// ring of shared-memory stages, with the rows of the O slices the density needs
// gathered the same way; builder warps lay out the operand that changes (the O
// slices of the list entries, or v X re-sliced from the X slices); one
// thread issues tcgen05.mma; epilogue warps read the accumulators with
// tcgen05.ld.  Stages, accumulators and per-tile buffers hand over through
// mbarriers, every wait bounded.  One persistent CTA per SM.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"
#include "pair.cuh"
#include "tc.cuh"

namespace etdm {

constexpr int kTP = 128;                 // points per tile (4 x 4 x 8)
constexpr int kNmax = 128;               // max list length per tile
// slices of the V operands, X^T (resident, per-function exponents over a
// group) and W = (v X)^T (per-row exponents over the group), and the highest
// order of slice products kept
constexpr int kVSlX = 3, kVSlW = 3, kVOrd = 3;
constexpr int kKs = 16;                  // K of one MMA (a "K step")
constexpr int kSlot = kNmax * kKs * 2;   // one BF16 slice of a K step, 128 rows (4 KB)

// padded list length of the V pass (a multiple of 16, at least 16: the MMA's N)
__host__ __device__ __forceinline__ int vpad(int n) { return n <= 16 ? 16 : ((n + 15) / 16) * 16; }
// K steps of the density pass (at least one, zero-filled, for an empty list)
__host__ __device__ __forceinline__ int rsteps(int n) { return n <= kKs ? 1 : (n + kKs - 1) / kKs; }

// ---- float-pair arithmetic and exact slicing -----------------------------------
// (explicit round-to-nearest intrinsics throughout: a product contracted with
// the following sum would break the error-free transformations)
// product of two float pairs (hi + lo): exact product by FMA, then renormalization
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.x, -p);
  const float t = __fadd_rn(e, __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
  const float s = __fadd_rn(p, t);
  return make_float2(s, __fsub_rn(t, __fsub_rn(s, p)));
}

// the same product left unnormalized (hi = fl(a.x b.x), |lo| <= 2 ulp(hi)), as
// slice4 takes it
__device__ __forceinline__ float2 df_mul_raw(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  return make_float2(p, __fadd_rn(__fmaf_rn(a.x, b.x, -p), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x))));
}

// sum of two float pairs with an exact TwoSum of the high parts
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  const float t = __fadd_rn(__fadd_rn(e, a.y), b.y);
  const float h = __fadd_rn(s, t);
  return make_float2(h, __fsub_rn(t, __fsub_rn(h, s)));
}

// x truncated toward zero to a 64-bit integer (|x| < 2^62) by integer shifts of
// its significand (no conversion instruction): x = m 2^e, m < 2^24
__device__ __forceinline__ long long f2ll_trunc(float x) {
  const uint32_t u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xFF) - 150;
  const unsigned long long m = (u & 0x7FFFFFu) | 0x800000u;
  unsigned long long v = e >= 0 ? (m << min(e, 39)) : (m >> min(-e, 63));
  v = (u & 0x7F800000u) ? v : 0ull;  // zero and subnormals
  return (u >> 31) ? -(long long)v : (long long)v;
}

// fixed-point unit 2^F of V: F = (exponent of the power of two above max|v|) - 46
__device__ __forceinline__ int vfix_exp(unsigned vmax_bits) {
  const float vm = __uint_as_float(vmax_bits);
  return vm > 0.f ? min(max(ilogbf(vm) + 1 - 46, -100), 60) : 0;
}

// ---- tiles, lists and staged basis factors ------------------------------------
__device__ __forceinline__ int tile_point(const GridGeom &g, int t, int p) {
  const int bz = t % g.nbz, by = (t / g.nbz) % g.nby, bx = t / (g.nbz * g.nby);
  const int i = bx * 4 + (p >> 5), j = by * 4 + ((p >> 3) & 3), k = bz * 8 + (p & 7);
  return (i < g.nx && j < g.ny && k < g.nz) ? (i * g.ny + j) * g.nz + k : -1;
}

// Per-tile staging of the separable basis factors (dynamic shared memory):
//   xy[(e, li*4+lj)] = (sq_x + sq_y, c_x c_y as a float pair, r_c^2 of the entry)
//   z [(e, lk)]      = (sq_z, c_z as a float pair, 0)
// so that a basis value costs one float-pair product and one cutoff test.
// Entry-major for the density slices, slot-major for the V slices.
constexpr int kStageXY = kNmax * 16;
constexpr int kStageBytes = (kNmax * 16 + kNmax * 8) * 16;  // 48 KB

template <bool TR>
__device__ __forceinline__ int xy_idx(int e, int s) { return TR ? s * kNmax + e : e * 16 + s; }
template <bool TR>
__device__ __forceinline__ int z_idx(int e, int s) { return TR ? s * kNmax + e : e * 8 + s; }

struct BuildShared {
  int mu[kNmax];          // image entries of the tile
  int ustart[kNmax + 1];  // first image entry of each function
  int nu;
  float sc[kTP];
};

// stage the tile's factors for its n image entries; points outside the grid
// get sq = inf, hence value 0; then group the entries by function
template <bool TR>
__device__ void stage_tile(const TcArgs &A, BuildShared &S, float4 *xy, float4 *zs, int t, int kb,
                           int n) {
  const GridGeom &g = A.g;
  const int bz = t % g.nbz, by = (t / g.nbz) % g.nby, bx = t / (g.nbz * g.nby);
  const int i0 = bx * 4, j0 = by * 4, k0 = bz * 8;
  const float4 out = make_float4(INFINITY, 0.f, 0.f, 0.f);
  for (int q = threadIdx.x; q < n * 24; q += blockDim.x) {
    const int e = TR ? q % n : q / 24, s = TR ? q / n : q % 24;
    const int key = A.keys[kb + e];
    const int mu = key >> 9;
    if (s < 16) {
      const int ix = ((key >> 6) & 7) - 4 + kImgMax, iy = ((key >> 3) & 7) - 4 + kImgMax;
      const int i = i0 + (s >> 2), j = j0 + (s & 3);
      const float4 xv = i < g.nx ? A.tab[0][((long)mu * kImgN + ix) * g.nx + i] : out;
      const float4 yv = j < g.ny ? A.tab[1][((long)mu * kImgN + iy) * g.ny + j] : out;
      const float2 c = df_mul(make_float2(xv.y, xv.z), make_float2(yv.y, yv.z));
      xy[xy_idx<TR>(e, s)] = make_float4(xv.x + yv.x, c.x, c.y, A.rc2f[mu]);
    } else {
      const int iz = (key & 7) - 4 + kImgMax;
      const int k = k0 + s - 16;
      zs[z_idx<TR>(e, s - 16)] = k < g.nz ? A.tab[2][((long)mu * kImgN + iz) * g.nz + k] : out;
    }
    if (s == 0) S.mu[e] = mu;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the list is sorted by function: images are adjacent
    int u = 0;
    for (int e = 0; e < n; ++e)
      if (e == 0 || S.mu[e] != S.mu[e - 1]) S.ustart[u++] = e;
    S.ustart[u] = n;
    S.nu = u;
  }
  __syncthreads();
}

// basis value of image entry e at tile point p as a float pair (about 44
// significant bits), zero beyond the cutoff radius
template <bool TR>
__device__ __forceinline__ float2 basis_val_df(const float4 *xy, const float4 *zs, int e, int p) {
  const int lxy = p >> 3, lk = p & 7;  // p = (li*4 + lj)*8 + lk
  const float4 a = xy[xy_idx<TR>(e, lxy)], b = zs[z_idx<TR>(e, lk)];
  if (!(a.x + b.x < a.w)) return make_float2(0.f, 0.f);
  return df_mul(make_float2(a.y, a.z), make_float2(b.y, b.z));
}

// value of function u (the sum of its images) at tile point p
template <bool TR>
__device__ __forceinline__ float2 func_val(const BuildShared &S, const float4 *xy, const float4 *zs,
                                           int u, int p) {
  float2 x = basis_val_df<TR>(xy, zs, S.ustart[u], p);
  for (int e = S.ustart[u] + 1; e < S.ustart[u + 1]; ++e) x = df_add(x, basis_val_df<TR>(xy, zs, e, p));
  return x;
}

// functions per tile (distinct mu in its sorted image list)
__global__ void count_unique_kernel(const int *tile_ptr, const int *keys, int n_tiles, int *nu) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
    int c = 0, last = -1;
    for (int e = tile_ptr[t]; e < tile_ptr[t + 1]; ++e) {
      const int mu = keys[e] >> 9;
      c += mu != last;
      last = mu;
    }
    nu[t] = c;
  }
}

// ---- set-up: density X slices (per-point exponents) ---------------------------
// For tile t, K step kk (functions kk*16 .. kk*16+15), slice k: block
// xr + (xr_off[t] + kk) * 16 KB + k * 4 KB, element (p, c) at kstep_off(p, c).
// Also writes the row exponents e_p (max_a |X_pa| < 2^(e_p - 1)).
__global__ void __launch_bounds__(256) xr_build_kernel(TcArgs A) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  float4 *xy = (float4 *)dsm, *zs = xy + kStageXY;
  __shared__ BuildShared S;
  for (int t = blockIdx.x; t < A.n_tiles; t += gridDim.x) {
    const int kb = A.tile_ptr[t], n = min(A.tile_ptr[t + 1] - kb, kNmax);
    stage_tile<false>(A, S, xy, zs, t, kb, n);
    const int nu = S.nu, nk = rsteps(nu);
    for (int p = threadIdx.x; p < kTP; p += blockDim.x) {
      float mx = 0.f;
      for (int u = 0; u < nu; ++u) mx = fmaxf(mx, fabsf(func_val<false>(S, xy, zs, u, p).x));
      const int e = slice_exp(mx);
      S.sc[p] = pow2f(8 - e);
      const int gp = tile_point(A.g, t, p);
      if (gp >= 0) A.rowexp[gp] = (signed char)e;
    }
    __syncthreads();
    uint8_t *dst = A.xr + (size_t)A.xr_off[t] * (4 * kSlot);
    for (int q = threadIdx.x; q < kTP * 2 * nk; q += blockDim.x) {
      const int p = q % kTP, gq = q / kTP;  // functions gq*8 .. gq*8+7
      const float sc = S.sc[p];
      uint32_t wd[4][4];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        float r[2][4];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const int a = gq * 8 + u + v;
          slice4(a < nu ? func_val<false>(S, xy, zs, a, p) : make_float2(0.f, 0.f), sc, r[v]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) wd[k][u >> 1] = pack_bf16(r[0][k], r[1][k]);
      }
      uint8_t *blk = dst + (size_t)(gq >> 1) * (4 * kSlot);
      const int off = kstep_off(p, (gq & 1) * 8);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        *(uint4 *)(blk + k * kSlot + off) = make_uint4(wd[k][0], wd[k][1], wd[k][2], wd[k][3]);
    }
    __syncthreads();
  }
}

// ---- set-up: V X^T slices (per-function exponents) -----------------------------
// V group g (tiles t0 .. t0 + nt - 1, union of np padded entries): for K step kk
// (points kk*16 .. kk*16+15 of the group, tile t0 + kk / 8), slice k < kVSlX:
// block xv + vg_xoff[g] * 256 + kk * np * 32 * kVSlX + k * np * 32, element (a, c)
// at kstep_off(a, c); rows a >= nu and functions absent from a tile's list are
// zero there.  vent[vg_eoff[g] + a] = (mu, 2^(e_a-8), bound of |X_pa| over the group, 0).

// row of function mu in the ascending union list umu[0, n) (mu is present)
__device__ __forceinline__ int union_row(const int *umu, int n, int mu) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (umu[m] < mu) lo = m + 1; else hi = m;
  }
  return lo;
}

__global__ void __launch_bounds__(256) xv_build_kernel(TcArgs A) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  float4 *xy = (float4 *)dsm, *zs = xy + kStageXY;
  __shared__ BuildShared S;
  __shared__ float bnd_s[kNmax], sa_s[kNmax];
  __shared__ int umu[kNmax], loc[kNmax];
  for (int g = blockIdx.x; g < A.n_vg; g += gridDim.x) {
    const int t0 = A.vg_t0[g], nt = A.vg_t0[g + 1] - t0, nu = A.vg_nu[g];
    const int e0 = A.vg_eoff[g], np = A.vg_eoff[g + 1] - e0;
    for (int a = threadIdx.x; a < np; a += blockDim.x) {
      umu[a] = A.vg_mu[e0 + a];
      bnd_s[a] = 0.f;
    }
    __syncthreads();
    for (int q = 0; q < nt; ++q) {  // separable bound of |X_pa| per tile, summed over images
      const int t = t0 + q, kb = A.tile_ptr[t], n = min(A.tile_ptr[t + 1] - kb, kNmax);
      stage_tile<true>(A, S, xy, zs, t, kb, n);
      for (int u = threadIdx.x; u < S.nu; u += blockDim.x) {
        float bnd = 0.f;
        for (int e = S.ustart[u]; e < S.ustart[u + 1]; ++e) {
          float mxy = 0.f, mz = 0.f;
          for (int s = 0; s < 16; ++s) mxy = fmaxf(mxy, xy[xy_idx<true>(e, s)].y);
          for (int s = 0; s < 8; ++s) mz = fmaxf(mz, zs[z_idx<true>(e, s)].y);
          bnd += mxy * mz * 1.0001f;
        }
        const int r = union_row(umu, nu, S.mu[S.ustart[u]]);
        bnd_s[r] = fmaxf(bnd_s[r], bnd * 1.0001f);
      }
      __syncthreads();
    }
    for (int a = threadIdx.x; a < np; a += blockDim.x) {
      const float bnd = bnd_s[a];
      const int ea = slice_exp(bnd);
      sa_s[a] = pow2f(8 - ea);
      A.vent[e0 + a] = make_float4(__int_as_float(a < nu ? umu[a] : 0), pow2f(ea - 8), bnd, 0.f);
    }
    uint8_t *base = A.xv + (size_t)A.vg_xoff[g] * 256;
    for (int q = 0; q < nt; ++q) {
      const int t = t0 + q;
      if (nt > 1) {  // (a one-tile group is still staged from the bound pass)
        const int kb = A.tile_ptr[t], n = min(A.tile_ptr[t + 1] - kb, kNmax);
        stage_tile<true>(A, S, xy, zs, t, kb, n);
      }
      for (int a = threadIdx.x; a < np; a += blockDim.x) loc[a] = -1;
      __syncthreads();
      for (int u = threadIdx.x; u < S.nu; u += blockDim.x) loc[union_row(umu, nu, S.mu[S.ustart[u]])] = u;
      __syncthreads();
      for (int qq = threadIdx.x; qq < np * 16; qq += blockDim.x) {
        const int a = qq % np, gq = qq / np;  // points gq*8 .. gq*8+7 of the tile
        const float sa = sa_s[a];
        const int u = loc[a];
        uint32_t wd[kVSlX][4];
#pragma unroll
        for (int uu = 0; uu < 8; uu += 2) {
          float r[2][4];
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int p = gq * 8 + uu + v;
            slice_n<kVSlX>(u >= 0 ? func_val<true>(S, xy, zs, u, p) : make_float2(0.f, 0.f), sa, r[v]);
          }
#pragma unroll
          for (int k = 0; k < kVSlX; ++k) wd[k][uu >> 1] = pack_bf16(r[0][k], r[1][k]);
        }
        uint8_t *blk = base + (size_t)(q * 8 + (gq >> 1)) * np * 32 * kVSlX;
        const int off = kstep_off(a, (gq & 1) * 8);
#pragma unroll
        for (int k = 0; k < kVSlX; ++k)
          *(uint4 *)(blk + k * np * 32 + off) = make_uint4(wd[k][0], wd[k][1], wd[k][2], wd[k][3]);
      }
      __syncthreads();
    }
  }
}

// ---- density ---------------------------------------------------------------
// Warp roles: 0-15 read the accumulators (lane quarter w % 4, column quarter
// w / 4), 16-19 lay out the O-slice operand of each K step, 20 streams the X
// slices and gathers the O-slice rows of the K step's 16 functions (one bulk
// copy per run of consecutive functions: the O slices are stored chunk by
// chunk, and the copy engine takes about one request per 90 cycles per SM),
// 21 issues the MMAs.  A job is (tile, chunk of <= 128 occupied orbitals).
constexpr int kRhoStages = 5;
constexpr int kRhoA = 4 * kSlot;        // X slices I0..I3 of a K step (16 KB, as stored)
constexpr int kRhoB = 3 * kSlot;        // O slices K0..K2 of a K step (12 KB)
constexpr int kRhoRow = kNmax * 8;      // room for one gathered O-slice row (<= 128 orbitals)
constexpr int kRhoG = kKs * kRhoRow;    // the K step's 16 rows (16 KB)
constexpr int kRhoStage = kRhoA + kRhoB + kRhoG;
constexpr int kRhoEpiW = 16, kRhoBldW = 4;
constexpr int kRhoParts = kRhoEpiW / 4;  // column parts per lane quarter
constexpr int kRhoEpi = kRhoEpiW * 32, kRhoBld = kRhoBldW * 32;
constexpr int kRhoThreads = kRhoEpi + kRhoBld + 64;

struct RhoBars {
  uint64_t tma_full[kRhoStages], bld_full[kRhoStages], empty[kRhoStages];
  uint64_t acc_full, acc_empty, part_full, part_empty, fin;
  uint32_t tbase;
  int stop;
  float2 part[kRhoParts - 1][kTP];
};

// phi = (acc0 + acc1 + acc2 + acc3) 2^g for 8 columns; their squares summed in
// FP32, the 8-term sum added to the float pair rs by TwoSum: the rounding of
// the running sum (the error that grows with the number of orbitals) stays
// at about 2^-44 of its value
__device__ __forceinline__ float2 rho_sum8(const uint32_t (&r)[32], const float *f, float2 rs) {
  float s8 = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float y = __uint_as_float(r[c]) +
              (__uint_as_float(r[8 + c]) + (__uint_as_float(r[16 + c]) + __uint_as_float(r[24 + c])));
    y *= f[c];
    s8 = fmaf(y, y, s8);
  }
  const float2 sm = pair::two_sum(rs.x, s8);
  return make_float2(sm.x, __fadd_rn(rs.y, sm.y));
}

// The jobs of this CTA in order, each record read one job ahead (the next
// job's tables are in registers when the current one ends).
struct JobStream {
  const TcJob *p;
  int n, j;
  TcJob next;
  __device__ __forceinline__ explicit JobStream(const TcBatch &B)
      : p(B.jobs + B.cta_ptr[blockIdx.x]),
        n(B.cta_ptr[blockIdx.x + 1] - B.cta_ptr[blockIdx.x]), j(0) {
    if (n > 0) next = p[0];
  }
  __device__ __forceinline__ bool get(TcJob &J) {
    if (j >= n) return false;
    J = next;
    if (++j < n) next = p[j];
    return true;
  }
};

__global__ void __launch_bounds__(kRhoThreads, 1) rho_tc_kernel(TcBatch B) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  __shared__ RhoBars R;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kRhoStages; ++s) {
      mbar_init(&R.tma_full[s], 1);
      mbar_init(&R.bld_full[s], kRhoBld);
      mbar_init(&R.empty[s], 1);
    }
    mbar_init(&R.acc_full, 1);
    mbar_init(&R.acc_empty, kRhoEpi);
    mbar_init(&R.part_full, (kRhoParts - 1) * kTP);
    mbar_init(&R.part_empty, kTP);
    mbar_init(&R.fin, 1);
    R.stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) tmem_alloc(&R.tbase);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = R.tbase;
  volatile int *stop = &R.stop;

  if (w == kRhoEpiW + kRhoBldW) {
    // ------------- bulk copies: X slices and the O-slice rows of each K step -------------
    int fill = 0;
    bool ok = true;
    JobStream js(B);
    TcJob J;
    while (ok && js.get(J)) {
      if (!B.active[J.a.x]) continue;
      const TcArgs &A = B.sys[J.a.x];
      const int mc = J.a.z;
      const int k0 = J.b.x, nk = J.b.y, nu = J.b.z;
      const int ocw = A.ocw;  // staged row length (even); the chunk's rows, ocw apart
      const uint2 *osl = A.Osl + (size_t)mc * A.g.M * ocw;
      // functions of the tile: lane l holds entries l, l + 32, l + 64, l + 96
      int mu4[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int a = lane + 32 * r;
        mu4[r] = a < nu ? A.tmu[J.b.w + a] : 0;
      }
      for (int kk = 0; kk < nk; ++kk, ++fill) {
        const int s = fill % kRhoStages, use = fill / kRhoStages;
        bool got = true;
        if (lane == 0 && use > 0) got = mbar_wait(&R.empty[s], (use - 1) & 1, stop);
        if (!__shfl_sync(0xffffffffu, got, 0)) { ok = false; break; }
        const int nrow = max(0, min(kKs, nu - kk * kKs));
        uint8_t *st = dsm + s * kRhoStage;
        if (lane == 0) {
          mbar_expect_tx(&R.tma_full[s], kRhoA + nrow * ocw * 8);
          bulk_g2s_stream(st, A.xr + (size_t)(k0 + kk) * kRhoA, kRhoA, &R.tma_full[s]);
        }
        __syncwarp();
        const int a = kk * kKs + (lane & 15), r = a >> 5;  // r is the same for the warp
        const int mv = r == 0 ? mu4[0] : r == 1 ? mu4[1] : r == 2 ? mu4[2] : mu4[3];
        const int mu = __shfl_sync(0xffffffffu, mv, a & 31);
        // row c of the staging area (rows ocw * 8 bytes apart) <- O-slice row mu_c
        // of the chunk; a run of consecutive functions is one copy
        const int mup = __shfl_up_sync(0xffffffffu, mu, 1);
        const bool cont = lane > 0 && lane < nrow && mu == mup + 1;
        const unsigned cb = __ballot_sync(0xffffffffu, cont);
        if (lane < nrow && !cont) {  // a run starts here: rows lane .. lane + len - 1
          const unsigned after = ~(cb >> (lane + 1));
          const int len = __ffs(after);  // 1 + the run's continued rows
          bulk_g2s(st + kRhoA + kRhoB + lane * ocw * 8, osl + (size_t)mu * ocw, len * ocw * 8,
                   &R.tma_full[s]);
        }
      }
    }
    if (lane == 0) {
      if (!ok) atomicExch((int *)stop, 1);
      // the copies still in flight land before the CTA exits
      for (int s = 0; s < kRhoStages && s < fill; ++s)
        mbar_wait(&R.tma_full[s], ((fill - 1 - s) / kRhoStages) & 1);
    }
  } else if (w == kRhoEpiW + kRhoBldW + 1) {
    // ---------------------------------- MMA issue ----------------------------------
    if (lane == 0) {
      int fill = 0, jp = 0;  // jp: jobs run (the accumulator hand-overs)
      bool ok = true;
      JobStream js(B);
      TcJob J;
      while (ok && js.get(J)) {
        if (!B.active[J.a.x]) continue;
        const TcArgs &A = B.sys[J.a.x];
        const int mc = J.a.z, nk = J.b.y;
        const int nm = min(kNmax, A.Nocc - mc * kNmax);
        const int nmpad = nm <= 32 ? 32 : ((nm + 31) / 32) * 32;
        if (jp > 0 && !mbar_wait(&R.acc_empty, (jp - 1) & 1, stop)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = idesc_bf16(nmpad), idesc2 = idesc_bf16(2 * nmpad);
        for (int kk = 0; kk < nk; ++kk, ++fill) {
          const int s = fill % kRhoStages, use = fill / kRhoStages;
          if (!mbar_wait(&R.tma_full[s], use & 1, stop) || !mbar_wait(&R.bld_full[s], use & 1, stop)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = su32(dsm + s * kRhoStage), b0 = a0 + kRhoA;
          uint64_t I[4], K[3];
#pragma unroll
          for (int k = 0; k < 4; ++k) I[k] = smem_desc(a0 + k * kSlot);
#pragma unroll
          for (int k = 0; k < 3; ++k) K[k] = smem_desc(b0 + k * nmpad * 32);
          // acc_o (order o) at column o * nmpad; I_i x [K_j; K_j+1] (N = 2 nmpad, the
          // slices lie nmpad rows apart) adds I_i K_j to acc_(i+j) and I_i K_j+1 to
          // acc_(i+j+1): the nine slice products of orders <= 3 in six MMAs
          const uint32_t acc = kk > 0, ac = (uint32_t)nmpad;
          mma_bf16(tmem, I[0], K[0], idesc2, acc);          // acc0 = I0 K0, acc1 = I0 K1
          mma_bf16(tmem + 2 * ac, I[0], K[2], idesc, acc);  // acc2 = I0 K2
          mma_bf16(tmem + ac, I[1], K[0], idesc2, 1u);      // acc1 += I1 K0, acc2 += I1 K1
          mma_bf16(tmem + 3 * ac, I[1], K[2], idesc, acc);  // acc3 = I1 K2
          mma_bf16(tmem + 2 * ac, I[2], K[0], idesc2, 1u);  // acc2 += I2 K0, acc3 += I2 K1
          mma_bf16(tmem + 3 * ac, I[3], K[0], idesc, 1u);   // acc3 += I3 K0
          mma_commit(&R.empty[s]);  // the stage is free once these MMAs complete
        }
        if (ok) mma_commit(&R.acc_full);
        ++jp;
      }
      if (!ok) atomicExch((int *)stop, 1);
      mma_commit(&R.fin);  // every MMA issued has completed before the TMEM is released
      mbar_wait(&R.fin, 0);
    }
  } else if (w >= kRhoEpiW) {
    // -------------- O-slice operand, B[m][a] = Oq[mu_a][m], from the gathered rows --------------
    const int bt = tid - kRhoEpi;
    int fill = 0;
    bool ok = true;
    JobStream js(B);
    TcJob J;
    while (ok && js.get(J)) {
      if (!B.active[J.a.x]) continue;
      const TcArgs &A = B.sys[J.a.x];
      const int mc = J.a.z, nk = J.b.y, nu = J.b.z;
      const int nm = min(kNmax, A.Nocc - mc * kNmax);
      const int ocw = A.ocw;  // staged row length (even)
      const int nmpad = nm <= 32 ? 32 : ((nm + 31) / 32) * 32;
      for (int kk = 0; kk < nk; ++kk, ++fill) {
        const int s = fill % kRhoStages, use = fill / kRhoStages;
        if (!mbar_wait(&R.tma_full[s], use & 1, stop)) { ok = false; break; }
        uint8_t *Bs = dsm + s * kRhoStage + kRhoA;
        const uint8_t *G = Bs + kRhoB;
        const int nrow = max(0, min(kKs, nu - kk * kKs));
        // a thread per orbital m: its 16 gathered entries (all loads issued
        // before the first use), laid out as the two 8-function halves of the
        // K step in each of the three slices
        const bool full = nrow == kKs;
        for (int m = bt; m < nmpad; m += kRhoBld) {
          uint32_t w01[kKs], w2[kKs];
          if (full && m < nm) {
#pragma unroll
            for (int c = 0; c < kKs; ++c) {
              const uint2 o = *(const uint2 *)(G + (c * ocw + m) * 8);
              w01[c] = o.x;
              w2[c] = o.y;
            }
          } else {
#pragma unroll
            for (int c = 0; c < kKs; ++c) {
              uint2 o = make_uint2(0u, 0u);
              if (c < nrow && m < nm) o = *(const uint2 *)(G + (c * ocw + m) * 8);
              w01[c] = o.x;
              w2[c] = o.y;
            }
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t *x = w01 + 8 * h, *y = w2 + 8 * h;
            const int off = kstep_off(m, h * 8);
            uint4 v0, v1, v2;
            v0.x = __byte_perm(x[0], x[1], 0x5410); v0.y = __byte_perm(x[2], x[3], 0x5410);
            v0.z = __byte_perm(x[4], x[5], 0x5410); v0.w = __byte_perm(x[6], x[7], 0x5410);
            v1.x = __byte_perm(x[0], x[1], 0x7632); v1.y = __byte_perm(x[2], x[3], 0x7632);
            v1.z = __byte_perm(x[4], x[5], 0x7632); v1.w = __byte_perm(x[6], x[7], 0x7632);
            v2.x = __byte_perm(y[0], y[1], 0x5410); v2.y = __byte_perm(y[2], y[3], 0x5410);
            v2.z = __byte_perm(y[4], y[5], 0x5410); v2.w = __byte_perm(y[6], y[7], 0x5410);
            *(uint4 *)(Bs + off) = v0;
            *(uint4 *)(Bs + nmpad * 32 + off) = v1;
            *(uint4 *)(Bs + 2 * nmpad * 32 + off) = v2;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&R.bld_full[s]);
      }
    }
    if (!ok) atomicExch((int *)stop, 1);
  } else {
    // ---------------------------- accumulator read-out ------------------------------
    // phi_pm = 2^(e_p + g_m - 16) y with y = acc0 + acc1 + acc2 + acc3;
    // rho_p = 2 sum_m phi_pm^2 (every term positive)
    const int quad = w & 3, part = w >> 2;
    const int pe = quad * 32 + lane;
    const uint32_t lanebits = (uint32_t)(quad * 32) << 16;
    float2 rsum = make_float2(0.f, 0.f);
    int ntile = 0, jp = 0;  // tiles finished (part buffer hand-overs), jobs run
    bool ok = true;
    JobStream js(B);
    TcJob J;
    while (ok && js.get(J)) {
      if (!B.active[J.a.x]) continue;
      const TcArgs &A = B.sys[J.a.x];
      const int t = J.a.y, mc = J.a.z;
      const int nm = min(kNmax, A.Nocc - mc * kNmax);
      const int nmpad = nm <= 32 ? 32 : ((nm + 31) / 32) * 32;
      const int gp = tile_point(A.g, t, pe);
      const int ep = gp >= 0 ? (int)A.rowexp[gp] : 0;
      ok = __all_sync(0xffffffffu, mbar_wait(&R.acc_full, jp & 1, stop));
      ++jp;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // this warp's column part (a quarter of the chunk) in pieces of 8; the
      // column scales 2^g_m come from the (zero-padded) global array of the
      // job's system
      const int cb = part * (nmpad / kRhoParts), ce = cb + nmpad / kRhoParts;
      const float *f = A.oscale + mc * kNmax;
      for (int c0 = cb; c0 < ce; c0 += 8) {
        uint32_t r[32];
        tmem_ld_issue(tmem + lanebits + c0, r, nmpad);
        tmem_ld_wait(r);
        rsum = rho_sum8(r, f + c0, rsum);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&R.acc_empty);
      if (mc == J.a.w - 1) {  // the tile is done: add the column parts
        if (part > 0) {
          if (ntile > 0) ok = mbar_wait(&R.part_empty, (ntile - 1) & 1, stop);
          R.part[part - 1][pe] = rsum;
          mbar_arrive(&R.part_full);
        } else {
          ok = mbar_wait(&R.part_full, ntile & 1, stop);
          float2 r = rsum;
#pragma unroll
          for (int q = 0; q < kRhoParts - 1; ++q) r = df_add(r, R.part[q][pe]);
          mbar_arrive(&R.part_empty);
          if (ok && gp >= 0) {
            A.rho[gp] = ldexp((double)r.x + (double)r.y, 2 * ep - 31);
            const int e2 = 2 * ep - 31;  // rho below 2^-100 is left out of the float pair
            if (e2 < -100) r = make_float2(0.f, 0.f);
            const float sc = pow2f(max(e2, -100));
            A.rhof[gp] = make_float2(r.x * sc, r.y * sc);
          }
        }
        rsum = make_float2(0.f, 0.f);
        ++ntile;
        ok = __all_sync(0xffffffffu, ok);
      }
    }
    if (!ok) atomicExch((int *)stop, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) tmem_dealloc(tmem);
  if (tid == 0 && R.stop) atomicExch(B.flags + FLAG_ERR, ETDM_ERR_TIMEOUT);
}

// ---- potential matrix ---------------------------------------------------------
// V_loc = dV X^T diag(v) X per group of tiles as D = W X^T on the tensor cores,
// W = (v X)^T (rows = union functions i, the accumulator lanes) and X^T
// (columns j), in kVSlW and kVSlX exact integer slices.  The slice products of
// order 0 go into one FP32 accumulator (exact: integers below 2^24 on the 2^0
// grid), those of orders 1 .. kVOrd into a second (about 2^-8 of the first, so
// its FP32 rounding is 2^-32 of V's scale).  Two accumulator pairs (4 x 128 TMEM
// columns) alternate between groups, so the read-out of one group overlaps the
// MMAs of the next.  Warp roles: 0-15 read the accumulators (lane quarter
// w % 4, every fourth 8-column chunk by w / 4) and add into V by fixed-point
// reductions; 16-23 build W from the X^T slices and v; 24 streams the X^T
// slices and the group buffers (v at the points, union entries); 25 issues the
// MMAs.  Lane i takes the columns j <= i and adds into V[mu_j][mu_i]
// (mu_j <= mu_i), so a warp's reductions run along a row of V.
constexpr int kVA = kVSlW * kSlot;  // W slices (128 rows)
constexpr int kVB = kVSlX * kSlot;  // X^T slices (np rows each, packed as stored)
constexpr int kVStage = kVA + kVB;
constexpr int kVStages = (200 * 1024) / kVStage;  // operand ring in 200 KB of shared memory
constexpr int kVEpiW = 16, kVBldW = 8;  // warps: 0-15 read-out, 16-23 build W
constexpr int kVEpi = kVEpiW * 32, kVBld = kVBldW * 32;
constexpr int kVThreads = kVEpi + kVBld + 64;
// tiles per V group at most (the group size is chosen per handle, <= this):
// an order-0 accumulator sums kVGmax * 128 products below 2^14 each, so 8
// keeps every partial sum within 2^24 (exact in FP32)
constexpr int kVGmax = 8;
constexpr int kVTileBuf = kVGmax * kTP * 8 + kNmax * 16;  // v pairs + union entries

struct VBars {
  uint64_t tma_full[kVStages], bld_full[kVStages], empty[kVStages];
  uint64_t tile_full[2], tile_empty[2], acc_full[2], acc_empty[2], fin;
  uint32_t tbase;
  int stop;
};

// max |v dV| over a group's points (all lanes of the calling warp get it)
__device__ __forceinline__ float tile_vmax(const float2 *vt, int n) {
  float m = 0.f;
  for (int p = (threadIdx.x & 31); p < n; p += 32) m = fmaxf(m, fabsf(vt[p].x));
  // non-negative floats order as their bit patterns
  return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));
}

// 8 columns of the two accumulators of a lane quarter; the wait is a separate
// statement that names the registers, so no use is scheduled before it
__device__ __forceinline__ void tmem_ld2_issue(uint32_t t0, uint32_t t1, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n\t"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(t0), "r"(t1));
}
__device__ __forceinline__ void tmem_ld2_wait(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

__global__ void __launch_bounds__(kVThreads, 1) vmat_tc_kernel(TcBatch B) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  uint8_t *tbuf = dsm + kVStages * kVStage;  // 2 group buffers: vt[nt * 128] float2, vent[np] float4
  __shared__ VBars R;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kVStages; ++s) {
      mbar_init(&R.tma_full[s], 1);
      mbar_init(&R.bld_full[s], kVBld);
      mbar_init(&R.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&R.tile_full[b], 1);
      mbar_init(&R.tile_empty[b], (kVEpi + kVBld) / 32);
      mbar_init(&R.acc_full[b], 1);
      mbar_init(&R.acc_empty[b], kVEpiW);
    }
    mbar_init(&R.fin, 1);
    R.stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) tmem_alloc(&R.tbase);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = R.tbase;
  // each CTA's jobs are a contiguous run of groups (of one system or a few):
  // CTAs running at the same time work in different parts of a box and rarely
  // add into the same entries of V
  volatile int *stop = &R.stop;
  constexpr int kSteps = kTP / kKs;  // 8 K steps of 16 points per tile of the group

  if (w == kVEpiW + kVBldW) {
    // ------------------------ bulk copies: tile buffers and X^T ------------------------
    if (lane == 0) {
      int fill = 0, it = 0;  // it: jobs run (the group buffer hand-overs)
      bool ok = true;
      JobStream js(B);
      TcJob J;
      while (ok && js.get(J)) {
        if (!B.active[J.a.x]) continue;
        const TcArgs &A = B.sys[J.a.x];
        const int mb = it & 1;
        const int t0 = J.a.z, nt = J.a.w, e0 = J.b.x, np = J.b.y;
        if (it >= 2 && !mbar_wait(&R.tile_empty[mb], ((it >> 1) - 1) & 1, stop)) { ok = false; break; }
        uint8_t *tb = tbuf + mb * kVTileBuf;
        mbar_expect_tx(&R.tile_full[mb], nt * kTP * 8 + np * 16);
        bulk_g2s(tb, A.vt + (size_t)t0 * kTP, nt * kTP * 8, &R.tile_full[mb]);
        bulk_g2s(tb + kVGmax * kTP * 8, A.vent + e0, np * 16, &R.tile_full[mb]);
        const uint8_t *src = A.xv + (size_t)J.b.w * 256;
        for (int kk = 0; kk < nt * kSteps; ++kk, ++fill) {
          const int s = fill % kVStages, use = fill / kVStages;
          if (use > 0 && !mbar_wait(&R.empty[s], (use - 1) & 1, stop)) { ok = false; break; }
          mbar_expect_tx(&R.tma_full[s], np * 32 * kVSlX);
          bulk_g2s_stream(dsm + s * kVStage + kVA, src + (size_t)kk * np * 32 * kVSlX, np * 32 * kVSlX,
                          &R.tma_full[s]);
        }
        ++it;
      }
      if (!ok) atomicExch((int *)stop, 1);
      // the copies still in flight land before the CTA exits
      for (int s = 0; s < kVStages && s < fill; ++s)
        mbar_wait(&R.tma_full[s], ((fill - 1 - s) / kVStages) & 1);
      for (int b = 0; b < 2 && b < it; ++b) mbar_wait(&R.tile_full[b], ((it - 1 - b) >> 1) & 1);
    }
  } else if (w == kVEpiW + kVBldW + 1) {
    // ---------------------------------- MMA issue ----------------------------------
    if (lane == 0) {
      int fill = 0, it = 0;
      bool ok = true;
      JobStream js(B);
      TcJob J;
      for (; ok && js.get(J); ++it) {
        if (!B.active[J.a.x]) { --it; continue; }
        const int buf = it & 1;
        const int nt = J.a.w, np = J.b.y;
        // the accumulator pair of group it - 2 has been read
        if (it >= 2 && !mbar_wait(&R.acc_empty[buf], ((it >> 1) - 1) & 1, stop)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = idesc_bf16(np);
        const uint32_t d0 = tmem + buf * 2 * kNmax, d1 = d0 + kNmax;
        for (int kk = 0; kk < nt * kSteps; ++kk, ++fill) {
          const int s = fill % kVStages, use = fill / kVStages;
          if (!mbar_wait(&R.tma_full[s], use & 1, stop) || !mbar_wait(&R.bld_full[s], use & 1, stop)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = su32(dsm + s * kVStage), b0 = a0 + kVA;
          uint64_t W[kVSlW], X[kVSlX];
#pragma unroll
          for (int k = 0; k < kVSlW; ++k) W[k] = smem_desc(a0 + k * kSlot);
#pragma unroll
          for (int k = 0; k < kVSlX; ++k) X[k] = smem_desc(b0 + k * np * 32);
          const uint32_t acc = kk > 0;
          mma_bf16(d0, W[0], X[0], idesc, acc);  // order 0
#pragma unroll
          for (int o = 1; o <= kVOrd; ++o)        // orders 1 .. kVOrd (W0 X1 first)
#pragma unroll
            for (int q = 0; q <= o; ++q)
              if (q < kVSlW && o - q < kVSlX)
                mma_bf16(d1, W[q], X[o - q], idesc, (o == 1 && q == 0) ? acc : 1u);
          mma_commit(&R.empty[s]);
        }
        if (ok) mma_commit(&R.acc_full[buf]);
      }
      if (!ok) atomicExch((int *)stop, 1);
      mma_commit(&R.fin);
      mbar_wait(&R.fin, 0);
    }
  } else if (w >= kVEpiW) {
    // -------------------- W = (v X)^T: rows b, 8 points of each K step ----------------------
    const int bt = tid - kVEpi;
    const int b = bt & 127, h = bt >> 7;
    int fill = 0, it = 0;
    bool ok = true;
    JobStream js(B);
    TcJob J;
    for (; ok && js.get(J); ++it) {
      if (!B.active[J.a.x]) { --it; continue; }
      const int mb = it & 1;
      const int nt = J.a.w, np = J.b.y, nu = J.b.z;
      ok = __all_sync(0xffffffffu, mbar_wait(&R.tile_full[mb], (it >> 1) & 1, stop));
      if (!ok) break;
      const uint8_t *tb = tbuf + mb * kVTileBuf;
      const float2 *vt = (const float2 *)tb;
      const float4 *ve = (const float4 *)(tb + kVGmax * kTP * 8);
      const float vmax = tile_vmax(vt, nt * kTP);
      // row b: X^T slices of x 2^(8 - e_b); W row exponent from the bound of
      // |v x| over the group
      float sb = 0.f;  // 2^(8 - e_w) 2^(e_b - 8): the X^T slices hold x 2^(8 - e_b)
      if (b < nu) {
        const float4 e = ve[b];
        sb = pow2f(8 - slice_exp(e.z * vmax * 1.0001f)) * e.y;
      }
      for (int kk = 0; kk < nt * kSteps; ++kk, ++fill) {
        const int s = fill % kVStages, use = fill / kVStages;
        if (use > 0 && !mbar_wait(&R.empty[s], (use - 1) & 1, stop)) { ok = false; break; }
        if (!mbar_wait(&R.tma_full[s], use & 1, stop)) { ok = false; break; }
        uint8_t *Ast = dsm + s * kVStage;
        const uint8_t *Bst = Ast + kVA;
        const int off = kstep_off(b, h * 8);
        uint4 o[kVSlW];
        if (b < nu) {
          uint4 xs[kVSlX];
#pragma unroll
          for (int k = 0; k < kVSlX; ++k) xs[k] = *(const uint4 *)(Bst + k * np * 32 + off);
          uint32_t ww[kVSlW][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {  // point pairs (2u, 2u + 1)
            float r[2][4];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              // the sliced x 2^(8 - e_b), exact: the slices' sum on the 2^-16 grid
              // below 2^8 (a fourth slice on the 2^-24 grid goes in the low part)
              float i[4];
#pragma unroll
              for (int k = 0; k < kVSlX; ++k) {
                const uint32_t sk = (&xs[k].x)[u];
                i[k] = __uint_as_float(v ? (sk & 0xFFFF0000u) : (sk << 16));
              }
              const float2 x = make_float2((i[0] + i[1]) + (kVSlX > 2 ? i[2] : 0.f), kVSlX > 3 ? i[3] : 0.f);
              slice_n<kVSlW>(df_mul_raw(x, vt[kk * kKs + h * 8 + 2 * u + v]), sb, r[v]);
            }
#pragma unroll
            for (int k = 0; k < kVSlW; ++k) ww[k][u] = pack_bf16(r[0][k], r[1][k]);
          }
#pragma unroll
          for (int k = 0; k < kVSlW; ++k) o[k] = make_uint4(ww[k][0], ww[k][1], ww[k][2], ww[k][3]);
        } else {
#pragma unroll
          for (int k = 0; k < kVSlW; ++k) o[k] = make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < kVSlW; ++k) *(uint4 *)(Ast + k * kSlot + off) = o[k];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&R.bld_full[s]);
      }
      ok = __all_sync(0xffffffffu, ok);
      if (lane == 0) mbar_arrive(&R.tile_empty[mb]);
    }
    if (!ok) atomicExch((int *)stop, 1);
  } else {
    // ------------------------- accumulator read-out into V ----------------------------
    // lane i of quarter w % 4 holds row i; columns j <= i of every fourth
    // 8-column chunk (by w / 4): y = acc0 + acc1 as a float pair, scaled to the
    // fixed-point unit, added into V[mu_j][mu_i]
    const int quad = w & 3, part = w >> 2;
    const int i = quad * 32 + lane;  // accumulator lane = W row
    const uint32_t lanebits = (uint32_t)(quad * 32) << 16;
    int it = 0;
    bool ok = true;
    JobStream js(B);
    TcJob J;
    for (; ok && js.get(J); ++it) {
      if (!B.active[J.a.x]) { --it; continue; }
      const TcArgs &A = B.sys[J.a.x];
      const int M = A.g.M;
      // fixed-point unit of the job's system (its max |v| from the potential pass)
      const int fixe = vfix_exp((unsigned)A.Vfix[(long)M * M]);
      const int mb = it & 1, buf = it & 1;
      const int nt = J.a.w, nu = J.b.z;
      ok = __all_sync(0xffffffffu, mbar_wait(&R.tile_full[mb], (it >> 1) & 1, stop) &&
                                       mbar_wait(&R.acc_full[buf], (it >> 1) & 1, stop));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint8_t *tb = tbuf + mb * kVTileBuf;
      const float4 *ve = (const float4 *)(tb + kVGmax * kTP * 8);
      const float vmax = tile_vmax((const float2 *)tb, nt * kTP);
      // 2^(e_i - 8 - F): W row scale over the fixed-point unit; mu of row i
      const float ub = i < nu ? pow2f(max(slice_exp(ve[i].z * vmax * 1.0001f) - 8 - fixe, -126)) : 0.f;
      const int mui = i < nu ? __float_as_int(ve[i].x) : 0;
      unsigned long long *const vrow = A.Vfix + mui;
      const uint32_t t0 = tmem + lanebits + buf * 2 * kNmax;
      const int jend = quad * 32 < nu ? min(quad * 32 + 32, nu) : 0;
      for (int c0 = part * 8; c0 < jend; c0 += 32) {
        uint32_t ra[16];
        tmem_ld2_issue(t0 + c0, t0 + kNmax + c0, ra);
        tmem_ld2_wait(ra);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int j = c0 + c;
          if (i < nu && j <= i) {
            const float4 ej = ve[j];
            const float f = ub * ej.y;  // exact: a product of powers of two
            const float2 y = pair::two_sum(__uint_as_float(ra[c]), __uint_as_float(ra[8 + c]));
            // a contribution below the fixed-point unit truncates to zero: nothing to add
            if (fabsf(y.x * f) >= 1.f) {
              const long long val = f2ll_trunc(y.x * f) + f2ll_trunc(y.y * f);
              atomicAdd(vrow + (long)__float_as_int(ej.x) * M, (unsigned long long)val);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&R.acc_empty[buf]);
        mbar_arrive(&R.tile_empty[mb]);
      }
    }
    if (!ok) atomicExch((int *)stop, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) tmem_dealloc(tmem);
  if (tid == 0 && R.stop) atomicExch(B.flags + FLAG_ERR, ETDM_ERR_TIMEOUT);
}

// V (upper triangle) from its fixed-point sums; blockIdx.y picks the system
__global__ void vfix_kernel(const VfArgs *av, const int *active) {
  if (!active[blockIdx.y]) return;
  const VfArgs &a = av[blockIdx.y];
  const int M = a.M;
  const int F = vfix_exp((unsigned)a.Vfix[(long)M * M]);
  const long MM = (long)M * M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MM;
       e += (long)gridDim.x * blockDim.x) {
    if (e / M > e % M) continue;
    a.Vout[e] = pair::split(ldexp((double)(long long)a.Vfix[e], F));
  }
}

// ---- set-up and per-evaluation helpers ------------------------------------------

// FP32 copies of the basis tables with norm^(1/3) folded into each factor
__global__ void tables_f32_kernel(const double *sq, const double *ex, const double *norm,
                                  int M, int n_ax, float4 *out) {
  long total = (long)M * kImgN * n_ax;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int mu = (int)(e / ((long)n_ax * kImgN));
    const double c = cbrt(norm[mu]) * ex[e];
    const float hi = (float)c;
    out[e] = make_float4((float)sq[e], hi, (float)(c - (double)hi), 0.f);
  }
}

// Column slices of the occupied orbitals O (M x N, float pairs from the dense
// chain): g_m = ilogb(max_mu |O_mu,m|) + 2, K0 + K1 + K2 = O 2^(8 - g) to 24 bits
// (K_k on the 2^-8k grid); dO = O - Oq (FP64) for the first-order energy
// correction sum (4 H O) o dO.
// O slicing, the first of two coalesced passes over the row-major O: the
// largest |O| of each column (orbital), as the bits of a non-negative double
// (which order as integers); a warp takes 32 consecutive columns over a run
// of 64 rows.  omax is zero on entry.
__global__ void __launch_bounds__(256) omax_kernel(const OsArgs *av, const int *active) {
  if (!active[blockIdx.y]) return;
  const OsArgs &a = av[blockIdx.y];
  const int M = a.M, N = a.N;
  const int ncg = (N + 31) / 32, nrc = (M + 63) / 64;
  const long items = (long)ncg * nrc;
  const int lane = threadIdx.x & 31;
  const long wstride = ((long)gridDim.x * blockDim.x) >> 5;
  for (long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < items; w += wstride) {
    const int m = (int)(w % ncg) * 32 + lane, r0 = (int)(w / ncg) * 64;
    if (m >= N) continue;
    const int r1 = min(r0 + 64, M);
    double mx = 0.0;
    for (int r = r0; r < r1; ++r) mx = fmax(mx, fabs(pair::to_double(a.O[(long)r * N + m])));
    atomicMax(a.omax + m, (unsigned long long)__double_as_longlong(mx));
  }
}

// The second pass: element (r, m) cut into three slices with the column's
// power of two 2^g (g from the column maximum), the remainder O - Oq, and
// the column scale (written by the thread of row 0).
__global__ void __launch_bounds__(256) oslice_kernel(const OsArgs *av, const int *active) {
  if (!active[blockIdx.y]) return;
  const OsArgs &a = av[blockIdx.y];
  const int M = a.M, N = a.N;
  const long MN = (long)M * N;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MN; e += (long)gridDim.x * blockDim.x) {
    const int r = (int)(e / N), m = (int)(e % N);
    const double mx = __longlong_as_double((long long)a.omax[m]);
    const int g = mx > 0.0 ? ilogb(mx) + 2 : 0;
    if (r == 0) a.oscale[m] = ldexpf(1.f, g);
    const double o = pair::to_double(a.O[e]);
    const double t0 = ldexp(o, 8 - g);
    const double r0 = rint(t0);
    const double t1 = (t0 - r0) * 256.0;
    const double r1 = rint(t1);
    const double t2 = (t1 - r1) * 256.0;
    const double r2 = rint(t2);
    const double q = ldexp(r0 + (r1 + r2 * (1.0 / 256.0)) * (1.0 / 256.0), g - 8);
    a.dO[e] = o - q;
    a.Osl[((long)(m / a.ocw) * M + r) * a.ocw + m % a.ocw] = make_uint2(
        (uint32_t)bf16_bits((float)r0) | ((uint32_t)bf16_bits((float)(r1 * (1.0 / 256.0))) << 16),
        (uint32_t)bf16_bits((float)(r2 * (1.0 / 65536.0))));
  }
}

TcArgs tc_args(etdm_handle *h) {
  TcArgs a{};
  a.g = h->geom_tc;
  a.n_tiles = h->n_tiles_tc;
  a.tile_ptr = h->d_tile_ptr_tc;
  a.keys = h->d_keys_tc;
  for (int ax = 0; ax < 3; ++ax) a.tab[ax] = h->d_tabf ? h->d_tabf + h->tab_off[ax] : nullptr;
  a.rc2f = h->d_rc2f;
  a.nu = h->d_nu_tc;
  a.xr_off = h->d_xr_off;
  a.mu_off = h->d_mu_off;
  a.tmu = h->d_tmu;
  a.n_vg = h->n_vg;
  a.vg_t0 = h->d_vg_t0;
  a.vg_nu = h->d_vg_nu;
  a.vg_eoff = h->d_vg_eoff;
  a.vg_xoff = h->d_vg_xoff;
  a.vg_mu = h->d_vg_mu;
  a.xr = h->d_xr;
  a.xv = h->d_xv;
  a.vent = h->d_vent;
  a.rowexp = h->d_rowexp;
  a.Osl = h->d_Osl;
  a.oscale = h->d_oscale;
  a.Nocc = h->N;
  a.NoccP = h->N + (h->N & 1);
  a.ocw = osl_width(h->N);
  a.rho = h->d_rho;
  a.rhof = h->d_rhof;
  a.v = h->d_vtot;
  a.vt = h->d_vt;
  a.Vfix = h->d_Vfix;
  a.dV = h->dV;
  a.flags = h->d_flags;
  return a;
}

cudaError_t launch_tables_f32(etdm_handle *h, cudaStream_t s) {
  for (int ax = 0; ax < 3; ++ax) {
    long total = (long)h->M * kImgN * h->n[ax];
    int blocks = (int)std::min<long>((total + 255) / 256, 4096);
    tables_f32_kernel<<<blocks, 256, 0, s>>>(h->d_sq + h->tab_off[ax], h->d_ex + h->tab_off[ax],
                                             h->d_norm, h->M, h->n[ax],
                                             h->d_tabf + h->tab_off[ax]);
  }
  return cudaGetLastError();
}

cudaError_t launch_count_unique(etdm_handle *h, int *d_nu, cudaStream_t s) {
  const int blocks = (h->n_tiles_tc + 255) / 256;
  count_unique_kernel<<<std::max(blocks, 1), 256, 0, s>>>(h->d_tile_ptr_tc, h->d_keys_tc,
                                                          h->n_tiles_tc, d_nu);
  return cudaGetLastError();
}

cudaError_t launch_xr_build(etdm_handle *h, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(xr_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStageBytes);
  if (e != cudaSuccess) return e;
  const int blocks = std::min(h->n_tiles_tc, 4 * h->num_sms);
  xr_build_kernel<<<blocks, 256, kStageBytes, s>>>(tc_args(h));
  return cudaGetLastError();
}

cudaError_t launch_xv_build(etdm_handle *h, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(xv_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStageBytes);
  if (e != cudaSuccess) return e;
  const int blocks = std::min(h->n_tiles_tc, 4 * h->num_sms);
  xv_build_kernel<<<blocks, 256, kStageBytes, s>>>(tc_args(h));
  return cudaGetLastError();
}

cudaError_t launch_operand_build(etdm_handle *h, cudaStream_t s) {
  cudaError_t e = launch_xr_build(h, s);
  if (e != cudaSuccess) return e;
  return launch_xv_build(h, s);
}

int tc_rho_steps(int nu) { return rsteps(nu); }
int tc_v_entries(int nu) { return vpad(nu); }
int tc_group_max() { return kVGmax; }
int tc_v_slices() { return kVSlX; }

OsArgs os_args(etdm_handle *h) {
  OsArgs a{};
  a.O = reinterpret_cast<const float2 *>(h->d_O);
  a.M = h->M; a.N = h->N; a.NP = h->N + (h->N & 1); a.ocw = osl_width(h->N);
  a.Osl = h->d_Osl; a.oscale = h->d_oscale; a.dO = h->d_dO;
  return a;
}

VfArgs vf_args(etdm_handle *h) {
  VfArgs a{};
  a.Vfix = h->d_Vfix; a.M = h->M; a.Vout = h->d_Vfin;
  return a;
}

cudaError_t launch_mixed_rho(const MixedPlan &P, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(P.omax, 0, P.omax_bytes, s);
  if (e != cudaSuccess) return e;
  {
    const long warps = (long)((P.os_maxN + 31) / 32) * ((P.os_maxMN / std::max(P.os_maxN, 1) + 63) / 64);
    const int bx = (int)std::max<long>(1, std::min<long>((warps + 7) / 8, 4096));
    omax_kernel<<<dim3(bx, P.n_sys), 256, 0, s>>>(P.os, P.active);
    const int bs = (int)std::max<long>(1, std::min<long>((P.os_maxMN + 255) / 256, 4096));
    oslice_kernel<<<dim3(bs, P.n_sys), 256, 0, s>>>(P.os, P.active);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sm = (size_t)kRhoStages * kRhoStage;
  e = cudaFuncSetAttribute(rho_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  rho_tc_kernel<<<P.rho.grid, kRhoThreads, sm, s>>>(P.rho);
  return cudaGetLastError();
}

cudaError_t launch_mixed_potential(const MixedPlan &P, cudaStream_t s) {
  // the V pass adds into zeroed fixed-point sums; the potential pass records max |v|
  cudaError_t e = cudaMemsetAsync(P.vfix, 0, P.vfix_bytes, s);
  if (e != cudaSuccess) return e;
  return launch_df_potential(P.dfl, P.df, P.active, s);
}

cudaError_t launch_mixed_vmat(const MixedPlan &P, cudaStream_t s) {
  const size_t sm = (size_t)kVStages * kVStage + 2 * (size_t)kVTileBuf;
  cudaError_t e = cudaFuncSetAttribute(vmat_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  vmat_tc_kernel<<<P.v.grid, kVThreads, sm, s>>>(P.v);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  vfix_kernel<<<dim3(P.vf_blocks, P.n_sys), 256, 0, s>>>(P.vf, P.active);
  return cudaGetLastError();
}

int tc_max_list() { return kNmax; }

}  // namespace etdm
