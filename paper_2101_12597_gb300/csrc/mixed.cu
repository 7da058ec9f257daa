// Mixed-precision grid passes on the 5th-generation tensor cores (tcgen05).
//
// basis -> grid density (Eq. 2, 3, 12) in orbital form: per 128-point tile
// (4 x 4 x 8) with a truncation list of n <= 128 function images,
//     phi = X O_loc  (128 x n x N_occ),  rho_p = 2 sum_m phi_pm^2 ,
// a sum of positive terms (the same density as sum X D X, whose terms cancel
// heavily in a non-orthogonal basis).  X rows and O columns are cut into exact
// integer slices held in BF16 ("Ozaki" splitting):
//     X_pa = 2^(e_p-8) (I0 + I1/2^8 + I2/2^16 + I3/2^24)   (X as a float pair),
//     O_am = 2^(g_m-8) (K0 + K1/2^8 + K2/2^16),    |I|, |K| <= 128.
// Every product of slices is an integer, and every accumulator (at most three
// products per K step, <= 128 entries of <= 2^14) stays below 2^24, so the
// four FP32 accumulators of slice order 0..3 in tensor memory are exact
// whatever rounding the accumulator applies (the tensor-core accumulator
// truncates).  X is resolved to about 2^-31 of its row maximum, which the
// cancellation in X O needs; the 24-bit quantization of O is coherent and is
// removed to first order in the energy by sum (4 V O) o (O - Oq) (dense
// reverse kernel); the rest (order >= 4 terms, FP32 square sums) is unbiased
// and incoherent across grid points.
//
// grid -> basis potential matrix (Eq. 11): V_ab = dV sum_p X_pa v_p X_pb with
// X^T and (v X)^T rows cut into four exact integer slices each (exponent per
// list entry from a separable bound over the tile) and slice orders 0..3 in
// four exact accumulators.  The gradient amplifies errors of V by the large
// Loewdin coefficients (O^T V O), so V is kept to about 2^-31 of its row
// scale; tiles are summed in per-CTA float-pair copies (no atomics) and the
// copies in FP64.
//
// Operands are staged in shared memory in the canonical no-swizzle K-major
// layout (8-row x 16-byte core matrices); one thread issues tcgen05.mma, the
// completion is tracked with tcgen05.commit on an mbarrier (bounded wait), and
// the accumulators are read back with tcgen05.ld.  One persistent CTA per SM.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace etdm {

constexpr int kRhoThreads = 512;   // 16 warps: 8 build-only, 8 also read TMEM
constexpr int kVThreads = 384;     // 12 warps (register budget of the V pass)
constexpr int kTP = 128;     // points per tile
constexpr int kNmax = 128;   // max padded list length
constexpr int kTmemCols = 512;
constexpr long kMbarSpin = 4000000;

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// canonical K-major no-swizzle offset of element (row, k) for a 128 x 128 BF16 operand
__device__ __forceinline__ int kmaj_off(int row, int k) {
  return (((row >> 3) * (kNmax / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}
// the same for a 128-row operand holding a K chunk of 64 columns
constexpr int kKc = 64;
constexpr int kChunkBytes = kTP * kKc * 2;
__device__ __forceinline__ int kmaj_off64(int row, int k) {
  return (((row >> 3) * (kKc / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo = (kNmax / 8) * 128) {
  const uint32_t lbo = 128;
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version (sm_100 family); no swizzle
  return d;
}

// kind::f16 with BF16 A and B, FP32 accumulate, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(mbar))
      : "memory");
}

// bounded wait for the mbarrier phase `parity`; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
  uint32_t done = 0;
  long it = 0;
  while (!done) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(su32(mbar)), "r"(parity)
        : "memory");
    if (++it > kMbarSpin) return false;
  }
  return true;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_val(uint16_t b) {
  return __uint_as_float((uint32_t)b << 16);
}

struct TcArgs {
  GridGeom g;  // 4 x 4 x 8 tiles
  int n_tiles;
  const int *tile_ptr, *keys;
  const float4 *tab[3];        // per axis [mu][img][i]: (sq, c hi, c lo, 0),
                               // c = norm^(1/3) exp(-alpha sq) as a float pair
  const float *rc2f;           // [M]
  const signed char *rowexp;   // [G]
  const uint2 *Osl;            // [M][N] bf16 slices of column-scaled O: x = K0 | K1 << 16, y = K2
  const float *oscale;         // [N] 2^g_m
  int Nocc;
  double *rho;                 // [G]
  const double *v;             // [G]
  float2 *Vpriv;               // [gridDim][M][M] per-CTA float-pair V (upper triangle)
  double dV;
  int *flags;
};

struct TileShared {
  int mu[kNmax];
  float fs[kNmax];
  float4 stage[kNmax * 16];  // per entry: 4 x-values, 4 y-values, 8 z-values
  float part[kTP];
  uint64_t mbar;
  uint32_t tbase;
  int n, npad, inside[kTP];
};

// index of slot s of entry e in the staged table: entry-major for the density
// pass (a warp shares the entry), slot-major for the V pass (a warp spans entries)
template <bool TR>
__device__ __forceinline__ int sidx(int e, int s) {
  return TR ? s * kNmax + e : e * 16 + s;
}

// stage the per-axis (sq, c exp(-alpha sq)) values of the tile for every entry
// (by the threads tid = 0 .. nthr-1 of the calling group)
template <bool TR>
__device__ void stage_tile(const TcArgs &A, TileShared &S, int t, int kb, int n, int tid,
                           int nthr) {
  const GridGeom &g = A.g;
  int bz = t % g.nbz, by = (t / g.nbz) % g.nby, bx = t / (g.nbz * g.nby);
  int i0 = bx * 4, j0 = by * 4, k0 = bz * 8;
  for (int q = tid; q < n * 16; q += nthr) {
    int e = q >> 4, s = q & 15;
    int key = A.keys[kb + e];
    int mu = key >> 9;
    int ix = ((key >> 6) & 7) - 4 + kImgMax, iy = ((key >> 3) & 7) - 4 + kImgMax,
        iz = (key & 7) - 4 + kImgMax;
    const float4 out = make_float4(INFINITY, 0.f, 0.f, 0.f);
    float4 val;
    if (s < 4) {
      int i = i0 + s;
      val = i < g.nx ? A.tab[0][((long)mu * kImgN + ix) * g.nx + i] : out;
    } else if (s < 8) {
      int j = j0 + s - 4;
      val = j < g.ny ? A.tab[1][((long)mu * kImgN + iy) * g.ny + j] : out;
    } else {
      int k = k0 + s - 8;
      val = k < g.nz ? A.tab[2][((long)mu * kImgN + iz) * g.nz + k] : out;
    }
    S.stage[sidx<TR>(e, s)] = val;
    if (s == 0) S.mu[e] = mu;
  }
  for (int p = tid; p < kTP; p += nthr) {
    int li = p >> 5, lj = (p >> 3) & 3, lk = p & 7;
    S.inside[p] = (i0 + li < g.nx && j0 + lj < g.ny && k0 + lk < g.nz)
                      ? ((i0 + li) * g.ny + (j0 + lj)) * g.nz + (k0 + lk)
                      : -1;
  }
}

template <bool TR>
__device__ __forceinline__ float basis_val(const TileShared &S, const float *rc2f, int e, int p) {
  int li = p >> 5, lj = (p >> 3) & 3, lk = p & 7;
  float4 x = S.stage[sidx<TR>(e, li)], y = S.stage[sidx<TR>(e, 4 + lj)],
         z = S.stage[sidx<TR>(e, 8 + lk)];
  float r2 = (x.x + y.x) + z.x;
  return r2 < rc2f[S.mu[e]] ? x.y * y.y * z.y : 0.f;
}

// float-pair (hi + lo) arithmetic: exact product by FMA, then renormalization
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  const float e = fmaf(a.x, b.x, -p);
  const float t = e + fmaf(a.x, b.y, a.y * b.x);
  const float s = p + t;
  return make_float2(s, t - (s - p));
}

// the same basis value as a float pair (about 44 significant bits); the hi
// part equals basis_val up to rounding
template <bool TR>
__device__ __forceinline__ float2 basis_val_df(const TileShared &S, const float *rc2f, int e,
                                               int p) {
  int li = p >> 5, lj = (p >> 3) & 3, lk = p & 7;
  float4 x = S.stage[sidx<TR>(e, li)], y = S.stage[sidx<TR>(e, 4 + lj)],
         z = S.stage[sidx<TR>(e, 8 + lk)];
  float r2 = (x.x + y.x) + z.x;
  if (!(r2 < rc2f[S.mu[e]])) return make_float2(0.f, 0.f);
  return df_mul(df_mul(make_float2(x.y, x.z), make_float2(y.y, y.z)), make_float2(z.y, z.z));
}

__device__ __forceinline__ void tmem_alloc(TileShared &S) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&S.tbase)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&S.mbar)), "r"(1)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(TileShared &S) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tbase),
                 "r"(kTmemCols)
                 : "memory");
}

// ---- density ---------------------------------------------------------------
__global__ void __launch_bounds__(kRhoThreads, 1) rho_tc_kernel(TcArgs A) {
  // one K chunk (64 list entries) of the operands at a time:
  // A = X slices I0..I3 (128 points x 64), B = O slices K0..K2 (<= 128 orbitals x 64)
  extern __shared__ __align__(1024) uint8_t dsm[];
  uint8_t *sA = dsm;
  uint8_t *sB = dsm + 4 * kChunkBytes;
  __shared__ TileShared S;
  tmem_alloc(S);
  const uint32_t tmem = S.tbase;
  uint32_t phase = 0;
  bool ok = true;
  const int w = threadIdx.x >> 5, quad = w & 3, half = w >> 2;
  const int pe = quad * 32 + (threadIdx.x & 31);  // epilogue point (TMEM lane)
  const uint32_t lane = (uint32_t)(quad * 32) << 16;
  for (int t = blockIdx.x; t < A.n_tiles && ok; t += gridDim.x) {
    const int kb = A.tile_ptr[t], n = A.tile_ptr[t + 1] - kb;
    if (n > kNmax) {  // rejected at set-up; never reached
      if (threadIdx.x == 0) atomicExch(A.flags + FLAG_ERR, ETDM_ERR_NUMERIC);
      continue;
    }
    const int nk = n <= 32 ? 2 : (n + 15) / 16;  // K steps of 16
    const int nkc = (nk + 3) / 4;                // K chunks of 64
    stage_tile<false>(A, S, t, kb, n, threadIdx.x, blockDim.x);
    __syncthreads();
    float rsum = 0.f;
    // occupied orbitals in chunks of up to 128 columns
    for (int m0 = 0; m0 < A.Nocc && ok; m0 += kNmax) {
      const int nm = min(kNmax, A.Nocc - m0);
      const int nmpad = nm <= 32 ? 32 : ((nm + 31) / 32) * 32;
      for (int m = threadIdx.x; m < nmpad; m += blockDim.x)
        S.fs[m] = m < nm ? A.oscale[m0 + m] : 0.f;
      for (int kc = 0; kc < nkc && ok; ++kc) {
        const int k0 = kc * kKc;
        // A: X slices of entries k0 .. k0 + 63; items (point, 8 entries)
        for (int q = threadIdx.x; q < kTP * (kKc / 8); q += blockDim.x) {
          const int p = q % kTP, c0 = (q / kTP) * 8;
          const int gp = S.inside[p];
          const int ep = gp >= 0 ? (int)A.rowexp[gp] : 0;
          uint16_t sl[4][8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int a = k0 + c0 + u;
            float2 x = (a < n && gp >= 0) ? basis_val_df<false>(S, A.rc2f, a, p) : make_float2(0.f, 0.f);
            // x 2^(8 - e_p) = r0 + r1/256 + r2/256^2 + r3/256^3 + O(2^-25)
            float h = ldexpf(x.x, 8 - ep), l = ldexpf(x.y, 8 - ep);
            float r0 = rintf(h);
            float tt = ((h - r0) + l) * 256.f;
            float r1 = rintf(tt);
            tt = (tt - r1) * 256.f;
            float r2 = rintf(tt);
            tt = (tt - r2) * 256.f;
            float r3 = rintf(tt);
            sl[0][u] = bf16_bits(r0); sl[1][u] = bf16_bits(r1);
            sl[2][u] = bf16_bits(r2); sl[3][u] = bf16_bits(r3);
          }
          const int off = kmaj_off64(p, c0);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            uint4 v;
            v.x = sl[k][0] | (sl[k][1] << 16); v.y = sl[k][2] | (sl[k][3] << 16);
            v.z = sl[k][4] | (sl[k][5] << 16); v.w = sl[k][6] | (sl[k][7] << 16);
            *(uint4 *)(sA + k * kChunkBytes + off) = v;
          }
        }
        // B: O slices, B[m][a] = O-slice[mu_a][m0 + m]; items (orbital, 8 entries)
        for (int q = threadIdx.x; q < nmpad * (kKc / 8); q += blockDim.x) {
          const int m = q % nmpad, c0 = (q / nmpad) * 8;
          uint32_t w01[8], w2[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int a = k0 + c0 + u;
            uint2 kk = (a < n && m < nm) ? A.Osl[(long)S.mu[a] * A.Nocc + m0 + m]
                                         : make_uint2(0u, 0u);
            w01[u] = kk.x;
            w2[u] = kk.y;
          }
          const int off = kmaj_off64(m, c0);
          uint4 v0, v1, v2;
          v0.x = (w01[0] & 0xFFFF) | (w01[1] << 16); v0.y = (w01[2] & 0xFFFF) | (w01[3] << 16);
          v0.z = (w01[4] & 0xFFFF) | (w01[5] << 16); v0.w = (w01[6] & 0xFFFF) | (w01[7] << 16);
          v1.x = (w01[0] >> 16) | (w01[1] & 0xFFFF0000u);
          v1.y = (w01[2] >> 16) | (w01[3] & 0xFFFF0000u);
          v1.z = (w01[4] >> 16) | (w01[5] & 0xFFFF0000u);
          v1.w = (w01[6] >> 16) | (w01[7] & 0xFFFF0000u);
          v2.x = w2[0] | (w2[1] << 16); v2.y = w2[2] | (w2[3] << 16);
          v2.z = w2[4] | (w2[5] << 16); v2.w = w2[6] | (w2[7] << 16);
          *(uint4 *)(sB + off) = v0;
          *(uint4 *)(sB + kChunkBytes + off) = v1;
          *(uint4 *)(sB + 2 * kChunkBytes + off) = v2;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t idesc = idesc_bf16(nmpad);
          const uint32_t a0 = su32(sA), b0 = su32(sB);
          const uint32_t sbo = (kKc / 8) * 128;
          const int ksteps = min(4, nk - kc * 4);
          for (int kk = 0; kk < ksteps; ++kk) {
            const uint32_t off = kk * 256;
            const uint64_t I0 = smem_desc(a0 + off, sbo), I1 = smem_desc(a0 + kChunkBytes + off, sbo),
                           I2 = smem_desc(a0 + 2 * kChunkBytes + off, sbo),
                           I3 = smem_desc(a0 + 3 * kChunkBytes + off, sbo);
            const uint64_t K0 = smem_desc(b0 + off, sbo), K1 = smem_desc(b0 + kChunkBytes + off, sbo),
                           K2 = smem_desc(b0 + 2 * kChunkBytes + off, sbo);
            const uint32_t acc = (kc > 0 || kk > 0);
            mma_bf16(tmem, I0, K0, idesc, acc);                  // order 0
            mma_bf16(tmem + kNmax, I0, K1, idesc, acc);          // order 1
            mma_bf16(tmem + kNmax, I1, K0, idesc, 1u);
            mma_bf16(tmem + 2 * kNmax, I0, K2, idesc, acc);      // order 2
            mma_bf16(tmem + 2 * kNmax, I1, K1, idesc, 1u);
            mma_bf16(tmem + 2 * kNmax, I2, K0, idesc, 1u);
            mma_bf16(tmem + 3 * kNmax, I1, K2, idesc, acc);      // order 3
            mma_bf16(tmem + 3 * kNmax, I2, K1, idesc, 1u);
            mma_bf16(tmem + 3 * kNmax, I3, K0, idesc, 1u);
          }
          mma_commit(&S.mbar);
        }
        ok = __syncthreads_and(mbar_wait(&S.mbar, phase)) != 0;
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      if (ok && w < 8) {  // warps 0..7 read TMEM (lane quarter w % 4, column half w / 4)
        // phi_pm = 2^(e_p + g_m - 16) y with y = acc0 + (acc1 + (acc2 + acc3/256)/256)/256;
        // rho_p = 2 sum_m phi_pm^2 (every term positive)
        const int cw = nmpad / 2;
        for (int c0 = half * cw; c0 < half * cw + cw; c0 += 16) {
          float y0[16], y1[16], y2[16], y3[16];
          tmem_ld16(tmem + lane + c0, y0);
          tmem_ld16(tmem + lane + kNmax + c0, y1);
          tmem_ld16(tmem + lane + 2 * kNmax + c0, y2);
          tmem_ld16(tmem + lane + 3 * kNmax + c0, y3);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float y = y0[j] + (y1[j] + (y2[j] + y3[j] * (1.f / 256.f)) * (1.f / 256.f)) *
                                  (1.f / 256.f);
            y *= S.fs[c0 + j];
            rsum = fmaf(y, y, rsum);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(A.flags + FLAG_ERR, ETDM_ERR_TIMEOUT);
      break;
    }
    if (half == 1) S.part[pe] = rsum;
    __syncthreads();
    if (half == 0) {
      const int gp = S.inside[pe];
      if (gp >= 0) {
        const int ep = (int)A.rowexp[gp];
        double r = (double)rsum + (double)S.part[pe];
        A.rho[gp] = ldexp(r, 2 * ep - 31);
      }
    }
    __syncthreads();
  }
  tmem_free(S);
}


// ---- potential matrix ---------------------------------------------------------
// sum of two float pairs (hi, lo) with an exact TwoSum of the high parts
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  const float e = (a.x - (s - bb)) + (b.x - bb);
  const float t = e + a.y + b.y;
  const float h = s + t;
  return make_float2(h, t - (h - s));
}

// exponent e with |x| 2^(8-e) < 128 for every |x| <= bound (0 for bound 0)
__device__ __forceinline__ int slice_exp(float bound) {
  return bound > 0.f ? ilogbf(bound) + 2 : 0;
}

// 4 integer slices of the float pair x 2^(8 - e) (|.| < 128): x 2^(8-e) =
// r0 + r1/256 + r2/256^2 + r3/256^3 + O(2^-25)
__device__ __forceinline__ void slice4(float2 x, int e, uint16_t *s) {
  float h = ldexpf(x.x, 8 - e), l = ldexpf(x.y, 8 - e);
  float r0 = rintf(h);
  float tt = ((h - r0) + l) * 256.f;
  float r1 = rintf(tt);
  tt = (tt - r1) * 256.f;
  float r2 = rintf(tt);
  tt = (tt - r2) * 256.f;
  float r3 = rintf(tt);
  s[0] = bf16_bits(r0); s[1] = bf16_bits(r1); s[2] = bf16_bits(r2); s[3] = bf16_bits(r3);
}

// ---- mbarrier helpers for the warp-specialized pipelines ---------------------
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// V_loc[a][b] = dV sum_p X_pa v_p X_pb on tensor cores with exact integer slices
// of X^T (rows a, exponent per entry from a bound over the tile) and (v X)^T
// (rows b); slice orders 0..3 in four FP32 accumulators (exact).  Warp roles:
// warps 0-7 build the operand slices of 32-point K chunks into two shared-memory
// stages; lane 0 of warp 8 issues the MMAs; warps 8-11 read the accumulators
// (lane quarter = warp % 4) and add V_loc into the CTA's private float-pair copy
// of the upper triangle of V.  A tile's MMAs start once the previous tile's
// accumulators are read; building overlaps both.
constexpr int kVProd = 256;              // producer threads (warps 0-7)
constexpr int kVEpi = 128;               // epilogue threads (warps 8-11)
constexpr int kVKc = 32;                 // points per K chunk
constexpr int kVSlice = kTP * kVKc * 2;  // one slice of one K chunk (8 KB)
constexpr int kVStage = 8 * kVSlice;     // X^T and (v X)^T, 4 slices each
constexpr int kVStages = 2;

__device__ __forceinline__ int kmaj_off32(int row, int k) {
  return (((row >> 3) * (kVKc / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

struct VMeta {  // per-tile data the epilogue needs (double-buffered)
  int mu[kNmax];
  int ea[kNmax], eb[kNmax];
  int rank[kNmax];
  int n, npad, maxrank;
};

__global__ void __launch_bounds__(kVThreads, 1) vmat_tc_kernel(TcArgs A) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  __shared__ TileShared S;  // producer-side staging (tables, points)
  __shared__ VMeta meta[2];
  __shared__ float2 vp[kTP];
  __shared__ float vmax_s;
  __shared__ __align__(8) uint64_t bar_full[kVStages], bar_empty[kVStages], bar_acc_full,
      bar_acc_empty, bar_meta_full[2], bar_meta_empty[2];
  __shared__ int stop;
  const int tid = threadIdx.x, w = tid >> 5;
  const int M = A.g.M;
  float2 *Vpriv = A.Vpriv + (long)blockIdx.x * M * M;
  if (tid == 0) {
    for (int s = 0; s < kVStages; ++s) { mbar_init(&bar_full[s], kVProd); mbar_init(&bar_empty[s], 1); }
    mbar_init(&bar_acc_full, 1);
    mbar_init(&bar_acc_empty, kVEpi);
    for (int s = 0; s < 2; ++s) { mbar_init(&bar_meta_full[s], kVProd); mbar_init(&bar_meta_empty[s], kVEpi); }
    stop = 0;
  }
  tmem_alloc(S);  // also fences the barrier initialization
  const uint32_t tmem = S.tbase;
  const int ntiles_cta = A.n_tiles > (int)blockIdx.x
                             ? (A.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                             : 0;
  if (w < 8) {
    // ------------------------------- producers -----------------------------------
    int fill = 0;  // K-chunk stage fills so far
    for (int it = 0; it < ntiles_cta; ++it) {
      const int t = blockIdx.x + it * gridDim.x;
      const int kb = A.tile_ptr[t], n = min(A.tile_ptr[t + 1] - kb, kNmax);
      const int npad = n <= 32 ? 32 : ((n + 31) / 32) * 32;
      const int mb = it & 1;
      if (it >= 2 && !mbar_wait(&bar_meta_empty[mb], ((it >> 1) - 1) & 1)) { atomicExch(&stop, 1); }
      if (*(volatile int *)&stop) break;
      VMeta &m = meta[mb];
      stage_tile<true>(A, S, t, kb, n, tid, kVProd);
      if (tid == 0) vmax_s = 0.f;
      named_sync(1, kVProd);
      for (int p = tid; p < kTP; p += kVProd) {
        const int gp = S.inside[p];
        const double vv = gp >= 0 ? A.v[gp] * A.dV : 0.0;
        const float hi = (float)vv;
        vp[p] = make_float2(hi, (float)(vv - (double)hi));
        atomicMax((int *)&vmax_s, __float_as_int(fabsf(hi)));  // non-negative floats order as ints
      }
      named_sync(1, kVProd);
      for (int a = tid; a < kNmax; a += kVProd) {
        float bnd = 0.f;
        int rk = 0;
        if (a < n) {
          float mx = 0.f, my = 0.f, mz = 0.f;
          for (int s = 0; s < 4; ++s) mx = fmaxf(mx, S.stage[sidx<true>(a, s)].y);
          for (int s = 4; s < 8; ++s) my = fmaxf(my, S.stage[sidx<true>(a, s)].y);
          for (int s = 8; s < 16; ++s) mz = fmaxf(mz, S.stage[sidx<true>(a, s)].y);
          bnd = mx * my * mz * 1.0001f;
          while (rk < a && S.mu[a - rk - 1] == S.mu[a]) ++rk;  // image rank among equal mu
        }
        m.mu[a] = a < n ? S.mu[a] : 0;
        m.ea[a] = slice_exp(bnd);
        m.eb[a] = slice_exp(bnd * vmax_s * 1.0001f);
        m.rank[a] = rk;
      }
      named_sync(1, kVProd);
      if (tid == 0) {
        int mr = 0;
        for (int a = 0; a < n; ++a) mr = max(mr, m.rank[a]);
        m.maxrank = mr;
        m.n = n;
        m.npad = npad;
      }
      for (int kc = 0; kc < kTP / kVKc; ++kc, ++fill) {
        const int s = fill % kVStages, use = fill / kVStages;
        if (use > 0 && !mbar_wait(&bar_empty[s], (use - 1) & 1)) { atomicExch(&stop, 1); break; }
        uint8_t *sA = dsm + s * kVStage, *sB = sA + 4 * kVSlice;
        for (int q = tid; q < npad * (kVKc / 8); q += kVProd) {
          const int a = q % npad, c0 = (q / npad) * 8;
          uint16_t xs[4][8], ws[4][8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int p = kc * kVKc + c0 + u;
            float2 x = (a < n && S.inside[p] >= 0) ? basis_val_df<true>(S, A.rc2f, a, p)
                                                   : make_float2(0.f, 0.f);
            float2 wv = df_mul(x, vp[p]);
            uint16_t s4[4];
            slice4(x, m.ea[a], s4);
#pragma unroll
            for (int k = 0; k < 4; ++k) xs[k][u] = s4[k];
            slice4(wv, m.eb[a], s4);
#pragma unroll
            for (int k = 0; k < 4; ++k) ws[k][u] = s4[k];
          }
          const int off = kmaj_off32(a, c0);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            uint4 v;
            v.x = xs[k][0] | (xs[k][1] << 16); v.y = xs[k][2] | (xs[k][3] << 16);
            v.z = xs[k][4] | (xs[k][5] << 16); v.w = xs[k][6] | (xs[k][7] << 16);
            *(uint4 *)(sA + k * kVSlice + off) = v;
            v.x = ws[k][0] | (ws[k][1] << 16); v.y = ws[k][2] | (ws[k][3] << 16);
            v.z = ws[k][4] | (ws[k][5] << 16); v.w = ws[k][6] | (ws[k][7] << 16);
            *(uint4 *)(sB + k * kVSlice + off) = v;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (kc == 0) mbar_arrive(&bar_meta_full[mb]);  // metadata written before chunk 0 is out
        mbar_arrive(&bar_full[s]);
      }
      if (*(volatile int *)&stop) break;
      named_sync(1, kVProd);  // the table buffer is reused by the next tile
    }
  } else {
    // ------------------------- MMA issue and epilogue ------------------------------
    const int quad = w & 3;
    const int ae = quad * 32 + (tid & 31);
    const uint32_t lane = (uint32_t)(quad * 32) << 16;
    int fill = 0;
    for (int it = 0; it < ntiles_cta; ++it) {
      const int mb = it & 1;
      bool ok = true;
      if (tid == kVProd) {  // lane 0 of warp 8
        if (it > 0) ok = mbar_wait(&bar_acc_empty, (it - 1) & 1);
        if (ok) ok = mbar_wait(&bar_meta_full[mb], (it >> 1) & 1);
        const int npad = ok ? meta[mb].npad : 32;
        for (int kc = 0; ok && kc < kTP / kVKc; ++kc) {
          const int s = (fill + kc) % kVStages, use = (fill + kc) / kVStages;
          ok = mbar_wait(&bar_full[s], use & 1);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t idesc = idesc_bf16(npad);
          const uint32_t a0 = su32(dsm + s * kVStage), b0 = a0 + 4 * kVSlice;
          const uint32_t sbo = (kVKc / 8) * 128;
          for (int kk = 0; kk < kVKc / 16; ++kk) {
            const uint32_t off = kk * 256;
            uint64_t X[4], W[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              X[k] = smem_desc(a0 + k * kVSlice + off, sbo);
              W[k] = smem_desc(b0 + k * kVSlice + off, sbo);
            }
            const uint32_t acc = (kc > 0 || kk > 0);
            mma_bf16(tmem, X[0], W[0], idesc, acc);                 // order 0
            mma_bf16(tmem + kNmax, X[0], W[1], idesc, acc);         // order 1
            mma_bf16(tmem + kNmax, X[1], W[0], idesc, 1u);
            mma_bf16(tmem + 2 * kNmax, X[0], W[2], idesc, acc);     // order 2
            mma_bf16(tmem + 2 * kNmax, X[1], W[1], idesc, 1u);
            mma_bf16(tmem + 2 * kNmax, X[2], W[0], idesc, 1u);
            mma_bf16(tmem + 3 * kNmax, X[0], W[3], idesc, acc);     // order 3
            mma_bf16(tmem + 3 * kNmax, X[1], W[2], idesc, 1u);
            mma_bf16(tmem + 3 * kNmax, X[2], W[1], idesc, 1u);
            mma_bf16(tmem + 3 * kNmax, X[3], W[0], idesc, 1u);
          }
          mma_commit(&bar_empty[s]);  // the stage is free once these MMAs complete
        }
        if (ok) mma_commit(&bar_acc_full);
        if (!ok) atomicExch(&stop, 1);
      }
      fill += kTP / kVKc;
      __syncwarp();
      if (*(volatile int *)&stop) break;
      // all epilogue threads: wait for the accumulators and the tile's metadata
      ok = mbar_wait(&bar_acc_full, it & 1) && mbar_wait(&bar_meta_full[mb], (it >> 1) & 1);
      if (!ok) { atomicExch(&stop, 1); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const VMeta &m = meta[mb];
      const int n = m.n, npad = m.npad;
      const int ma = ae < n ? m.mu[ae] : 0, ra = ae < n ? m.rank[ae] : -1;
      // values of row ae, in 16-column chunks; rows of equal mu (images) add into
      // the same targets, so they take turns by image rank
      for (int r = 0; r <= m.maxrank; ++r) {
        for (int c0 = 0; c0 < npad; c0 += 16) {
          float y0[16], y1[16], y2[16], y3[16];
          tmem_ld16(tmem + lane + c0, y0);
          tmem_ld16(tmem + lane + kNmax + c0, y1);
          tmem_ld16(tmem + lane + 2 * kNmax + c0, y2);
          tmem_ld16(tmem + lane + 3 * kNmax + c0, y3);
          if (ra == r) {
            float2 val[16], old[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int b = c0 + j;
              const int sc = m.ea[ae] + m.eb[b < n ? b : 0] - 16;
              float lo = (y1[j] + (y2[j] + y3[j] * (1.f / 256.f)) * (1.f / 256.f)) * (1.f / 256.f);
              float hi = y0[j] + lo;
              lo = lo - (hi - y0[j]);
              val[j] = make_float2(ldexpf(hi, sc), ldexpf(lo, sc));
              if (b < n && b >= ae && m.mu[b] == ma && b != ae) {  // both orders of an image pair
                val[j].x *= 2.f;
                val[j].y *= 2.f;
              }
            }
            // adjacent columns of equal mu (images) share a target: fold them first
            bool live[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) live[j] = (c0 + j >= ae && c0 + j < n);
            if (m.maxrank > 0) {
#pragma unroll
              for (int j = 15; j > 0; --j)
                if (live[j] && live[j - 1] && m.mu[c0 + j] == m.mu[c0 + j - 1]) {
                  val[j - 1] = df_add(val[j - 1], val[j]);
                  live[j] = false;
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j)
              old[j] = live[j] ? Vpriv[(long)ma * M + m.mu[c0 + j]] : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (live[j]) Vpriv[(long)ma * M + m.mu[c0 + j]] = df_add(old[j], val[j]);
          }
        }
        if (m.maxrank > 0) named_sync(2, kVEpi);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&bar_acc_empty);
      mbar_arrive(&bar_meta_empty[mb]);
    }
  }
  if (*(volatile int *)&stop && tid == 0) atomicExch(A.flags + FLAG_ERR, ETDM_ERR_TIMEOUT);
  tmem_free(S);
}

// H_upper[mu][nu] = sum over CTA copies of (hi + lo), FP64, mu <= nu
__global__ void vpriv_reduce_kernel(const float2 *Vpriv, int ncopies, int M, double *Vout) {
  const long MM = (long)M * M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MM;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / M), c = (int)(e % M);
    if (i > c) continue;
    double s = 0.0;
    for (int k = 0; k < ncopies; ++k) {
      const float2 v = Vpriv[(long)k * MM + e];
      s += (double)v.x + (double)v.y;
    }
    Vout[e] = s;
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

// per grid point: exponent e_p with max_a |X_pa| < 2^(e_p - 1) (same FP32 values
// as the density kernel computes)
__global__ void __launch_bounds__(256) rowexp_kernel(TcArgs A, signed char *rowexp) {
  __shared__ TileShared S;
  for (int t = blockIdx.x; t < A.n_tiles; t += gridDim.x) {
    const int kb = A.tile_ptr[t], n = A.tile_ptr[t + 1] - kb;
    stage_tile<false>(A, S, t, kb, min(n, kNmax), threadIdx.x, blockDim.x);
    __syncthreads();
    for (int p = threadIdx.x; p < kTP; p += blockDim.x) {
      const int gp = S.inside[p];
      if (gp < 0) continue;
      float mx = 0.f;
      for (int a = 0; a < min(n, kNmax); ++a) mx = fmaxf(mx, fabsf(basis_val<false>(S, A.rc2f, a, p)));
      rowexp[gp] = (signed char)(mx > 0.f ? ilogbf(mx) + 2 : 0);
    }
    __syncthreads();
  }
}

// Column slices of the occupied orbitals O (M x N): g_m = ilogb(max_mu |O_mu,m|)
// + 2, K0 + K1/256 + K2/65536 = O 2^(8 - g) to 24 bits; dO = O - Oq (FP64) for
// the first-order energy correction sum (4 H O) o dO.
__global__ void __launch_bounds__(256) oslice_kernel(const double *O, int M, int N, uint2 *Osl,
                                                     float *oscale, double *dO) {
  const int m = blockIdx.x;
  double mx = 0.0;
  for (int r = threadIdx.x; r < M; r += blockDim.x) mx = fmax(mx, fabs(O[(long)r * N + m]));
  __shared__ double red[256];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  mx = red[0];
  const int g = mx > 0.0 ? ilogb(mx) + 2 : 0;
  if (threadIdx.x == 0) oscale[m] = ldexpf(1.f, g);
  for (int r = threadIdx.x; r < M; r += blockDim.x) {
    const double o = O[(long)r * N + m];
    const double t0 = ldexp(o, 8 - g);
    const double r0 = rint(t0);
    const double t1 = (t0 - r0) * 256.0;
    const double r1 = rint(t1);
    const double t2 = (t1 - r1) * 256.0;
    const double r2 = rint(t2);
    const double q = ldexp(r0 + (r1 + r2 * (1.0 / 256.0)) * (1.0 / 256.0), g - 8);
    dO[(long)r * N + m] = o - q;
    Osl[(long)r * N + m] =
        make_uint2((uint32_t)bf16_bits((float)r0) | ((uint32_t)bf16_bits((float)r1) << 16),
                   (uint32_t)bf16_bits((float)r2));
  }
}

static TcArgs tc_args(etdm_handle *h) {
  TcArgs a{};
  a.g = h->geom_tc;
  a.n_tiles = h->n_tiles_tc;
  a.tile_ptr = h->d_tile_ptr_tc;
  a.keys = h->d_keys_tc;
  for (int ax = 0; ax < 3; ++ax) a.tab[ax] = h->d_tabf + h->tab_off[ax];
  a.rc2f = h->d_rc2f;
  a.rowexp = h->d_rowexp;
  a.Osl = h->d_Osl;
  a.oscale = h->d_oscale;
  a.Nocc = h->N;
  a.rho = h->d_rho;
  a.v = h->d_vtot;
  a.Vpriv = h->d_Vpriv;
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

cudaError_t launch_rowexp(etdm_handle *h, cudaStream_t s) {
  TcArgs a = tc_args(h);
  rowexp_kernel<<<std::min(h->n_tiles_tc, 8 * h->num_sms), 256, 0, s>>>(a, h->d_rowexp);
  return cudaGetLastError();
}

cudaError_t launch_oslice(etdm_handle *h, cudaStream_t s) {
  oslice_kernel<<<h->N, 256, 0, s>>>(h->d_O, h->M, h->N, h->d_Osl, h->d_oscale, h->d_dO);
  return cudaGetLastError();
}

cudaError_t launch_rho_tc(etdm_handle *h, cudaStream_t s) {
  const size_t sm = 7 * (size_t)kChunkBytes;
  cudaError_t e = cudaFuncSetAttribute(rho_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  rho_tc_kernel<<<std::min(h->n_tiles_tc, h->num_sms), kRhoThreads, sm, s>>>(tc_args(h));
  return cudaGetLastError();
}

cudaError_t launch_vmat_tc(etdm_handle *h, cudaStream_t s) {
  const size_t sm = (size_t)kVStages * kVStage;
  cudaError_t e = cudaFuncSetAttribute(vmat_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int copies = std::min(h->n_tiles_tc, h->n_vcopies);
  const size_t MM = (size_t)h->M * h->M;
  e = cudaMemsetAsync(h->d_Vpriv, 0, (size_t)copies * MM * sizeof(float2), s);
  if (e != cudaSuccess) return e;
  vmat_tc_kernel<<<copies, kVThreads, sm, s>>>(tc_args(h));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  vpriv_reduce_kernel<<<256, 256, 0, s>>>(h->d_Vpriv, copies, h->M, h->d_Vfin);
  return cudaGetLastError();
}

int tc_max_list() { return kNmax; }

}  // namespace etdm
