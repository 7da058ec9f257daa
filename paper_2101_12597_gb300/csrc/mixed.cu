// Mixed-precision grid passes on the 5th-generation tensor cores (tcgen05).
//
// basis -> grid density (Eq. 2, 12): per 128-point tile (4 x 4 x 8) with a
// truncation list of n <= 128 function images,
//     Y = X D_loc  (128 x n x n),  rho_p = sum_b X_pb Y_pb .
// X rows and D columns are cut into exact integer slices held in BF16
// ("Ozaki" splitting): X_pa = 2^(e_p-8) (I0 + I1/2^8 + I2/2^16),
// D_ab = 2^(f_b-8) (J0 + J1/2^8), |I|, |J| <= 128.  Every product of slices is
// an integer and every sum over a (<= 128 terms of <= 2^14) stays below 2^24,
// so the three FP32 accumulators in tensor memory
//     acc0 = I0 J0,  acc1 = I0 J1 + I1 J0,  acc2 = I1 J1 + I2 J0
// are exact whatever rounding the accumulator applies.  The remaining errors
// (dropped 2^-24 terms, FP32 row dot) are unbiased and incoherent across grid
// points; the quantization of D (16 bits) is coherent and is removed to first
// order in the energy with Tr(V (D - Dq)) (dense reverse kernel).
//
// grid -> basis potential matrix (Eq. 11): V_ab = dV sum_p X_pa v_p X_pb with
// X and v X as BF16 hi + lo pairs (three products, one FP32 accumulator); it
// only feeds the gradient and the first-order energy correction.
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

constexpr int kTcThreads = 256;
constexpr int kTP = 128;     // points per tile
constexpr int kNmax = 128;   // max padded list length
constexpr int kTmemCols = 512;
constexpr int kSliceBytes = kTP * kNmax * 2;  // one 128 x 128 BF16 operand
constexpr long kMbarSpin = 4000000;

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// canonical K-major no-swizzle offset of element (row, k) for a 128 x 128 BF16 operand
__device__ __forceinline__ int kmaj_off(int row, int k) {
  return (((row >> 3) * (kNmax / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  const uint32_t lbo = 128, sbo = (kNmax / 8) * 128;
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
  const float2 *tab[3];        // per axis [mu][img][i]: (sq, norm^(1/3) exp(-alpha sq))
  const float *rc2f;           // [M]
  const signed char *rowexp;   // [G]
  const uint32_t *J;           // [M][M] bf16 pairs (J0 low, J1 high) of row-scaled D
  const float *fscale;         // [M] 2^f_nu
  double *rho;                 // [G]
  const double *v;             // [G]
  float *Vacc;                 // [M][M] upper triangle
  double dV;
  int *flags;
};

struct TileShared {
  int mu[kNmax];
  float fs[kNmax];
  float2 stage[kNmax][16];  // per entry: 4 x-values, 4 y-values, 8 z-values
  float part[kTP];
  uint64_t mbar;
  uint32_t tbase;
  int n, npad, inside[kTP];
};

// stage the per-axis (sq, c exp(-alpha sq)) values of the tile for every entry
__device__ void stage_tile(const TcArgs &A, TileShared &S, int t, int kb, int n) {
  const GridGeom &g = A.g;
  int bz = t % g.nbz, by = (t / g.nbz) % g.nby, bx = t / (g.nbz * g.nby);
  int i0 = bx * 4, j0 = by * 4, k0 = bz * 8;
  for (int q = threadIdx.x; q < n * 16; q += blockDim.x) {
    int e = q >> 4, s = q & 15;
    int key = A.keys[kb + e];
    int mu = key >> 9;
    int ix = ((key >> 6) & 7) - 4 + kImgMax, iy = ((key >> 3) & 7) - 4 + kImgMax,
        iz = (key & 7) - 4 + kImgMax;
    float2 val;
    if (s < 4) {
      int i = i0 + s;
      val = i < g.nx ? A.tab[0][((long)mu * kImgN + ix) * g.nx + i] : make_float2(INFINITY, 0.f);
    } else if (s < 8) {
      int j = j0 + s - 4;
      val = j < g.ny ? A.tab[1][((long)mu * kImgN + iy) * g.ny + j] : make_float2(INFINITY, 0.f);
    } else {
      int k = k0 + s - 8;
      val = k < g.nz ? A.tab[2][((long)mu * kImgN + iz) * g.nz + k] : make_float2(INFINITY, 0.f);
    }
    S.stage[e][s] = val;
    if (s == 0) {
      S.mu[e] = mu;
      S.fs[e] = A.fscale ? A.fscale[mu] : 0.f;
    }
  }
  for (int p = threadIdx.x; p < kTP; p += blockDim.x) {
    int li = p >> 5, lj = (p >> 3) & 3, lk = p & 7;
    S.inside[p] = (i0 + li < g.nx && j0 + lj < g.ny && k0 + lk < g.nz)
                      ? ((i0 + li) * g.ny + (j0 + lj)) * g.nz + (k0 + lk)
                      : -1;
  }
}

__device__ __forceinline__ float basis_val(const TileShared &S, const float *rc2f, int e, int p) {
  int li = p >> 5, lj = (p >> 3) & 3, lk = p & 7;
  float2 x = S.stage[e][li], y = S.stage[e][4 + lj], z = S.stage[e][8 + lk];
  float r2 = (x.x + y.x) + z.x;
  return r2 < rc2f[S.mu[e]] ? x.y * y.y * z.y : 0.f;
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
__global__ void __launch_bounds__(kTcThreads, 1) rho_tc_kernel(TcArgs A) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  uint8_t *sA = dsm;                     // 3 slices I0, I1, I2
  uint8_t *sB = dsm + 3 * kSliceBytes;   // 2 slices J0, J1
  __shared__ TileShared S;
  tmem_alloc(S);
  const uint32_t tmem = S.tbase;
  uint32_t phase = 0;
  bool ok = true;
  for (int t = blockIdx.x; t < A.n_tiles && ok; t += gridDim.x) {
    const int kb = A.tile_ptr[t], n = A.tile_ptr[t + 1] - kb;
    const int npad = n <= 32 ? 32 : ((n + 31) / 32) * 32;
    if (n > kNmax) {  // rejected at set-up; never reached
      if (threadIdx.x == 0) atomicExch(A.flags + FLAG_ERR, ETDM_ERR_NUMERIC);
      continue;
    }
    stage_tile(A, S, t, kb, n);
    __syncthreads();
    // A slices: items (p, 8 consecutive entries)
    for (int q = threadIdx.x; q < kTP * (npad / 8); q += blockDim.x) {
      const int p = q % kTP, a0 = (q / kTP) * 8;
      const int gp = S.inside[p];
      const int ep = gp >= 0 ? (int)A.rowexp[gp] : 0;
      uint16_t s0[8], s1[8], s2[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        int a = a0 + u;
        float x = (a < n && gp >= 0) ? basis_val(S, A.rc2f, a, p) : 0.f;
        float t0 = ldexpf(x, 8 - ep);
        float r0 = rintf(t0);
        float t1 = (t0 - r0) * 256.f;
        float r1 = rintf(t1);
        float t2 = (t1 - r1) * 256.f;
        float r2 = rintf(t2);
        s0[u] = bf16_bits(r0); s1[u] = bf16_bits(r1); s2[u] = bf16_bits(r2);
      }
      const int off = kmaj_off(p, a0);
      uint4 v0, v1, v2;
      v0.x = s0[0] | (s0[1] << 16); v0.y = s0[2] | (s0[3] << 16);
      v0.z = s0[4] | (s0[5] << 16); v0.w = s0[6] | (s0[7] << 16);
      v1.x = s1[0] | (s1[1] << 16); v1.y = s1[2] | (s1[3] << 16);
      v1.z = s1[4] | (s1[5] << 16); v1.w = s1[6] | (s1[7] << 16);
      v2.x = s2[0] | (s2[1] << 16); v2.y = s2[2] | (s2[3] << 16);
      v2.z = s2[4] | (s2[5] << 16); v2.w = s2[6] | (s2[7] << 16);
      *(uint4 *)(sA + off) = v0;
      *(uint4 *)(sA + kSliceBytes + off) = v1;
      *(uint4 *)(sA + 2 * kSliceBytes + off) = v2;
    }
    // B slices: B[b][a] = J[mu_b][mu_a]
    for (int q = threadIdx.x; q < npad * (npad / 8); q += blockDim.x) {
      const int b = q % npad, a0 = (q / npad) * 8;
      uint32_t w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        int a = a0 + u;
        w[u] = (a < n && b < n) ? A.J[(long)S.mu[b] * A.g.M + S.mu[a]] : 0u;
      }
      const int off = kmaj_off(b, a0);
      uint4 v0, v1;
      v0.x = (w[0] & 0xFFFF) | (w[1] << 16); v0.y = (w[2] & 0xFFFF) | (w[3] << 16);
      v0.z = (w[4] & 0xFFFF) | (w[5] << 16); v0.w = (w[6] & 0xFFFF) | (w[7] << 16);
      v1.x = (w[0] >> 16) | (w[1] & 0xFFFF0000u); v1.y = (w[2] >> 16) | (w[3] & 0xFFFF0000u);
      v1.z = (w[4] >> 16) | (w[5] & 0xFFFF0000u); v1.w = (w[6] >> 16) | (w[7] & 0xFFFF0000u);
      *(uint4 *)(sB + off) = v0;
      *(uint4 *)(sB + kSliceBytes + off) = v1;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = idesc_bf16(npad);
      const uint32_t a0 = su32(sA), b0 = su32(sB);
      for (int kk = 0; kk < npad / 16; ++kk) {
        const uint32_t off = kk * 256;
        const uint64_t I0 = smem_desc(a0 + off), I1 = smem_desc(a0 + kSliceBytes + off),
                       I2 = smem_desc(a0 + 2 * kSliceBytes + off);
        const uint64_t J0 = smem_desc(b0 + off), J1 = smem_desc(b0 + kSliceBytes + off);
        const uint32_t acc = kk > 0;
        mma_bf16(tmem, I0, J0, idesc, acc);
        mma_bf16(tmem + kNmax, I0, J1, idesc, acc);
        mma_bf16(tmem + kNmax, I1, J0, idesc, 1u);
        mma_bf16(tmem + 2 * kNmax, I1, J1, idesc, acc);
        mma_bf16(tmem + 2 * kNmax, I2, J0, idesc, 1u);
      }
      mma_commit(&S.mbar);
    }
    ok = __syncthreads_and(mbar_wait(&S.mbar, phase)) != 0;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(A.flags + FLAG_ERR, ETDM_ERR_TIMEOUT);
      break;
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) ..; warps 0-3 and 4-7 split columns
    {
      const int w = threadIdx.x >> 5, quad = w & 3, half = w >> 2;
      const int p = quad * 32 + (threadIdx.x & 31);
      const uint32_t lane = (uint32_t)(quad * 32) << 16;
      const int cw = npad / 2;
      float sum = 0.f;
      for (int c0 = half * cw; c0 < half * cw + cw; c0 += 16) {
        float y0[16], y1[16], y2[16];
        tmem_ld16(tmem + lane + c0, y0);
        tmem_ld16(tmem + lane + kNmax + c0, y1);
        tmem_ld16(tmem + lane + 2 * kNmax + c0, y2);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int b = c0 + j;
          const int off = kmaj_off(p, b);
          float x = bf16_val(*(const uint16_t *)(sA + off)) +
                    bf16_val(*(const uint16_t *)(sA + kSliceBytes + off)) * (1.f / 256.f) +
                    bf16_val(*(const uint16_t *)(sA + 2 * kSliceBytes + off)) * (1.f / 65536.f);
          float y = y0[j] + (y1[j] + y2[j] * (1.f / 256.f)) * (1.f / 256.f);
          float fsb = b < n ? S.fs[b] : 0.f;
          sum = fmaf(x * y, fsb, sum);
        }
      }
      if (half == 1) S.part[p] = sum;
      __syncthreads();
      if (half == 0) {
        const int gp = S.inside[p];
        if (gp >= 0) {
          const int ep = (int)A.rowexp[gp];
          double r = (double)sum + (double)S.part[p];
          A.rho[gp] = ldexp(r, 2 * ep - 24);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  tmem_free(S);
}

// ---- potential matrix ---------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1) vmat_tc_kernel(TcArgs A) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  uint8_t *sA = dsm;                     // X^T hi, lo  (rows a, K = points)
  uint8_t *sB = dsm + 2 * kSliceBytes;   // (v X)^T hi, lo
  __shared__ TileShared S;
  __shared__ float vp[kTP];
  tmem_alloc(S);
  const uint32_t tmem = S.tbase;
  uint32_t phase = 0;
  bool ok = true;
  const int M = A.g.M;
  for (int t = blockIdx.x; t < A.n_tiles && ok; t += gridDim.x) {
    const int kb = A.tile_ptr[t], n = A.tile_ptr[t + 1] - kb;
    const int npad = n <= 32 ? 32 : ((n + 31) / 32) * 32;
    if (n > kNmax) {
      if (threadIdx.x == 0) atomicExch(A.flags + FLAG_ERR, ETDM_ERR_NUMERIC);
      continue;
    }
    stage_tile(A, S, t, kb, n);
    __syncthreads();
    for (int p = threadIdx.x; p < kTP; p += blockDim.x) {
      const int gp = S.inside[p];
      vp[p] = gp >= 0 ? (float)(A.v[gp] * A.dV) : 0.f;
    }
    __syncthreads();
    // items (entry a, 8 consecutive points)
    for (int q = threadIdx.x; q < npad * (kTP / 8); q += blockDim.x) {
      const int a = q % npad, p0 = (q / npad) * 8;
      uint16_t xh[8], xl[8], wh[8], wl[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int p = p0 + u;
        float x = (a < n && S.inside[p] >= 0) ? basis_val(S, A.rc2f, a, p) : 0.f;
        float w = x * vp[p];
        xh[u] = bf16_bits(x);
        xl[u] = bf16_bits(x - bf16_val(xh[u]));
        wh[u] = bf16_bits(w);
        wl[u] = bf16_bits(w - bf16_val(wh[u]));
      }
      const int off = kmaj_off(a, p0);
      uint4 v;
      v.x = xh[0] | (xh[1] << 16); v.y = xh[2] | (xh[3] << 16);
      v.z = xh[4] | (xh[5] << 16); v.w = xh[6] | (xh[7] << 16);
      *(uint4 *)(sA + off) = v;
      v.x = xl[0] | (xl[1] << 16); v.y = xl[2] | (xl[3] << 16);
      v.z = xl[4] | (xl[5] << 16); v.w = xl[6] | (xl[7] << 16);
      *(uint4 *)(sA + kSliceBytes + off) = v;
      v.x = wh[0] | (wh[1] << 16); v.y = wh[2] | (wh[3] << 16);
      v.z = wh[4] | (wh[5] << 16); v.w = wh[6] | (wh[7] << 16);
      *(uint4 *)(sB + off) = v;
      v.x = wl[0] | (wl[1] << 16); v.y = wl[2] | (wl[3] << 16);
      v.z = wl[4] | (wl[5] << 16); v.w = wl[6] | (wl[7] << 16);
      *(uint4 *)(sB + kSliceBytes + off) = v;
    }
    // rows a >= npad of the M = 128 operand stay as set below
    for (int q = threadIdx.x; q < (kNmax - npad) * (kTP / 8); q += blockDim.x) {
      const int a = npad + q % (kNmax - npad), p0 = (q / (kNmax - npad)) * 8;
      const int off = kmaj_off(a, p0);
      *(uint4 *)(sA + off) = make_uint4(0, 0, 0, 0);
      *(uint4 *)(sA + kSliceBytes + off) = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = idesc_bf16(npad);
      const uint32_t a0 = su32(sA), b0 = su32(sB);
      for (int kk = 0; kk < kTP / 16; ++kk) {
        const uint32_t off = kk * 256;
        const uint64_t Xh = smem_desc(a0 + off), Xl = smem_desc(a0 + kSliceBytes + off);
        const uint64_t Wh = smem_desc(b0 + off), Wl = smem_desc(b0 + kSliceBytes + off);
        mma_bf16(tmem, Xh, Wh, idesc, kk > 0);
        mma_bf16(tmem, Xh, Wl, idesc, 1u);
        mma_bf16(tmem, Xl, Wh, idesc, 1u);
      }
      mma_commit(&S.mbar);
    }
    ok = __syncthreads_and(mbar_wait(&S.mbar, phase)) != 0;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(A.flags + FLAG_ERR, ETDM_ERR_TIMEOUT);
      break;
    }
    {
      const int w = threadIdx.x >> 5, quad = w & 3, half = w >> 2;
      const int a = quad * 32 + (threadIdx.x & 31);
      const uint32_t lane = (uint32_t)(quad * 32) << 16;
      const int cw = npad / 2;
      const int ma = a < n ? S.mu[a] : 0;
      for (int c0 = half * cw; c0 < half * cw + cw; c0 += 16) {
        float val[16];
        tmem_ld16(tmem + lane + c0, val);  // whole warp, converged (.sync.aligned)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int b = c0 + j;
          if (a < n && b >= a && b < n) {
            const int mb = S.mu[b];
            float s = val[j];
            if (ma == mb && a != b) s *= 2.f;
            if (s != 0.f) atomicAdd(A.Vacc + (long)ma * M + mb, s);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  tmem_free(S);
}

// ---- set-up and per-evaluation helpers ------------------------------------------

// FP32 copies of the basis tables with norm^(1/3) folded into each factor
__global__ void tables_f32_kernel(const double *sq, const double *ex, const double *norm,
                                  int M, int n_ax, float2 *out) {
  long total = (long)M * kImgN * n_ax;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int mu = (int)(e / ((long)n_ax * kImgN));
    out[e] = make_float2((float)sq[e], (float)(cbrt(norm[mu]) * ex[e]));
  }
}

// per grid point: exponent e_p with max_a |X_pa| < 2^(e_p - 1) (same FP32 values
// as the density kernel computes)
__global__ void __launch_bounds__(kTcThreads) rowexp_kernel(TcArgs A, signed char *rowexp) {
  __shared__ TileShared S;
  for (int t = blockIdx.x; t < A.n_tiles; t += gridDim.x) {
    const int kb = A.tile_ptr[t], n = A.tile_ptr[t + 1] - kb;
    stage_tile(A, S, t, kb, min(n, kNmax));
    __syncthreads();
    for (int p = threadIdx.x; p < kTP; p += blockDim.x) {
      const int gp = S.inside[p];
      if (gp < 0) continue;
      float mx = 0.f;
      for (int a = 0; a < min(n, kNmax); ++a) mx = fmaxf(mx, fabsf(basis_val(S, A.rc2f, a, p)));
      rowexp[gp] = (signed char)(mx > 0.f ? ilogbf(mx) + 2 : 0);
    }
    __syncthreads();
  }
}

// Row slices of D: f_nu = ilogb(max |D_nu,:|) + 2, J0 + J1/256 = D 2^(8 - f) to
// 16 bits; dD = D - Dq (FP64) for the first-order energy correction.
__global__ void __launch_bounds__(256) dslice_kernel(const double *D, int M, uint32_t *J,
                                                     float *fscale, double *dD) {
  const int nu = blockIdx.x;
  double mx = 0.0;
  for (int c = threadIdx.x; c < M; c += blockDim.x) mx = fmax(mx, fabs(D[(long)nu * M + c]));
  __shared__ double red[256];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  mx = red[0];
  const int f = mx > 0.0 ? ilogb(mx) + 2 : 0;
  if (threadIdx.x == 0) fscale[nu] = ldexpf(1.f, f);
  for (int c = threadIdx.x; c < M; c += blockDim.x) {
    const double d = D[(long)nu * M + c];
    const double t0 = ldexp(d, 8 - f);
    const double r0 = rint(t0);
    const double t1 = (t0 - r0) * 256.0;
    const double r1 = rint(t1);
    const double q = ldexp(r0 + r1 * (1.0 / 256.0), f - 8);
    dD[(long)nu * M + c] = d - q;
    J[(long)nu * M + c] = (uint32_t)bf16_bits((float)r0) | ((uint32_t)bf16_bits((float)r1) << 16);
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
  a.J = h->d_J;
  a.fscale = h->d_fscale;
  a.rho = h->d_rho;
  a.v = h->d_vtot;
  a.Vacc = h->d_Vacc;
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
  rowexp_kernel<<<std::min(h->n_tiles_tc, 8 * h->num_sms), kTcThreads, 0, s>>>(a, h->d_rowexp);
  return cudaGetLastError();
}

cudaError_t launch_dslice(etdm_handle *h, cudaStream_t s) {
  dslice_kernel<<<h->M, 256, 0, s>>>(h->d_D, h->M, h->d_J, h->d_fscale, h->d_dD);
  return cudaGetLastError();
}

cudaError_t launch_rho_tc(etdm_handle *h, cudaStream_t s) {
  const size_t sm = 5 * (size_t)kSliceBytes;
  cudaError_t e = cudaFuncSetAttribute(rho_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  rho_tc_kernel<<<std::min(h->n_tiles_tc, h->num_sms), kTcThreads, sm, s>>>(tc_args(h));
  return cudaGetLastError();
}

cudaError_t launch_vmat_tc(etdm_handle *h, cudaStream_t s) {
  const size_t sm = 4 * (size_t)kSliceBytes;
  cudaError_t e = cudaFuncSetAttribute(vmat_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(h->d_Vacc, 0, (size_t)h->M * h->M * sizeof(float), s);
  if (e != cudaSuccess) return e;
  vmat_tc_kernel<<<std::min(h->n_tiles_tc, h->num_sms), kTcThreads, sm, s>>>(tc_args(h));
  return cudaGetLastError();
}

int tc_max_list() { return kNmax; }

}  // namespace etdm
