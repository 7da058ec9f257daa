// Tensor-core products of the mixed path's dense chains (Eq. 7 O = C0 U, the
// exp(A) series, T O, V O, C0^T Gbar and the reverse pass), run inside the
// cooperative dense kernels on float-pair matrices.
//
// A product out = alpha op(A) op(B) (+ epilogue terms) of float pairs (about
// 47 bits) is evaluated in BF16 slices:
//   row i of op(A) and column j of op(B) are scaled by powers of two
//   2^(8-e_i), 2^(8-f_j) (|scaled| < 128) and cut into five slices each, r_t
//   a multiple of 2^-8t with an integer numerator of at most 129 (exact in
//   BF16, slice5);
//   the 15 slice products of orders t + u <= 4 go into four FP32 sums in
//   tensor memory: one each for the orders 0, 1 and 2, and one for the orders
//   3 and 4 together;
//   the B slices of a K step lie one after another in shared memory, so
//   A_q times [B_0 .. B_(3-q)] (one MMA of N = 64 (4 - q)) puts the orders
//   q .. 3 at columns 64 q .. 192 at once; the five order-4 products A_q
//   B_(4-q) add into the order-3 sum: 9 MMAs per K step of 16;
//   every product of slices is an integer of at most 129^2 in units of its
//   order, so the sums of orders 0 .. 2 (at most three products per K
//   element) are exact over 21 K steps (336 elements: 3 x 336 x 129^2 <
//   2^24) whatever rounding the accumulator applies; the epilogue reads the
//   four sums every 21 K steps and adds them into float-pair sums; the FP32
//   rounding of the order 3-4 sum is about 2^-48 of |A||B| per element;
//   the dropped orders >= 5 are about 2^-40 of |A||B| per term.
// Tensor memory holds two buffers of the four sums (256 columns each): the
// MMAs of one chunk run while the epilogue reads the previous one.
// Roles (warps of the 512-thread block): warp 0 streams the slices of a K
// step (one 20 KB and one 10 KB bulk copy) into a five-stage ring, warp 1
// issues the MMAs, warps 8-15 read the sums (lane quarter w % 4, 32-column
// half (w - 8) / 4) and write the outputs with the phase's epilogue terms.
// Every wait is bounded.
#pragma once

#include "pair.cuh"
#include "tc.cuh"

namespace etdm {

constexpr int kGS = 5;                   // BF16 slices per operand
constexpr int kGN = 64;                  // output tile columns (MMA N); rows: 128
constexpr int kGA = kGS * 4096;          // A slices of one K step (128 rows x 16): 20 KB
constexpr int kGB = kGS * 2048;          // B slices of one K step (64 rows x 16): 10 KB
constexpr int kGStage = kGA + kGB;
constexpr int kGStages = 5;
constexpr int kGChunk = 21;              // K steps per chunk (exact order 0-2 sums)
constexpr int kGSet = 256;               // tensor-memory columns of one buffer of the four sums
constexpr int kGDyn = kGStages * kGStage;  // dynamic shared memory, 150 KB
constexpr int kGEpiW0 = 8;               // first read-out warp

__host__ __device__ __forceinline__ long gpad(long x, long q) { return (x + q - 1) / q * q; }

// Workspace of the tensor-core products (device memory, one product at a time)
struct GemmWs {
  uint8_t *asl;  // A slices: [row block][K step][slice][4 KB], canonical K-major layout
  uint8_t *bsl;  // B slices: [column block][K step][slice][2 KB]
  int *rexp;     // per row of op(A): bits of max |value| (then the slice exponent)
  int *cexp;     // per column of op(B)
};

// mbarriers of the tensor-core products, initialized once per kernel, and the
// roles' running counts (stage fills, exact chunks, final waits), carried
// from one product to the next so that every wait names its phase exactly
struct GemmSmem {
  uint64_t full[kGStages], empty[kGStages];
  uint64_t acc_full[2], acc_empty[2], fin;  // per tensor-memory buffer
  int stop;
  int fill_copy, fill_mma, chunk_mma, chunk_epi, fins;
};

// tensor-core context of one block of a cooperative dense kernel
struct TcCtx {
  GemmWs ws;
  uint8_t *dyn;     // dynamic shared memory (the stage ring)
  GemmSmem *S;
  uint32_t tmem;    // 512 columns, allocated for the kernel's lifetime
};

// row (column) maxima of |op(X)| as float bits, atomicMax per segment of K;
// `rowmajor` when the rows of op(X) are contiguous in memory.  Each thread has
// eight loads in flight.
template <class F>
__device__ void tc_maxima(F fetch, int rows, int K, bool rowmajor, int *out, long gtid,
                          long gstride) {
  if (rowmajor) {  // a warp per (row, 256 consecutive k)
    const long segs = (K + 255) / 256;
    const long items = (long)rows * segs * 32;
    for (long e = gtid; e < items; e += gstride) {
      const int lane = (int)(e & 31);
      const long w = e >> 5;
      const int i = (int)(w / segs), k0 = (int)(w % segs) * 256 + lane;
      float m = 0.f;
      if (k0 + 224 < K) {  // the eight loads unconditional, all issued before the first use
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = fetch(i, k0 + 32 * u).x;
#pragma unroll
        for (int u = 0; u < 8; ++u) m = fmaxf(m, fabsf(x[u]));
      } else {
        for (int k = k0; k < K; k += 32) m = fmaxf(m, fabsf(fetch(i, k).x));
      }
      m = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));
      if (lane == 0) atomicMax(out + i, __float_as_int(m));
    }
  } else {  // the lanes of a warp: 32 consecutive rows, 32 consecutive k each
    const long segs = (K + 31) / 32;
    const long items = (long)((rows + 31) / 32) * segs * 32;
    for (long e = gtid; e < items; e += gstride) {
      const long w = e >> 5;
      const int i = (int)(w / segs) * 32 + (int)(e & 31), k0 = (int)(w % segs) * 32;
      if (i >= rows) continue;
      float m = 0.f;
      if (k0 + 32 <= K) {
#pragma unroll
        for (int u0 = 0; u0 < 32; u0 += 8) {
          float x[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) x[u] = fetch(i, k0 + u0 + u).x;
#pragma unroll
          for (int u = 0; u < 8; ++u) m = fmaxf(m, fabsf(x[u]));
        }
      } else {
        for (int k = k0; k < K; ++k) m = fmaxf(m, fabsf(fetch(i, k).x));
      }
      atomicMax(out + i, __float_as_int(m));
    }
  }
}

// slices of op(X) (rows x K) into the canonical layout: blocks of `br` rows x
// 16 K, one block per slice, kGS blocks of br*32 bytes per (row block, K step);
// padding rows and K are zero.  A thread slices 8 consecutive K of one row
// (a K group); the warp's stores fill whole 128-byte core matrices: 8 rows x
// 4 K groups per warp when rows are contiguous in memory, else 32 consecutive
// rows at one K group.
template <class F>
__device__ void tc_slice(F fetch, int rows, int K, int br, bool rowmajor, const int *exps,
                         uint8_t *dst, long gtid, long gstride) {
  const int nrb = (rows + br - 1) / br, nks = (K + 15) / 16, ng = nks * 2;
  const long nrows = (long)nrb * br;  // a multiple of 8
  const int ngq = (ng + 3) / 4;
  const long items = rowmajor ? nrows / 8 * ngq * 32 : nrows * ng;
  const int bb = br * 32;  // bytes of one slice block
  for (long e = gtid; e < items; e += gstride) {
    int i, g;
    if (rowmajor) {
      const int lane = (int)(e & 31);
      const long w = e >> 5;
      i = (int)(w / ngq) * 8 + (lane & 7);
      g = (int)(w % ngq) * 4 + (lane >> 3);
      if (g >= ng) continue;
    } else {
      g = (int)(e / nrows);
      i = (int)(e % nrows);
    }
    const int k0 = g * 8;
    float sc = 0.f;
    if (i < rows) sc = pow2f(8 - slice_exp(__int_as_float(exps[i])));
    float2 x[8];
    if (i < rows && k0 + 8 <= K) {  // the eight loads issued before the first use
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = fetch(i, k0 + u);
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        x[u] = (i < rows && k0 + u < K) ? fetch(i, k0 + u) : make_float2(0.f, 0.f);
    }
    uint32_t wd[kGS][4];
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      float r[2][kGS];
      slice5(x[u], sc, r[0]);
      slice5(x[u + 1], sc, r[1]);
#pragma unroll
      for (int t = 0; t < kGS; ++t) wd[t][u >> 1] = pack_bf16(r[0][t], r[1][t]);
    }
    const int rb = i / br, rr = i % br, ks = g >> 1;
    uint8_t *blk = dst + ((long)rb * nks + ks) * kGS * bb;
    const int off = kstep_off(rr, (g & 1) * 8);
#pragma unroll
    for (int t = 0; t < kGS; ++t)
      *(uint4 *)(blk + t * bb + off) = make_uint4(wd[t][0], wd[t][1], wd[t][2], wd[t][3]);
  }
}

}  // namespace etdm
