// Device helpers shared by the kernels of libetdm.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace etdm {

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned *p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for kernels launched cooperatively (all blocks resident).
// bar[0] counts arrivals, bar[1] is the generation.  The block's writes are
// published by thread 0's release-ordered arrival (after the block barrier) and
// seen by the other blocks through their acquire loads of the generation.  The
// wait is bounded: after kSpinLimit polls the block records ETDM_ERR_TIMEOUT in
// flags[FLAG_ERR] and the barrier returns false; callers then return.  A grid of
// one block needs only the block barrier.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *flags) {
  __syncthreads();
  if (gridDim.x * gridDim.y * gridDim.z == 1) return true;  // one block: the block barrier is all
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = ld_acquire_gpu(bar + 1);
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned arrived = atom_add_acq_rel_gpu(bar, 1u);
    if (arrived == nb - 1) {
      st_relaxed_gpu(bar, 0u);          // reset for the next use, ordered before
      st_release_gpu(bar + 1, g + 1);   // the release of the new generation
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

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0) {
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) red[0] = t;
  }
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// Sum of red[0, n) by the whole block; every thread gets the total.
__device__ __forceinline__ double block_sum_of(const double *red, int n) {
  double t = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) t += red[b];
  return block_sum(t);
}

}  // namespace etdm
