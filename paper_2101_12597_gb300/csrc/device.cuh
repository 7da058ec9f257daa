// Device helpers shared by the kernels of libetdm.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace etdm {

// Grid-wide barrier for kernels launched cooperatively (all blocks resident).
// bar[0] counts arrivals, bar[1] is the generation.  The wait is bounded:
// after kSpinLimit polls the block records ETDM_ERR_TIMEOUT in flags[FLAG_ERR]
// and the barrier returns false; callers then return.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *flags) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned *gen = bar + 1;
    unsigned g = *gen;
    __threadfence();
    unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nb - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long it = 0;
      while (*gen == g) {
        if (++it > kSpinLimit) {
          atomicExch(flags + FLAG_ERR, ETDM_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int *)(flags + FLAG_ERR) == ETDM_ERR_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// Sum of v over the block (all threads get the result).  blockDim.x <= 1024.
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

}  // namespace etdm
