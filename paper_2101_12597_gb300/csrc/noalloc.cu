// Allocation-free L-BFGS two-loop direction (etdm_lbfgs_direction_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// search direction: code running inside a stream capture whose memory pool is
// frozen, host frameworks that hand out only pre-registered buffers, and
// embedded drivers that forbid cudaMalloc after start-up.  This entry point
// computes the same direction as the handle's etdm_lbfgs_step, from a pair
// history the caller keeps, with its reduction scratch in a fixed file-scope
// device array instead of handle-owned memory.  It calls no cudaMalloc,
// cudaFree or allocating library routine.
//
// The scratch array lives in every GPU that loads the library until the
// process exits.  All calls share it and it keeps the last call's contents:
// the barrier words and the status word are cleared at the start of each
// call, and calls that overlap on the GPU (two streams, or two host threads)
// race on it.  The status word records a device-side failure of the last call
// (a grid barrier that gave up, or a pair without positive curvature);
// etdm_lbfgs_direction_noalloc_status reads it without allocating.
#include <cooperative_groups.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "device.cuh"
#include "internal.h"

namespace etdm {

constexpr int kNaMaxPairs = 16;      // maximum number of (s, y) pairs
constexpr int kNaMaxBlocks = 256;    // partial sums held per reduction
constexpr int kNaThreads = 256;
constexpr int kNaDevices = 64;
// layout: [0, 256) bytes: barrier count, generation, error flag; then
// kNaMaxBlocks doubles of block partials
constexpr size_t kNaScratchBytes = 256 + kNaMaxBlocks * sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

struct NaArgs {
  const double *g, *s, *y, *h0;
  double *p;
  long n;
  int m;
  unsigned *bar;
  int *flags;
  double *red;
};

__device__ double na_dot(const NaArgs &a, double part, bool *ok) {
  part = block_sum(part);
  if (threadIdx.x == 0) a.red[blockIdx.x] = part;
  if (!grid_barrier(a.bar, a.flags)) { *ok = false; return 0.0; }
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += a.red[b];
    tot = t;
  }
  __syncthreads();
  double r = tot;
  if (!grid_barrier(a.bar, a.flags)) { *ok = false; return 0.0; }
  return r;
}

// p = -H g by the two-loop recursion over pairs oldest (0) .. newest (m-1),
// with the diagonal initial inverse Hessian h0; p doubles as the work vector.
// A pair whose curvature y.s is not positive and finite makes the direction
// meaningless: the kernel records ETDM_ERR_NUMERIC in the status word and
// returns (every block sees the same sum, so all of them stop together).
__global__ void __launch_bounds__(kNaThreads) lbfgs_noalloc_kernel(NaArgs a) {
  const long n = a.n;
  const long gtid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long gstride = (long)gridDim.x * blockDim.x;
  bool ok = true;
  double rho[kNaMaxPairs], alph[kNaMaxPairs];
  for (int i = 0; i < a.m; ++i) {
    const double *si = a.s + (long)i * n, *yi = a.y + (long)i * n;
    double part = 0.0;
    for (long e = gtid; e < n; e += gstride) part += yi[e] * si[e];
    double ys = na_dot(a, part, &ok);
    if (!ok) return;
    if (!(ys > 0.0) || isinf(ys)) {
      if (gtid == 0) atomicExch(a.flags + FLAG_ERR, ETDM_ERR_NUMERIC);
      return;
    }
    rho[i] = 1.0 / ys;
  }
  for (long e = gtid; e < n; e += gstride) a.p[e] = a.g[e];
  for (int i = a.m - 1; i >= 0; --i) {
    const double *si = a.s + (long)i * n, *yi = a.y + (long)i * n;
    double part = 0.0;
    for (long e = gtid; e < n; e += gstride) part += si[e] * a.p[e];
    double sq = na_dot(a, part, &ok);
    if (!ok) return;
    alph[i] = rho[i] * sq;
    for (long e = gtid; e < n; e += gstride) a.p[e] -= alph[i] * yi[e];
  }
  for (long e = gtid; e < n; e += gstride) a.p[e] *= a.h0[e];
  for (int i = 0; i < a.m; ++i) {
    const double *si = a.s + (long)i * n, *yi = a.y + (long)i * n;
    double part = 0.0;
    for (long e = gtid; e < n; e += gstride) part += yi[e] * a.p[e];
    double yr = na_dot(a, part, &ok);
    if (!ok) return;
    const double coef = alph[i] - rho[i] * yr;
    for (long e = gtid; e < n; e += gstride) a.p[e] += coef * si[e];
  }
  for (long e = gtid; e < n; e += gstride) a.p[e] = -a.p[e];
}

namespace {

struct NaDevice {
  bool ready = false;
  unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
  int blocks_max = 0;
};

std::mutex g_na_mutex;
NaDevice g_na[kNaDevices];

int na_fail(int code, const std::string &msg) {
  set_unbound_error(msg);
  return code;
}

}  // namespace

}  // namespace etdm

using namespace etdm;

namespace etdm {
namespace {

// The device's scratch address and launch size, looked up once per device with
// that device current (the array's host-side name is not a device address).
int na_device(NaDevice **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaDevices)
    return na_fail(ETDM_ERR_CUDA, "no current CUDA device");
  NaDevice *d = &g_na[dev];
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!d->ready) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess)
      return na_fail(ETDM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    int sms = 0, bps = 0, coop = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, lbfgs_noalloc_kernel, kNaThreads,
                                                      0) != cudaSuccess ||
        !coop || bps < 1)
      return na_fail(ETDM_ERR_CUDA, "cannot size the cooperative two-loop kernel");
    d->scratch = (unsigned char *)ptr;
    d->blocks_max = std::min(kNaMaxBlocks, sms * bps);
    d->ready = true;
  }
  *out = d;
  return ETDM_OK;
}

}  // namespace
}  // namespace etdm

extern "C" int etdm_lbfgs_direction_noalloc(const double *g_dev, const double *s_dev,
                                            const double *y_dev, int32_t m, int64_t n,
                                            const double *h0_dev, double *p_dev,
                                            void *stream) {
  if (m < 0 || m > kNaMaxPairs)
    return na_fail(ETDM_ERR_INVALID_ARG,
                   "m must be in [0, " + std::to_string(kNaMaxPairs) + "] (scratch limit)");
  if (n < 0 || n > (int64_t)1 << 40) return na_fail(ETDM_ERR_INVALID_ARG, "n out of range");
  if (n == 0) return ETDM_OK;
  if (!g_dev || !h0_dev || !p_dev || (m > 0 && (!s_dev || !y_dev)))
    return na_fail(ETDM_ERR_INVALID_ARG, "g, h0, p (and s, y when m > 0) are required");
  NaDevice *d = nullptr;
  int rc = na_device(&d);
  if (rc != ETDM_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // barrier words and the status word must start at zero
  cudaError_t e = cudaMemsetAsync(d->scratch, 0, 256, s);
  if (e != cudaSuccess)
    return na_fail(ETDM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  NaArgs a;
  a.g = g_dev; a.s = s_dev; a.y = y_dev; a.h0 = h0_dev; a.p = p_dev;
  a.n = (long)n; a.m = m;
  a.bar = (unsigned *)d->scratch;
  a.flags = (int *)(d->scratch + 64);
  a.red = (double *)(d->scratch + 256);
  const long want = (n + 4L * kNaThreads - 1) / (4L * kNaThreads);
  const int blocks = (int)std::max(1L, std::min((long)d->blocks_max, want));
  void *args[] = {&a};
  e = cudaLaunchCooperativeKernel((void *)lbfgs_noalloc_kernel, dim3(blocks), dim3(kNaThreads),
                                  args, 0, s);
  if (e != cudaSuccess)
    return na_fail(ETDM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return ETDM_OK;
}

extern "C" int etdm_lbfgs_direction_noalloc_status(void *stream) {
  NaDevice *d = nullptr;
  int rc = na_device(&d);
  if (rc != ETDM_OK) return rc;
  // wait for the calls queued on `stream`, then copy the status word into a
  // local (a pageable copy: no pinned staging buffer, nothing allocated)
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  int word = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&word, d->scratch + 64, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess)
    return na_fail(ETDM_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
  if (word == ETDM_ERR_TIMEOUT)
    return na_fail(ETDM_ERR_TIMEOUT,
                   "the last allocation-free direction gave up at a grid barrier "
                   "(blocks not co-resident?); its output is incomplete");
  if (word == ETDM_ERR_NUMERIC)
    return na_fail(ETDM_ERR_NUMERIC,
                   "the last allocation-free direction met a pair with y.s <= 0 (or not "
                   "finite); its output is incomplete");
  if (word != 0) return na_fail(word, "the last allocation-free direction failed on the device");
  return ETDM_OK;
}
