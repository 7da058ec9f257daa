// Host-side helpers shared by the set-up code of libetdm: the error type
// that the C ABI turns into a status code, CUDA call checking and device
// allocations owned by a handle (freed by etdm_free).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace etdm {

struct Fail {
  int code;
  std::string msg;
};

#define CUDA_TRY(expr)                                                            \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess)                                                        \
      throw ::etdm::Fail{ETDM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)}; \
  } while (0)

// count elements of device memory owned by h, zero-filled
template <typename T>
T *dalloc(etdm_handle *h, size_t count) {
  void *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Fail{ETDM_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) +
                                 " bytes failed: " + cudaGetErrorString(e)};
  }
  h->allocs.push_back(p);
  CUDA_TRY(cudaMemset(p, 0, count * sizeof(T)));
  return (T *)p;
}

// release one allocation of h early (nullptr: nothing)
inline void dfree(etdm_handle *h, void *p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i] == p) {
      cudaFree(p);
      h->allocs.erase(h->allocs.begin() + i);
      return;
    }
}

// a device copy of n host elements, owned by h
template <typename T>
T *dupload(etdm_handle *h, const T *src, size_t n) {
  T *d = dalloc<T>(h, n);
  if (n) CUDA_TRY(cudaMemcpy(d, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return d;
}

// The device tables of the mixed path's grid stages over the systems `subs`
// (one system: the handle itself; a batch: its members), allocated in owner.
// batch = false keeps the single-system work order: density tiles dealt to the
// CTAs round-robin, V groups in equal contiguous runs; batch = true balances
// the CTAs by a cost model (longest jobs first for the density, contiguous
// cost-balanced runs for V).
// vfix (vfix_bytes) holds every system's fixed-point V sums: the systems'
// d_Vfix arrays must lie inside it.
void build_mixed_plan(etdm_handle *owner, const std::vector<etdm_handle *> &subs,
                      const int *d_active, int *d_flags, bool batch,
                      unsigned long long *vfix, size_t vfix_bytes, MixedPlan *P);

// Optional stage timing: events around a stage on the calling stream.
struct StageTimer {
  etdm_handle *h;
  cudaStream_t s;
  int stage;
  cudaEvent_t e0 = nullptr;
  StageTimer(etdm_handle *hh, cudaStream_t ss, int st) : h(hh), s(ss), stage(st) {
    if (h->profiling) {
      CUDA_TRY(cudaEventCreate(&e0));
      CUDA_TRY(cudaEventRecord(e0, s));
    }
  }
  void done() {
    if (!h->profiling) return;
    cudaEvent_t e1;
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaEventRecord(e1, s));
    h->prof_events.push_back({stage, {e0, e1}});
  }
};

// V groups of at most vg_max tiles, their tables and X^T slices (capi.cu)
void build_vgroups(etdm_handle *h, int vg_max, cudaStream_t s);

// L-BFGS memory, line-search buffers and reduction scratch for h->nvar
// variables (capi.cu).
void alloc_opt_buffers(etdm_handle *h);

// Single-system pieces of the C ABI (capi.cu) that the batch reuses.
void init_system(etdm_handle *h, const etdm_system *sys, const etdm_options *opt);
void eval_system(etdm_handle *h, const double *a, double *E, double *g, cudaStream_t s);
void release_handle(etdm_handle *h);

// Batches of systems (batch.cu).
void init_batch(etdm_handle *h, const etdm_system *sys, int n_sys, const etdm_options *opt);
void batch_energy_grad(etdm_handle *h, const double *a, double *E, double *g, cudaStream_t s);
void batch_energy_grad_host(etdm_handle *h, const double *a, double *E, double *g);
void batch_minimize(etdm_handle *h, double *a, int n_steps, double *E_hist, double *alpha_hist,
                    int32_t *trials_hist, cudaStream_t s);
void batch_check(etdm_handle *h, cudaStream_t s);
void batch_release(etdm_handle *h);

}  // namespace etdm
