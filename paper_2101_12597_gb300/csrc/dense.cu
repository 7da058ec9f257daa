// Dense algebra of one ETDM evaluation: exp(A) for the occupied-virtual
// parametrization (Eq. 36-37), O = C0 U, D = O F O^T (Eq. 12), and the
// analytic gradient dE/dA_ov (Eq. 14) by reverse-mode differentiation of the
// same steps; plus the L-BFGS two-loop update (Sec. 3.1) and the diagonal
// preconditioner (Eq. 33-34).
//
// cos sqrt(P) and sin sqrt(P)/sqrt(P) (P = A_ov A_ov^T) are entire functions
// of P.  They are evaluated without an eigendecomposition: Taylor series of
// Q = P / 4^j with spectral radius rho(Q) <= 1, then j doubling steps
//   cos 2x = 1 + 4k + 2k^2 (k = cos x - 1),  sin 2x / 2x = (sin x / x) cos x,
// which keep the small quantity k = cos x - 1 without cancellation.  P is
// symmetric, so the truncation error of a series in Q (and of its derivative)
// is bounded through rho(Q), and rho(P) <= |P^m|_F^(1/m) for every m: j is
// taken from the smallest of |P|_F, |P^2|_F^(1/2) and |P^4|_F^(1/4), the powers
// the series needs anyway (for a P with many comparable eigenvalues the
// Frobenius norm alone overstates rho by up to sqrt(N)).  The two
// degree-10 series are evaluated by Paterson-Stockmeyer blocking: Q^2, Q^3,
// Q^4, blocks B_i = sum_r c_{4i+r} Q^r (r < 4), and Horner in Q^4,
//   p(Q) = B_0 + Q^4 (B_1 + Q^4 B_2),
// four dependent product steps instead of nine; the reverse pass follows the
// same graph backwards.
//
// Each chain of small dependent products runs as ONE cooperative launch over
// all SMs with a bounded grid barrier between products.  The chains are
// written once over an element type R: double for the FP64 path, and float
// pairs (pair.cuh) for the mixed path, whose products then run on the FP32
// pipes (FP64 is the scarce resource on this GPU: about 1.7 FMA per clock per
// SM).  Both element types are 8 bytes, so the workspaces are shared; in the
// float-pair instantiation the matrices of the chain hold (hi, lo) pairs and
// only A (in), g (out), dO and the energy terms stay FP64.
#include <algorithm>
#include <cooperative_groups.h>
#include <math.h>

#include "device.cuh"
#include "internal.h"
#include "pair.cuh"
#include "tcgemm.cuh"

namespace etdm {

constexpr int BM = 8, BN = 16, BK = 16, NT = 512;
constexpr int NG = 128;       // threads of one K group (one output each)
constexpr int KG = NT / NG;   // K groups: a tile's K chunks go round-robin to the groups
static_assert(kTaylor >= 8 && kTaylor <= 11, "Paterson-Stockmeyer blocks assume degree 8..11");
// The blocks that run one chain together: either a cooperative grid (one
// system per launch, a bounded grid barrier between dependent products) or a
// single block of a batched launch (one system per block, where the block
// barrier is all the chain needs).
struct Coop {
  int rank, size;
  unsigned *bar;
  int *flags;
  const struct TcRun *tc = nullptr;  // tensor-core products of large phases (mixed path)
  __device__ __forceinline__ bool sync() const {
    if (size == 1) {
      __syncthreads();
      return true;
    }
    return grid_barrier(bar, flags);
  }
};
__device__ __forceinline__ Coop grid_coop(unsigned *bar, int *flags) {
  return Coop{(int)blockIdx.x, (int)gridDim.x, bar, flags, nullptr};
}
__device__ __forceinline__ Coop block_coop() { return Coop{0, 1, nullptr, nullptr, nullptr}; }

// the tensor-core context and the size from which a phase's products use it
struct TcRun {
  TcCtx ctx;
  long long min_work;  // m n k of the largest product of a call
};

// slots of the forward series workspace Qk
enum { kQ1 = 0, kQ2, kQ3, kQ4, kBc2, kBs2, kTc, kTs, kQslots };
// slots of the reverse workspace Wr
enum { kQ4b = 0, kTcb, kTsb, kBc2b, kBs2b, kQ1bB, kQ2bB, kQ3b, kQ2b, kQ1bt, kQ1b, kWslots };

// ---- the two element types --------------------------------------------------
// ld/st: an element of a matrix held in R; ld_f64: an element of an FP64 matrix
// converted to R; dbl: the value as FP64; fma(s, x, y) = s x + y with an FP64
// scalar s; scale2: multiplication by a power of two.
template <class R> struct Num;
template <> struct Num<double> {
  static constexpr bool kPair = false;
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double from(double x) { return x; }
  static __device__ __forceinline__ double dbl(double x) { return x; }
  static __device__ __forceinline__ double ld(const void *p, long e) { return static_cast<const double *>(p)[e]; }
  static __device__ __forceinline__ double ld_f64(const void *p, long e) { return static_cast<const double *>(p)[e]; }
  static __device__ __forceinline__ void st(void *p, long e, double v) { static_cast<double *>(p)[e] = v; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double fma(double s, double x, double y) { return s * x + y; }
  static __device__ __forceinline__ double scale2(double x, double s) { return s * x; }
};
template <> struct Num<float2> {
  static constexpr bool kPair = true;
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ float2 from(double x) { return pair::split(x); }
  static __device__ __forceinline__ double dbl(float2 x) { return pair::to_double(x); }
  static __device__ __forceinline__ float2 ld(const void *p, long e) { return static_cast<const float2 *>(p)[e]; }
  static __device__ __forceinline__ float2 ld_f64(const void *p, long e) {
    return pair::split(static_cast<const double *>(p)[e]);
  }
  static __device__ __forceinline__ void st(void *p, long e, float2 v) { static_cast<float2 *>(p)[e] = v; }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return pair::add(a, b); }
  static __device__ __forceinline__ float2 fma(double s, float2 x, float2 y) {
    return pair::add(pair::mul(pair::split(s), x), y);
  }
  static __device__ __forceinline__ float2 scale2(float2 x, double s) { return pair::scale2(x, (float)s); }
};

// Four independent multiply-add chains of one output (latency hiding).
template <class R> struct Mac;
template <> struct Mac<double> {
  double c[4];
  __device__ __forceinline__ Mac() : c{0.0, 0.0, 0.0, 0.0} {}
  __device__ __forceinline__ void step(int u, double a, double b) { c[u] = fma(a, b, c[u]); }
  __device__ __forceinline__ double total() const { return (c[0] + c[1]) + (c[2] + c[3]); }
};
template <> struct Mac<float2> {
  float h[4], l[4];
  __device__ __forceinline__ Mac() : h{0.f, 0.f, 0.f, 0.f}, l{0.f, 0.f, 0.f, 0.f} {}
  __device__ __forceinline__ void step(int u, float2 a, float2 b) { pair::mac(h[u], l[u], a, b); }
  __device__ __forceinline__ float2 total() const {
    return pair::add(pair::add(make_float2(h[0], l[0]), make_float2(h[1], l[1])),
                     pair::add(make_float2(h[2], l[2]), make_float2(h[3], l[3])));
  }
};

template <class R>
__device__ __forceinline__ R opA(const Prod &P, int i, int k) {
  long e = P.ta ? (long)k * P.lda + i : (long)i * P.lda + k;
  if (P.f64 & 4) e = i <= k ? (long)i * P.lda + k : (long)k * P.lda + i;  // symmetric, upper stored
  return (P.f64 & 1) ? Num<R>::ld_f64(P.A, e) : Num<R>::ld(P.A, e);
}
template <class R>
__device__ __forceinline__ R opB(const Prod &P, int k, int j) {
  const long e = P.tb ? (long)j * P.ldb + k : (long)k * P.ldb + j;
  return (P.f64 & 2) ? Num<R>::ld_f64(P.B, e) : Num<R>::ld(P.B, e);
}

// One output tile (BM x BN) of a phase.  The block's KG groups of 128 threads
// (one output each) take the K chunks round-robin and add their partial sums
// at the end, which divides the dependent multiply-add chain of a tile by KG.
// Each group double-buffers its chunks in shared memory: the next chunk's
// global loads are in flight in registers while the current one is multiplied.  Not inlined: every phase of
// a chain runs the same copy of this code, which stays in the instruction
// cache (inlined at each of the chain's call sites, the first chunk of every
// phase waited on instruction fetch for several microseconds).
constexpr int kLa = BM * BK / NG, kLb = BK * BN / NG;  // elements per thread per chunk
template <class R>
__device__ __noinline__ void phase_tile(const Phase &ph, int tile, R (*As)[2][BM][BK + 1],
                           R (*Bs)[2][BK][BN + 1], R (*part)[NG], double *sq) {
  using X = Num<R>;
  const int tilesN = (ph.n + BN - 1) / BN;
  const int r0 = (tile / tilesN) * BM, c0 = (tile % tilesN) * BN;
  const int tid = threadIdx.x % NG, grp = threadIdx.x / NG;
  const int ty = tid / BN, tx = tid % BN;
  const int i = r0 + ty, j = c0 + tx;
  const int nch = (ph.k + BK - 1) / BK, nit = nch > grp ? (nch - grp + KG - 1) / KG : 0;
  R acc = X::zero();
  for (int q = 0; q < ph.np; ++q) {
    const Prod P = ph.p[q];
    if (P.alpha == 0.0) continue;
    // this thread's load slots: (row, k) of A and (k, col) of B within a chunk
    int ai[kLa], ak[kLa], bk[kLb], bj[kLb];
#pragma unroll
    for (int u = 0; u < kLa; ++u) {
      const int e = tid + u * NG;
      if (P.ta) { ak[u] = e / BM; ai[u] = e % BM; } else { ai[u] = e / BK; ak[u] = e % BK; }
    }
#pragma unroll
    for (int u = 0; u < kLb; ++u) {
      const int e = tid + u * NG;
      if (P.tb) { bj[u] = e / BK; bk[u] = e % BK; } else { bk[u] = e / BN; bj[u] = e % BN; }
    }
    R ra[kLa], rb[kLb];
    auto load = [&](int c) {  // chunk c (zeros beyond K)
      const int k0 = c * BK;
#pragma unroll
      for (int u = 0; u < kLa; ++u) {
        const int gi = r0 + ai[u], gk = k0 + ak[u];
        ra[u] = (gi < ph.m && gk < ph.k) ? opA<R>(P, gi, gk) : X::zero();
      }
#pragma unroll
      for (int u = 0; u < kLb; ++u) {
        const int gk = k0 + bk[u], gj = c0 + bj[u];
        rb[u] = (gk < ph.k && gj < ph.n) ? opB<R>(P, gk, gj) : X::zero();
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int u = 0; u < kLa; ++u) As[grp][buf][ai[u]][ak[u]] = ra[u];
#pragma unroll
      for (int u = 0; u < kLb; ++u) Bs[grp][buf][bk[u]][bj[u]] = rb[u];
    };
    if (nit > 0) {
      load(grp);
      store(0);
    }
    __syncthreads();
    Mac<R> mac;
    const int nitm = (nch + KG - 1) / KG;  // iterations of the busiest group (block-uniform)
    for (int it = 0; it < nitm; ++it) {  // this group's chunks grp, grp + KG, ...
      const int buf = it & 1;
      const bool more = it + 1 < nit;
      if (more) load(KG * (it + 1) + grp);
      if (it < nit) {
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u) mac.step(u, As[grp][buf][ty][kk + u], Bs[grp][buf][kk + u][tx]);
        }
      }
      if (more) store(buf ^ 1);
      __syncthreads();
    }
    acc = X::fma(P.alpha, mac.total(), acc);
  }
  if (grp > 0) part[grp - 1][tid] = acc;
  __syncthreads();
  if (grp == 0 && i < ph.m && j < ph.n) {
    R v = acc;
#pragma unroll
    for (int q = 0; q < KG - 1; ++q) v = X::add(v, part[q][tid]);
    for (int q = 0; q < ph.nc; ++q) v = X::fma(ph.beta[q], X::ld(ph.C[q], (long)i * ph.ldc[q] + j), v);
    if (i == j) v = X::add(v, X::from(ph.diag));
    const long o = (long)i * ph.ldo + j;
    if (ph.out64) static_cast<double *>(ph.out)[o] = X::dbl(v);
    else X::st(ph.out, o, v);
    if (sq) {  // running sum of squares of this thread's outputs
      const double d = X::dbl(v);
      *sq += d * d;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ int phase_tiles(const Phase &ph) {
  if (ph.m <= 0 || ph.n <= 0) return 0;
  return ((ph.m + BM - 1) / BM) * ((ph.n + BN - 1) / BN);
}

// ---- large output tiles for large matrices ------------------------------------
// 64 x 64 outputs per block, K chunks of 16 double-buffered, each of the 512
// threads 4 rows x 2 columns: six shared-memory loads per eight multiply-adds
// (the 8 x 16 tiles above load two per one, and keep every SM busy only on
// small matrices).  A phase takes them when it has at least four per block.
constexpr int LBM = 64, LBN = 64, LBK = 16;
static_assert(NT == 512 && (LBM / 4) * (LBN / 2) == NT, "16 x 32 threads, 4 x 2 outputs each");

template <class R> struct Mac8;
template <> struct Mac8<double> {
  double c[8];
  __device__ __forceinline__ Mac8() : c{0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0} {}
  __device__ __forceinline__ void step(int u, double a, double b) { c[u] = fma(a, b, c[u]); }
  __device__ __forceinline__ double get(int u) const { return c[u]; }
};
template <> struct Mac8<float2> {
  float h[8], l[8];
  __device__ __forceinline__ Mac8() : h{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, l{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f} {}
  __device__ __forceinline__ void step(int u, float2 a, float2 b) { pair::mac(h[u], l[u], a, b); }
  __device__ __forceinline__ float2 get(int u) const { return make_float2(h[u], l[u]); }
};

__device__ __forceinline__ int big_tiles(const Phase &ph) {
  if (ph.m <= 0 || ph.n <= 0) return 0;
  return ((ph.m + LBM - 1) / LBM) * ((ph.n + LBN - 1) / LBN);
}
__device__ __forceinline__ bool use_big(const Phase &ph, int nb) { return big_tiles(ph) >= 4 * nb; }
__device__ __forceinline__ int ntiles(const Phase &ph, int nb) {
  return use_big(ph, nb) ? big_tiles(ph) : phase_tiles(ph);
}

template <class R>
__device__ __noinline__ void phase_tile_big(const Phase &ph, int tile, R (*As)[LBK][LBM + 1],
                                            R (*Bs)[LBK][LBN + 1], double *sq) {
  using X = Num<R>;
  const int tilesN = (ph.n + LBN - 1) / LBN;
  const int r0 = (tile / tilesN) * LBM, c0 = (tile % tilesN) * LBN;
  const int tid = threadIdx.x, ty = tid / 32, tx = tid % 32;  // rows ty*4 + r, columns tx + 32 c
  const int nch = (ph.k + LBK - 1) / LBK;
  R acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = X::zero();
  for (int q = 0; q < ph.np; ++q) {
    const Prod P = ph.p[q];
    if (P.alpha == 0.0) continue;
    // load slots (two elements of A's and of B's chunk per thread), along the
    // stored rows of each operand
    int ai[2], ak[2], bk[2], bj[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * NT;
      if (P.ta) { ak[u] = e / LBM; ai[u] = e % LBM; } else { ai[u] = e / LBK; ak[u] = e % LBK; }
      if (P.tb) { bj[u] = e / LBK; bk[u] = e % LBK; } else { bk[u] = e / LBN; bj[u] = e % LBN; }
    }
    R ra[2], rb[2];
    auto load = [&](int c) {
      const int k0 = c * LBK;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int gi = r0 + ai[u], gk = k0 + ak[u];
        ra[u] = (gi < ph.m && gk < ph.k) ? opA<R>(P, gi, gk) : X::zero();
        const int hk = k0 + bk[u], gj = c0 + bj[u];
        rb[u] = (hk < ph.k && gj < ph.n) ? opB<R>(P, hk, gj) : X::zero();
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        As[buf][ak[u]][ai[u]] = ra[u];
        Bs[buf][bk[u]][bj[u]] = rb[u];
      }
    };
    load(0);
    store(0);
    __syncthreads();
    Mac8<R> mac;
    for (int it = 0; it < nch; ++it) {
      const int buf = it & 1;
      const bool more = it + 1 < nch;
      if (more) load(it + 1);
#pragma unroll 4
      for (int kk = 0; kk < LBK; ++kk) {
        R a[4], b[2];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[buf][kk][ty * 4 + r];
#pragma unroll
        for (int c = 0; c < 2; ++c) b[c] = Bs[buf][kk][tx + 32 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 2; ++c) mac.step(r * 2 + c, a[r], b[c]);
      }
      if (more) store(buf ^ 1);
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = X::fma(P.alpha, mac.get(u), acc[u]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = r0 + ty * 4 + r, j = c0 + tx + 32 * c;
      if (i < ph.m && j < ph.n) {
        R v = acc[r * 2 + c];
        for (int q = 0; q < ph.nc; ++q) v = X::fma(ph.beta[q], X::ld(ph.C[q], (long)i * ph.ldc[q] + j), v);
        if (i == j) v = X::add(v, X::from(ph.diag));
        const long o = (long)i * ph.ldo + j;
        if (ph.out64) static_cast<double *>(ph.out)[o] = X::dbl(v);
        else X::st(ph.out, o, v);
        if (sq) {
          const double d = X::dbl(v);
          *sq += d * d;
        }
      }
    }
  __syncthreads();
}

// Run independent phases over one shared tile index space (no barrier); with
// sq, each thread adds the squares of the outputs it wrote to *sq.
// The phase descriptors are copied once into shared memory: every thread holds
// its own copy in its stack frame, and reading that local memory in each tile's
// prologue and epilogue missed L1 (512 threads x 2 KB per SM).  The small and
// the large tiles share one shared-memory buffer.
constexpr int kSmallTileBytes = (KG * 2 * BM * (BK + 1) + KG * 2 * BK * (BN + 1) + (KG - 1) * NG) * 8;
constexpr int kBigTileBytes = (2 * LBK * (LBM + 1) + 2 * LBK * (LBN + 1)) * 8;
constexpr int kTileBytes = kSmallTileBytes > kBigTileBytes ? kSmallTileBytes : kBigTileBytes;
static_assert(kTileBytes >= 8 * 32 * 16 * 8, "the tensor-core epilogue stages 8 warps x 32 x 16 float pairs here");

template <class R>
__device__ __noinline__ void run_phases_tc(const Coop &cp, const Phase *sph, int count, double *sq,
                                           float2 *stage);

template <class R, bool TCK = false>
__device__ __forceinline__ void run_phases(const Coop &cp, const Phase *ph, int count,
                                           double *sq = nullptr) {
  static_assert(sizeof(R) == 8, "8-byte elements");
  __shared__ __align__(16) unsigned char tsm[kTileBytes];
  __shared__ Phase sph[3];
  __syncthreads();  // the previous user of sph is done
  if (threadIdx.x == 0)
    for (int c = 0; c < count; ++c) sph[c] = ph[c];
  __syncthreads();
  if constexpr (TCK) {  // large products on the tensor cores
    long long work = 0;
    for (int c = 0; c < count; ++c)
      work = max(work, (long long)sph[c].m * sph[c].n * sph[c].k);
    if (cp.tc && work >= cp.tc->min_work) {
      run_phases_tc<R>(cp, sph, count, sq, reinterpret_cast<float2 *>(tsm));  // tsm: 32 KB staging
      return;
    }
  }
  R *const base = reinterpret_cast<R *>(tsm);
  auto *As = reinterpret_cast<R (*)[2][BM][BK + 1]>(base);
  auto *Bs = reinterpret_cast<R (*)[2][BK][BN + 1]>(base + KG * 2 * BM * (BK + 1));
  auto *part = reinterpret_cast<R (*)[NG]>(base + KG * 2 * BM * (BK + 1) + KG * 2 * BK * (BN + 1));
  auto *Al = reinterpret_cast<R (*)[LBK][LBM + 1]>(base);
  auto *Bl = reinterpret_cast<R (*)[LBK][LBN + 1]>(base + 2 * LBK * (LBM + 1));
  int total = 0;
  for (int c = 0; c < count; ++c) total += ntiles(sph[c], cp.size);
  for (int t = cp.rank; t < total; t += cp.size) {
    int c = 0, base_t = 0;
    while (t - base_t >= ntiles(sph[c], cp.size)) { base_t += ntiles(sph[c], cp.size); ++c; }
    if (use_big(sph[c], cp.size)) phase_tile_big<R>(sph[c], t - base_t, Al, Bl, sq);
    else phase_tile<R>(sph[c], t - base_t, As, Bs, part, sq);
  }
}

// ---- tensor-core products of large phases (float pairs; tcgemm.cuh) ----------
// one 8-column load of a single accumulator (lane quarter of the warp)
__device__ __forceinline__ void tmem_ld8(uint32_t t, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(t)
      : "memory");
}

// where a bounded wait of the tensor-core products gave up: the first one is
// recorded in the status words 2 (1: stage free, 2: read-out done, 3: stage
// filled, 4: accumulators ready) and 3 (the stage fill or chunk count)
__device__ __forceinline__ void tc_gave_up(const Coop &cp, int where, int count) {
  if (atomicCAS(cp.flags + 2, 0, where) == 0) cp.flags[3] = count;
}

// out (m x n) of product q of phase P, on this CTA's tiles (see tcgemm.cuh);
// `first`: the phase's first product (writes alpha AB + epilogue terms), else
// adds alpha AB to out; `last`: accumulates the squares of the outputs in *sq
__device__ __noinline__ void tc_tiles(const Coop &cp, const Phase &P, const Prod &pr, bool first,
                                      bool last, double *sq, float2 *stage) {
  const TcCtx &C = cp.tc->ctx;
  GemmSmem &S = *C.S;
  const int m = P.m, n = P.n, K = P.k;
  // scalars in registers: the MMA and copy loops read no memory between their
  // asm statements (which clobber memory)
  const uint32_t tmem = C.tmem;
  uint8_t *const dyn = C.dyn;
  const uint8_t *const asl = C.ws.asl, *const bsl = C.ws.bsl;
  const int *const rexp = C.ws.rexp, *const cexp = C.ws.cexp;
  const int rank = cp.rank, size = cp.size;
  const int ncb = (n + kGN - 1) / kGN, nks = (K + 15) / 16;
  const int ntiles = ((m + 127) / 128) * ncb;
  const int nch = (nks + kGChunk - 1) / kGChunk;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  // the barriers live for the whole kernel; the counts of the previous
  // products give each wait its phase
  const int fill0_copy = S.fill_copy, fill0_mma = S.fill_mma;
  const int ch0_mma = S.chunk_mma, ch0_epi = S.chunk_epi, fins = S.fins;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  volatile int *stop = &S.stop;

  if (w == 0) {
    // --------------------- bulk copies of the slices of each K step ---------------------
    if (lane == 0) {
      // the slices were written by generic stores (before the grid barrier)
      asm volatile("fence.proxy.async.global;" ::: "memory");
      int fill = fill0_copy;
      bool ok = true;
      for (int t = rank; t < ntiles && ok; t += size) {
        const int rb = t / ncb, cb = t % ncb;
        const uint8_t *ab = asl + (size_t)rb * nks * kGA;
        const uint8_t *bb = bsl + (size_t)cb * nks * kGB;
        for (int ks = 0; ks < nks; ++ks, ++fill) {
          const int s = fill % kGStages, use = fill / kGStages;
          if (use > 0 && !mbar_wait(&S.empty[s], (use - 1) & 1, stop)) {
            tc_gave_up(cp, 1, fill);
            ok = false;
            break;
          }
          mbar_expect_tx(&S.full[s], kGStage);
          bulk_g2s(dyn + s * kGStage, ab + (size_t)ks * kGA, kGA, &S.full[s]);
          bulk_g2s(dyn + s * kGStage + kGA, bb + (size_t)ks * kGB, kGB, &S.full[s]);
        }
      }
      if (!ok) atomicExch((int *)stop, 1);
      // the copies still in flight land before the call ends
      for (int q = 0; q < kGStages && q < fill - fill0_copy; ++q) {
        const int f = fill - 1 - q;
        mbar_wait(&S.full[f % kGStages], (f / kGStages) & 1);
      }
      S.fill_copy = fill;
    }
  } else if (w == 1) {
    // ------------------------------------ MMA issue ------------------------------------
    if (lane == 0) {
      // instruction descriptors of N = 256, 192, 128, 64 (index 4 - N / 64)
      const uint32_t id256 = idesc_bf16(256), id192 = idesc_bf16(192), id128 = idesc_bf16(128),
                     id64 = idesc_bf16(64);
      int fill = fill0_mma, ch = ch0_mma;
      bool ok = true;
      for (int t = rank; t < ntiles && ok; t += size) {
        for (int ks = 0; ks < nks; ++ks, ++fill) {
          const int kc = ks % kGChunk, b = ch & 1;
          if (kc == 0 && ch >= 2) {  // the read-out of this buffer's previous chunk is done
            if (!mbar_wait(&S.acc_empty[b], ((ch >> 1) - 1) & 1, stop)) {
              tc_gave_up(cp, 2, ch);
              ok = false;
              break;
            }
          }
          const int s = fill % kGStages, use = fill / kGStages;
          if (!mbar_wait(&S.full[s], use & 1, stop)) {
            tc_gave_up(cp, 3, fill);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = su32(dyn + s * kGStage), b0 = a0 + kGA;
          const uint32_t d = tmem + b * kGSet;
          const uint64_t B0 = smem_desc(b0);
          // A_q against B_0 .. B_(3-q) (consecutive in shared memory) lands the
          // orders q .. 3 at columns 64 q .. 192: one MMA per q; the first of a
          // chunk starts the four sums afresh
          mma_bf16(d, smem_desc(a0), B0, id256, kc == 0 ? 0u : 1u);
          mma_bf16(d + 64, smem_desc(a0 + 4096), B0, id192, 1u);
          mma_bf16(d + 128, smem_desc(a0 + 8192), B0, id128, 1u);
          mma_bf16(d + 192, smem_desc(a0 + 12288), B0, id64, 1u);
          // the order-4 products A_q B_(4-q) into the order-3 sum (FP32)
#pragma unroll
          for (int q = 0; q < kGS; ++q)
            mma_bf16(d + 192, smem_desc(a0 + q * 4096), smem_desc(b0 + (4 - q) * 2048), id64, 1u);
          mma_commit(&S.empty[s]);
          if (kc == kGChunk - 1 || ks == nks - 1) {
            mma_commit(&S.acc_full[b]);
            ++ch;
          }
        }
      }
      if (!ok) atomicExch((int *)stop, 1);
      mma_commit(&S.fin);  // every MMA issued has completed when the call ends
      mbar_wait(&S.fin, fins & 1);
      S.fill_mma = fill;
      S.chunk_mma = ch;
      S.fins = fins + 1;
    }
  } else if (w >= kGEpiW0) {
    // ---------------------------- read-out and outputs ----------------------------
    const int e = w - kGEpiW0, quad = w & 3, half = e >> 2;
    const uint32_t lanebits = (uint32_t)(quad * 32) << 16;
    const float2 al = pair::split(pr.alpha), diag = pair::split(P.diag);
    const long ldo = P.ldo;
    void *const out = P.out;
    const int out64 = P.out64, nc = P.nc;
    int ch = ch0_epi;
    bool ok = true;
    double sql = 0.0;
    for (int t = rank; t < ntiles && ok; t += size) {
      const int rb = t / ncb, cb = t % ncb;
      float2 acc[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = make_float2(0.f, 0.f);
      for (int c = 0; c < nch; ++c, ++ch) {
        const int b = ch & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&S.acc_full[b], (ch >> 1) & 1, stop));
        if (!ok) {
          if (lane == 0) tc_gave_up(cp, 4, ch);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int cg = 0; cg < 4; ++cg) {  // 8 columns of the four sums
          uint32_t r[32];
          tmem_ld_issue(tmem + b * kGSet + lanebits + half * 32 + cg * 8, r, kGN);
          tmem_ld_wait(r);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // the exact integers of orders 0 .. 2 (each on its own 2^-8o grid)
            // and the FP32 sum of orders 3 and 4
            const float2 y = pair::two_sum(__uint_as_float(r[j]), __uint_as_float(r[8 + j]));
            const float lo = __fadd_rn(y.y, __fadd_rn(__uint_as_float(r[16 + j]), __uint_as_float(r[24 + j])));
            acc[cg * 8 + j] = pair::add(acc[cg * 8 + j], make_float2(y.x, lo));
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.acc_empty[b]);
      }
      if (!ok) break;
      // out = alpha 2^(e_i - 8) 2^(f_j - 8) acc (+ epilogue terms on the first
      // product); the warp's 32 x 32 block goes out through shared memory in two
      // passes of 16 columns, so that each load and store of the outputs and the
      // epilogue terms covers two 128-byte row pieces
      const int i0 = rb * 128 + quad * 32;
      {
        const float si = i0 + lane < m ? pow2f(slice_exp(__int_as_float(rexp[i0 + lane])) - 8) : 0.f;
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = pair::scale2(acc[c], si);
      }
      float2 *stg = stage + e * 512;  // this warp's 32 x 16 buffer (XOR-swizzled columns)
      const int jc = lane & 15;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 16; ++c) stg[lane * 16 + (c ^ (lane & 15))] = acc[16 * p + c];
        __syncwarp();
        const int j = cb * kGN + half * 32 + 16 * p + jc;
        if (j >= n) continue;
        const float sj = pow2f(slice_exp(__int_as_float(cexp[j])) - 8);
#pragma unroll 4
        for (int rr = 0; rr < 16; ++rr) {
          const int r = 2 * rr + (lane >> 4), i = i0 + r;
          if (i >= m) continue;
          float2 v = pair::mul(al, pair::scale2(stg[r * 16 + (jc ^ (r & 15))], sj));
          const long o = (long)i * ldo + j;
          if (first) {
            for (int q = 0; q < nc; ++q)
              v = pair::add(pair::mul(pair::split(P.beta[q]),
                                      static_cast<const float2 *>(P.C[q])[(long)i * P.ldc[q] + j]),
                            v);
            if (i == j) v = pair::add(v, diag);
          } else {
            v = pair::add(v, out64 ? pair::split(static_cast<const double *>(out)[o])
                                   : static_cast<const float2 *>(out)[o]);
          }
          if (out64) static_cast<double *>(out)[o] = pair::to_double(v);
          else static_cast<float2 *>(out)[o] = v;
          if (last && sq) {
            const double d = pair::to_double(v);
            sql += d * d;
          }
        }
      }
    }
    if (!ok) atomicExch((int *)stop, 1);
    if (sq) *sq += sql;
    if (e == 0 && lane == 0) S.chunk_epi = ch;  // (every read-out warp counts the same)
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && S.stop) atomicExch(cp.flags + FLAG_ERR, ETDM_ERR_TIMEOUT);
}

// Element (i, k) of op(X) as a float pair, the storage fixed at compile time
// (the slicing passes then issue their loads back to back): FMT bit 0 FP64
// (else float pairs), bit 1 symmetric with the upper triangle stored;
// T: op(X) = X^T.
template <int FMT, int T>
struct OpX {
  const void *p;
  long ld;
  __device__ __forceinline__ float2 operator()(int i, int k) const {
    long e;
    if constexpr ((FMT & 2) != 0) e = i <= k ? (long)i * ld + k : (long)k * ld + i;
    else e = T ? (long)k * ld + i : (long)i * ld + k;
    if constexpr ((FMT & 1) == 0) return static_cast<const float2 *>(p)[e];
    else return pair::split(static_cast<const double *>(p)[e]);
  }
};

// calls g(accessor, rowmajor) with the accessor of op(A) (rows i, columns k)
// or of op(B)^T (rows j, columns k)
template <class G>
__device__ __forceinline__ void with_op(const void *p, long ld, int trans, int fmt, G g) {
  if (fmt == 3) g(OpX<3, 0>{p, ld}, true);
  else if (fmt == 2) g(OpX<2, 0>{p, ld}, true);
  else if (fmt == 1) {
    if (trans) g(OpX<1, 1>{p, ld}, false);
    else g(OpX<1, 0>{p, ld}, true);
  } else {
    if (trans) g(OpX<0, 1>{p, ld}, false);
    else g(OpX<0, 0>{p, ld}, true);
  }
}

// A call of run_phases on the tensor cores: the phases one after another,
// each product sliced (exponents, then slices, into the workspace) and
// multiplied; grid barriers between the steps.  Only the float-pair chains
// take this path.
template <class R>
__device__ __noinline__ void run_phases_tc(const Coop &cp, const Phase *tph, int count, double *sq,
                                           float2 *stage) {
  if constexpr (!Num<R>::kPair) {
    return;
  } else {
    const GemmWs &W = cp.tc->ctx.ws;
    const long gtid = (long)cp.rank * blockDim.x + threadIdx.x;
    const long gstride = (long)cp.size * blockDim.x;
    for (int c = 0; c < count; ++c) {
      const Phase &P = tph[c];
      int first = -1, last = -1;
      for (int q = 0; q < P.np; ++q)
        if (P.p[q].alpha != 0.0) {
          if (first < 0) first = q;
          last = q;
        }
      if (first < 0) continue;  // (every phase of the chains has a product)
      for (int q = first; q <= last; ++q) {
        const Prod &pr = P.p[q];  // (shared memory)
        if (pr.alpha == 0.0) continue;
        for (long e = gtid; e < P.m; e += gstride) W.rexp[e] = 0;
        for (long e = gtid; e < P.n; e += gstride) W.cexp[e] = 0;
        if (!cp.sync()) return;
        // op(A): rows i; op(B)^T: rows j (op(B)^T = B when tb, else B^T)
        const int fa = (pr.f64 & 1) | ((pr.f64 & 4) ? 2 : 0), fb = (pr.f64 & 2) ? 1 : 0;
        const int m = P.m, n = P.n, K = P.k;
        with_op(pr.A, pr.lda, pr.ta, fa, [&](auto x, bool rm) {
          tc_maxima(x, m, K, rm, W.rexp, gtid, gstride);
        });
        with_op(pr.B, pr.ldb, !pr.tb, fb, [&](auto x, bool rm) {
          tc_maxima(x, n, K, rm, W.cexp, gtid, gstride);
        });
        if (!cp.sync()) return;
        with_op(pr.A, pr.lda, pr.ta, fa, [&](auto x, bool rm) {
          tc_slice(x, m, K, 128, rm, W.rexp, W.asl, gtid, gstride);
        });
        with_op(pr.B, pr.ldb, !pr.tb, fb, [&](auto x, bool rm) {
          tc_slice(x, n, K, kGN, rm, W.cexp, W.bsl, gtid, gstride);
        });
        asm volatile("fence.proxy.async.global;" ::: "memory");  // generic writes -> bulk copies
        if (!cp.sync()) return;
        tc_tiles(cp, P, pr, q == first, q == last, sq, stage);
        // the next product rewrites the workspace (and adds to these outputs)
        if ((q < last || c + 1 < count) && !cp.sync()) return;
      }
    }
  }
}

__device__ __forceinline__ Prod mk(const void *A, int lda, int ta, const void *B, int ldb,
                                   int tb, double alpha) {
  Prod p;
  p.A = A; p.B = B; p.lda = lda; p.ldb = ldb; p.ta = ta; p.tb = tb; p.alpha = alpha; p.f64 = 0;
  return p;
}

__device__ __forceinline__ Phase mkphase(int m, int n, int k, void *out, int ldo) {
  Phase ph;
  ph.m = m; ph.n = n; ph.k = k; ph.np = 0;
  ph.nc = 0;
  ph.diag = 0.0; ph.out = out; ph.ldo = ldo; ph.out64 = 0;
  return ph;
}

__device__ __forceinline__ void addc(Phase &ph, const void *c, int ld, double beta) {
  ph.C[ph.nc] = c; ph.ldc[ph.nc] = ld; ph.beta[ph.nc] = beta; ++ph.nc;
}

// In place, for each of the n N x N row-major matrices X: X <- s (X + X^T).
// A block takes a pair of 32 x 32 tiles (I, J), I <= J, reads both and writes
// both, so no element is read after another block has rewritten it.  The
// reverse pass uses it to keep the cotangents of the symmetric intermediates
// symmetric (the chain's intermediates are symmetric functions of P, and P =
// A A^T moves only in symmetric directions, so only the symmetric part of a
// cotangent reaches the gradient); a pair X K + K X then is Y + Y^T with the
// one product Y = X K.
template <class R>
__device__ void sym_pass(const Coop &cp, double *const *mats, int n, int N, double s) {
  using X = Num<R>;
  __shared__ R ta[32][33], tb[32][33];
  const int nt = (N + 31) / 32;
  const long pairs = (long)nt * (nt + 1) / 2;
  for (long w = cp.rank; w < pairs * n; w += cp.size) {
    R *const Xm = reinterpret_cast<R *>(mats[w / pairs]);
    long p = w % pairs;
    int I = 0;
    while (p >= nt - I) { p -= nt - I; ++I; }
    const int J = I + (int)p;
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
      const int r = e >> 5, c = e & 31;
      const int i1 = I * 32 + r, j1 = J * 32 + c, i2 = J * 32 + r, j2 = I * 32 + c;
      ta[r][c] = (i1 < N && j1 < N) ? X::ld(Xm, (long)i1 * N + j1) : X::zero();
      tb[r][c] = (i2 < N && j2 < N) ? X::ld(Xm, (long)i2 * N + j2) : X::zero();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
      const int r = e >> 5, c = e & 31;
      const int i1 = I * 32 + r, j1 = J * 32 + c, i2 = J * 32 + r, j2 = I * 32 + c;
      if (i1 < N && j1 < N) X::st(Xm, (long)i1 * N + j1, X::scale2(X::add(ta[r][c], tb[c][r]), s));
      if (I != J && i2 < N && j2 < N)
        X::st(Xm, (long)i2 * N + j2, X::scale2(X::add(tb[r][c], ta[c][r]), s));
    }
    __syncthreads();
  }
}

#define BARRIER_OR_RETURN()   \
  do {                        \
    if (!cp.sync()) return;   \
  } while (0)

// Forward: P, j, Q^k, Taylor series, doublings, U_occ = [cos sqrt P; -A^T s(P)],
// O = C0 U_occ, then D = 2 O O^T and H <- T (FP64 grid passes) or T O (mixed).
template <class R, bool TCK = false>
__device__ void dense_forward(const DenseArgs &a, const Coop &cp) {
  using X = Num<R>;
  const int M = a.M, N = a.N, V = a.V;
  const long NN = (long)N * N;
  const long gtid = (long)cp.rank * blockDim.x + threadIdx.x;
  const long gstride = (long)cp.size * blockDim.x;
  __shared__ int sh_j, sh_jf;
  __shared__ double sh_sc;
  // A_ov as R: the float-pair engine converts the FP64 input once, in the first phase
  const void *const Ar = X::kPair ? (const void *)a.Af : (const void *)a.A;

  {  // P = A_ov A_ov^T (reads the FP64 A); each block sums the squares of its outputs
    if (X::kPair)
      for (long e = gtid; e < (long)N * V; e += gstride) X::st(a.Af, e, X::ld_f64(a.A, e));
    Phase ph = mkphase(N, N, V, a.P, N);
    ph.np = 1; ph.p[0] = mk(a.A, V, 0, a.A, V, 1, 1.0); ph.p[0].f64 = 3;
    double sq = 0.0;
    run_phases<R, TCK>(cp, &ph, 1, &sq);
    sq = block_sum(sq);
    if (threadIdx.x == 0) a.red[cp.rank] = sq;
  }
  BARRIER_OR_RETURN();
  {  // the range check |P|_F <= 4^kJmax (every block sums the partials in the same order)
    const double t = block_sum_of(a.red, cp.size);
    double nrm = sqrt(t);
    int j = 0;
    while (nrm > 1.0 && j <= kJmax) { nrm *= 0.25; ++j; }
    if (!(t == t) || isinf(t)) j = kJmax + 1;
    if (threadIdx.x == 0) sh_jf = j;
  }
  __syncthreads();
  const int JF = sh_jf;  // the doublings |P|_F alone would take
  if (JF > kJmax) {
    if (gtid == 0) atomicExch(a.flags + FLAG_ERR, ETDM_ERR_NUMERIC);
    return;
  }
  double *const Qs = a.Qk;
  auto slot = [&](int k) { return Qs + (long)k * NN; };
  // P^2, P^3 and P^4 unscaled (|P|_F <= 4^8 keeps |P^4| below 2^64), with the
  // squares of P^2 and P^4 summed for the bounds on rho(P)
  {
    Phase ph = mkphase(N, N, N, slot(kQ2), N);
    ph.np = 1; ph.p[0] = mk(a.P, N, 0, a.P, N, 0, 1.0);
    double sq = 0.0;
    run_phases<R, TCK>(cp, &ph, 1, &sq);
    sq = block_sum(sq);
    if (threadIdx.x == 0) a.red[cp.size + cp.rank] = sq;
  }
  BARRIER_OR_RETURN();
  {
    Phase ph[2];
    ph[0] = mkphase(N, N, N, slot(kQ3), N);
    ph[0].np = 1; ph[0].p[0] = mk(a.P, N, 0, slot(kQ2), N, 0, 1.0);
    ph[1] = mkphase(N, N, N, slot(kQ4), N);
    ph[1].np = 1; ph[1].p[0] = mk(slot(kQ2), N, 0, slot(kQ2), N, 0, 1.0);
    run_phases<R, TCK>(cp, ph, 2);
  }
  BARRIER_OR_RETURN();
  {
    double sq = 0.0;
    for (long e = gtid; e < NN; e += gstride) {
      const double x = X::dbl(X::ld(slot(kQ4), e));
      sq += x * x;
    }
    sq = block_sum(sq);
    if (threadIdx.x == 0) a.red[2 * cp.size + cp.rank] = sq;
  }
  BARRIER_OR_RETURN();
  {  // j from the smallest bound on rho(P)
    const double t1 = block_sum_of(a.red, cp.size);
    const double t2 = block_sum_of(a.red + cp.size, cp.size);
    const double t4 = block_sum_of(a.red + 2 * cp.size, cp.size);
    double rho = fmin(sqrt(t1), fmin(sqrt(sqrt(t2)), sqrt(sqrt(sqrt(t4)))));
    if (!(rho == rho)) rho = sqrt(t1);
    int j = 0;
    while (rho > 1.0 && j < JF) { rho *= 0.25; ++j; }
    if (threadIdx.x == 0) {
      sh_j = j;
      sh_sc = ldexp(1.0, -2 * j);
    }
  }
  __syncthreads();
  const int J = sh_j;
  const double sc = sh_sc;
  if (gtid == 0) { a.flags[FLAG_J] = J; a.scal[0] = sc; }
  // Q^r = sc^r P^r in place (powers of two: exact), Q = sc P kept for the
  // reverse pass; the products below use P with the scale in their
  // coefficients.  Paterson-Stockmeyer blocks B_i = sum_r c_{4i+r} Q^r (r < 4)
  // enter the products below as epilogue terms; B_2 is also stored for the
  // reverse pass
  auto cf = [&](const double *c, int k) { return k <= kTaylor ? c[k] : 0.0; };
  const double sc2 = sc * sc, sc3 = sc2 * sc, sc4 = sc2 * sc2;
  for (long e = gtid; e < NN; e += gstride) {
    const int i = (int)(e / N), c = (int)(e % N);
    const R q1 = X::scale2(X::ld(a.P, e), sc), q2 = X::scale2(X::ld(slot(kQ2), e), sc2),
            q3 = X::scale2(X::ld(slot(kQ3), e), sc3), q4 = X::scale2(X::ld(slot(kQ4), e), sc4);
    X::st(slot(kQ1), e, q1);
    X::st(slot(kQ2), e, q2);
    X::st(slot(kQ3), e, q3);
    X::st(slot(kQ4), e, q4);
    const R q[4] = {X::from(i == c ? 1.0 : 0.0), q1, q2, q3};
    R bc = X::zero(), bs = X::zero();
    for (int r = 0; r < 4; ++r) {
      bc = X::fma(cf(a.ck, 8 + r), q[r], bc);
      bs = X::fma(cf(a.sk, 8 + r), q[r], bs);
    }
    X::st(slot(kBc2), e, bc);
    X::st(slot(kBs2), e, bs);
  }
  BARRIER_OR_RETURN();
  {  // T = B_1 + Q^4 B_2 (B_2 stored by the pass above)
    Phase ph[2];
    const double *co[2] = {a.ck, a.sk};
    double *const out[2] = {slot(kTc), slot(kTs)};
    const int b2[2] = {kBc2, kBs2};
    for (int w = 0; w < 2; ++w) {
      const double *c = co[w];
      ph[w] = mkphase(N, N, N, out[w], N);
      ph[w].np = 1; ph[w].p[0] = mk(slot(kQ4), N, 0, slot(b2[w]), N, 0, 1.0);
      addc(ph[w], a.P, N, cf(c, 5) * sc);
      addc(ph[w], slot(kQ2), N, cf(c, 6));
      addc(ph[w], slot(kQ3), N, cf(c, 7));
      ph[w].diag = cf(c, 4);
    }
    run_phases<R, TCK>(cp, ph, 2);
  }
  BARRIER_OR_RETURN();
  {  // k = cos sqrt(Q) - 1 = B_0 + Q^4 T_c, s = sin sqrt(Q) / sqrt(Q) = B_0 + Q^4 T_s
    Phase ph[2];
    const double *co[2] = {a.ck, a.sk};
    double *const out[2] = {a.Kt, a.St};
    const double *tt[2] = {slot(kTc), slot(kTs)};
    for (int w = 0; w < 2; ++w) {
      const double *c = co[w];
      ph[w] = mkphase(N, N, N, out[w], N);
      ph[w].np = 1; ph[w].p[0] = mk(slot(kQ4), N, 0, tt[w], N, 0, 1.0);
      addc(ph[w], a.P, N, cf(c, 1) * sc);
      addc(ph[w], slot(kQ2), N, cf(c, 2));
      addc(ph[w], slot(kQ3), N, cf(c, 3));
      ph[w].diag = cf(c, 0);
    }
    run_phases<R, TCK>(cp, ph, 2);
  }
  BARRIER_OR_RETURN();
  for (int t = 0; t < J; ++t) {  // doubling: k' = 4k + 2k^2, s' = s + s k
    const double *Kc = a.Kt + (long)t * NN, *Sc = a.St + (long)t * NN;
    Phase ph[2];
    ph[0] = mkphase(N, N, N, a.Kt + (long)(t + 1) * NN, N);
    ph[0].np = 1; ph[0].p[0] = mk(Kc, N, 0, Kc, N, 0, 2.0);
    addc(ph[0], Kc, N, 4.0);
    ph[1] = mkphase(N, N, N, a.St + (long)(t + 1) * NN, N);
    ph[1].np = 1; ph[1].p[0] = mk(Sc, N, 0, Kc, N, 0, 1.0);
    addc(ph[1], Sc, N, 1.0);
    run_phases<R, TCK>(cp, ph, 2);
    BARRIER_OR_RETURN();
  }
  {
    const double *KJ = a.Kt + (long)J * NN, *SJ = a.St + (long)J * NN;
    for (long e = gtid; e < NN; e += gstride) {
      int i = (int)(e / N), c = (int)(e % N);
      X::st(a.Uocc, e, X::add(X::ld(KJ, e), X::from(i == c ? 1.0 : 0.0)));
    }
    Phase ph = mkphase(V, N, N, a.Uocc + NN, N);  // -A^T s(P)
    ph.np = 1; ph.p[0] = mk(Ar, V, 1, SJ, N, 0, -1.0);
    run_phases<R, TCK>(cp, &ph, 1);
  }
  BARRIER_OR_RETURN();
  {
    Phase ph = mkphase(M, N, M, a.O, N);  // O = C0 U_occ
    ph.np = 1; ph.p[0] = mk(a.C0, M, 0, a.Uocc, N, 0, 1.0);
    run_phases<R, TCK>(cp, &ph, 1);
  }
  BARRIER_OR_RETURN();
  if (a.Vacc) {  // mixed path: the density comes from O on the grid; T O for the kinetic energy and dE/dO
    Phase ph = mkphase(M, N, M, a.TO, N);
    ph.np = 1; ph.p[0] = mk(a.T, M, 0, a.O, N, 0, 1.0);
    run_phases<R, TCK>(cp, &ph, 1);
  } else {
    Phase ph = mkphase(M, M, N, a.D, M);  // D = 2 O O^T (Eq. 12, f = 2)
    ph.np = 1; ph.p[0] = mk(a.O, N, 0, a.O, N, 1, 2.0);
    run_phases<R, TCK>(cp, &ph, 1);
    const long MM = (long)M * M;
    for (long e = gtid; e < MM; e += gstride) X::st(a.H, e, X::ld(a.T, e));
  }
}

template <class R>
__global__ void __launch_bounds__(NT) dense_forward_kernel(DenseArgs a) {
  dense_forward<R>(a, grid_coop(a.bar, a.flags));
}

// Batched: block b runs the chains of systems order[b], order[b + gridDim], ...
// (largest first) one after another, each system on this block alone; systems
// whose active flag is 0 are skipped.
template <class R>
__global__ void __launch_bounds__(NT) dense_forward_batch_kernel(const DenseArgs *av, const int *order,
                                                                 int n, const int *active) {
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    const int i = order[q];
    if (active[i]) dense_forward<R>(av[i], block_coop());
  }
}

// Reverse: E = Tr(D T) + grid terms; dE/dO = 4 H O; dE/dU = C0^T (4 H O);
// (mixed path: Tr(D T) = 2 sum O o (T O), 4 H O = 4 T O + 4 V O);
// back through U_occ, the doublings, the Taylor powers and P = A A^T.
template <class R, bool TCK = false>
__device__ void dense_reverse(const DenseArgs &a, int want_grad, const Coop &cp) {
  using X = Num<R>;
  const int M = a.M, N = a.N, V = a.V;
  const long NN = (long)N * N, MM = (long)M * M;
  const long gtid = (long)cp.rank * blockDim.x + threadIdx.x;
  const long gstride = (long)cp.size * blockDim.x;
  const bool mixed = a.Vacc != nullptr;
  const long MN = (long)M * N;
  const void *const Ar = X::kPair ? (const void *)a.Af : (const void *)a.A;  // set by the forward
  if (mixed) {
    // Tr(D T) = 2 sum O o (T O) (the kinetic energy is exact: O as computed,
    // only the grid energy saw Oq); Gbar = dE/dO = 4 V O + 4 T O with V read
    // from its upper triangle; the first-order correction of the density's O
    // quantization, sum (4 V O) o (O - Oq) = sum Gbar o dO - 4 sum (T O) o dO
    double s = 0.0, c = 0.0;
    for (long e = gtid; e < MN; e += gstride) {
      const double to = X::dbl(X::ld(a.TO, e));
      s += 2.0 * X::dbl(X::ld(a.O, e)) * to;
      c += to * a.dO[e];
    }
    s = block_sum(s);
    c = block_sum(c);
    if (threadIdx.x == 0) { a.red[cp.rank] = s; a.red[cp.size + cp.rank] = -4.0 * c; }
    Phase ph = mkphase(M, N, M, a.Gbar, N);
    ph.np = 1; ph.p[0] = mk(a.Vacc, M, 0, a.O, N, 0, 4.0); ph.p[0].f64 = 4;  // A symmetric (upper)
    addc(ph, a.TO, N, 4.0);
    run_phases<R, TCK>(cp, &ph, 1);
    BARRIER_OR_RETURN();
    double c2 = 0.0;
    for (long e = gtid; e < MN; e += gstride) c2 += X::dbl(X::ld(a.Gbar, e)) * a.dO[e];
    c2 = block_sum(c2);
    if (threadIdx.x == 0) a.red[2 * cp.size + cp.rank] = c2;
    if (want_grad) {
      Phase pu = mkphase(M, N, M, a.Ubar, N);  // Ubar = C0^T Gbar
      pu.np = 1; pu.p[0] = mk(a.C0, M, 1, a.Gbar, N, 0, 1.0);
      run_phases<R, TCK>(cp, &pu, 1);
    }
    BARRIER_OR_RETURN();
  } else {
    double s = 0.0;
    for (long e = gtid; e < MM; e += gstride) s += X::dbl(X::ld(a.D, e)) * X::dbl(X::ld(a.T, e));
    if (want_grad) {  // the grid pass accumulated the upper triangle of H
      for (long e = gtid; e < MM; e += gstride) {
        int i = (int)(e / M), c = (int)(e % M);
        if (i > c) X::st(a.H, e, X::ld(a.H, (long)c * M + i));
      }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) a.red[cp.rank] = s;
    BARRIER_OR_RETURN();
    if (want_grad) {
      Phase ph = mkphase(M, N, M, a.Gbar, N);  // Gbar = dE/dO = 4 H O
      ph.np = 1; ph.p[0] = mk(a.H, M, 0, a.O, N, 0, 4.0);
      run_phases<R, TCK>(cp, &ph, 1);
      BARRIER_OR_RETURN();
      Phase pu = mkphase(M, N, M, a.Ubar, N);  // Ubar = C0^T Gbar
      pu.np = 1; pu.p[0] = mk(a.C0, M, 1, a.Gbar, N, 0, 1.0);
      run_phases<R, TCK>(cp, &pu, 1);
      BARRIER_OR_RETURN();
    }
  }
  if (cp.rank == 0) {  // energy terms: tree sums over the block partials, all threads of block 0
    double kin = 0.0, corr = 0.0, t3[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < cp.size; b += blockDim.x) {
      kin += a.red[b];
      if (mixed) corr += a.red[cp.size + b] + a.red[2 * cp.size + b];
    }
    for (int b = threadIdx.x; b < a.n_gridpart; b += blockDim.x)
      for (int q = 0; q < 3; ++q) t3[q] += a.gridpart[3 * b + q];
    kin = block_sum(kin);
    corr = block_sum(corr);
    for (int q = 0; q < 3; ++q) t3[q] = block_sum(t3[q]);
    if (threadIdx.x == 0) {
      const double E = kin + t3[0] + t3[1] + t3[2] + corr;
      a.eterms[0] = kin; a.eterms[1] = t3[0]; a.eterms[2] = t3[1]; a.eterms[3] = t3[2] + corr;
      if (a.E) *a.E = E;
      if (!(E == E) || isinf(E)) atomicExch(a.flags + FLAG_ERR, ETDM_ERR_NUMERIC);
    }
  }
  if (!want_grad) return;
  const int J = a.flags[FLAG_J];
  const double sc = a.scal[0];
  const double *Ubv = a.Ubar + NN;  // rows N..M-1 (V x N)
  {
    Phase ph[2];
    ph[0] = mkphase(N, N, V, a.Sbar[0], N);  // Sbar_J = -A Ubar_v
    ph[0].np = 1; ph[0].p[0] = mk(Ar, V, 0, Ubv, N, 0, -1.0);
    ph[1] = mkphase(N, V, N, a.Abar, V);     // Abar = -S_J Ubar_v^T
    ph[1].np = 1; ph[1].p[0] = mk(a.St + (long)J * NN, N, 0, Ubv, N, 1, -1.0);
    run_phases<R, TCK>(cp, ph, 2);
  }
  BARRIER_OR_RETURN();
  // symmetric cotangents of k_J (Ubar_o, the first N rows of Ubar, which the
  // residual below still reads) and of s_J
  {
    for (long e = gtid; e < NN; e += gstride) X::st(a.Kbar[1], e, X::ld(a.Ubar, e));
    BARRIER_OR_RETURN();
    double *const m2[2] = {a.Kbar[1], a.Sbar[0]};
    sym_pass<R>(cp, m2, 2, N, 0.5);
  }
  BARRIER_OR_RETURN();
  const double *kb = a.Kbar[1];
  const double *sb = a.Sbar[0];
  int pp = 0;
  for (int t = J - 1; t >= 0; --t) {
    // k' = 4k + 2k^2, s' = s + s k with kbar', sbar' symmetric:
    //   kbar = 4 kbar' + 2 (kbar' k + k kbar') + sym(s sbar') = Z + Z^T,
    //          Z = 2 kbar' + 2 kbar' k + s sbar' / 2,
    //   sbar = sbar' + sym(sbar' k) = W + W^T,  W = sbar' / 2 + sbar' k / 2
    const double *Kc = a.Kt + (long)t * NN, *Sc = a.St + (long)t * NN;
    double *kbo = a.Kbar[pp], *sbo = a.Sbar[1 - pp];
    Phase ph[2];
    ph[0] = mkphase(N, N, N, sbo, N);
    ph[0].np = 1; ph[0].p[0] = mk(sb, N, 0, Kc, N, 0, 0.5);
    addc(ph[0], sb, N, 0.5);
    ph[1] = mkphase(N, N, N, kbo, N);
    ph[1].np = 2;
    ph[1].p[0] = mk(kb, N, 0, Kc, N, 0, 2.0);
    ph[1].p[1] = mk(Sc, N, 0, sb, N, 0, 0.5);
    addc(ph[1], kb, N, 2.0);
    run_phases<R, TCK>(cp, ph, 2);
    BARRIER_OR_RETURN();
    double *const m2[2] = {kbo, sbo};
    sym_pass<R>(cp, m2, 2, N, 1.0);
    BARRIER_OR_RETURN();
    kb = kbo; sb = sbo; pp = 1 - pp;
  }
  // back through k = B_0 + Q^4 T_c, s = B_0 + Q^4 T_s (all forward matrices are
  // symmetric, so for C = X Y: Xbar += Cbar Y, Ybar += X Cbar)
  const double *const Qs = a.Qk;
  auto slot = [&](int k) { return Qs + (long)k * NN; };
  auto wr = [&](int k) { return a.Wr + (long)k * NN; };
  {
    Phase ph[3];
    ph[0] = mkphase(N, N, N, wr(kQ4b), N);  // Q4bar = kbar T_c + sbar T_s
    ph[0].np = 2;
    ph[0].p[0] = mk(kb, N, 0, slot(kTc), N, 0, 1.0);
    ph[0].p[1] = mk(sb, N, 0, slot(kTs), N, 0, 1.0);
    ph[1] = mkphase(N, N, N, wr(kTcb), N);  // T_c bar = Q^4 kbar
    ph[1].np = 1; ph[1].p[0] = mk(slot(kQ4), N, 0, kb, N, 0, 1.0);
    ph[2] = mkphase(N, N, N, wr(kTsb), N);  // T_s bar = Q^4 sbar
    ph[2].np = 1; ph[2].p[0] = mk(slot(kQ4), N, 0, sb, N, 0, 1.0);
    run_phases<R, TCK>(cp, ph, 3);
  }
  BARRIER_OR_RETURN();
  {  // back through T = B_1 + Q^4 B_2
    Phase ph[3];
    ph[0] = mkphase(N, N, N, wr(kQ4b), N);  // Q4bar += T_c bar B_c2 + T_s bar B_s2
    ph[0].np = 2;
    ph[0].p[0] = mk(wr(kTcb), N, 0, slot(kBc2), N, 0, 1.0);
    ph[0].p[1] = mk(wr(kTsb), N, 0, slot(kBs2), N, 0, 1.0);
    addc(ph[0], wr(kQ4b), N, 1.0);
    ph[1] = mkphase(N, N, N, wr(kBc2b), N);  // B_c2 bar = Q^4 T_c bar
    ph[1].np = 1; ph[1].p[0] = mk(slot(kQ4), N, 0, wr(kTcb), N, 0, 1.0);
    ph[2] = mkphase(N, N, N, wr(kBs2b), N);  // B_s2 bar = Q^4 T_s bar
    ph[2].np = 1; ph[2].p[0] = mk(slot(kQ4), N, 0, wr(kTsb), N, 0, 1.0);
    run_phases<R, TCK>(cp, ph, 3);
  }
  BARRIER_OR_RETURN();
  // the blocks' cotangents to the powers: Q^r bar = sum_i c_{4i+r} B_ci bar + s_{4i+r} B_si bar
  for (long e = gtid; e < NN; e += gstride) {
    const R bcb[3] = {X::ld(kb, e), X::ld(wr(kTcb), e), X::ld(wr(kBc2b), e)};
    const R bsb[3] = {X::ld(sb, e), X::ld(wr(kTsb), e), X::ld(wr(kBs2b), e)};
    R qb[4] = {X::zero(), X::zero(), X::zero(), X::zero()};
    for (int b = 0; b < 3; ++b)
      for (int r = 1; r < 4; ++r) {
        const int k = 4 * b + r;
        if (k <= kTaylor) qb[r] = X::fma(a.ck[k], bcb[b], X::fma(a.sk[k], bsb[b], qb[r]));
      }
    X::st(wr(kQ1bB), e, qb[1]);
    X::st(wr(kQ2bB), e, qb[2]);
    X::st(wr(kQ3b), e, qb[3]);
  }
  BARRIER_OR_RETURN();
  {  // the cotangents of Q^4, Q^3 and the blocks' parts of Qbar, Q2bar made symmetric
    double *const m4[4] = {wr(kQ4b), wr(kQ3b), wr(kQ1bB), wr(kQ2bB)};
    sym_pass<R>(cp, m4, 4, N, 0.5);
  }
  BARRIER_OR_RETURN();
  {  // back through Q^4 = Q^2 Q^2 and Q^3 = Q Q^2:
     //   Q2bar = Q2bar_B + (Q4bar Q^2 + Q^2 Q4bar) + sym(Q Q3bar) = Z + Z^T,
     //           Z = Q2bar_B / 2 + Q4bar Q^2 + Q Q3bar / 2,
     //   Qbar_t = Q1bar_B + sym(Q3bar Q^2) = Zt + Zt^T,  Zt = Q1bar_B / 2 + Q3bar Q^2 / 2
    Phase ph[2];
    ph[0] = mkphase(N, N, N, wr(kQ2b), N);
    ph[0].np = 2;
    ph[0].p[0] = mk(wr(kQ4b), N, 0, slot(kQ2), N, 0, 1.0);
    ph[0].p[1] = mk(slot(kQ1), N, 0, wr(kQ3b), N, 0, 0.5);
    addc(ph[0], wr(kQ2bB), N, 0.5);
    ph[1] = mkphase(N, N, N, wr(kQ1bt), N);
    ph[1].np = 1; ph[1].p[0] = mk(wr(kQ3b), N, 0, slot(kQ2), N, 0, 0.5);
    addc(ph[1], wr(kQ1bB), N, 0.5);
    run_phases<R, TCK>(cp, ph, 2);
  }
  BARRIER_OR_RETURN();
  {
    double *const m2[2] = {wr(kQ2b), wr(kQ1bt)};
    sym_pass<R>(cp, m2, 2, N, 1.0);
  }
  BARRIER_OR_RETURN();
  {  // back through Q^2 = Q Q: Qbar = Qbar_t + Q2bar Q + Q Q2bar = Z + Z^T, Z = Qbar_t / 2 + Q2bar Q
    Phase ph = mkphase(N, N, N, wr(kQ1b), N);
    ph.np = 1; ph.p[0] = mk(wr(kQ2b), N, 0, slot(kQ1), N, 0, 1.0);
    addc(ph, wr(kQ1bt), N, 0.5);
    run_phases<R, TCK>(cp, &ph, 1);
  }
  BARRIER_OR_RETURN();
  {
    double *const m1[1] = {wr(kQ1b)};
    sym_pass<R>(cp, m1, 1, N, 1.0);
  }
  BARRIER_OR_RETURN();
  {  // Q = sc P: g = Abar + (Pbar + Pbar^T) A = Abar + 2 sc Qbar A (Qbar symmetric), written as FP64
    Phase ph = mkphase(N, V, N, a.g, V);
    ph.np = 1; ph.p[0] = mk(wr(kQ1b), N, 0, Ar, V, 0, 2.0 * sc);
    addc(ph, a.Abar, V, 1.0);
    ph.out64 = 1;
    run_phases<R, TCK>(cp, &ph, 1);
  }
  if (!a.resid) return;
  // Eq. 45 in the orthonormal basis of C0 (C0^T S C0 = I): the occupied
  // orbitals are U_occ, H psi_i has the coefficients (C0^T H C0 U)_i =
  // Ubar_i / 4 and lambda = U^T (Ubar / 4), so the residual is
  // R / 4 with R = Ubar - U_occ (U_occ^T Ubar), and Eq. 45 = (1/N_e) sum f_i
  // |R_i / 4|^2 = |R|^2 / (8 N_e) with f = 2, N_e = 2 N.  X in the first
  // reverse workspace slot and R in Gbar (both free by now).
  BARRIER_OR_RETURN();
  {
    Phase ph = mkphase(N, N, M, wr(kQ4b), N);  // X = U_occ^T Ubar
    ph.np = 1; ph.p[0] = mk(a.Uocc, N, 1, a.Ubar, N, 0, 1.0);
    run_phases<R, TCK>(cp, &ph, 1);
  }
  BARRIER_OR_RETURN();
  {
    Phase ph = mkphase(M, N, N, a.Gbar, N);  // R = Ubar - U_occ X
    ph.np = 1; ph.p[0] = mk(a.Uocc, N, 0, wr(kQ4b), N, 0, -1.0);
    addc(ph, a.Ubar, N, 1.0);
    double sq = 0.0;
    run_phases<R, TCK>(cp, &ph, 1, &sq);
    sq = block_sum(sq);
    if (threadIdx.x == 0) a.red[3 * cp.size + cp.rank] = sq;
  }
  BARRIER_OR_RETURN();
  if (cp.rank == 0) {
    const double t = block_sum_of(a.red + 3 * cp.size, cp.size);
    if (threadIdx.x == 0) *a.resid = t / (16.0 * N);
  }
}

template <class R>
__global__ void __launch_bounds__(NT) dense_reverse_kernel(DenseArgs a, int want_grad) {
  dense_reverse<R>(a, want_grad, grid_coop(a.bar, a.flags));
}

template <class R>
__global__ void __launch_bounds__(NT) dense_reverse_batch_kernel(const DenseArgs *av, const int *order,
                                                                 int n, const int *active) {
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    const int i = order[q];
    if (active[i]) dense_reverse<R>(av[i], 1, block_coop());
  }
}

// The float-pair chains with their large products on the tensor cores: one
// block per SM (the stage ring's dynamic shared memory leaves room for no
// second block), 512 tensor-memory columns held for the kernel's lifetime.
__device__ __forceinline__ void tc_setup(const DenseArgs &a, TcRun &run, GemmSmem &gS,
                                         uint8_t *dyn, uint32_t *slot) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) {
      mbar_init(&gS.full[s], 1);
      mbar_init(&gS.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&gS.acc_full[b], 1);
      mbar_init(&gS.acc_empty[b], 8);  // one arrival per read-out warp
    }
    mbar_init(&gS.fin, 1);
    gS.stop = 0;
    gS.fill_copy = gS.fill_mma = gS.chunk_mma = gS.chunk_epi = gS.fins = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(slot);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  run.ctx.ws = GemmWs{a.tc_asl, a.tc_bsl, a.tc_rexp, a.tc_cexp};
  run.ctx.dyn = dyn;
  run.ctx.S = &gS;
  run.ctx.tmem = *slot;
  run.min_work = a.tc_min_work;
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem);
}

__global__ void __launch_bounds__(NT) dense_forward_tc_kernel(DenseArgs a) {
  extern __shared__ __align__(1024) uint8_t gdyn[];
  __shared__ GemmSmem gS;
  __shared__ uint32_t slot;
  TcRun run;
  tc_setup(a, run, gS, gdyn, &slot);
  Coop cp = grid_coop(a.bar, a.flags);
  cp.tc = &run;
  dense_forward<float2, true>(a, cp);
  tc_teardown(run.ctx.tmem);
}

__global__ void __launch_bounds__(NT) dense_reverse_tc_kernel(DenseArgs a, int want_grad) {
  extern __shared__ __align__(1024) uint8_t gdyn[];
  __shared__ GemmSmem gS;
  __shared__ uint32_t slot;
  TcRun run;
  tc_setup(a, run, gS, gdyn, &slot);
  Coop cp = grid_coop(a.bar, a.flags);
  cp.tc = &run;
  dense_reverse<float2, true>(a, want_grad, cp);
  tc_teardown(run.ctx.tmem);
}

// One product C = op(A) op(B) of FP64 matrices on the tensor-core path (the
// building block of the chains' large products), as a cooperative launch.
__global__ void __launch_bounds__(NT) pair_gemm_kernel(Phase ph, DenseArgs a) {
  extern __shared__ __align__(1024) uint8_t gdyn[];
  __shared__ GemmSmem gS;
  __shared__ uint32_t slot;
  TcRun run;
  tc_setup(a, run, gS, gdyn, &slot);
  Coop cp = grid_coop(a.bar, a.flags);
  cp.tc = &run;
  run.min_work = 0;
  run_phases<float2, true>(cp, &ph, 1);
  tc_teardown(run.ctx.tmem);
}

// Plain (non-cooperative) product for set-up work.
__global__ void __launch_bounds__(NT) gemm_kernel(Phase ph) {
  run_phases<double>(grid_coop(nullptr, nullptr), &ph, 1);
}

// ---- L-BFGS two-loop (Sec. 3.1) with H0 = P^(k) (Eq. 33-34) ---------------
__device__ __forceinline__ double precond_elem(const double *eps, int N, int V, long e,
                                               double gamma, double beta) {
  int i = (int)(e / V), jv = (int)(e % V);
  double d = (eps[i] - eps[N + jv]) * 2.0;  // (e_i - e_j)(f_i - f_j), f = 2 / 0
  return 1.0 / (2.0 * (1.0 - gamma) * fabs(d) + gamma * beta);
}

// P^(k) of variable e: the occupied-virtual form above, or (full A over
// k-points) from the per-variable parts 2 (1 - gamma) |(e_i - e_j)(f_i - f_j)|
// and w_k (Eq. 33 with the k-point weight on beta, Sec. 3.3).
__device__ __forceinline__ double precond_of(const LbfgsArgs &a, long e, double beta) {
  if (a.pden) return 1.0 / (a.pden[e] + a.gamma * beta * a.pw[e]);
  return precond_elem(a.eps, a.N, a.V, e, a.gamma, beta);
}

// Dot product of the whole grid: every block gets the same value.  The block
// partials alternate between two halves of red[] (2 * gridDim entries each,
// room for two sums), so one barrier suffices: a block can only write a half
// again after the next call's barrier, which every block reaches after reading
// this call's sums.
__device__ double grid_dot_finish(const LbfgsArgs &a, const Coop &cp, double part, int *parity,
                                  bool *ok) {
  double *red = a.red + (*parity) * 2 * cp.size;
  *parity ^= 1;
  part = block_sum(part);
  if (threadIdx.x == 0) red[cp.rank] = part;
  if (!cp.sync()) { *ok = false; return 0.0; }
  return block_sum_of(red, cp.size);
}

__device__ void lbfgs_two_loop(const LbfgsArgs &a, const Coop &cp) {
  const long n = a.n;
  const int m = a.m;
  const long gtid = (long)cp.rank * blockDim.x + threadIdx.x;
  const long gstride = (long)cp.size * blockDim.x;
  double *st = a.state;
  int count = (int)st[0], head = (int)st[1];
  const bool have_prev = st[2] != 0.0;
  double beta = st[3];
  bool ok = true;
  int par = 0;
  if (have_prev) {  // candidate pair into slot `head`
    double *sn = a.s + (long)head * n, *yn = a.y + (long)head * n;
    double p1 = 0.0, p2 = 0.0;
    for (long e = gtid; e < n; e += gstride) {
      double sv = a.a[e] - a.aprev[e], yv = a.g[e] - a.gprev[e];
      sn[e] = sv; yn[e] = yv;
      p1 += sv * yv; p2 += yv * yv;
    }
    double sy = grid_dot_finish(a, cp, p1, &par, &ok); if (!ok) return;
    double yy = grid_dot_finish(a, cp, p2, &par, &ok); if (!ok) return;
    if (sy > 1e-30) {
      beta = yy / sy;
      st[4 + head] = 1.0 / sy;  // rho of the slot (identical in every block)
      head = (head + 1) % m;
      count = count < m ? count + 1 : m;
    }
  }
  for (long e = gtid; e < n; e += gstride) {
    a.aprev[e] = a.a[e];
    a.gprev[e] = a.g[e];
    a.q[e] = a.g[e];
  }
  // first loop: newest to oldest
  double alph[16];
  for (int c = 0; c < count; ++c) {
    int slot = (head - 1 - c + 2 * m) % m;
    const double *sv = a.s + (long)slot * n, *yv = a.y + (long)slot * n;
    double part = 0.0;
    for (long e = gtid; e < n; e += gstride) part += sv[e] * a.q[e];
    double sq = grid_dot_finish(a, cp, part, &par, &ok); if (!ok) return;
    double al = st[4 + slot] * sq;
    alph[c] = al;
    for (long e = gtid; e < n; e += gstride) a.q[e] -= al * yv[e];
  }
  // r = H0 q
  for (long e = gtid; e < n; e += gstride)
    a.q[e] *= precond_of(a, e, beta);
  // second loop: oldest to newest
  for (int c = count - 1; c >= 0; --c) {
    int slot = (head - 1 - c + 2 * m) % m;
    const double *sv = a.s + (long)slot * n, *yv = a.y + (long)slot * n;
    double part = 0.0;
    for (long e = gtid; e < n; e += gstride) part += yv[e] * a.q[e];
    double yr = grid_dot_finish(a, cp, part, &par, &ok); if (!ok) return;
    double be = st[4 + slot] * yr;
    double coef = alph[c] - be;
    for (long e = gtid; e < n; e += gstride) a.q[e] += coef * sv[e];
  }
  for (long e = gtid; e < n; e += gstride) a.p[e] = -a.q[e];
  if (!cp.sync()) return;
  if (gtid == 0) {
    st[0] = count; st[1] = head; st[2] = 1.0; st[3] = beta;
  }
}

__global__ void __launch_bounds__(256) lbfgs_kernel(LbfgsArgs a) {
  lbfgs_two_loop(a, grid_coop(a.bar, a.flags));
}

// Batched: block b runs the two-loop of systems b, b + gridDim, ... whose dir
// flag is set, each on this block alone; reset[i] first erases the system's
// memory (no pairs, no previous point; beta kept), as after a direction that
// was not a descent direction.
__global__ void __launch_bounds__(256) lbfgs_batch_kernel(const LbfgsArgs *av, const int *dir,
                                                          const int *reset, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    if (!dir[i]) continue;
    const LbfgsArgs &a = av[i];
    __syncthreads();  // the previous system's reads of its state are done
    if (reset[i] && threadIdx.x == 0) {
      a.state[0] = 0.0;
      a.state[1] = 0.0;
      a.state[2] = 0.0;
    }
    __syncthreads();
    lbfgs_two_loop(a, block_coop());
  }
}

// The same two-loop when every thread of the grid owns at most kLbPer
// elements (every system up to water32, spread over all SMs: the FP64 work
// per SM stays small) and m <= kLbMaxM: the elements of a, g, the previous
// point and the stored pairs are loaded once into registers, all loads in
// flight together, so the loops wait on no global memory, and the two dot
// products of a new pair share one grid barrier.
constexpr int kLbPer = 2, kLbMaxM = 6;

// Two dot products of the whole grid in one barrier (every block gets both).
__device__ double2 grid_dot2_finish(LbfgsArgs &a, double p1, double p2, int *parity, bool *ok) {
  double *red = a.red + (*parity) * 2 * gridDim.x;
  *parity ^= 1;
  p1 = block_sum(p1);
  p2 = block_sum(p2);
  if (threadIdx.x == 0) { red[blockIdx.x] = p1; red[gridDim.x + blockIdx.x] = p2; }
  if (!grid_barrier(a.bar, a.flags)) { *ok = false; return make_double2(0.0, 0.0); }
  const double r1 = block_sum_of(red, gridDim.x);
  return make_double2(r1, block_sum_of(red + gridDim.x, gridDim.x));
}

__global__ void __launch_bounds__(256) lbfgs_reg_kernel(LbfgsArgs a) {
  const long n = a.n;
  const int m = a.m;
  const long gtid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long gstride = (long)gridDim.x * blockDim.x;
  const double *st = a.state;
  int count = (int)st[0], head = (int)st[1];
  const bool have_prev = st[2] != 0.0;
  double beta = st[3];
  double rho[kLbMaxM], alph[kLbMaxM];
  for (int k = 0; k < m; ++k) rho[k] = st[4 + k];
  long e[kLbPer];
  bool in[kLbPer];
  double q[kLbPer], sv[kLbMaxM][kLbPer], yv[kLbMaxM][kLbPer];
#pragma unroll
  for (int u = 0; u < kLbPer; ++u) {
    e[u] = gtid + u * gstride;
    in[u] = e[u] < n;
    q[u] = in[u] ? a.g[e[u]] : 0.0;
#pragma unroll
    for (int k = 0; k < kLbMaxM; ++k) {
      const bool use = in[u] && k < m;
      sv[k][u] = use ? a.s[(long)k * n + e[u]] : 0.0;
      yv[k][u] = use ? a.y[(long)k * n + e[u]] : 0.0;
    }
  }
  bool ok = true;
  int par = 0, new_slot = -1;
  if (have_prev) {  // candidate pair into slot `head`
    double ns[kLbPer], ny[kLbPer], p1 = 0.0, p2 = 0.0;
#pragma unroll
    for (int u = 0; u < kLbPer; ++u) {
      ns[u] = in[u] ? a.a[e[u]] - a.aprev[e[u]] : 0.0;
      ny[u] = in[u] ? q[u] - a.gprev[e[u]] : 0.0;
      p1 += ns[u] * ny[u];
      p2 += ny[u] * ny[u];
    }
    const double2 d = grid_dot2_finish(a, p1, p2, &par, &ok);
    if (!ok) return;
    if (d.x > 1e-30) {
#pragma unroll
      for (int k = 0; k < kLbMaxM; ++k)
        if (k == head) {
#pragma unroll
          for (int u = 0; u < kLbPer; ++u) {
            sv[k][u] = ns[u];
            yv[k][u] = ny[u];
            if (in[u]) { a.s[(long)k * n + e[u]] = ns[u]; a.y[(long)k * n + e[u]] = ny[u]; }
          }
        }
      beta = d.y / d.x;
      rho[head] = 1.0 / d.x;
      new_slot = head;
      head = (head + 1) % m;
      count = count < m ? count + 1 : m;
    }
  }
#pragma unroll
  for (int u = 0; u < kLbPer; ++u)
    if (in[u]) { a.aprev[e[u]] = a.a[e[u]]; a.gprev[e[u]] = q[u]; }
  for (int c = 0; c < count; ++c) {  // first loop: newest to oldest
    const int sl = (head - 1 - c + 2 * m) % m;
    double part = 0.0;
#pragma unroll
    for (int k = 0; k < kLbMaxM; ++k)
      if (k == sl) {
#pragma unroll
        for (int u = 0; u < kLbPer; ++u) part += sv[k][u] * q[u];
      }
    const double al = rho[sl] * grid_dot_finish(a, grid_coop(a.bar, a.flags), part, &par, &ok);
    if (!ok) return;
    alph[c] = al;
#pragma unroll
    for (int k = 0; k < kLbMaxM; ++k)
      if (k == sl) {
#pragma unroll
        for (int u = 0; u < kLbPer; ++u) q[u] -= al * yv[k][u];
      }
  }
#pragma unroll
  for (int u = 0; u < kLbPer; ++u)  // r = H0 q
    if (in[u]) q[u] *= precond_of(a, e[u], beta);
  for (int c = count - 1; c >= 0; --c) {  // second loop: oldest to newest
    const int sl = (head - 1 - c + 2 * m) % m;
    double part = 0.0;
#pragma unroll
    for (int k = 0; k < kLbMaxM; ++k)
      if (k == sl) {
#pragma unroll
        for (int u = 0; u < kLbPer; ++u) part += yv[k][u] * q[u];
      }
    const double coef = alph[c] - rho[sl] * grid_dot_finish(a, grid_coop(a.bar, a.flags), part, &par, &ok);
    if (!ok) return;
#pragma unroll
    for (int k = 0; k < kLbMaxM; ++k)
      if (k == sl) {
#pragma unroll
        for (int u = 0; u < kLbPer; ++u) q[u] += coef * sv[k][u];
      }
  }
#pragma unroll
  for (int u = 0; u < kLbPer; ++u)
    if (in[u]) a.p[e[u]] = -q[u];
  if (!grid_barrier(a.bar, a.flags)) return;  // every block has read the state
  if (gtid == 0) {
    double *stw = a.state;
    stw[0] = count; stw[1] = head; stw[2] = 1.0; stw[3] = beta;
    if (new_slot >= 0) stw[4 + new_slot] = rho[new_slot];
  }
}

__global__ void precond_kernel(LbfgsArgs a, const double *g, double *pg) {
  const double beta = a.state[3];
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < a.n;
       e += (long)gridDim.x * blockDim.x)
    pg[e] = precond_of(a, e, beta) * g[e];
}

// Dot product of the line-search scalars in two deterministic stages: each
// block sums a fixed grid-stride share, then one block adds the partials in
// index order.
__global__ void __launch_bounds__(256) dot_part_kernel(const double *x, const double *y, long n,
                                                       double *part) {
  double s = 0.0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    s += x[e] * y[e];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void __launch_bounds__(kDotBlocks) dot_final_kernel(const double *part, int nb, double *out) {
  double s = (int)threadIdx.x < nb ? part[threadIdx.x] : 0.0;
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void axpy_kernel(const double *x, double alpha, const double *p, double *out,
                            long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    out[e] = x[e] + alpha * p[e];
}

__global__ void permute_cols_kernel(const double *src, const int *perm, double *dst, int M) {
  long MM = (long)M * M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MM;
       e += (long)gridDim.x * blockDim.x) {
    int r = (int)(e / M), c = (int)(e % M);
    dst[e] = src[(long)r * M + perm[c]];
  }
}

// out[j] = sum_{m,n} C[m][j] Hm[m][n] C[n][j]
__global__ void __launch_bounds__(256) diag_quad_kernel(const double *C, const double *Hm,
                                                        double *out, int M) {
  int j = blockIdx.x;
  double s = 0.0;
  for (long e = threadIdx.x; e < (long)M * M; e += blockDim.x) {
    int r = (int)(e / M), c = (int)(e % M);
    s += C[(long)r * M + j] * Hm[e] * C[(long)c * M + j];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) out[j] = s;
}

__global__ void ns_prep_kernel(const double *S, double *Y, double *Zm, double c, int M) {
  long MM = (long)M * M;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MM;
       e += (long)gridDim.x * blockDim.x) {
    int r = (int)(e / M), q = (int)(e % M);
    Y[e] = S[e] / c;
    Zm[e] = (r == q) ? 1.0 : 0.0;
  }
}

__global__ void __launch_bounds__(1024) resid_kernel(const double *ZY, double *out, int M) {
  double mx = 0.0;
  for (long e = threadIdx.x; e < (long)M * M; e += blockDim.x) {
    int r = (int)(e / M), q = (int)(e % M);
    double d = fabs(ZY[e] - (r == q ? 1.0 : 0.0));
    if (!(d <= mx)) mx = d;  // NaN propagates
  }
  __shared__ double red[1024];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double o = red[threadIdx.x + s];
      if (!(o <= red[threadIdx.x])) red[threadIdx.x] = o;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void __launch_bounds__(1024) max_rowsum_kernel(const double *S, double *out, int M) {
  double mx = 0.0;
  for (int r = threadIdx.x; r < M; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < M; ++c) s += fabs(S[(long)r * M + c]);
    mx = fmax(mx, s);
  }
  __shared__ double red[1024];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void scale_copy_kernel(const double *src, double *dst, double c, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    dst[e] = c * src[e];
}

// ---- host wrappers ----------------------------------------------------------

// The mixed path's evaluations run the chains on float pairs; the set-up
// evaluation and the FP64 path on FP64.
static bool dense_pairs(const etdm_handle *h) {
  return h->precision == ETDM_PREC_MIXED && !h->in_setup;
}

DenseArgs dense_args(etdm_handle *h, const double *a) {
  DenseArgs d{};
  const bool pairs = dense_pairs(h);
  d.M = h->M; d.N = h->N; d.V = h->V;
  d.A = a;
  d.Af = pairs ? reinterpret_cast<double *>(h->d_Af) : nullptr;
  d.P = h->d_P; d.Qk = h->d_Qk; d.Kt = h->d_Kt; d.St = h->d_St;
  d.Uocc = h->d_Uocc; d.O = h->d_O; d.D = h->d_D; d.H = h->d_H; d.TO = h->d_TO;
  d.C0 = pairs ? (const void *)h->d_C0p : (const void *)h->d_C0;
  d.T = pairs ? (const void *)h->d_Tp : (const void *)h->d_T;
  d.Gbar = h->d_Gbar; d.Ubar = h->d_Ubar;
  d.Kbar[0] = h->d_bar2[0]; d.Kbar[1] = h->d_bar2[1];
  d.Sbar[0] = h->d_bar2[2]; d.Sbar[1] = h->d_bar2[3];
  d.Abar = h->d_Abar; d.Wr = h->d_Wr;
  d.eterms = h->d_eterms;
  d.gridpart = h->d_gridpart; d.n_gridpart = h->n_gridpart;
  if (pairs) { d.Vacc = h->d_Vfin; d.dO = h->d_dO; }
  d.tc_asl = h->d_tc_asl; d.tc_bsl = h->d_tc_bsl;
  d.tc_rexp = h->d_tc_rexp; d.tc_cexp = h->d_tc_cexp;
  d.tc_min_work = h->tc_min_work;
  d.red = h->d_red; d.flags = h->d_flags; d.bar = h->d_bar; d.scal = h->d_scal;
  // c_k = (-1)^k/(2k)!, s_k = (-1)^k/(2k+1)!
  double f = 1.0;
  d.ck[0] = 0.0; d.sk[0] = 1.0;
  for (int k = 1; k <= kTaylor; ++k) {
    double f2k = f * (2 * k);                 // (2k)!  (f = (2k-1)!)
    double f2k1 = f2k * (2 * k + 1);          // (2k+1)!
    double sg = (k % 2) ? -1.0 : 1.0;
    d.ck[k] = sg / f2k;
    d.sk[k] = sg / f2k1;
    f = f2k1;
  }
  return d;
}

cudaError_t launch_dense_forward(etdm_handle *h, const double *a, cudaStream_t s) {
  DenseArgs d = dense_args(h, a);
  void *args[] = {&d};
  h->pairs_last = dense_pairs(h);
  if (dense_pairs(h) && h->dense_tc)
    return cudaLaunchCooperativeKernel((const void *)dense_forward_tc_kernel, dim3(h->coop_blocks),
                                       dim3(NT), args, kGDyn, s);
  const void *fn = dense_pairs(h) ? (const void *)dense_forward_kernel<float2>
                                  : (const void *)dense_forward_kernel<double>;
  return cudaLaunchCooperativeKernel(fn, dim3(h->coop_blocks), dim3(NT), args, 0, s);
}

cudaError_t launch_dense_reverse(etdm_handle *h, const double *a, double *g, double *E,
                                 cudaStream_t s) {
  DenseArgs d = dense_args(h, a);
  d.g = g; d.E = E;
  d.resid = (h->want_resid && g) ? h->d_dot + 3 : nullptr;  // Eq. 45 with the energy
  int want = g != nullptr;
  void *args[] = {&d, &want};
  if (dense_pairs(h) && h->dense_tc)
    return cudaLaunchCooperativeKernel((const void *)dense_reverse_tc_kernel, dim3(h->coop_blocks),
                                       dim3(NT), args, kGDyn, s);
  const void *fn = dense_pairs(h) ? (const void *)dense_reverse_kernel<float2>
                                  : (const void *)dense_reverse_kernel<double>;
  return cudaLaunchCooperativeKernel(fn, dim3(h->coop_blocks), dim3(NT), args, 0, s);
}

__global__ void to_pairs_kernel(const double *src, float2 *dst, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    dst[e] = pair::split(src[e]);
}
__global__ void from_pairs_kernel(const float2 *src, double *dst, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    dst[e] = pair::to_double(src[e]);
}

cudaError_t launch_to_pairs(const double *src, float2 *dst, long n, cudaStream_t s) {
  to_pairs_kernel<<<(int)std::min<long>((n + 255) / 256, 1024), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}
cudaError_t launch_from_pairs(const float2 *src, double *dst, long n, cudaStream_t s) {
  from_pairs_kernel<<<(int)std::min<long>((n + 255) / 256, 1024), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_gemm(const Phase &ph, cudaStream_t s) {
  int tiles = ((ph.m + BM - 1) / BM) * ((ph.n + BN - 1) / BN);
  if (tiles <= 0) return cudaSuccess;
  gemm_kernel<<<tiles, NT, 0, s>>>(ph);
  return cudaGetLastError();
}

cudaError_t launch_lbfgs(etdm_handle *h, const double *a, const double *g, double *p,
                         cudaStream_t s) {
  LbfgsArgs d = lbfgs_args(h, a, g, p);
  void *args[] = {&d};
  if (d.n <= (long)h->lb_blocks * 256 * kLbPer && d.m <= kLbMaxM)  // registers hold every element
    return cudaLaunchCooperativeKernel((void *)lbfgs_reg_kernel, dim3(h->lb_blocks), dim3(256), args,
                                       0, s);
  return cudaLaunchCooperativeKernel((void *)lbfgs_kernel, dim3(h->lb_blocks), dim3(256), args,
                                     0, s);
}

cudaError_t launch_precond(etdm_handle *h, const double *g, double *pg, cudaStream_t s) {
  const LbfgsArgs d = lbfgs_args(h, nullptr, g, pg);
  int blocks = (int)((d.n + 255) / 256);
  if (blocks > 4 * h->num_sms) blocks = 4 * h->num_sms;
  if (blocks < 1) blocks = 1;
  precond_kernel<<<blocks, 256, 0, s>>>(d, g, pg);
  return cudaGetLastError();
}

cudaError_t launch_dot(const double *x, const double *y, long n, double *out, double *part,
                       cudaStream_t s) {
  const int nb = (int)std::max(1L, std::min<long>(kDotBlocks, (n + 255) / 256));
  dot_part_kernel<<<nb, 256, 0, s>>>(x, y, n, part);
  dot_final_kernel<<<1, kDotBlocks, 0, s>>>(part, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_axpy(const double *x, double alpha, const double *p, double *out, long n,
                        cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  axpy_kernel<<<blocks, 256, 0, s>>>(x, alpha, p, out, n);
  return cudaGetLastError();
}

cudaError_t launch_permute_cols(const double *src, const int *perm, double *dst, int M,
                                cudaStream_t s) {
  permute_cols_kernel<<<256, 256, 0, s>>>(src, perm, dst, M);
  return cudaGetLastError();
}

cudaError_t launch_diag_quad(const double *C, const double *Hm, double *out, int M,
                             cudaStream_t s) {
  diag_quad_kernel<<<M, 256, 0, s>>>(C, Hm, out, M);
  return cudaGetLastError();
}

cudaError_t launch_ns_prep(const double *S, double *Y, double *Zm, double c, int M,
                           cudaStream_t s) {
  ns_prep_kernel<<<256, 256, 0, s>>>(S, Y, Zm, c, M);
  return cudaGetLastError();
}

cudaError_t launch_resid(const double *ZY, double *out, int M, cudaStream_t s) {
  resid_kernel<<<1, 1024, 0, s>>>(ZY, out, M);
  return cudaGetLastError();
}

cudaError_t launch_max_rowsum(const double *S, double *out, int M, cudaStream_t s) {
  max_rowsum_kernel<<<1, 1024, 0, s>>>(S, out, M);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(const double *src, double *dst, double c, long n,
                              cudaStream_t s) {
  scale_copy_kernel<<<256, 256, 0, s>>>(src, dst, c, n);
  return cudaGetLastError();
}

LbfgsArgs lbfgs_args(etdm_handle *h, const double *a, const double *g, double *p) {
  LbfgsArgs d{};
  d.n = h->nvar; d.N = h->N; d.V = h->V; d.m = h->lbfgs_m;
  d.a = a; d.g = g; d.p = p;
  d.pden = h->d_kpden; d.pw = h->d_kpw;
  d.s = h->d_s; d.y = h->d_y; d.aprev = h->d_aprev; d.gprev = h->d_gprev; d.q = h->d_q;
  d.state = h->d_lbstate; d.eps = h->d_eps; d.gamma = h->gamma;
  d.red = h->d_red; d.bar = h->d_bar; d.flags = h->d_flags;
  return d;
}

cudaError_t launch_dense_batch(const DenseArgs *av, const int *order, int n, const int *active,
                               int grid, bool pairs, bool reverse, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (reverse) {
    if (pairs) dense_reverse_batch_kernel<float2><<<grid, NT, 0, s>>>(av, order, n, active);
    else dense_reverse_batch_kernel<double><<<grid, NT, 0, s>>>(av, order, n, active);
  } else {
    if (pairs) dense_forward_batch_kernel<float2><<<grid, NT, 0, s>>>(av, order, n, active);
    else dense_forward_batch_kernel<double><<<grid, NT, 0, s>>>(av, order, n, active);
  }
  return cudaGetLastError();
}

cudaError_t launch_lbfgs_batch(const LbfgsArgs *av, const int *dir, const int *reset, int n,
                               int grid, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  lbfgs_batch_kernel<<<grid, 256, 0, s>>>(av, dir, reset, n);
  return cudaGetLastError();
}

int occupancy_dense(int *bps) {
  const void *fns[4] = {(const void *)dense_forward_kernel<double>, (const void *)dense_reverse_kernel<double>,
                        (const void *)dense_forward_kernel<float2>, (const void *)dense_reverse_kernel<float2>};
  int best = 1 << 30;
  for (const void *f : fns) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, NT, 0) != cudaSuccess) return -1;
    best = std::min(best, b);
  }
  *bps = best;
  return 0;
}

int occupancy_dense_tc(int *bps) {
  const void *fns[2] = {(const void *)dense_forward_tc_kernel, (const void *)dense_reverse_tc_kernel};
  int best = 1 << 30;
  for (const void *f : fns) {
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kGDyn) != cudaSuccess)
      return -1;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, NT, kGDyn) != cudaSuccess) return -1;
    best = std::min(best, b);
  }
  *bps = best;
  return 0;
}

cudaError_t launch_pair_gemm(const double *A, const double *B, double *C, int m, int n, int k,
                             int ta, int tb, uint8_t *asl, uint8_t *bsl, int *rexp, int *cexp,
                             unsigned *bar, int *flags, int blocks, cudaStream_t s) {
  Phase ph{};
  ph.m = m; ph.n = n; ph.k = k; ph.np = 1;
  ph.p[0] = Prod{A, B, ta ? m : k, tb ? k : n, ta, tb, 1.0, 3};
  ph.out = C; ph.ldo = n; ph.out64 = 1;
  DenseArgs d{};
  d.tc_asl = asl; d.tc_bsl = bsl; d.tc_rexp = rexp; d.tc_cexp = cexp;
  d.bar = bar; d.flags = flags;
  void *args[] = {&ph, &d};
  cudaError_t e = cudaFuncSetAttribute((const void *)pair_gemm_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kGDyn);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void *)pair_gemm_kernel, dim3(blocks), dim3(NT), args,
                                     kGDyn, s);
}

size_t dense_tc_asl_bytes(long M) { return (size_t)kGS * gpad(M, 128) * gpad(M, 16) * 2; }
size_t dense_tc_bsl_bytes(long M) { return (size_t)kGS * gpad(M, kGN) * gpad(M, 16) * 2; }

int occupancy_lbfgs(int *bps) {
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, lbfgs_kernel, 256, 0) != cudaSuccess)
    return -1;
  return 0;
}

}  // namespace etdm
