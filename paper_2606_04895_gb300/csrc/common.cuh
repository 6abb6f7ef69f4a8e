// common.cuh -- device-side types shared by the sampling kernels of libbst.
//
// Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Every draw is keyed
// by (seed) and addressed by the counter (chain, iteration, purpose, block), so
// a chain's stream does not depend on how chains are tiled or how many steps a
// launch takes.  Uniforms are ((x >> 8) + 1/2) 2^-24 (open interval, exact in
// float), normals come from Box-Muller on consecutive uniform pairs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bst.h"  // include/ is on the include path

namespace bst {

constexpr int kMaxD = 32;          // largest parameter dimension
constexpr int kMaxDepthNuts = 10;  // largest NUTS depth
constexpr double kNutsDeltaMax = 1000.0;

// Third word of the Philox counter.
enum Purpose : uint32_t {
  kXi = 1,           // proposal noise / momentum
  kAccept = 2,       // Metropolis uniform / NUTS slice variable
  kNutsDir = 3,      // doubling direction
  kNutsSel = 4,      // in-subtree merge
  kNutsTop = 5,      // top-level progressive selection
  kAiesPartner = 6,  // partner walker
  kAiesZ = 7         // stretch factor
};

// Launch modes of the chain-tile kernels.
enum Mode : int {
  kModeMH = BST_MH,
  kModeMALA = BST_MALA,
  kModeHMC = BST_HMC,
  kModeNUTS = BST_NUTS,
  kModeAIES = BST_AIES,
  kModeLoglike = 16,  // external theta rows -> logL (+ grad)
  kModeRefresh = 17   // chain state z -> log pi, grad (after init / adaptation)
};

// Device status bits.
enum StatusBits : int { kStatusTimeout = 1, kStatusBadArg = 2 };

struct Philox {
  static __device__ __forceinline__ void block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, uint32_t out[4]) {
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
      const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
      const uint32_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
      x0 = n0;
      x1 = lo1;
      x2 = n2;
      x3 = lo0;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
  }
};

template <typename R>
__device__ __forceinline__ R u01(uint32_t x) {
  return (static_cast<R>(x >> 8) + R(0.5)) * R(1.0 / 16777216.0);
}

// Uniform number idx of stream (chain, iter, purpose): word idx % 4 of block idx / 4.
template <typename R>
__device__ __forceinline__ R draw_uniform(uint64_t seed, uint32_t chain, uint32_t iter,
                                          uint32_t purpose, uint32_t idx) {
  uint32_t w[4];
  Philox::block(seed, chain, iter, purpose, idx >> 2, w);
  return u01<R>(w[idx & 3u]);
}

__device__ __forceinline__ void box_muller(float u0, float u1, float &a, float &b) {
  const float r = sqrtf(-2.0f * logf(u0));
  float s, c;
  sincospif(2.0f * u1, &s, &c);
  a = r * c;
  b = r * s;
}
__device__ __forceinline__ void box_muller(double u0, double u1, double &a, double &b) {
  const double r = sqrt(-2.0 * log(u0));
  double s, c;
  sincospi(2.0 * u1, &s, &c);
  a = r * c;
  b = r * s;
}

// Normals k = 0..n-1 of stream (chain, iter, purpose); normal k comes from block k / 4.
template <typename R>
__device__ __forceinline__ void draw_normals(uint64_t seed, uint32_t chain, uint32_t iter,
                                             uint32_t purpose, int n, R *out) {
  for (int b = 0; 4 * b < n; ++b) {
    uint32_t w[4];
    Philox::block(seed, chain, iter, purpose, static_cast<uint32_t>(b), w);
    R v[4];
    box_muller(u01<R>(w[0]), u01<R>(w[1]), v[0], v[1]);
    box_muller(u01<R>(w[2]), u01<R>(w[3]), v[2], v[3]);
    for (int k = 0; k < 4 && 4 * b + k < n; ++k) out[4 * b + k] = v[k];
  }
}

// Whitening (x = mu + L z) and prior (box, N(0,1) on flagged dims), device view.  The
// values are copied into the kernel parameters (the step kernels take their StepArgs as a
// __grid_constant__ parameter), so every thread reads them through the constant cache.
template <typename R>
struct TargetView {
  int d;
  double logdet;   // sum_i log L_ii
  int any_gauss;
  R mu[kMaxD];          // [d]
  R L[kMaxD * kMaxD];   // [d][d] row-major (first d*d entries), lower triangular
  R lower[kMaxD];       // [d]
  R upper[kMaxD];       // [d]
  int gauss[kMaxD];     // [d]

  // x = mu + L z; returns the log prior (0 / -inf / -x_g.x_g/2).
  // (z is read once into registers: the triangular product is unrolled over kMaxD with the
  // same summation order as a plain loop over j <= i)
  __device__ __noinline__ double to_x_prior(const R *z, R *x) const {
    R zr[kMaxD];
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) zr[j] = j < d ? z[j] : R(0);
    bool inside = true;
    double lp = 0.0;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
      if (i < d) {
        R s = mu[i];
#pragma unroll
        for (int j = 0; j <= i; ++j) s += L[i * d + j] * zr[j];
        x[i] = s;
        if (!(s >= lower[i] && s <= upper[i])) inside = false;
        if (any_gauss && gauss[i]) lp -= 0.5 * static_cast<double>(s) * static_cast<double>(s);
      }
    }
    return inside ? lp : -INFINITY;
  }
  // g += L^T (-x on Gaussian dims)
  __device__ __forceinline__ void add_prior_grad(const R *x, R *g) const {
    if (!any_gauss) return;
    for (int j = 0; j < d; ++j) {
      R s = 0;
      for (int i = j; i < d; ++i)
        if (gauss[i]) s -= L[i * d + j] * x[i];
      g[j] += s;
    }
  }
};

// Persistent per-chain state plus the per-row evaluation buffers.
template <typename R>
struct ChainState {
  R *z;    // [n_chains][dp] whitened position
  R *g;    // [n_chains][dp] grad log pi_z
  R *lp;   // [n_chains]     log pi_z
  uint32_t *iter;
  double *acc_stat;
  unsigned long long *accepts, *evals, *divs;
  R *ze;   // [n_rows][ze_ld] point to evaluate (z-space, or x-space in loglike mode)
  R *lle;  // [n_rows]        logL at ze
  R *gle;  // [n_rows][gle_ld] grad of logL at ze (w.r.t. ze)
  int ze_ld, gle_ld;
  R *work;         // [n_chains][work_stride] per-kernel temporaries
  int work_stride;
  int *steps_done;  // [n_chains] iterations completed in this launch
};

template <typename R>
struct StepArgs {
  int mode;
  int n_chains, n_rows, d, dp;
  double eps;
  int n_leapfrog, n_steps, max_depth, aies_walkers, thin;
  double aies_a;
  uint64_t seed;
  int need_grad;
  TargetView<R> tgt;
  ChainState<R> st;
  R *samples;  // [n_steps / thin][n_chains][d] x-space, or nullptr
  // loglike mode
  const R *ext_in;
  R *ext_logl, *ext_grad;
  // Welford (covariance adaptation, FP64 tile accumulators)
  int welford_on;
  double *wf;       // [n_tiles][wf_stride]
  int wf_stride;
  R *xbuf;          // [n_rows][dp]
  int *status;
};

// Per-chain work row: kDworkOffsetVecs vectors of dp reals (NUTS trajectory ends,
// selected point, per-level pending subtrees), then kDworkDoubles doubles.
constexpr int kDworkOffsetVecs = 9 + 4 * kMaxDepthNuts;
constexpr int kDworkDoubles = 32;
template <typename R>
constexpr int work_stride_elems(int dp) {
  return kDworkOffsetVecs * dp + kDworkDoubles * static_cast<int>(sizeof(double) / sizeof(R));
}

// Welford tile record layout (doubles): n, mean[32], M2[32*32], batch count, batch mean[32],
// batch M2[32*32].
constexpr int kWfN = 0, kWfMean = 1, kWfM2 = 33, kWfBn = 33 + 1024, kWfBMean = kWfBn + 1,
              kWfBM2 = kWfBMean + 32, kWfStride = kWfBM2 + 1024;

__device__ __forceinline__ void set_status(int *status, int bits) {
  if (status) atomicOr(status, bits);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace bst
