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
#include <cuda_fp16.h>
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
  // (8: initial walker positions, drawn by init_positions_kernel)
};

// Launch modes of the chain-tile kernels.
enum Mode : int {
  kModeMH = BST_MH,
  kModeMALA = BST_MALA,
  kModeHMC = BST_HMC,
  kModeNUTS = BST_NUTS,
  kModeNUTS_MN = BST_NUTS_MULTINOMIAL,
  kModeAIES = BST_AIES,
  kModeAIES_DE = BST_AIES_DE,
  kModeLoglike = 16,  // external theta rows -> logL (+ grad)
  kModeRefresh = 17   // chain state z -> log pi, grad (after init / adaptation)
};

// Device status bits.
enum StatusBits : int { kStatusTimeout = 1, kStatusBadArg = 2 };

// The ensemble moves (stretch and differential evolution) share the walker layout and the
// alternation of halves.
__host__ __device__ constexpr bool is_ensemble_mode(int mode) { return mode == kModeAIES || mode == kModeAIES_DE; }
// The two NUTS variants share the tree machine.
__host__ __device__ constexpr bool is_nuts_mode(int mode) { return mode == kModeNUTS || mode == kModeNUTS_MN; }

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
// Entries beyond d are zero (mu, L, bounds, flags), so loops unrolled past d add exact zeros.
template <typename R>
struct TargetView {
  int d;
  double logdet;   // sum_i log L_ii
  int any_gauss;
  R mu[kMaxD];          // [d]
  R L[kMaxD * kMaxD];   // L_ij at i * kMaxD + j, lower triangular
  R lower[kMaxD];       // [d]
  R upper[kMaxD];       // [d]
  int gauss[kMaxD];     // [d]
  // smooth bounds (Sec. 3.1): pen_iw[i] = 1 / w_i > 0 replaces dim i's hard box by the factor
  // exp(-r_i^2 / 2), r_i = (x_i - clamp(x_i, lower_i, upper_i)) / w_i
  int any_pen;
  R pen_iw[kMaxD];

  // x = mu + L z over DM >= d entries; returns the log prior (0 / -inf outside the box /
  // -x_g.x_g / 2 over the flagged dims, minus r.r / 2 over the dims with a smooth bound, as four
  // partial sums of R added in FP64).  XOUT stores x (DM entries); with grad,
  // g[j] -= sum_{i >= j} L_ij p_i with p_i = x_i (Gaussian dims) + r_i / w_i (smooth bounds): the
  // gradient of the prior terms through x = mu + L z, Algorithm 1.  Fully unrolled, so every element of mu and
  // L is a constant-bank operand of its FMA.  x is accumulated column by column (z_j streamed,
  // each x_i still summed over j in ascending order) and the gradient row by row, so about DM
  // values are live at a time.
  template <int DM, bool XOUT, class VZ, class VG>
  __device__ __forceinline__ double eval(VZ z, R *x, VG g, bool grad) const {
    R xs[DM];
#pragma unroll
    for (int i = 0; i < DM; ++i) xs[i] = mu[i];
#pragma unroll
    for (int j = 0; j < DM; ++j) {
      const R zj = j < d ? static_cast<R>(z[j]) : R(0);
#pragma unroll
      for (int i = j; i < DM; ++i) xs[i] += L[i * kMaxD + j] * zj;
    }
    R part[4] = {R(0), R(0), R(0), R(0)};
    bool inside = true;
#pragma unroll
    for (int i = 0; i < DM; ++i) {
      if (XOUT) x[i] = xs[i];
      const bool pen = any_pen && pen_iw[i] > R(0);
      if (i < d && !pen && !(xs[i] >= lower[i] && xs[i] <= upper[i])) inside = false;
      R p = gauss[i] ? xs[i] : R(0);
      R q = p * p;
      if (pen) {
        const R out = xs[i] < lower[i] ? xs[i] - lower[i] : (xs[i] > upper[i] ? xs[i] - upper[i] : R(0));
        const R r = out * pen_iw[i];
        q += r * r;
        p += r * pen_iw[i];
      }
      xs[i] = p;
      part[i & 3] += q;
    }
    if (grad && (any_gauss || any_pen)) {
#pragma unroll
      for (int j = 0; j < DM; ++j) {
        R sg = R(0);
#pragma unroll
        for (int i = j; i < DM; ++i) sg += L[i * kMaxD + j] * xs[i];
        if (j < d) g[j] -= sg;
      }
    }
    const double lp = -0.5 * ((static_cast<double>(part[0]) + static_cast<double>(part[1])) +
                              (static_cast<double>(part[2]) + static_cast<double>(part[3])));
    return inside ? lp : -INFINITY;
  }
  // The same quantities with loops over d (FP64 state, where the loop overhead is small next
  // to the arithmetic); the prior is summed in order.
  template <bool XOUT, class VZ, class VG>
  __device__ __forceinline__ double eval_loop(VZ z, R *x, VG g, bool grad) const {
    R xg[kMaxD];
    bool inside = true;
    double lp = 0.0;
    for (int i = 0; i < d; ++i) {
      R s = mu[i];
      for (int j = 0; j <= i; ++j) s += L[i * kMaxD + j] * z[j];
      if (XOUT) x[i] = s;
      const bool pen = any_pen && pen_iw[i] > R(0);
      if (!pen && !(s >= lower[i] && s <= upper[i])) inside = false;
      xg[i] = gauss[i] ? s : R(0);
      lp -= 0.5 * static_cast<double>(xg[i]) * static_cast<double>(xg[i]);
      if (pen) {
        const R out = s < lower[i] ? s - lower[i] : (s > upper[i] ? s - upper[i] : R(0));
        const R r = out * pen_iw[i];
        lp -= 0.5 * static_cast<double>(r) * static_cast<double>(r);
        xg[i] += r * pen_iw[i];
      }
    }
    if (grad && (any_gauss || any_pen))
      for (int j = 0; j < d; ++j) {
        R sg = R(0);
        for (int i = j; i < d; ++i) sg += L[i * kMaxD + j] * xg[i];
        g[j] -= sg;
      }
    return inside ? lp : -INFINITY;
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
  // Point to evaluate (z-space, or x-space in loglike mode) and grad of logL there (w.r.t. ze):
  // with ld > 0 row-major [n_rows][ld] (a caller's theta rows), with ld == 0 chain-blocked with
  // dp elements per row (row_off / row_es below).
  R *ze;
  R *lle;  // [n_rows] logL at ze
  R *gle;
  int ze_ld, gle_ld;
  // Per-chain temporaries of the general sampler code, chain-blocked: kDworkOffsetVecs vectors
  // of kMaxD reals (vector k, element i is element k * kMaxD + i), and kDworkDoubles doubles.
  R *work;
  double *dwork;
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

// Chain-blocked layout of the per-chain buffers of the general sampler code: chains in blocks
// of kChainBlock; element e (of n_e per chain) of chain c at
//     (c / kChainBlock) * kChainBlock * n_e + e * kChainBlock + c % kChainBlock,
// so the threads of a warp (consecutive chains) touch one line per element, and an element
// index known at compile time is an immediate offset.
constexpr int kChainBlock = 32;
__host__ __device__ __forceinline__ size_t blk_off(int c, int n_e) {
  return static_cast<size_t>(c / kChainBlock) * kChainBlock * static_cast<size_t>(n_e) + (c % kChainBlock);
}
__host__ __device__ __forceinline__ size_t chains_padded(int n) {
  return static_cast<size_t>((n + kChainBlock - 1) / kChainBlock) * kChainBlock;
}
// element 0 of row r of ze / gle and the element stride (ld > 0: row-major, else chain-blocked)
__device__ __forceinline__ size_t row_off(int ld, int r, int dp) {
  return ld > 0 ? static_cast<size_t>(r) * ld : blk_off(r, dp);
}
__device__ __forceinline__ int row_es(int ld) { return ld > 0 ? 1 : kChainBlock; }

// Per-chain work: kDworkOffsetVecs vectors of kMaxD reals (NUTS trajectory ends, selected point,
// per-level pending subtrees; HMC z1 q1 g1), then kDworkDoubles doubles; the buffer holds the
// vectors of all (padded) chains, then their doubles.
constexpr int kDworkOffsetVecs = 9 + 4 * kMaxDepthNuts;
constexpr int kDworkDoubles = 32;
template <typename R>
constexpr size_t work_elems_per_chain() {
  return static_cast<size_t>(kDworkOffsetVecs) * kMaxD + kDworkDoubles * (sizeof(double) / sizeof(R));
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
