// sampler.cuh -- per-chain proposal / accept state machines.
//
// A chain-tile kernel alternates
//     pre(row)   -> write the point to evaluate into ze[row]      (proposal)
//     engine     -> lle[row] = logL(ze[row]), gle[row] = grad     (emulator / analytic)
//     post(row)  -> Metropolis / Hamiltonian / tree bookkeeping    (accept)
// so one likelihood evaluation of a whole tile of chains is in flight at a
// time.  Everything here is per chain, O(d) or O(d^2), and runs on the threads
// that own the chains.  Every decision (Metropolis accept, NUTS slice, Delta_max
// and U-turn tests) is the one of the FP64 expression formed from the working-
// precision state.  With FP32 state it is first taken in FP32, with a bound on
// the FP32 rounding error of each side; only a comparison closer than its bound
// is evaluated in FP64 (FP64 arithmetic runs at a small fraction of the FP32
// rate on this part).
//
// Target in whitened coordinates (paper Sec. 2.2, Eq. (2.12), Algorithm 1):
//     x = mu + L z,   log pi_z(z) = logL(x) + log prior(x) + sum_i log L_ii.
#pragma once

#include <stddef.h>

#include "common.cuh"

namespace bst {

// A per-chain vector with its element stride S known at compile time: S = 1 for a state row,
// S = kChainBlock for the chain-blocked buffers (a warp's consecutive chains read one line per
// element; every offset within a vector is an immediate).
template <typename T, int S>
struct Vec {
  T *p;
  __device__ __forceinline__ T &operator[](int i) const { return p[i * S]; }
};
template <typename R>
using Row = Vec<R, 1>;
template <typename R>
using Blk = Vec<R, kChainBlock>;

// The vector loops run in chunks of kVc elements: a chunk is loaded before any of it is stored,
// so its loads are in flight together (the vectors may alias as far as the compiler knows).
// Accessors are Vec or a thread's array.
constexpr int kVc = 8;

template <typename R, class A>
__device__ __forceinline__ void vload(const A &v, int i0, int n, R (&t)[kVc]) {
#pragma unroll
  for (int u = 0; u < kVc; ++u)
    if (u < n) t[u] = v[i0 + u];
}
template <typename R, class A>
__device__ __forceinline__ void vstore(const A &v, int i0, int n, const R (&t)[kVc]) {
#pragma unroll
  for (int u = 0; u < kVc; ++u)
    if (u < n) v[i0 + u] = t[u];
}

template <typename R, class D, class S>
__device__ __forceinline__ void vcopy(D dst, S src, int d) {
#pragma unroll 1
  for (int i0 = 0; i0 < d; i0 += kVc) {
    const int n = min(kVc, d - i0);
    R t[kVc];
    vload(src, i0, n, t);
    vstore(dst, i0, n, t);
  }
}
template <typename R, class D0, class S0, class D1, class S1>
__device__ __forceinline__ void vcopy2(D0 d0, S0 s0, D1 d1, S1 s1, int d) {
#pragma unroll 1
  for (int i0 = 0; i0 < d; i0 += kVc) {
    const int n = min(kVc, d - i0);
    R t0[kVc], t1[kVc];
    vload(s0, i0, n, t0);
    vload(s1, i0, n, t1);
    vstore(d0, i0, n, t0);
    vstore(d1, i0, n, t1);
  }
}
// qh = qe + e/2 ge; zn = zs + e qh  (first half of a leapfrog step)
template <typename R, class QH, class ZN, class QE, class GE, class ZS>
__device__ __forceinline__ void half_kick_drift(QH qh, ZN zn, QE qe, GE ge, ZS zs, R e, int d) {
#pragma unroll 1
  for (int i0 = 0; i0 < d; i0 += kVc) {
    const int n = min(kVc, d - i0);
    R q[kVc], g[kVc], z[kVc];
    vload(qe, i0, n, q);
    vload(ge, i0, n, g);
    vload(zs, i0, n, z);
#pragma unroll
    for (int u = 0; u < kVc; ++u) {
      q[u] = q[u] + R(0.5) * e * g[u];
      z[u] = z[u] + e * q[u];
    }
    vstore(qh, i0, n, q);
    vstore(zn, i0, n, z);
  }
}
// second half: qend = qh + e/2 gn, zend = zn, gend = gn; returns |qend|^2 summed in R
template <typename R, class ZE, class QE, class GE, class QH, class ZN, class GN>
__device__ __forceinline__ R half_kick_store(ZE zend, QE qend, GE gend, QH qh, ZN zn, GN gn, R e, int d) {
  R qq = R(0);
#pragma unroll 1
  for (int i0 = 0; i0 < d; i0 += kVc) {
    const int n = min(kVc, d - i0);
    R q[kVc], z[kVc], g[kVc];
    vload(qh, i0, n, q);
    vload(zn, i0, n, z);
    vload(gn, i0, n, g);
#pragma unroll
    for (int u = 0; u < kVc; ++u) {
      q[u] = q[u] + R(0.5) * e * g[u];
      if (u < n) qq += q[u] * q[u];
    }
    vstore(zend, i0, n, z);
    vstore(qend, i0, n, q);
    vstore(gend, i0, n, g);
  }
  return qq;
}
// dst = zc + a u (+ b v)
template <typename R, class D, class ZC, class U>
__device__ __forceinline__ void vaxpy(D dst, ZC zc, R a, U u, int d) {
#pragma unroll 1
  for (int i0 = 0; i0 < d; i0 += kVc) {
    const int n = min(kVc, d - i0);
    R t[kVc], w[kVc];
    vload(zc, i0, n, t);
    vload(u, i0, n, w);
#pragma unroll
    for (int k = 0; k < kVc; ++k) t[k] = t[k] + a * w[k];
    vstore(dst, i0, n, t);
  }
}
template <typename R, class D, class ZC, class U, class V>
__device__ __forceinline__ void vaxpby(D dst, ZC zc, R a, U u, R b, V v, int d) {
#pragma unroll 1
  for (int i0 = 0; i0 < d; i0 += kVc) {
    const int n = min(kVc, d - i0);
    R t[kVc], w[kVc], x[kVc];
    vload(zc, i0, n, t);
    vload(u, i0, n, w);
    vload(v, i0, n, x);
#pragma unroll
    for (int k = 0; k < kVc; ++k) t[k] = t[k] + a * w[k] + b * x[k];
    vstore(dst, i0, n, t);
  }
}
// q1 += e/2 g1; z1 += e q1; zp = z1
template <typename R, class Z1, class Q1, class G1, class ZP>
__device__ __forceinline__ void kick_drift_inplace(Z1 z1, Q1 q1, G1 g1, ZP zp, R e, int d) {
#pragma unroll 1
  for (int i0 = 0; i0 < d; i0 += kVc) {
    const int n = min(kVc, d - i0);
    R q[kVc], g[kVc], z[kVc];
    vload(q1, i0, n, q);
    vload(g1, i0, n, g);
    vload(z1, i0, n, z);
#pragma unroll
    for (int u = 0; u < kVc; ++u) {
      q[u] = q[u] + R(0.5) * e * g[u];
      z[u] = z[u] + e * q[u];
    }
    vstore(q1, i0, n, q);
    vstore(z1, i0, n, z);
    vstore(zp, i0, n, z);
  }
}

// No U-turn between two trajectory points (Hoffman & Gelman 2014, Eq. (9) with identity mass):
// sum_i v (a_i - b_i) p_i >= 0 and sum_i v (a_i - b_i) q_i >= 0, as FP64 sums of the products of
// the working-precision values.  FP32 state: FP32 sums first, with the bound (d + 4) 2^-23 times
// the sum of |terms| on their error (twice the recursive-summation bound); a sum within its
// bound of zero sends the test to the FP64 loop.
template <typename R, class VA, class VB, class VP, class VQ>
__device__ __forceinline__ bool no_uturn(VA za, VB zb, VP p, VQ q, double v, int d) {
  if constexpr (sizeof(R) == 4) {
    const float vf = static_cast<float>(v);
    float s1 = 0.f, s2 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 1
    for (int i0 = 0; i0 < d; i0 += kVc) {
      const int n = min(kVc, d - i0);
      float A[kVc], B[kVc], P[kVc], Q[kVc];
      vload(za, i0, n, A);
      vload(zb, i0, n, B);
      vload(p, i0, n, P);
      vload(q, i0, n, Q);
#pragma unroll
      for (int u = 0; u < kVc; ++u)
        if (u < n) {
          const float dz = vf * (A[u] - B[u]);
          const float t1 = dz * P[u], t2 = dz * Q[u];
          s1 += t1;
          s2 += t2;
          a1 += fabsf(t1);
          a2 += fabsf(t2);
        }
    }
    const float k = static_cast<float>(d + 4) * 0x1p-23f;
    const float e1 = k * a1, e2 = k * a2;
    if (s1 > e1 && s2 > e2) return true;
    if (s1 < -e1 || s2 < -e2) return false;
  }
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < d; ++i) {
    const double dz = v * (static_cast<double>(za[i]) - zb[i]);
    s1 += dz * p[i];
    s2 += dz * q[i];
  }
  return s1 >= 0.0 && s2 >= 0.0;
}

// log(exp(a) + exp(b)) without overflow: max + log1p(exp(min - max)); -inf when both are.
__device__ __forceinline__ double log_add_exp(double a, double b) {
  const double hi = a > b ? a : b, lo = a > b ? b : a;
  if (hi == -INFINITY) return -INFINITY;
  return hi + log1p(exp(lo - hi));
}

// U: unrolled whitening / prior for FP32 state (the tcgen05 kernel); the CUDA-core kernel,
// whose time is all in its emulator GEMMs, takes the loop form, which needs far fewer registers.
template <typename R, bool U = true>
struct Chain {
  // FP32 state: FP32-first decisions (see the header)
  static constexpr bool kF32 = sizeof(R) == 4;
  const StepArgs<R> &a;
  __device__ Chain(const StepArgs<R> &args) : a(args) {}

  // state rows (row-major), then the chain-blocked evaluation rows and work buffers
  __device__ Row<R> z(int c) const { return Row<R>{a.st.z + static_cast<size_t>(c) * a.dp}; }
  __device__ Row<R> g(int c) const { return Row<R>{a.st.g + static_cast<size_t>(c) * a.dp}; }
  __device__ Blk<R> ze(int r) const { return Blk<R>{a.st.ze + blk_off(r, a.dp)}; }
  __device__ Blk<R> gle(int r) const { return Blk<R>{a.st.gle + blk_off(r, a.dp)}; }
  __device__ Blk<R> wv(int c, int k) const {
    return Blk<R>{a.st.work + blk_off(c, kDworkOffsetVecs * kMaxD) + k * (kMaxD * kChainBlock)};
  }
  __device__ Blk<double> dw(int c) const { return Blk<double>{a.st.dwork + blk_off(c, kDworkDoubles)}; }

  static __device__ double accept_prob(double la) {
    if (!(la == la)) return 0.0;
    return la >= 0.0 ? 1.0 : exp(la);
  }
  // min(1, alpha) from an FP32 log alpha: the acceptance statistic, which only feeds step-size
  // adaptation
  static __device__ float accept_prob32(float la) { return la >= 0.f ? 1.f : (la == la ? expf(la) : 0.f); }

  // x = mu + L z, log prior and its gradient: FP32 state TargetView::eval unrolled to 8 or
  // kMaxD entries (constant-bank operands), FP64 state plain loops over d
  // (TargetView::eval_loop).  (Each kernel has two call sites: log pi in post(), the x-space
  // record in finish().)
  template <bool XOUT, class VZ, class VG>
  __device__ __forceinline__ double prior(VZ zv, R *x, VG gadd, bool grad) const {
    if constexpr (kF32 && U) {
      if (a.d <= 8) return a.tgt.template eval<8, XOUT>(zv, x, gadd, grad);
      return a.tgt.template eval<kMaxD, XOUT>(zv, x, gadd, grad);
    } else {
      return a.tgt.template eval_loop<XOUT>(zv, x, gadd, grad);
    }
  }

  // x-space sample record and Welford hand-off after a chain finishes an iteration.
  __device__ void record(int c, int row, int step) const {
    const bool smp = a.samples && ((step + 1) % a.thin) == 0;
    if (!smp && !a.welford_on) return;
    const int d = a.d;
    R x[kMaxD];
    prior<true>(z(c), x, static_cast<R *>(nullptr), false);
    if (smp) {
      R *dst = a.samples + (static_cast<size_t>(step / a.thin) * a.n_chains + c) * d;
      for (int i = 0; i < d; ++i) dst[i] = x[i];
    }
    if (a.welford_on) {
      R *xb = a.xbuf + static_cast<size_t>(row) * a.dp;
      for (int i = 0; i < d; ++i) xb[i] = x[i];
    }
  }

  // log pi_z and, with grad, grad log pi_z (into the thread's array gout) at the evaluated
  // point of row r
  __device__ double logpi(int r, bool grad, R *gout) const {
    if (grad) vcopy<R>(gout, gle(r), a.d);
    const double lpr = prior<false>(ze(r), static_cast<R *>(nullptr), gout, grad);
    return static_cast<double>(a.st.lle[r]) + lpr + a.tgt.logdet;
  }

  __device__ void count(int c, bool accepted, double stat, int evals) const {
    a.st.acc_stat[c] += stat;
    a.st.accepts[c] += accepted ? 1ull : 0ull;
    a.st.evals[c] += static_cast<unsigned long long>(evals);
  }

  // Metropolis decision log u < la for MH / MALA / AIES.  FP64 state: la64() and log u in FP64.
  // FP32 state: la32 with the bound err on its rounding error (relative to la64()) against
  // logf(u) (u has 25 significant bits; 2^-20 |log u| covers logf), FP64 only inside the bound.
  template <class F>
  __device__ __forceinline__ bool metropolis(int c, uint32_t it, float la32, float err, F la64,
                                             double &stat) const {
    if constexpr (kF32) {
      const float u32 = draw_uniform<float>(a.seed, static_cast<uint32_t>(c), it, kAccept, 0);
      const float lu32 = logf(u32);
      const float gap = la32 - lu32;
      const float e2 = err + 0x1p-20f * fabsf(lu32) + 0x1p-22f;
      stat = static_cast<double>(accept_prob32(la32));
      if (gap > e2) return true;
      if (gap < -e2) return false;
      return log(static_cast<double>(u32)) < la64();
    } else {
      const double la = la64();
      stat = accept_prob(la);
      return log(draw_uniform<double>(a.seed, static_cast<uint32_t>(c), it, kAccept, 0)) < la;
    }
  }

  // ---------------------------------------------------------------- MH
  // Random walk in whitened units: z' = z + eps xi.
  __device__ __noinline__ bool mh_pre(int c) const {
    if (a.st.steps_done[c] >= a.n_steps) return false;
    R xi[kMaxD];
    draw_normals<R>(a.seed, c, a.st.iter[c], kXi, a.d, xi);
    vaxpy<R>(ze(c), z(c), static_cast<R>(a.eps), xi, a.d);
    return true;
  }
  __device__ __noinline__ bool mh_post(int c, double lpp) const {
    const uint32_t it = a.st.iter[c];
    const double lpc = static_cast<double>(a.st.lp[c]);
    bool acc;
    double stat = 0.0;
    if (lpp == -INFINITY) {
      acc = false;  // log alpha = -inf (or NaN): the FP64 comparison is false
    } else {
      const float lpp32 = static_cast<float>(lpp), lp32 = static_cast<float>(lpc);
      const float la32 = lpp32 - lp32;
      const float err = 0x1p-22f * (3.f * (fabsf(lpp32) + fabsf(lp32)) + 4.f);
      acc = metropolis(c, it, la32, err, [&] { return lpp - lpc; }, stat);
    }
    if (acc) {
      vcopy<R>(z(c), ze(c), a.d);
      a.st.lp[c] = static_cast<R>(lpp);
    }
    count(c, acc, stat, 1);
    return true;
  }

  // ---------------------------------------------------------------- MALA
  // Eq. (2.3): z' = z + eps grad + sqrt(2 eps) xi; q(a|b) = N(a; b + eps grad(b), 2 eps I).
  __device__ __noinline__ bool mala_pre(int c) const {
    if (a.st.steps_done[c] >= a.n_steps) return false;
    R xi[kMaxD];
    draw_normals<R>(a.seed, c, a.st.iter[c], kXi, a.d, xi);
    const R e = static_cast<R>(a.eps), s = static_cast<R>(sqrt(2.0 * a.eps));
    vaxpby<R>(ze(c), z(c), e, g(c), s, xi, a.d);
    return true;
  }
  __device__ __noinline__ bool mala_post(int c, double lpp, const R *gp) const {
    const int d = a.d;
    const uint32_t it = a.st.iter[c];
    const Row<R> zc = z(c), gc = g(c);
    const Blk<R> zp = ze(c);
    const double e = a.eps;
    const double lpc = static_cast<double>(a.st.lp[c]);
    // log alpha = log pi(z') - log pi(z) + log q(z|z') - log q(z'|z), in FP64
    auto la64 = [&] {
      double fwd = 0.0, rev = 0.0;
      for (int i = 0; i < d; ++i) {
        const double f = static_cast<double>(zp[i]) - zc[i] - e * gc[i];
        const double r = static_cast<double>(zc[i]) - zp[i] - e * gp[i];
        fwd += f * f;
        rev += r * r;
      }
      return lpp - lpc + (fwd - rev) / (4.0 * e);
    };
    bool acc;
    double stat = 0.0;
    if (kF32 && lpp == -INFINITY) {
      acc = false;
    } else if constexpr (kF32) {
      // FP32 log alpha and its rounding bound (the sums of squares, e*g, the differences and
      // the final combination, with a factor 4 of margin)
      const float ef = static_cast<float>(e);
      float fwd = 0.f, rev = 0.f, fab = 0.f, rab = 0.f;
#pragma unroll 1
      for (int i0 = 0; i0 < d; i0 += kVc) {
        const int n = min(kVc, d - i0);
        float P[kVc], Z[kVc], G[kVc], GP[kVc];
        vload(zp, i0, n, P);
        vload(zc, i0, n, Z);
        vload(gc, i0, n, G);
        vload(gp, i0, n, GP);
#pragma unroll
        for (int u = 0; u < kVc; ++u)
          if (u < n) {
            const float eg = ef * G[u], egp = ef * GP[u];
            const float f = P[u] - Z[u] - eg;
            const float r = Z[u] - P[u] - egp;
            const float fa = fabsf(P[u]) + fabsf(Z[u]) + fabsf(eg);
            const float ra = fabsf(Z[u]) + fabsf(P[u]) + fabsf(egp);
            fwd += f * f;
            rev += r * r;
            fab += fa * fa;
            rab += ra * ra;
          }
      }
      const float inv4e = 0.25f / ef;
      const float lpp32 = static_cast<float>(lpp), lp32 = static_cast<float>(lpc);
      const float la32 = (lpp32 - lp32) + (fwd - rev) * inv4e;
      const float err = 0x1p-22f * (static_cast<float>(d + 10) * (fab + rab) * inv4e +
                                    3.f * (fabsf(lpp32) + fabsf(lp32)) + 4.f);
      acc = metropolis(c, it, la32, err, la64, stat);
    } else {
      acc = metropolis(c, it, 0.f, 0.f, la64, stat);
    }
    if (acc) {
      vcopy2<R>(zc, zp, gc, gp, d);
      a.st.lp[c] = static_cast<R>(lpp);
    }
    count(c, acc, stat, 1);
    return true;
  }

  // ---------------------------------------------------------------- HMC
  // Identity mass in whitened space (Eqs. (2.7)-(2.8)); leapfrog; accept on H0 - H1.
  // work vectors: 0 z1, 1 q1, 2 g1; dwork: 0 leapfrogs done, 1 H0.
  __device__ __noinline__ bool hmc_pre(int c) const {
    if (a.st.steps_done[c] >= a.n_steps) return false;
    const Blk<double> dwc = dw(c);
    const Blk<R> z1 = wv(c, 0), q1 = wv(c, 1), g1 = wv(c, 2);
    const R e = static_cast<R>(a.eps);
    if (dwc[0] == 0.0) {
      R q[kMaxD];
      draw_normals<R>(a.seed, c, a.st.iter[c], kXi, a.d, q);
      double qq = 0.0;  // once per trajectory: FP64
      for (int i = 0; i < a.d; ++i) qq += static_cast<double>(q[i]) * q[i];
      vcopy2<R>(z1, z(c), g1, g(c), a.d);
      vcopy<R>(q1, q, a.d);
      dwc[1] = -static_cast<double>(a.st.lp[c]) + 0.5 * qq;
    }
    kick_drift_inplace<R>(z1, q1, g1, ze(c), e, a.d);
    return true;
  }
  __device__ __noinline__ bool hmc_post(int c, double lp1, const R *gl) const {
    const int d = a.d;
    const Blk<double> dwc = dw(c);
    const Blk<R> q1 = wv(c, 1), g1 = wv(c, 2);
    const R e = static_cast<R>(a.eps);
    // q1 += e/2 g (closing the leapfrog); g1 = g, the gradient at z1
    R qq = R(0);
#pragma unroll 1
    for (int i0 = 0; i0 < d; i0 += kVc) {
      const int n = min(kVc, d - i0);
      R q[kVc], gg[kVc];
      vload(q1, i0, n, q);
      vload(gl, i0, n, gg);
#pragma unroll
      for (int u = 0; u < kVc; ++u) {
        q[u] = q[u] + R(0.5) * e * gg[u];
        if (u < n) qq += q[u] * q[u];
      }
      vstore(q1, i0, n, q);
      vstore(g1, i0, n, gg);
    }
    const double nlf = dwc[0] + 1.0;
    a.st.evals[c] += 1ull;
    if (nlf < a.n_leapfrog) {
      dwc[0] = nlf;
      return false;
    }
    dwc[0] = 0.0;
    const double h0 = dwc[1];
    const uint32_t it = a.st.iter[c];
    const double u = draw_uniform<double>(a.seed, c, it, kAccept, 0);
    const double lu = log(u);  // once per trajectory
    // H1 = -log pi(z1) + |q1|^2 / 2; FP32 state: |q1|^2 in FP32 within (d + 4) 2^-24 |q1|^2
    // of the FP64 sum, which is formed only when la is that close to log u
    double la = h0 - (-lp1 + 0.5 * static_cast<double>(qq));
    bool acc;
    if (kF32 && la - lu > (d + 4) * 0x1p-24 * static_cast<double>(qq) +
                              0x1p-50 * (fabs(h0) + fabs(lp1) + static_cast<double>(qq) + fabs(lu))) {
      acc = true;
    } else if (kF32 && la - lu < -((d + 4) * 0x1p-24 * static_cast<double>(qq) +
                                   0x1p-50 * (fabs(h0) + fabs(lp1) + static_cast<double>(qq) + fabs(lu)))) {
      acc = false;
    } else {
      if (kF32) {
        double q2 = 0.0;
        for (int i = 0; i < d; ++i) q2 += static_cast<double>(q1[i]) * q1[i];
        la = h0 - (-lp1 + 0.5 * q2);
      }
      acc = lu < la;
    }
    const double stat = kF32 ? static_cast<double>(accept_prob32(static_cast<float>(la))) : accept_prob(la);
    if (acc) {
      vcopy2<R>(z(c), wv(c, 0), g(c), g1, d);
      a.st.lp[c] = static_cast<R>(lp1);
    }
    count(c, acc, stat, 0);
    return true;
  }

  // ---------------------------------------------------------------- NUTS
  // Hoffman & Gelman (2014) Algorithm 3, unrolled into one leapfrog per call:
  // the tree of the current doubling is built leaf by leaf; pending left
  // siblings wait on a per-level stack and are merged (candidate kept with
  // probability n''/(n'+n''), U-turn check of the merged span) when their right
  // sibling completes.  work vectors: 0 zm 1 qm 2 gm 3 zp 4 qp 5 gp 6 zs 7 gs
  // 8 qh, level i: 9+4i first z, 10+4i first q, 11+4i cand z, 12+4i cand g.
  // dwork: 0 new-iteration flag, 1 log u - H0, 2 H0, 3 n, 4 lp of selected,
  // 5 acceptance-stat sum, 6 j, 7 v, 8 m_sub, 9 leaves, 10 diverged, 11 moved,
  // 12+i cand lp, 22+i node n.  Multinomial variant (kModeNUTS_MN): dwork 3 and 22+i hold log
  // weights log sum exp(H0 - H) instead of the counts n (the start point: log 1 = 0).
  __device__ __noinline__ bool nuts_pre(int c) const {
    if (a.st.steps_done[c] >= a.n_steps) return false;
    const Blk<double> dwc = dw(c);
    const int d = a.d;
    const uint32_t it = a.st.iter[c];
    if (dwc[0] != 0.0) {
      R q0[kMaxD];
      draw_normals<R>(a.seed, c, it, kXi, d, q0);
      double qq = 0.0;  // once per iteration: FP64
      for (int i = 0; i < d; ++i) qq += static_cast<double>(q0[i]) * q0[i];
      const double H0 = -static_cast<double>(a.st.lp[c]) + 0.5 * qq;
      dwc[2] = H0;
      dwc[1] = log(draw_uniform<double>(a.seed, c, it, kAccept, 0)) - H0;
      // both trajectory ends and the selected point start at (z, q0, g): one pass over z, g
      const Row<R> zc = z(c), gc = g(c);
#pragma unroll 1
      for (int i0 = 0; i0 < d; i0 += kVc) {
        const int n = min(kVc, d - i0);
        R tz[kVc], tg[kVc], tq[kVc];
        vload(zc, i0, n, tz);
        vload(gc, i0, n, tg);
        vload(q0, i0, n, tq);
        vstore(wv(c, 0), i0, n, tz);
        vstore(wv(c, 3), i0, n, tz);
        vstore(wv(c, 6), i0, n, tz);
        vstore(wv(c, 2), i0, n, tg);
        vstore(wv(c, 5), i0, n, tg);
        vstore(wv(c, 7), i0, n, tg);
        vstore(wv(c, 1), i0, n, tq);
        vstore(wv(c, 4), i0, n, tq);
      }
      dwc[3] = a.mode == kModeNUTS_MN ? 0.0 : 1.0;
      dwc[4] = static_cast<double>(a.st.lp[c]);
      dwc[5] = 0.0;
      dwc[6] = 0.0;
      dwc[7] = draw_uniform<double>(a.seed, c, it, kNutsDir, 0) < 0.5 ? -1.0 : 1.0;
      dwc[8] = 0.0;
      dwc[9] = 0.0;
      dwc[10] = 0.0;
      dwc[11] = 0.0;
      dwc[0] = 0.0;
    }
    const bool back = dwc[7] < 0.0;
    const R e = static_cast<R>(dwc[7] * a.eps);
    half_kick_drift<R>(wv(c, 8), ze(c), wv(c, back ? 1 : 4), wv(c, back ? 2 : 5), wv(c, back ? 0 : 3), e, d);
    return true;
  }

  // returns whether the iteration ends (nuts_finish follows)
  __device__ bool nuts_leaf(int c, double lpn, const R *gn) const {
    const Blk<double> dwc = dw(c);
    const int d = a.d;
    // the chain's scalars in one batch of loads, ahead of the leaf's vector stores
    const uint32_t it = a.st.iter[c];
    const unsigned long long n_ev = a.st.evals[c];
    const double v = dwc[7], leaves = dwc[9] + 1.0, log_u = dwc[1], H0 = dwc[2], stat0 = dwc[5];
    const int m_sub = static_cast<int>(dwc[8]);
    const int j = static_cast<int>(dwc[6]);
    const bool back = v < 0.0;
    const R e = static_cast<R>(v * a.eps);
    const Blk<R> zend = wv(c, back ? 0 : 3), qend = wv(c, back ? 1 : 4), gend = wv(c, back ? 2 : 5);
    const R qq = half_kick_store<R>(zend, qend, gend, wv(c, 8), ze(c), gn, e, d);
    a.st.evals[c] = n_ev + 1ull;
    dwc[9] = leaves;
    const int leaf = static_cast<int>(leaves);
    // H of the new leaf; FP32 state: |q|^2 in FP32, within errH of the FP64 H
    double Hl = -lpn + 0.5 * static_cast<double>(qq);
    const bool mn = a.mode == kModeNUTS_MN;
    bool nlb, sl;
    if (mn) {
      // multinomial: the leaf's log weight H0 - H (FP64 from the working-precision state);
      // divergent when H - H0 exceeds Delta_max
      if (kF32) {
        double q2 = 0.0;
        for (int i = 0; i < d; ++i) q2 += static_cast<double>(qend[i]) * qend[i];
        Hl = -lpn + 0.5 * q2;
      }
      nlb = true;
      sl = Hl - H0 < kNutsDeltaMax;
    } else {
      const double t = log_u + Hl;
      const double errH = kF32 ? (d + 4) * 0x1p-24 * static_cast<double>(qq) +
                                     0x1p-50 * (fabs(lpn) + static_cast<double>(qq) + fabs(log_u) + kNutsDeltaMax)
                               : 0.0;
      const bool sure = kF32 && (t < -errH || t > errH) && (t < kNutsDeltaMax - errH || t > kNutsDeltaMax + errH);
      if (sure) {
        nlb = t < 0.0;
        sl = t < kNutsDeltaMax;
      } else {
        if (kF32) {
          double q2 = 0.0;
          for (int i = 0; i < d; ++i) q2 += static_cast<double>(qend[i]) * qend[i];
          Hl = -lpn + 0.5 * q2;
        }
        nlb = log_u <= -Hl;
        sl = log_u < kNutsDeltaMax - Hl;
      }
    }
    dwc[5] = stat0 + (kF32 ? static_cast<double>(accept_prob32(static_cast<float>(H0 - Hl))) : accept_prob(H0 - Hl));
    const double nl = mn ? H0 - Hl : (nlb ? 1.0 : 0.0);
    if (!sl) {
      dwc[10] = 1.0;
      return true;
    }
    // current node = the new leaf; first = leaf, candidate = leaf
    int first_src = -1, cand_src = -1;
    double node_n = nl;
    int lvl = 0;
    while ((m_sub >> lvl) & 1) {
      // merge pending left sibling at level lvl with the node
      const double ln = dwc[22 + lvl];
      const double u = draw_uniform<double>(a.seed, c, it, kNutsSel,
                                            static_cast<uint32_t>(8 * (leaf - 1) + lvl + 1));
      // slice: counts, take the right half's candidate with probability n'' / (n' + n'');
      // multinomial: log weights, probability w'' / (w' + w'')
      const double ntot = mn ? log_add_exp(ln, node_n) : ln + node_n;
      const bool take_right = mn ? u < exp(node_n - ntot) : (ntot > 0.0 && u * ntot < node_n);
      if (!take_right) cand_src = lvl;
      // U-turn check of the merged span [left.first .. leaf]
      const bool ok = no_uturn<R>(zend, wv(c, 9 + 4 * lvl), wv(c, 10 + 4 * lvl), qend, v, d);
      first_src = lvl;
      node_n = ntot;
      ++lvl;
      if (!ok) return true;
    }
    // candidate vectors of the node
    const Blk<R> cz = cand_src < 0 ? zend : wv(c, 11 + 4 * cand_src);
    const Blk<R> cg = cand_src < 0 ? gend : wv(c, 12 + 4 * cand_src);
    const double clp = cand_src < 0 ? lpn : dwc[12 + cand_src];
    if (lvl == j) {
      // the subtree of this doubling is complete: progressive top-level selection
      const double ut = draw_uniform<double>(a.seed, c, it, kNutsTop, static_cast<uint32_t>(j));
      if (mn ? ut < exp(node_n - dwc[3]) : ut * dwc[3] < node_n) {
        vcopy2<R>(wv(c, 6), cz, wv(c, 7), cg, d);
        dwc[4] = clp;
        dwc[11] = 1.0;
      }
      dwc[3] = mn ? log_add_exp(dwc[3], node_n) : dwc[3] + node_n;
      const bool ok = no_uturn<R>(wv(c, 3), wv(c, 0), wv(c, 1), wv(c, 4), 1.0, d);
      const int jn = j + 1;
      dwc[6] = jn;
      if (!ok || jn >= a.max_depth) return true;
      dwc[7] = draw_uniform<double>(a.seed, c, it, kNutsDir, static_cast<uint32_t>(jn)) < 0.5 ? -1.0 : 1.0;
      dwc[8] = 0.0;
    } else {
      // park the node as the pending left sibling at level lvl
      const Blk<R> fz = first_src < 0 ? zend : wv(c, 9 + 4 * first_src);
      const Blk<R> fq = first_src < 0 ? qend : wv(c, 10 + 4 * first_src);
      if (first_src != lvl) vcopy2<R>(wv(c, 9 + 4 * lvl), fz, wv(c, 10 + 4 * lvl), fq, d);
      if (cand_src != lvl) vcopy2<R>(wv(c, 11 + 4 * lvl), cz, wv(c, 12 + 4 * lvl), cg, d);
      dwc[12 + lvl] = clp;
      dwc[22 + lvl] = node_n;
      dwc[8] = m_sub + 1;
    }
    return false;
  }

  __device__ bool nuts_finish(int c) const {
    const Blk<double> dwc = dw(c);
    vcopy2<R>(z(c), wv(c, 6), g(c), wv(c, 7), a.d);
    a.st.lp[c] = static_cast<R>(dwc[4]);
    const double leaves = dwc[9];
    a.st.acc_stat[c] += leaves > 0.0 ? dwc[5] / leaves : 0.0;
    a.st.accepts[c] += dwc[11] != 0.0 ? 1ull : 0ull;
    a.st.divs[c] += dwc[10] != 0.0 ? 1ull : 0ull;
    dwc[0] = 1.0;
    return true;
  }
  __device__ __noinline__ bool nuts_post(int c, double lpn, const R *gn) const { return nuts_leaf(c, lpn, gn) && nuts_finish(c); }

  // ---------------------------------------------------------------- AIES
  // Goodman-Weare stretch move (Sec. 2.3): y = z_j + Z (z_i - z_j),
  // Z = (u (a - 1) + 1)^2 / a (Eq. (2.15)); accept with min(1, Z^(d-1) pi(y)/pi(z_i)).
  // Row r moves walker k = r % (W/2) of half h of ensemble r / (W/2).  dwork 0: Z.
  __device__ int aies_walker(int r, int h) const {
    const int half = a.aies_walkers / 2;
    return (r / half) * a.aies_walkers + h * half + (r % half);
  }
  __device__ __noinline__ bool aies_pre(int r, int h) const {
    const int i = aies_walker(r, h);
    if (a.st.steps_done[i] >= a.n_steps) return false;
    const int half = a.aies_walkers / 2;
    const int base = (r / half) * a.aies_walkers + (1 - h) * half;
    const uint32_t it = a.st.iter[i];
    const double up = draw_uniform<double>(a.seed, i, it, kAiesPartner, 0);
    int jj = static_cast<int>(up * half);
    if (jj > half - 1) jj = half - 1;
    const int jw = base + jj;
    const Row<R> zi = z(i), zj = z(jw);
    const Blk<R> y = ze(r);
    if (a.mode == kModeAIES_DE) {
      // differential evolution (Sec. 2.3, after Eq. (2.15)): y = z_i + gamma (z_j - z_k), k != j
      // uniform over the other half (uniform 1 of the partner stream, skipping j), gamma =
      // (1 + sigma_gamma eta) 2.38 / sqrt(2 d) with eta normal 0 of the scale stream
      const double uk = draw_uniform<double>(a.seed, i, it, kAiesPartner, 1);
      int kk = static_cast<int>(uk * (half - 1));
      if (kk > half - 2) kk = half - 2;
      if (kk >= jj) ++kk;
      const Row<R> zk = z(base + kk);
      R eta;
      draw_normals<R>(a.seed, i, it, kAiesZ, 1, &eta);
      const R gam = (R(1) + static_cast<R>(a.eps) * eta) * static_cast<R>(2.38 / sqrt(2.0 * a.d));
#pragma unroll 1
      for (int q = 0; q < a.d; ++q) y[q] = zi[q] + gam * (zj[q] - zk[q]);
      return true;
    }
    const double uz = draw_uniform<double>(a.seed, i, it, kAiesZ, 0);
    const double t = uz * (a.aies_a - 1.0) + 1.0;
    const double Z = a.aies_a == 2.0 ? t * t * 0.5 : t * t / a.aies_a;  // (x 0.5 is exact)
    dw(i)[0] = Z;
    const R Zr = static_cast<R>(Z);
#pragma unroll 1
    for (int q0 = 0; q0 < a.d; q0 += kVc) {
      R A[kVc], B[kVc];
#pragma unroll
      for (int u = 0; u < kVc; ++u)
        if (q0 + u < a.d) {
          A[u] = zi[q0 + u];
          B[u] = zj[q0 + u];
        }
#pragma unroll
      for (int u = 0; u < kVc; ++u)
        if (q0 + u < a.d) y[q0 + u] = B[u] + Zr * (A[u] - B[u]);
    }
    return true;
  }
  __device__ __noinline__ bool aies_post(int r, int h, double lpy) const {
    const int i = aies_walker(r, h);
    if (a.mode == kModeAIES_DE) return de_post(r, h, lpy);
    const double Z = dw(i)[0];
    const double lpc = static_cast<double>(a.st.lp[i]);
    const uint32_t it = a.st.iter[i];
    const int d = a.d;
    auto la64 = [&] { return (d - 1) * log(Z) + lpy - lpc; };
    bool acc;
    double stat = 0.0;
    if (kF32 && lpy == -INFINITY) {
      acc = false;
    } else if constexpr (kF32) {
      // logf(Z) to 2 ulp plus 2^-24 from rounding Z, times (d - 1); the FP32 sums to a factor 4
      const float lz = logf(static_cast<float>(Z));
      const float lpy32 = static_cast<float>(lpy), lp32 = static_cast<float>(lpc);
      const float la32 = static_cast<float>(d - 1) * lz + (lpy32 - lp32);
      const float err = static_cast<float>(d - 1) * (0x1p-21f * fabsf(lz) + 0x1p-22f) +
                        0x1p-21f * (fabsf(lpy32) + fabsf(lp32) + static_cast<float>(d - 1) * fabsf(lz));
      acc = metropolis(i, it, la32, err, la64, stat);
    } else {
      acc = metropolis(i, it, 0.f, 0.f, la64, stat);
    }
    if (acc) {
      vcopy<R>(z(i), ze(r), d);
      a.st.lp[i] = static_cast<R>(lpy);
    }
    count(i, acc, stat, 1);
    return true;
  }

  // Differential-evolution decision: the move is symmetric, log alpha = log pi(y) - log pi(z_i).
  __device__ __noinline__ bool de_post(int r, int h, double lpy) const {
    const int i = aies_walker(r, h);
    const double lpc = static_cast<double>(a.st.lp[i]);
    const uint32_t it = a.st.iter[i];
    auto la64 = [&] { return lpy - lpc; };
    bool acc;
    double stat = 0.0;
    if (kF32 && lpy == -INFINITY) {
      acc = false;
    } else if constexpr (kF32) {
      const float lpy32 = static_cast<float>(lpy), lp32 = static_cast<float>(lpc);
      const float la32 = lpy32 - lp32;
      const float err = 0x1p-21f * (fabsf(lpy32) + fabsf(lp32));
      acc = metropolis(i, it, la32, err, la64, stat);
    } else {
      acc = metropolis(i, it, 0.f, 0.f, la64, stat);
    }
    if (acc) {
      vcopy<R>(z(i), ze(r), a.d);
      a.st.lp[i] = static_cast<R>(lpy);
    }
    count(i, acc, stat, 1);
    return true;
  }

  // ---------------------------------------------------------------- batch modes
  __device__ bool refresh_pre(int c) const {
    if (a.st.steps_done[c] >= 1) return false;
    vcopy<R>(ze(c), z(c), a.d);
    return true;
  }
  __device__ bool refresh_post(int c, double lp, const R *gp) const {
    a.st.lp[c] = static_cast<R>(lp);
    vcopy<R>(g(c), gp, a.d);
    a.st.steps_done[c] = 1;
    return true;
  }

  // common end of an iteration: counters, sample record
  __device__ void finish(int c, int row) const {
    const int s = a.st.steps_done[c];
    a.st.iter[c] += 1u;
    record(c, row, s);
    a.st.steps_done[c] = s + 1;
  }

  // Dispatch. pre returns whether the row needs an evaluation; post returns whether
  // the chain of the row completed an iteration (for the covariance accumulator).  The
  // per-kernel bodies are separate functions (__noinline__), so that their temporaries do not
  // add up in the caller; log pi (and its gradient) and the record are evaluated here, where
  // the whitening factor is read from the kernel parameters as constant-bank operands.
  __device__ bool pre(int row, int h) const {
    switch (a.mode) {
      case kModeMH: return mh_pre(row);
      case kModeMALA: return mala_pre(row);
      case kModeHMC: return hmc_pre(row);
      case kModeNUTS:
      case kModeNUTS_MN: return nuts_pre(row);
      case kModeAIES:
      case kModeAIES_DE: return aies_pre(row, h);
      case kModeRefresh: return refresh_pre(row);
      default: return false;
    }
  }
  __device__ bool post(int row, int h) const {
    // log pi (and its gradient) at the evaluated point, then the kernel's decision, then the
    // end of the chain's iteration if it completed one
    R gp[kMaxD];
    const bool grad = a.mode != kModeMH && !is_ensemble_mode(a.mode);
    const double lp = logpi(row, grad, gp);
    int c = row;
    bool done;
    switch (a.mode) {
      case kModeMH: done = mh_post(row, lp); break;
      case kModeMALA: done = mala_post(row, lp, gp); break;
      case kModeHMC: done = hmc_post(row, lp, gp); break;
      case kModeNUTS:
      case kModeNUTS_MN: done = nuts_post(row, lp, gp); break;
      case kModeAIES:
      case kModeAIES_DE:
        c = aies_walker(row, h);
        done = aies_post(row, h, lp);
        break;
      case kModeRefresh: return refresh_post(row, lp, gp);
      default: return false;
    }
    if (done) finish(c, row);
    return done;
  }
};

// ---------------------------------------------------------------- register-resident MALA / MH / HMC
// For d <= 8 the BF16 engine keeps a chain's position, gradient and log density in the
// registers of the thread that owns the chain for the whole launch (the point under
// evaluation, its gradient and the MALA noise / HMC momentum in shared memory), instead of
// reading them back from the state arrays around every evaluation.  Proposals (Eq. (2.3),
// the random walk, and the leapfrog of Eqs. (2.7)-(2.8)), Philox streams and accept decisions
// are those of mala_* / mh_* / hmc_* above; the state arrays are written through on every
// change, so they are current after each step.
//
// The decision log u < log alpha is first taken in FP32: for MALA / MH log alpha is formed
// in FP32 together with a bound on its rounding error relative to the FP64 expression of
// mala_post / mh_post (HMC forms H0 - H1 in FP64 as hmc_post does), log u with logf, and only
// when |log alpha - log u| is inside the bound is the FP64 comparison evaluated, so the
// outcome is always the FP64 one.  The acceptance statistic min(1, alpha) that feeds
// step-size adaptation is summed from the FP32 log alpha.
template <typename R>
struct RegChain8 {
  static constexpr int DB = 8;
  R z[DB], g[DB];
  // point under evaluation (MALA / MH proposal, HMC z1), grad logL there (HMC g1), and the
  // next MALA proposal's noise (have_xi) or the HMC momentum q1: DB entries each in the
  // caller's shared memory
  R *zp, *gp, *xi;
  R lp, e, s;
  uint32_t iter;
  int steps;
  int nlf;    // HMC: leapfrogs of the current trajectory done
  double h0;  // HMC: H at the start of the trajectory
  double acc_stat, lpr, u;
  unsigned long long n_acc, n_ev;
  float lu32;
  bool inside, prepped, have_xi;
  // the last decision's memory side (record): pending, accepted, with gradient, step index
  bool rec_pending, rec_acc, rec_grad;
  int rec_step;

  __device__ void load(const StepArgs<R> &a, int c, R *zp_smem, R *gp_smem, R *xi_smem) {
    zp = zp_smem;
    gp = gp_smem;
    xi = xi_smem;
    const R *zc = a.st.z + static_cast<size_t>(c) * a.dp, *gc = a.st.g + static_cast<size_t>(c) * a.dp;
#pragma unroll
    for (int i = 0; i < DB; ++i) {
      z[i] = i < a.d ? zc[i] : R(0);
      g[i] = i < a.d ? gc[i] : R(0);
      zp[i] = R(0);
      gp[i] = R(0);
    }
    lp = a.st.lp[c];
    iter = a.st.iter[c];
    acc_stat = a.st.acc_stat[c];
    n_acc = a.st.accepts[c];
    n_ev = a.st.evals[c];
    steps = 0;
    nlf = 0;
    h0 = 0.0;
    e = static_cast<R>(a.eps);
    s = static_cast<R>(sqrt(2.0 * a.eps));
    prepped = have_xi = false;
    rec_pending = rec_acc = rec_grad = false;
    rec_step = 0;
  }

  // dst[0..d) = v[0..d): one thread per chain writes its own row, so the stores do not coalesce
  // across the warp; with d == 8 and a 16-byte aligned row two 16-byte stores do it.
  static __device__ __forceinline__ void store_row(R *dst, const R *v, int d) {
    if (sizeof(R) == 4 && d == 8 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
      float4 *q = reinterpret_cast<float4 *>(dst);
      q[0] = make_float4(v[0], v[1], v[2], v[3]);
      q[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
      for (int i = 0; i < DB; ++i)
        if (i < d) dst[i] = v[i];
    }
  }
  // x = mu + L v on the first d entries (same summation order as TargetView::eval)
  static __device__ __forceinline__ void to_x(const StepArgs<R> &a, const R *v, R *x) {
#pragma unroll
    for (int i = 0; i < DB; ++i) {
      R acc = R(0);
      if (i < a.d) {
        acc = a.tgt.mu[i];
#pragma unroll
        for (int j = 0; j <= i; ++j) acc += a.tgt.L[i * kMaxD + j] * v[j];
      }
      x[i] = acc;
    }
  }
  // normals 0..DB-1 of stream (c, it, kXi), as draw_normals
  static __device__ __forceinline__ void normals(const StepArgs<R> &a, int c, uint32_t it, R *out) {
#pragma unroll
    for (int b = 0; b < DB / 4; ++b) {
      R v[4] = {R(0), R(0), R(0), R(0)};
      if (4 * b < a.d) {
        uint32_t w[4];
        Philox::block(a.seed, static_cast<uint32_t>(c), it, kXi, static_cast<uint32_t>(b), w);
        box_muller(u01<R>(w[0]), u01<R>(w[1]), v[0], v[1]);
        box_muller(u01<R>(w[2]), u01<R>(w[3]), v[2], v[3]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) out[4 * b + k] = v[k];
    }
  }

  // Proposal z' written to zp (and to the state's evaluation row).
  __device__ bool pre(const StepArgs<R> &a, int c, bool mala) {
    if (steps >= a.n_steps) return false;
    if (!have_xi) normals(a, c, iter, xi);
    have_xi = false;
#pragma unroll
    for (int i = 0; i < DB; ++i)
      if (i < a.d) zp[i] = mala ? z[i] + e * g[i] + s * xi[i] : z[i] + e * xi[i];
    return true;
  }

  // Distance of x_i outside [lower_i, upper_i] (0 inside).
  static __device__ __forceinline__ R bound_excess(const TargetView<R> &t, R x, int i) {
    return x < t.lower[i] ? x - t.lower[i] : (x > t.upper[i] ? x - t.upper[i] : R(0));
  }
  // gz += the gradient (through x = mu + L z) of the Gaussian prior terms and the smooth-bound
  // penalties at the point zv: gz_j -= sum_{i >= j} L_ij p_i, p_i = x_i (Gaussian dims) +
  // r_i / w_i (smooth bounds).
  __device__ void prior_grad(const StepArgs<R> &a, const R *zv, R *gz) const {
    const int d = a.d;
    R xp[DB];
    to_x(a, zv, xp);
#pragma unroll
    for (int i = 0; i < DB; ++i) {
      R p = (i < d && a.tgt.gauss[i]) ? xp[i] : R(0);
      if (i < d && a.tgt.any_pen && a.tgt.pen_iw[i] > R(0))
        p += bound_excess(a.tgt, xp[i], i) * a.tgt.pen_iw[i] * a.tgt.pen_iw[i];
      xp[i] = p;
    }
#pragma unroll
    for (int j = 0; j < DB; ++j)
      if (j < d) {
        R sg = 0;
#pragma unroll
        for (int i = j; i < DB; ++i)
          if (i < d) sg -= a.tgt.L[i * kMaxD + j] * xp[i];
        gz[j] += sg;
      }
  }

  // The part of post that does not depend on the evaluation in flight: x of the proposal and
  // its prior term, the accept uniform, and the noise of the next iteration's proposal.
  __device__ void prep(const StepArgs<R> &a, int c) {
    R xp[DB];
    to_x(a, zp, xp);
    inside = true;
    lpr = 0.0;
#pragma unroll
    for (int i = 0; i < DB; ++i)
      if (i < a.d) {
        const bool pen = a.tgt.any_pen && a.tgt.pen_iw[i] > R(0);
        if (!pen && !(xp[i] >= a.tgt.lower[i] && xp[i] <= a.tgt.upper[i])) inside = false;
        if (a.tgt.any_gauss && a.tgt.gauss[i]) lpr -= 0.5 * static_cast<double>(xp[i]) * static_cast<double>(xp[i]);
        if (pen) {
          const R r = bound_excess(a.tgt, xp[i], i) * a.tgt.pen_iw[i];
          lpr -= 0.5 * static_cast<double>(r) * static_cast<double>(r);
        }
      }
    u = draw_uniform<double>(a.seed, static_cast<uint32_t>(c), iter, kAccept, 0);
    lu32 = logf(static_cast<float>(u));
    prepped = true;
  }
  __device__ void prep_next(const StepArgs<R> &a, int c) {
    if (a.mode == kModeHMC) return;
    if (steps + 1 < a.n_steps) {
      normals(a, c, iter + 1u, xi);
      have_xi = true;
    }
  }

  // HMC: one leapfrog of the current trajectory (a new trajectory draws its momentum);
  // z1 goes to zp for evaluation.  Same operations as hmc_pre.
  __device__ bool hmc_pre(const StepArgs<R> &a, int c) {
    if (steps >= a.n_steps) return false;
    R *q1 = xi, *g1 = gp, *z1 = zp;
    if (nlf == 0) {
      normals(a, c, iter, q1);
      double qq = 0.0;
#pragma unroll
      for (int i = 0; i < DB; ++i)
        if (i < a.d) {
          qq += static_cast<double>(q1[i]) * q1[i];
          z1[i] = z[i];
          g1[i] = g[i];
        }
      h0 = -static_cast<double>(lp) + 0.5 * qq;
    }
#pragma unroll
    for (int i = 0; i < DB; ++i)
      if (i < a.d) {
        q1[i] += R(0.5) * e * g1[i];
        z1[i] += e * q1[i];
      }
    return true;
  }
  // HMC: close the leapfrog (gp holds grad logL at z1); after n_leapfrog of them, the
  // accept of hmc_post.  Returns whether the trajectory (an iteration) completed.
  __device__ bool hmc_post(const StepArgs<R> &a, int c, int row, R lle, bool defer) {
    const TargetView<R> &t = a.tgt;
    const int d = a.d;
    const bool last = nlf + 1 >= a.n_leapfrog;
    if (!prepped) prep(a, c);
    prepped = false;
    R *q1 = xi, *g1 = gp, *z1 = zp;
    if (rec_pending) record(a, c, row);
    const double lp1 = static_cast<double>(lle) + (inside ? lpr : -INFINITY) + t.logdet;
    if (t.any_gauss || t.any_pen) prior_grad(a, z1, g1);
    double qq = 0.0;
#pragma unroll
    for (int i = 0; i < DB; ++i)
      if (i < d) {
        q1[i] += R(0.5) * e * g1[i];
        qq += static_cast<double>(q1[i]) * q1[i];
      }
    n_ev += 1ull;
    nlf += 1;
    if (!last) return false;
    nlf = 0;
    const double h1 = -lp1 + 0.5 * qq;
    const double la = h0 - h1;
    const float la32 = static_cast<float>(la);
    const float err = 0x1p-21f * (1.f + fabsf(lu32));  // log u by logf; la is the FP64 value
    const float gap = la32 - lu32;
    bool acc;
    if (!(la == la)) acc = false;
    else if (gap > err) acc = true;
    else if (gap < -err) acc = false;
    else acc = log(u) < la;
    const float p = la32 >= 0.f ? 1.f : (la32 == la32 ? expf(la32) : 0.f);
    return finish_step(a, c, row, acc, p, z1, g1, lp1, true, defer);
  }

  // End of an iteration, shared by the three kernels: the new state in registers (the next
  // proposal needs only these), then record() writes it through: state, counters, iteration
  // counter, sample record and Welford hand-off.  With `defer` the engine calls record()
  // later, while the next evaluation is in flight (never with the covariance accumulator on,
  // which reads the record right after the decision).
  __device__ bool finish_step(const StepArgs<R> &a, int c, int row, bool acc, float p, const R *znew,
                              const R *gnew, double lpnew, bool with_grad, bool defer) {
    if (acc) {
#pragma unroll
      for (int i = 0; i < DB; ++i)
        if (i < a.d) {
          z[i] = znew[i];
          if (with_grad) g[i] = gnew[i];
        }
      lp = static_cast<R>(lpnew);
    }
    acc_stat += static_cast<double>(p);
    n_acc += acc ? 1ull : 0ull;
    rec_acc = acc;
    rec_grad = with_grad;
    rec_step = steps;
    iter += 1u;
    steps += 1;
    rec_pending = true;
    if (!defer) record(a, c, row);
    return true;
  }
  __device__ void record(const StepArgs<R> &a, int c, int row) {
    if (!rec_pending) return;
    rec_pending = false;
    const int d = a.d;
    R x[DB];
    to_x(a, z, x);  // x-space record of the new position
    if (rec_acc) {
      store_row(a.st.z + static_cast<size_t>(c) * a.dp, z, d);
      if (rec_grad) store_row(a.st.g + static_cast<size_t>(c) * a.dp, g, d);
      a.st.lp[c] = lp;
    }
    a.st.acc_stat[c] = acc_stat;
    a.st.accepts[c] = n_acc;
    a.st.evals[c] = n_ev;
    a.st.iter[c] = iter;
    if (a.samples && ((rec_step + 1) % a.thin) == 0)
      store_row(a.samples + (static_cast<size_t>(rec_step / a.thin) * a.n_chains + c) * d, x, d);
    if (a.welford_on) store_row(a.xbuf + static_cast<size_t>(row) * a.dp, x, d);
    a.st.steps_done[c] = steps;
  }

  // lle = logL at zp; gp (MALA) holds grad logL at zp.  Returns true (an iteration completed).
  __device__ bool post(const StepArgs<R> &a, int c, int row, R lle, bool mala, bool defer) {
    const TargetView<R> &t = a.tgt;
    const int d = a.d;
    if (rec_pending) record(a, c, row);
    if (!prepped) prep(a, c);
    prepped = false;
    // log pi_z(zp) and its gradient (logpi_eval)
    const double lpp = static_cast<double>(lle) + (inside ? lpr : -INFINITY) + t.logdet;
    if (mala && (t.any_gauss || t.any_pen)) prior_grad(a, zp, gp);
    bool acc;
    float p;
    if (!inside) {
      acc = false;  // log alpha = -inf
      p = 0.f;
    } else {
      float fwd = 0.f, rev = 0.f, fab = 0.f, rab = 0.f;
      if (mala) {
#pragma unroll
        for (int i = 0; i < DB; ++i)
          if (i < d) {
            const float f = static_cast<float>(zp[i]) - static_cast<float>(z[i]) - static_cast<float>(e * g[i]);
            const float r = static_cast<float>(z[i]) - static_cast<float>(zp[i]) - static_cast<float>(e * gp[i]);
            const float fa = fabsf(static_cast<float>(zp[i])) + fabsf(static_cast<float>(z[i])) +
                             fabsf(static_cast<float>(e * g[i]));
            const float ra = fabsf(static_cast<float>(z[i])) + fabsf(static_cast<float>(zp[i])) +
                             fabsf(static_cast<float>(e * gp[i]));
            fwd += f * f;
            rev += r * r;
            fab += fa * fa;
            rab += ra * ra;
          }
      }
      const float inv4e = mala ? 0.25f / static_cast<float>(a.eps) : 0.f;
      const float lpp32 = static_cast<float>(lpp), lp32 = static_cast<float>(lp);
      const float la32 = (lpp32 - lp32) + (fwd - rev) * inv4e;
      // FP32 rounding of the sums of squares, of e*g, of the differences and of the final
      // combination, with a factor 4 of margin; u has 25 significant bits (log u to 2^-24).
      const float err = 0x1p-22f * (static_cast<float>(d + 10) * (fab + rab) * inv4e +
                                    3.f * (fabsf(lpp32) + fabsf(lp32)) + 4.f * fabsf(lu32) + 4.f);
      const float gap = la32 - lu32;
      if (gap > err) acc = true;
      else if (gap < -err) acc = false;
      else {
        // the FP64 expression of mala_post / mh_post
        double la = lpp - static_cast<double>(lp);
        if (mala) {
          const double ed = a.eps;
          double fw = 0.0, rv = 0.0;
#pragma unroll
          for (int i = 0; i < DB; ++i)
            if (i < d) {
              const double f = static_cast<double>(zp[i]) - z[i] - ed * g[i];
              const double r = static_cast<double>(z[i]) - zp[i] - ed * gp[i];
              fw += f * f;
              rv += r * r;
            }
          la += (fw - rv) / (4.0 * ed);
        }
        acc = log(u) < la;
      }
      p = la32 >= 0.f ? 1.f : (la32 == la32 ? expf(la32) : 0.f);
    }
    n_ev += 1ull;
    return finish_step(a, c, row, acc, p, zp, gp, lpp, mala, defer);
  }
};

}  // namespace bst
