// sampler.cuh -- per-chain proposal / accept state machines.
//
// A chain-tile kernel alternates
//     pre(row)   -> write the point to evaluate into ze[row]      (proposal)
//     engine     -> lle[row] = logL(ze[row]), gle[row] = grad     (emulator / analytic)
//     post(row)  -> Metropolis / Hamiltonian / tree bookkeeping    (accept)
// so one likelihood evaluation of a whole tile of chains is in flight at a
// time.  Everything here is per chain, O(d) or O(d^2), and runs on the threads
// that own the chains; the log-acceptance ratios and Hamiltonian energies are
// formed in FP64 from the working-precision state.
//
// Target in whitened coordinates (paper Sec. 2.2, Eq. (2.12), Algorithm 1):
//     x = mu + L z,   log pi_z(z) = logL(x) + log prior(x) + sum_i log L_ii.
#pragma once

#include "common.cuh"

namespace bst {

// Per-chain vector loops over the state rows (global memory).  The rows are distinct, so the
// parameters are restrict-qualified: the loads of one loop can all be in flight at once
// instead of each waiting behind the previous iteration's stores.
template <typename R>
__device__ __forceinline__ void vcopy(R *__restrict__ dst, const R *__restrict__ src, int d) {
#pragma unroll 4
  for (int i = 0; i < d; ++i) dst[i] = src[i];
}
template <typename R>
__device__ __forceinline__ void vcopy2(R *__restrict__ d0, const R *__restrict__ s0, R *__restrict__ d1,
                                       const R *__restrict__ s1, int d) {
#pragma unroll 4
  for (int i = 0; i < d; ++i) {
    d0[i] = s0[i];
    d1[i] = s1[i];
  }
}
// qh = qe + e/2 ge; zn = ze + e qh  (first half of a leapfrog step)
template <typename R>
__device__ __forceinline__ void half_kick_drift(R *__restrict__ qh, R *__restrict__ zn, const R *__restrict__ qe,
                                                const R *__restrict__ ge, const R *__restrict__ zs, R e, int d) {
#pragma unroll 4
  for (int i = 0; i < d; ++i) {
    qh[i] = qe[i] + R(0.5) * e * ge[i];
    zn[i] = zs[i] + e * qh[i];
  }
}
// second half: qend = qh + e/2 gn, zend = zn, gend = gn; returns |qend|^2 (FP64 sum)
template <typename R>
__device__ __forceinline__ double half_kick_store(R *__restrict__ zend, R *__restrict__ qend, R *__restrict__ gend,
                                                  const R *__restrict__ qh, const R *__restrict__ zn,
                                                  const R *__restrict__ gn, R e, int d) {
  double qq = 0.0;
#pragma unroll 4
  for (int i = 0; i < d; ++i) {
    const R qn = qh[i] + R(0.5) * e * gn[i];
    qq += static_cast<double>(qn) * qn;
    zend[i] = zn[i];
    qend[i] = qn;
    gend[i] = gn[i];
  }
  return qq;
}

// zp = zc + a u + b v
template <typename R>
__device__ __forceinline__ void vaxpby(R *__restrict__ zp, const R *__restrict__ zc, R a, const R *__restrict__ u, R b,
                                       const R *__restrict__ v, int d) {
#pragma unroll 4
  for (int i = 0; i < d; ++i) zp[i] = zc[i] + a * u[i] + b * v[i];
}
// q1 += e/2 g1; z1 += e q1; zp = z1
template <typename R>
__device__ __forceinline__ void kick_drift_inplace(R *__restrict__ z1, R *__restrict__ q1, const R *__restrict__ g1,
                                                   R *__restrict__ zp, R e, int d) {
#pragma unroll 4
  for (int i = 0; i < d; ++i) {
    const R q = q1[i] + R(0.5) * e * g1[i];
    const R z = z1[i] + e * q;
    q1[i] = q;
    z1[i] = z;
    zp[i] = z;
  }
}

template <typename R>
struct Chain {
  const StepArgs<R> &a;
  __device__ Chain(const StepArgs<R> &args) : a(args) {}

  __device__ R *z(int c) const { return a.st.z + static_cast<size_t>(c) * a.dp; }
  __device__ R *g(int c) const { return a.st.g + static_cast<size_t>(c) * a.dp; }
  __device__ R *ze(int r) const { return a.st.ze + static_cast<size_t>(r) * a.dp; }
  __device__ R *gle(int r) const { return a.st.gle + static_cast<size_t>(r) * a.dp; }
  __device__ R *wv(int c, int k) const {
    return a.st.work + static_cast<size_t>(c) * a.st.work_stride + static_cast<size_t>(k) * a.dp;
  }

  static __device__ double accept_prob(double la) {
    if (!(la == la)) return 0.0;
    return la >= 0.0 ? 1.0 : exp(la);
  }

  // x-space sample record and Welford hand-off after a chain finishes an iteration.
  __device__ void record(int c, int row, int step) const {
    const int d = a.d;
    R x[kMaxD];
    a.tgt.to_x_prior(z(c), x);
    if (a.samples && ((step + 1) % a.thin) == 0) {
      R *dst = a.samples + (static_cast<size_t>(step / a.thin) * a.n_chains + c) * d;
      for (int i = 0; i < d; ++i) dst[i] = x[i];
    }
    if (a.welford_on) {
      R *xb = a.xbuf + static_cast<size_t>(row) * a.dp;
      for (int i = 0; i < d; ++i) xb[i] = x[i];
    }
  }

  // log pi_z and grad log pi_z at the evaluated point of row r (x written to xo).
  __device__ double logpi_eval(int r, R *gout, R *xo) const {
    const double lpr = a.tgt.to_x_prior(ze(r), xo);
    const double lp = static_cast<double>(a.st.lle[r]) + lpr + a.tgt.logdet;
    if (gout) {
      vcopy(gout, static_cast<const R *>(gle(r)), a.d);
      a.tgt.add_prior_grad(xo, gout);
    }
    return lp;
  }

  __device__ void count(int c, bool accepted, double la, int evals) const {
    a.st.acc_stat[c] += accept_prob(la);
    a.st.accepts[c] += accepted ? 1ull : 0ull;
    a.st.evals[c] += static_cast<unsigned long long>(evals);
  }

  // ---------------------------------------------------------------- MH
  // Random walk in whitened units: z' = z + eps xi.
  __device__ bool mh_pre(int c) const {
    if (a.st.steps_done[c] >= a.n_steps) return false;
    R xi[kMaxD];
    draw_normals<R>(a.seed, c, a.st.iter[c], kXi, a.d, xi);
    const R e = static_cast<R>(a.eps);
    R *zc = z(c), *zp = ze(c);
    {
      R *__restrict__ dst = zp;
      const R *__restrict__ src = zc;
#pragma unroll 4
      for (int i = 0; i < a.d; ++i) dst[i] = src[i] + e * xi[i];
    }
    return true;
  }
  __device__ bool mh_post(int c) const {
    R x[kMaxD];
    const double lpp = logpi_eval(c, nullptr, x);
    const uint32_t it = a.st.iter[c];
    const double la = lpp - static_cast<double>(a.st.lp[c]);
    const double u = draw_uniform<double>(a.seed, c, it, kAccept, 0);
    const bool acc = log(u) < la;
    if (acc) {
      vcopy(z(c), static_cast<const R *>(ze(c)), a.d);
      a.st.lp[c] = static_cast<R>(lpp);
    }
    count(c, acc, la, 1);
    finish(c, c);
    return true;
  }

  // ---------------------------------------------------------------- MALA
  // Eq. (2.3): z' = z + eps grad + sqrt(2 eps) xi; q(a|b) = N(a; b + eps grad(b), 2 eps I).
  __device__ bool mala_pre(int c) const {
    if (a.st.steps_done[c] >= a.n_steps) return false;
    R xi[kMaxD];
    draw_normals<R>(a.seed, c, a.st.iter[c], kXi, a.d, xi);
    const R e = static_cast<R>(a.eps), s = static_cast<R>(sqrt(2.0 * a.eps));
    vaxpby(ze(c), static_cast<const R *>(z(c)), e, static_cast<const R *>(g(c)), s, static_cast<const R *>(xi), a.d);
    return true;
  }
  __device__ bool mala_post(int c) const {
    R x[kMaxD], gp[kMaxD];
    const double lpp = logpi_eval(c, gp, x);
    const uint32_t it = a.st.iter[c];
    R *zc = z(c), *gc = g(c), *zp = ze(c);
    const double e = a.eps;
    double fwd = 0.0, rev = 0.0;
    for (int i = 0; i < a.d; ++i) {
      const double f = static_cast<double>(zp[i]) - zc[i] - e * gc[i];
      const double r = static_cast<double>(zc[i]) - zp[i] - e * gp[i];
      fwd += f * f;
      rev += r * r;
    }
    // log q(z|z') - log q(z'|z)
    const double la = lpp - static_cast<double>(a.st.lp[c]) + (fwd - rev) / (4.0 * e);
    const double u = draw_uniform<double>(a.seed, c, it, kAccept, 0);
    const bool acc = log(u) < la;
    if (acc) {
      vcopy2(zc, static_cast<const R *>(zp), gc, static_cast<const R *>(gp), a.d);
      a.st.lp[c] = static_cast<R>(lpp);
    }
    count(c, acc, la, 1);
    finish(c, c);
    return true;
  }

  // ---------------------------------------------------------------- HMC
  // Identity mass in whitened space (Eqs. (2.7)-(2.8)); leapfrog; accept on H0 - H1.
  // work vectors: 0 z1, 1 q1, 2 g1; dwork: 0 leapfrogs done, 1 H0.
  __device__ double *dwork_ptr(int c) const;

  __device__ bool hmc_pre(int c) const {
    if (a.st.steps_done[c] >= a.n_steps) return false;
    double *dw = dwork_ptr(c);
    R *z1 = wv(c, 0), *q1 = wv(c, 1), *g1 = wv(c, 2);
    const R e = static_cast<R>(a.eps);
    if (dw[0] == 0.0) {
      R q[kMaxD];
      draw_normals<R>(a.seed, c, a.st.iter[c], kXi, a.d, q);
      double qq = 0.0;
      for (int i = 0; i < a.d; ++i) qq += static_cast<double>(q[i]) * q[i];
      vcopy2(z1, static_cast<const R *>(z(c)), g1, static_cast<const R *>(g(c)), a.d);
      vcopy(q1, static_cast<const R *>(q), a.d);
      dw[1] = -static_cast<double>(a.st.lp[c]) + 0.5 * qq;
    }
    kick_drift_inplace(z1, q1, static_cast<const R *>(g1), ze(c), e, a.d);
    return true;
  }
  __device__ bool hmc_post(int c) const {
    double *dw = dwork_ptr(c);
    R *z1 = wv(c, 0), *q1 = wv(c, 1), *g1 = wv(c, 2);
    R x[kMaxD];
    const double lp1 = logpi_eval(c, g1, x);
    const R e = static_cast<R>(a.eps);
    double qq = 0.0;
    for (int i = 0; i < a.d; ++i) {
      q1[i] += R(0.5) * e * g1[i];
      qq += static_cast<double>(q1[i]) * q1[i];
    }
    dw[0] += 1.0;
    a.st.evals[c] += 1ull;
    if (dw[0] < a.n_leapfrog) return false;
    dw[0] = 0.0;
    const double H1 = -lp1 + 0.5 * qq;
    const double la = dw[1] - H1;
    const uint32_t it = a.st.iter[c];
    const double u = draw_uniform<double>(a.seed, c, it, kAccept, 0);
    const bool acc = log(u) < la;
    if (acc) {
      vcopy2(z(c), static_cast<const R *>(z1), g(c), static_cast<const R *>(g1), a.d);
      a.st.lp[c] = static_cast<R>(lp1);
    }
    count(c, acc, la, 0);
    finish(c, c);
    return true;
  }

  // ---------------------------------------------------------------- NUTS
  // Hoffman & Gelman (2014) Algorithm 3, unrolled into one leapfrog per call:
  // the tree of the current doubling is built leaf by leaf; pending left
  // siblings wait on a per-level stack and are merged (candidate kept with
  // probability n''/(n'+n''), U-turn check of the merged span) when their right
  // sibling completes.  work vectors: 0 zm 1 qm 2 gm 3 zp 4 qp 5 gp 6 zs 7 gs
  // 8 qh, level i: 9+4i first z, 10+4i first q, 11+4i cand z, 12+4i cand g.
  // dwork: 0 new-iteration flag, 1 log u, 2 H0, 3 n, 4 lp of selected,
  // 5 acceptance-stat sum, 6 j, 7 v, 8 m_sub, 9 leaves, 10 diverged, 11 moved,
  // 12+i cand lp, 22+i node n.
  __device__ bool nuts_pre(int c) const {
    if (a.st.steps_done[c] >= a.n_steps) return false;
    double *dw = dwork_ptr(c);
    const int d = a.d;
    const uint32_t it = a.st.iter[c];
    if (dw[0] != 0.0) {
      R q0[kMaxD];
      draw_normals<R>(a.seed, c, it, kXi, d, q0);
      double qq = 0.0;
      for (int i = 0; i < d; ++i) qq += static_cast<double>(q0[i]) * q0[i];
      const double H0 = -static_cast<double>(a.st.lp[c]) + 0.5 * qq;
      dw[2] = H0;
      dw[1] = log(draw_uniform<double>(a.seed, c, it, kAccept, 0)) - H0;
      R *zc = z(c), *gc = g(c);
      R *zm = wv(c, 0), *qm = wv(c, 1), *gm = wv(c, 2), *zp = wv(c, 3), *qp = wv(c, 4),
        *gp = wv(c, 5), *zs = wv(c, 6), *gs = wv(c, 7);
      vcopy2(zm, static_cast<const R *>(zc), gm, static_cast<const R *>(gc), d);
      vcopy2(zp, static_cast<const R *>(zc), gp, static_cast<const R *>(gc), d);
      vcopy2(zs, static_cast<const R *>(zc), gs, static_cast<const R *>(gc), d);
      vcopy2(qm, static_cast<const R *>(q0), qp, static_cast<const R *>(q0), d);
      dw[3] = 1.0;
      dw[4] = static_cast<double>(a.st.lp[c]);
      dw[5] = 0.0;
      dw[6] = 0.0;
      dw[7] = draw_uniform<double>(a.seed, c, it, kNutsDir, 0) < 0.5 ? -1.0 : 1.0;
      dw[8] = 0.0;
      dw[9] = 0.0;
      dw[10] = 0.0;
      dw[11] = 0.0;
      dw[0] = 0.0;
    }
    const bool back = dw[7] < 0.0;
    const R e = static_cast<R>(dw[7] * a.eps);
    R *ze_ = wv(c, back ? 0 : 3), *qe = wv(c, back ? 1 : 4), *ge = wv(c, back ? 2 : 5);
    R *qh = wv(c, 8), *zn = ze(c);
    half_kick_drift(qh, zn, static_cast<const R *>(qe), static_cast<const R *>(ge), static_cast<const R *>(ze_), e, d);
    return true;
  }

  __device__ bool nuts_post(int c) const {
    double *dw = dwork_ptr(c);
    const int d = a.d;
    const uint32_t it = a.st.iter[c];
    const bool back = dw[7] < 0.0;
    const double v = dw[7];
    const R e = static_cast<R>(v * a.eps);
    R x[kMaxD], gn[kMaxD];
    const double lpn = logpi_eval(c, gn, x);
    R *qh = wv(c, 8), *zn = ze(c);
    R *zend = wv(c, back ? 0 : 3), *qend = wv(c, back ? 1 : 4), *gend = wv(c, back ? 2 : 5);
    const double qq = half_kick_store(zend, qend, gend, static_cast<const R *>(qh), static_cast<const R *>(zn),
                                      static_cast<const R *>(gn), e, d);
    a.st.evals[c] += 1ull;
    dw[9] += 1.0;
    const int leaf = static_cast<int>(dw[9]);
    const double Hl = -lpn + 0.5 * qq;
    dw[5] += accept_prob(dw[2] - Hl);
    const double log_u = dw[1];
    const double nl = (log_u <= -Hl) ? 1.0 : 0.0;
    const bool sl = log_u < kNutsDeltaMax - Hl;
    if (!sl) {
      dw[10] = 1.0;
      return nuts_finish(c);
    }
    // current node = the new leaf; first = leaf, candidate = leaf
    int first_src = -1, cand_src = -1;
    double node_n = nl;
    const int m_sub = static_cast<int>(dw[8]);
    const int j = static_cast<int>(dw[6]);
    int lvl = 0;
    while ((m_sub >> lvl) & 1) {
      // merge pending left sibling at level lvl with the node
      const double ln = dw[22 + lvl];
      const double u = draw_uniform<double>(a.seed, c, it, kNutsSel,
                                            static_cast<uint32_t>(8 * (leaf - 1) + lvl + 1));
      const double ntot = ln + node_n;
      const bool take_right = ntot > 0.0 && u * ntot < node_n;
      if (!take_right) cand_src = lvl;
      // U-turn check of the merged span [left.first .. leaf]
      const R *fz = wv(c, 9 + 4 * lvl), *fq = wv(c, 10 + 4 * lvl);
      double s1 = 0.0, s2 = 0.0;
      for (int i = 0; i < d; ++i) {
        const double dz = v * (static_cast<double>(zend[i]) - fz[i]);
        s1 += dz * fq[i];
        s2 += dz * qend[i];
      }
      first_src = lvl;
      node_n = ntot;
      ++lvl;
      if (!(s1 >= 0.0 && s2 >= 0.0)) return nuts_finish(c);
    }
    // candidate vectors of the node
    const R *cz = cand_src < 0 ? zend : wv(c, 11 + 4 * cand_src);
    const R *cg = cand_src < 0 ? gend : wv(c, 12 + 4 * cand_src);
    const double clp = cand_src < 0 ? lpn : dw[12 + cand_src];
    if (lvl == j) {
      // the subtree of this doubling is complete: progressive top-level selection
      const double ut = draw_uniform<double>(a.seed, c, it, kNutsTop, static_cast<uint32_t>(j));
      if (ut * dw[3] < node_n) {
        vcopy2(wv(c, 6), cz, wv(c, 7), cg, d);
        dw[4] = clp;
        dw[11] = 1.0;
      }
      dw[3] += node_n;
      const R *zm = wv(c, 0), *qm = wv(c, 1), *zp = wv(c, 3), *qp = wv(c, 4);
      double s1 = 0.0, s2 = 0.0;
      for (int i = 0; i < d; ++i) {
        const double dz = static_cast<double>(zp[i]) - zm[i];
        s1 += dz * qm[i];
        s2 += dz * qp[i];
      }
      const int jn = j + 1;
      dw[6] = jn;
      if (!(s1 >= 0.0 && s2 >= 0.0) || jn >= a.max_depth) return nuts_finish(c);
      dw[7] = draw_uniform<double>(a.seed, c, it, kNutsDir, static_cast<uint32_t>(jn)) < 0.5 ? -1.0 : 1.0;
      dw[8] = 0.0;
    } else {
      // park the node as the pending left sibling at level lvl
      R *pz = wv(c, 9 + 4 * lvl), *pq = wv(c, 10 + 4 * lvl), *pcz = wv(c, 11 + 4 * lvl),
        *pcg = wv(c, 12 + 4 * lvl);
      const R *fz = first_src < 0 ? zend : wv(c, 9 + 4 * first_src);
      const R *fq = first_src < 0 ? qend : wv(c, 10 + 4 * first_src);
      if (first_src != lvl) vcopy2(pz, fz, pq, fq, d);
      if (cand_src != lvl) vcopy2(pcz, cz, pcg, cg, d);
      dw[12 + lvl] = clp;
      dw[22 + lvl] = node_n;
      dw[8] = m_sub + 1;
    }
    return false;
  }

  __device__ bool nuts_finish(int c) const {
    double *dw = dwork_ptr(c);
    R *zc = z(c), *gc = g(c), *zs = wv(c, 6), *gs = wv(c, 7);
    for (int i = 0; i < a.d; ++i) {
      zc[i] = zs[i];
      gc[i] = gs[i];
    }
    a.st.lp[c] = static_cast<R>(dw[4]);
    const double leaves = dw[9];
    a.st.acc_stat[c] += leaves > 0.0 ? dw[5] / leaves : 0.0;
    a.st.accepts[c] += dw[11] != 0.0 ? 1ull : 0ull;
    a.st.divs[c] += dw[10] != 0.0 ? 1ull : 0ull;
    dw[0] = 1.0;
    finish(c, c);
    return true;
  }

  // ---------------------------------------------------------------- AIES
  // Goodman-Weare stretch move (Sec. 2.3): y = z_j + Z (z_i - z_j),
  // Z = (u (a - 1) + 1)^2 / a (Eq. (2.15)); accept with min(1, Z^(d-1) pi(y)/pi(z_i)).
  // Row r moves walker k = r % (W/2) of half h of ensemble r / (W/2).
  __device__ int aies_walker(int r, int h) const {
    const int half = a.aies_walkers / 2;
    return (r / half) * a.aies_walkers + h * half + (r % half);
  }
  __device__ bool aies_pre(int r, int h) const {
    const int i = aies_walker(r, h);
    if (a.st.steps_done[i] >= a.n_steps) return false;
    const int half = a.aies_walkers / 2;
    const int base = (r / half) * a.aies_walkers + (1 - h) * half;
    const uint32_t it = a.st.iter[i];
    const double up = draw_uniform<double>(a.seed, i, it, kAiesPartner, 0);
    int jj = static_cast<int>(up * half);
    if (jj > half - 1) jj = half - 1;
    const int jw = base + jj;
    const double uz = draw_uniform<double>(a.seed, i, it, kAiesZ, 0);
    const double t = uz * (a.aies_a - 1.0) + 1.0;
    const double Z = t * t / a.aies_a;
    dwork_ptr(i)[0] = Z;
    const R *__restrict__ zi = z(i);
    const R *__restrict__ zj = z(jw);
    R *__restrict__ y = ze(r);
    const R Zr = static_cast<R>(Z);
#pragma unroll 4
    for (int q = 0; q < a.d; ++q) y[q] = zj[q] + Zr * (zi[q] - zj[q]);
    return true;
  }
  __device__ bool aies_post(int r, int h) const {
    const int i = aies_walker(r, h);
    R x[kMaxD];
    const double lpy = logpi_eval(r, nullptr, x);
    const double Z = dwork_ptr(i)[0];
    const double la = (a.d - 1) * log(Z) + lpy - static_cast<double>(a.st.lp[i]);
    const uint32_t it = a.st.iter[i];
    const double u = draw_uniform<double>(a.seed, i, it, kAccept, 0);
    const bool acc = log(u) < la;
    if (acc) {
      vcopy(z(i), static_cast<const R *>(ze(r)), a.d);
      a.st.lp[i] = static_cast<R>(lpy);
    }
    count(i, acc, la, 1);
    finish(i, r);
    return true;
  }

  // ---------------------------------------------------------------- batch modes
  __device__ bool refresh_pre(int c) const {
    if (a.st.steps_done[c] >= 1) return false;
    R *zc = z(c), *zp = ze(c);
    for (int i = 0; i < a.d; ++i) zp[i] = zc[i];
    return true;
  }
  __device__ bool refresh_post(int c) const {
    R x[kMaxD], gp[kMaxD];
    const double lp = logpi_eval(c, gp, x);
    a.st.lp[c] = static_cast<R>(lp);
    R *gc = g(c);
    for (int i = 0; i < a.d; ++i) gc[i] = gp[i];
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
  // the chain of the row completed an iteration (for the covariance accumulator).
  __device__ bool pre(int row, int h) const {
    switch (a.mode) {
      case kModeMH: return mh_pre(row);
      case kModeMALA: return mala_pre(row);
      case kModeHMC: return hmc_pre(row);
      case kModeNUTS: return nuts_pre(row);
      case kModeAIES: return aies_pre(row, h);
      case kModeRefresh: return refresh_pre(row);
      default: return false;
    }
  }
  __device__ bool post(int row, int h) const {
    switch (a.mode) {
      case kModeMH: return mh_post(row);
      case kModeMALA: return mala_post(row);
      case kModeHMC: return hmc_post(row);
      case kModeNUTS: return nuts_post(row);
      case kModeAIES: return aies_post(row, h);
      case kModeRefresh: return refresh_post(row);
      default: return false;
    }
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
  // x = mu + L v on the first d entries (same summation order as TargetView::to_x_prior)
  static __device__ __forceinline__ void to_x(const StepArgs<R> &a, const R *v, R *x) {
#pragma unroll
    for (int i = 0; i < DB; ++i) {
      R acc = R(0);
      if (i < a.d) {
        acc = a.tgt.mu[i];
#pragma unroll
        for (int j = 0; j <= i; ++j) acc += a.tgt.L[i * a.d + j] * v[j];
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
        if (!(xp[i] >= a.tgt.lower[i] && xp[i] <= a.tgt.upper[i])) inside = false;
        if (a.tgt.any_gauss && a.tgt.gauss[i]) lpr -= 0.5 * static_cast<double>(xp[i]) * static_cast<double>(xp[i]);
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
    if (t.any_gauss) {
      R xp[DB];
      to_x(a, z1, xp);
#pragma unroll
      for (int j = 0; j < DB; ++j)
        if (j < d) {
          R sg = 0;
#pragma unroll
          for (int i = j; i < DB; ++i)
            if (i < d && a.tgt.gauss[i]) sg -= a.tgt.L[i * a.d + j] * xp[i];
          g1[j] += sg;
        }
    }
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
    if (mala && t.any_gauss) {
      R xp[DB];
      to_x(a, zp, xp);
#pragma unroll
      for (int j = 0; j < DB; ++j)
        if (j < d) {
          R sg = 0;
#pragma unroll
          for (int i = j; i < DB; ++i)
            if (i < d && a.tgt.gauss[i]) sg -= a.tgt.L[i * a.d + j] * xp[i];
          gp[j] += sg;
        }
    }
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

// Double-precision per-chain scratch lives after the R vectors of the work row.
template <typename R>
__device__ double *Chain<R>::dwork_ptr(int c) const {
  char *base = reinterpret_cast<char *>(a.st.work + static_cast<size_t>(c) * a.st.work_stride);
  const size_t vec_bytes = static_cast<size_t>(kDworkOffsetVecs) * a.dp * sizeof(R);
  return reinterpret_cast<double *>(base + vec_bytes);
}

}  // namespace bst
