/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Sources followed, in the order of this file:
 *  - Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 *    easy as 1, 2, 3", SC'11 (the Philox S-box and key schedule).
 *  - Box-Muller normals: Box & Muller (1958).
 *  - Whitened target: paper Sec. 2.2, Eqs. (2.4)-(2.5) and (2.12), Algorithm 1:
 *    log pi_z(z) = log pi_x(mu + L z) + log|det L|.
 *  - Analytic "theory map" likelihood: f(x) = A tanh(B x_c + c) + N x_n with
 *    a Gaussian chi^2 (the synthetic stand-in for the paper's Planck + BAO
 *    likelihood, Sec. 4).
 *  - Emulator: tanh multilayer perceptron predicting a standardised chi^2
 *    (stand-in for the CLiENT likelihood emulator, Sec. 1 and Sec. 4), with
 *    its input gradient by reverse-mode differentiation.
 *  - MH: random-walk proposal in whitened units (Sec. 2, Sec. 4).
 *  - MALA: proposal of Sec. 2.1, Eq. (2.3), with the Metropolis-Hastings
 *    correction for the Gaussian proposal N(z + eps grad, 2 eps I).
 *  - HMC: Hamiltonian of Eq. (2.1) with identity mass in whitened space
 *    (Eqs. (2.7)-(2.8)), leapfrog integrator, Metropolis accept on Delta H.
 *  - NUTS: Hoffman & Gelman (2014) Algorithm 3 (slice variable, doubling in a
 *    random direction, U-turn test, progressive top-level selection), as
 *    described in Sec. 2.1; the multinomial variant (Betancourt 2017, "A
 *    Conceptual Introduction to Hamiltonian Monte Carlo", Appendix A) draws the
 *    point from the trajectory with weights exp(-H) instead of a slice.
 *  - AIES: Goodman & Weare (2010) stretch move, Sec. 2.3, Eqs. (2.13)-(2.15);
 *    the differential-evolution move of Sec. 2.3 (after Eq. (2.15)).
 *  - Covariance adaptation: pooled covariance, Cholesky factorisation with
 *    diagonal regularisation (Sec. 3.2); Chan, Golub & LeVeque (1979) merge.
 *  - Adam: Kingma & Ba (2015), Algorithm 1.
 *  - ESS: multi-chain effective sample size with Geyer's initial monotone
 *    sequence (Gelman et al., Bayesian Data Analysis 3rd ed., Sec. 11.5).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11)                                     */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 24-bit uniform on the open interval (0, 1): ((x >> 8) + 1/2) 2^-24. */
static double u01(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

static void block(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t purpose, uint32_t b,
                  uint32_t out[4]) {
  uint32_t ctr[4] = {chain, iter, purpose, b};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

double orc_uniform(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t purpose, uint32_t idx) {
  uint32_t w[4];
  block(seed, chain, iter, purpose, idx / 4u, w);
  return u01(w[idx % 4u]);
}

/* Normals k = 4b .. 4b+3 come from block b: Box-Muller on (u0,u1), (u2,u3). */
void orc_normals(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t purpose, int n, double *out) {
  for (int b = 0; 4 * b < n; ++b) {
    uint32_t w[4];
    block(seed, chain, iter, purpose, (uint32_t)b, w);
    double u[4] = {u01(w[0]), u01(w[1]), u01(w[2]), u01(w[3])};
    double v[4];
    for (int p = 0; p < 2; ++p) {
      double r = sqrt(-2.0 * log(u[2 * p]));
      double a = 2.0 * M_PI * u[2 * p + 1];
      v[2 * p] = r * cos(a);
      v[2 * p + 1] = r * sin(a);
    }
    for (int k = 0; k < 4 && 4 * b + k < n; ++k) out[4 * b + k] = v[k];
  }
}

/* Round to the nearest bfloat16 value (8 significant bits), ties to even. */
double orc_bf16_round(double v) {
  if (v == 0.0 || !isfinite(v)) return v;
  int e;
  double m = frexp(v, &e);         /* v = m 2^e, 0.5 <= |m| < 1 */
  double s = ldexp(m, 8);          /* 8 significant bits -> integer part */
  double r = nearbyint(s);         /* default rounding mode: to nearest, ties even */
  return ldexp(r, e - 8);
}

/* Round to the nearest IEEE 754 binary16 value (11 significant bits, exponent range
 * 2^-14 .. 2^15, subnormals in steps of 2^-24), ties to even; |v| >= 65520 gives inf. */
double orc_fp16_round(double v) {
  if (v == 0.0 || !isfinite(v)) return v;
  const double a = fabs(v);
  if (a >= 65520.0) return v > 0 ? INFINITY : -INFINITY;
  if (a < ldexp(1.0, -14)) return ldexp(nearbyint(ldexp(v, 24)), -24);
  int e;
  double m = frexp(v, &e);         /* v = m 2^e, 0.5 <= |m| < 1 */
  return ldexp(nearbyint(ldexp(m, 11)), e - 11);
}

/* Operand rounding of the emulation modes: 1 BF16, 2 FP16, else exact. */
static double oround(double v, int mode) {
  return mode == 1 ? orc_bf16_round(v) : (mode == 2 ? orc_fp16_round(v) : v);
}

/* ------------------------------------------------------------------------ */
/* Likelihoods                                                              */
/* ------------------------------------------------------------------------ */

/* Analytic likelihood: r = data - f(x); logL = -||r||^2 / (2 sigma^2). */
static double analytic_logl(const orc_model *m, const double *x, double *grad) {
  const int H = m->n_hidden, n = m->n_data, dc = m->d_c, dn = m->d - m->d_c;
  double *t = (double *)malloc(sizeof(double) * (size_t)H);
  double *r = (double *)malloc(sizeof(double) * (size_t)n);
  for (int k = 0; k < H; ++k) {
    double a = m->c[k];
    for (int j = 0; j < dc; ++j) a += m->B[k * dc + j] * x[j];
    t[k] = m->linear ? a : tanh(a);
  }
  double chi2 = 0.0;
  for (int i = 0; i < n; ++i) {
    double f = 0.0;
    for (int k = 0; k < H; ++k) f += m->A[i * H + k] * t[k];
    for (int j = 0; j < dn; ++j) f += m->N[i * dn + j] * x[dc + j];
    r[i] = m->data[i] - f;
    chi2 += r[i] * r[i];
  }
  const double s2 = m->sigma * m->sigma;
  if (grad) {
    /* d logL / dx_c = B^T [ (1 - t^2) (A^T r) ] / sigma^2; d/dx_n = N^T r / sigma^2 */
    for (int j = 0; j < m->d; ++j) grad[j] = 0.0;
    for (int k = 0; k < H; ++k) {
      double atr = 0.0;
      for (int i = 0; i < n; ++i) atr += m->A[i * H + k] * r[i];
      double dk = (m->linear ? 1.0 : (1.0 - t[k] * t[k])) * atr / s2;
      for (int j = 0; j < dc; ++j) grad[j] += m->B[k * dc + j] * dk;
    }
    for (int j = 0; j < dn; ++j) {
      double ntr = 0.0;
      for (int i = 0; i < n; ++i) ntr += m->N[i * dn + j] * r[i];
      grad[dc + j] = ntr / s2;
    }
  }
  free(t);
  free(r);
  return -0.5 * chi2 / s2;
}

/* Emulator: u = (x - m_in)/s_in; h_1 = tanh(W_1 u + b_1); h_l = tanh(W_l h_{l-1} + b_l);
 * out = w_o . h_D + b_o; chi2_hat = out_s out + out_m (linear output) or
 * out_floor + exp(out_s out + out_m) (log output); logL = -chi2_hat / 2.  The gradient of
 * the log output is that of the linear one times exp(out_s out + out_m) (chain rule).
 * BF16 mode: operands of the hidden-to-hidden products (W_2..W_D, h_1..h_{D-1})
 * and every adjoint vector delta_1..delta_D are rounded to bfloat16; the input
 * layer, the output layer and all sums are exact.  FP16 mode rounds the same
 * operands to binary16, and seeds the adjoint with -w_o (1 - h_D^2) / 2 (without
 * out_s, which scales the input gradient instead: the tensor-core engine keeps
 * the FP16 adjoint vectors away from the range limit that way).               */
static double emulator_logl(const orc_model *m, const double *x, double *grad) {
  const int d = m->d, D = m->depth, w = m->width, bf = m->bf16;
  const double *P = m->params;
  double *u = (double *)malloc(sizeof(double) * (size_t)d);
  double *h = (double *)malloc(sizeof(double) * (size_t)D * (size_t)w); /* h_l rows */
  const double **W = (const double **)malloc(sizeof(double *) * (size_t)(D + 1));
  const double **b = (const double **)malloc(sizeof(double *) * (size_t)(D + 1));
  const double *p = P;
  for (int l = 1; l <= D; ++l) {
    int fan_in = (l == 1) ? d : w;
    W[l] = p; p += (size_t)w * (size_t)fan_in;
    b[l] = p; p += w;
  }
  const double *wo = p; p += w;
  const double bo = *p;

  for (int j = 0; j < d; ++j) u[j] = (x[j] - m->in_m[j]) / m->in_s[j];
  for (int l = 1; l <= D; ++l) {
    double *hl = h + (size_t)(l - 1) * w;
    for (int k = 0; k < w; ++k) {
      double a = b[l][k];
      if (l == 1) {
        for (int j = 0; j < d; ++j) a += W[1][k * d + j] * u[j];
      } else {
        const double *hp = h + (size_t)(l - 2) * w;
        for (int j = 0; j < w; ++j) {
          double wkj = W[l][(size_t)k * w + j];
          a += oround(wkj, bf) * hp[j];
        }
      }
      hl[k] = tanh(a);
    }
    if (bf && l < D)
      for (int k = 0; k < w; ++k) hl[k] = oround(hl[k], bf);
  }
  const double *hD = h + (size_t)(D - 1) * w;
  double out = bo;
  for (int k = 0; k < w; ++k) out += wo[k] * hD[k];
  const double arg = m->out_s * out + m->out_m;
  const double tfac = m->out_log ? exp(arg) : 1.0; /* d chi2_hat / d arg */
  const double chi2 = m->out_log ? m->out_floor + tfac : arg;

  if (grad) {
    double *dl = (double *)malloc(sizeof(double) * (size_t)w);
    double *dn = (double *)malloc(sizeof(double) * (size_t)w);
    const double c = (bf == 2) ? -0.5 : -0.5 * m->out_s; /* d logL / d out (FP16: without out_s) */
    const double gscale = tfac * ((bf == 2) ? m->out_s : 1.0);
    for (int k = 0; k < w; ++k) {
      dl[k] = c * wo[k] * (1.0 - hD[k] * hD[k]);
      if (bf) dl[k] = oround(dl[k], bf);
    }
    for (int l = D; l >= 2; --l) {
      const double *hp = h + (size_t)(l - 2) * w;
      for (int j = 0; j < w; ++j) {
        double s = 0.0;
        for (int k = 0; k < w; ++k) {
          double wkj = W[l][(size_t)k * w + j];
          s += oround(wkj, bf) * dl[k];
        }
        dn[j] = s * (1.0 - hp[j] * hp[j]);
        if (bf) dn[j] = oround(dn[j], bf);
      }
      memcpy(dl, dn, sizeof(double) * (size_t)w);
    }
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int k = 0; k < w; ++k) s += W[1][k * d + j] * dl[k];
      grad[j] = s / m->in_s[j] * gscale;
    }
    free(dl);
    free(dn);
  }
  free(u);
  free(h);
  free(W);
  free(b);
  return -0.5 * chi2;
}

double orc_loglike(const orc_model *m, const double *x, double *grad_x) {
  return m->lik_kind == ORC_LIK_ANALYTIC ? analytic_logl(m, x, grad_x) : emulator_logl(m, x, grad_x);
}

void orc_loglike_batch(const orc_model *m, int n, const double *x, double *logl, double *grad) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n; ++i)
    logl[i] = orc_loglike(m, x + (size_t)i * m->d, grad ? grad + (size_t)i * m->d : NULL);
}

/* Whitened log target, Eq. (2.12) / Algorithm 1:
 *   x = mu + L z;  log pi_z = logL(x) + log prior(x) + sum_i log L_ii.
 * The prior is a hard box (0 inside, -inf outside) times N(0,1) on the dims
 * flagged gauss (constant terms dropped).  The gradient returned is that of
 * logL + the Gaussian prior, mapped to z by L^T, and is defined outside the
 * box as well (leapfrog points outside the box keep moving).
 * Smooth bounds (Sec. 3.1, the likelihood extended outside the box by a smooth
 * exponential penalty): on a dim with pen_w[i] > 0 the box does not reject;
 * instead the density is multiplied by exp(-r_i^2 / 2), r_i = the distance of
 * x_i outside [lower_i, upper_i] divided by pen_w[i] (0 inside), whose log is
 * continuous with a continuous gradient -r_i / pen_w[i] at the bounds.        */
double orc_logpost_z(const orc_model *m, const double *z, double *grad_z, double *x_out) {
  const int d = m->d;
  double *x = (double *)malloc(sizeof(double) * (size_t)d);
  double *gx = (double *)malloc(sizeof(double) * (size_t)d);
  for (int i = 0; i < d; ++i) {
    double s = m->mu[i];
    for (int j = 0; j <= i; ++j) s += m->L[i * d + j] * z[j];
    x[i] = s;
  }
  double lp = orc_loglike(m, x, grad_z ? gx : NULL);
  int inside = 1;
  for (int i = 0; i < d; ++i) {
    if (m->pen_w && m->pen_w[i] > 0.0) {
      const double out = x[i] < m->lower[i] ? x[i] - m->lower[i] : (x[i] > m->upper[i] ? x[i] - m->upper[i] : 0.0);
      const double r = out / m->pen_w[i];
      lp += -0.5 * r * r;
      if (grad_z) gx[i] += -r / m->pen_w[i];
    } else if (!(x[i] >= m->lower[i] && x[i] <= m->upper[i])) {
      inside = 0;
    }
    if (m->gauss && m->gauss[i]) {
      lp += -0.5 * x[i] * x[i];
      if (grad_z) gx[i] += -x[i];
    }
  }
  double logdet = 0.0;
  for (int i = 0; i < d; ++i) logdet += log(fabs(m->L[i * d + i]));
  lp += logdet;
  if (!inside) lp = -INFINITY;
  if (grad_z) {
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int i = j; i < d; ++i) s += m->L[i * d + j] * gx[i];
      grad_z[j] = s;
    }
  }
  if (x_out) memcpy(x_out, x, sizeof(double) * (size_t)d);
  free(x);
  free(gx);
  return lp;
}

void orc_logpost_batch(const orc_model *m, int n, const double *z, double *lp, double *grad) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n; ++i)
    lp[i] = orc_logpost_z(m, z + (size_t)i * m->d, grad ? grad + (size_t)i * m->d : NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* Samplers                                                                 */
/* ------------------------------------------------------------------------ */
static double dot(int d, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < d; ++i) s += a[i] * b[i];
  return s;
}

static void to_x(const orc_model *m, const double *z, double *x) {
  for (int i = 0; i < m->d; ++i) {
    double s = m->mu[i];
    for (int j = 0; j <= i; ++j) s += m->L[i * m->d + j] * z[j];
    x[i] = s;
  }
}

/* Metropolis decision shared by MH, MALA, HMC and AIES: accept iff log u < log alpha;
 * a NaN log alpha rejects.                                                   */
static int metropolis(double log_alpha, double u) { return log(u) < log_alpha; }

static double accept_prob(double log_alpha) {
  if (!(log_alpha == log_alpha)) return 0.0;
  return log_alpha >= 0.0 ? 1.0 : exp(log_alpha);
}

typedef struct {
  double log_alpha, log_u;
  int accepted;
  int depth, nleaf, diverged;
  double margin; /* NUTS: smallest decision margin of the iteration (test bookkeeping) */
} step_out;

/* Random-walk MH in whitened units: z' = z + eps xi, xi ~ N(0, I). */
static void mh_step(const orc_model *m, const orc_step_params *p, uint32_t chain, uint32_t it,
                    double *z, double *lp, double *g, step_out *o, double *work) {
  const int d = m->d;
  double *xi = work, *zp = work + d;
  orc_normals(p->seed, chain, it, ORC_P_XI, d, xi);
  for (int i = 0; i < d; ++i) zp[i] = z[i] + p->eps * xi[i];
  double lpp = orc_logpost_z(m, zp, NULL, NULL);
  double la = lpp - *lp;
  double u = orc_uniform(p->seed, chain, it, ORC_P_ACCEPT, 0);
  o->log_alpha = la;
  o->log_u = log(u);
  o->accepted = metropolis(la, u);
  if (o->accepted) {
    memcpy(z, zp, sizeof(double) * (size_t)d);
    *lp = lpp;
  }
  (void)g;
}

/* MALA, Eq. (2.3): z' = z + eps grad + sqrt(2 eps) xi; q(a|b) = N(a; b + eps grad(b), 2 eps I). */
static void mala_step(const orc_model *m, const orc_step_params *p, uint32_t chain, uint32_t it,
                      double *z, double *lp, double *g, step_out *o, double *work) {
  const int d = m->d;
  const double eps = p->eps;
  double *xi = work, *zp = work + d, *gp = work + 2 * d;
  orc_normals(p->seed, chain, it, ORC_P_XI, d, xi);
  for (int i = 0; i < d; ++i) zp[i] = z[i] + eps * g[i] + sqrt(2.0 * eps) * xi[i];
  double lpp = orc_logpost_z(m, zp, gp, NULL);
  double fwd = 0.0, rev = 0.0; /* ||z' - z - eps g||^2, ||z - z' - eps g'||^2 */
  for (int i = 0; i < d; ++i) {
    double a = zp[i] - z[i] - eps * g[i];
    double b = z[i] - zp[i] - eps * gp[i];
    fwd += a * a;
    rev += b * b;
  }
  double log_q_fwd = -fwd / (4.0 * eps); /* log q(z'|z) */
  double log_q_rev = -rev / (4.0 * eps); /* log q(z|z') */
  double la = lpp - *lp + log_q_rev - log_q_fwd;
  double u = orc_uniform(p->seed, chain, it, ORC_P_ACCEPT, 0);
  o->log_alpha = la;
  o->log_u = log(u);
  o->accepted = metropolis(la, u);
  if (o->accepted) {
    memcpy(z, zp, sizeof(double) * (size_t)d);
    memcpy(g, gp, sizeof(double) * (size_t)d);
    *lp = lpp;
  }
}

/* HMC: q ~ N(0, I) (identity mass in whitened space, Eq. (2.7)); L leapfrog steps of
 * H(z, q) = -log pi_z(z) + q.q/2 (Eq. (2.8)); accept with probability min(1, exp(H0 - H1)). */
static void hmc_step(const orc_model *m, const orc_step_params *p, uint32_t chain, uint32_t it,
                     double *z, double *lp, double *g, step_out *o, double *work) {
  const int d = m->d;
  const double eps = p->eps;
  double *q = work, *z1 = work + d, *g1 = work + 2 * d;
  orc_normals(p->seed, chain, it, ORC_P_XI, d, q);
  const double H0 = -(*lp) + 0.5 * dot(d, q, q);
  memcpy(z1, z, sizeof(double) * (size_t)d);
  memcpy(g1, g, sizeof(double) * (size_t)d);
  double lp1 = *lp;
  for (int s = 0; s < p->n_leapfrog; ++s) {
    for (int i = 0; i < d; ++i) q[i] += 0.5 * eps * g1[i];
    for (int i = 0; i < d; ++i) z1[i] += eps * q[i];
    lp1 = orc_logpost_z(m, z1, g1, NULL);
    for (int i = 0; i < d; ++i) q[i] += 0.5 * eps * g1[i];
  }
  const double H1 = -lp1 + 0.5 * dot(d, q, q);
  double la = H0 - H1;
  double u = orc_uniform(p->seed, chain, it, ORC_P_ACCEPT, 0);
  o->log_alpha = la;
  o->log_u = log(u);
  o->accepted = metropolis(la, u);
  if (o->accepted) {
    memcpy(z, z1, sizeof(double) * (size_t)d);
    memcpy(g, g1, sizeof(double) * (size_t)d);
    *lp = lp1;
  }
}

/* Plain leapfrog integrator used by HMC (exposed for the reversibility pins). */
double orc_leapfrog(const orc_model *m, double *z, double *q, double *g, double eps, int n) {
  const int d = m->d;
  double lp = 0.0;
  for (int s = 0; s < n; ++s) {
    for (int i = 0; i < d; ++i) q[i] += 0.5 * eps * g[i];
    for (int i = 0; i < d; ++i) z[i] += eps * q[i];
    lp = orc_logpost_z(m, z, g, NULL);
    for (int i = 0; i < d; ++i) q[i] += 0.5 * eps * g[i];
  }
  return lp;
}

/* ---- NUTS (Hoffman & Gelman 2014, Algorithm 3), written recursively. ---- */
#define NUTS_DELTA_MAX 1000.0

typedef struct {
  const orc_model *m;
  const orc_step_params *p;
  uint32_t chain, it;
  double log_u;     /* log of the slice variable                    */
  int leaf;         /* leapfrogs taken so far in this iteration     */
  int diverged;
  double H0;
  double acc_sum;   /* sum over leaves of min(1, exp(H0 - H))       */
  int multinomial;  /* weights exp(H0 - H) instead of the slice      */
  double margin;    /* smallest distance of a decision from its threshold so far: log-scale
                     * tests (slice, Delta_max, multinomial weights) in absolute units,
                     * uniform-against-ratio tests in probability units, U-turn dot products
                     * relative to the sum of the magnitudes of their terms.  Bookkeeping for
                     * the parity tests only; no decision depends on it.                  */
} nuts_ctx;

typedef struct {
  double *zm, *qm, *gm;   /* backward end (theta-, r-) and its gradient */
  double *zp, *qp, *gp;   /* forward end  (theta+, r+) and its gradient */
  double *zc, *gc;        /* candidate theta' and its gradient          */
  double lpc;
  double n;               /* n'  */
  double lw;              /* multinomial: log of the summed leaf weights exp(H0 - H) */
  int s;                  /* s'  */
} nuts_tree;

static double *nalloc(int d) { return (double *)malloc(sizeof(double) * (size_t)d); }
static double log_add_exp(double a, double b) {
  const double hi = a > b ? a : b, lo = a > b ? b : a;
  return hi + log1p(exp(lo - hi));
}
static void tree_alloc(nuts_tree *t, int d) {
  t->zm = nalloc(d); t->qm = nalloc(d); t->gm = nalloc(d);
  t->zp = nalloc(d); t->qp = nalloc(d); t->gp = nalloc(d);
  t->zc = nalloc(d); t->gc = nalloc(d);
}
static void tree_free(nuts_tree *t) {
  free(t->zm); free(t->qm); free(t->gm); free(t->zp); free(t->qp); free(t->gp);
  free(t->zc); free(t->gc);
}

static void note_margin(double *margin, double m) {
  m = fabs(m);
  if (m < *margin) *margin = m;
}

/* U-turn criterion: (theta+ - theta-) . r- >= 0 and (theta+ - theta-) . r+ >= 0.
 * margin (may be NULL) receives the relative distance of the two products from 0. */
static int no_uturn_m(int d, const double *zm, const double *qm, const double *zp, const double *qp,
                      double *margin) {
  double a = 0.0, b = 0.0, aa = 0.0, bb = 0.0;
  for (int i = 0; i < d; ++i) {
    double dz = zp[i] - zm[i];
    a += dz * qm[i];
    b += dz * qp[i];
    aa += fabs(dz * qm[i]);
    bb += fabs(dz * qp[i]);
  }
  if (margin) {
    note_margin(margin, aa > 0.0 ? a / aa : 1.0);
    note_margin(margin, bb > 0.0 ? b / bb : 1.0);
  }
  return a >= 0.0 && b >= 0.0;
}
static int no_uturn(int d, const double *zm, const double *qm, const double *zp, const double *qp) {
  return no_uturn_m(d, zm, qm, zp, qp, NULL);
}

/* BuildTree(theta, r, u, v, j, eps).  Input: the state (z, q, g) to extend from.
 * The uniform that decides each in-subtree merge is keyed by the index of the last
 * leapfrog of the merged node and its level: idx = 8 * leaf + level.            */
static void build_tree(nuts_ctx *c, const double *z, const double *q, const double *g, int v,
                       int j, nuts_tree *out) {
  const orc_model *m = c->m;
  const int d = m->d;
  if (j == 0) {
    const double e = v * c->p->eps;
    double *q1 = out->qp, *z1 = out->zp, *g1 = out->gp;
    for (int i = 0; i < d; ++i) q1[i] = q[i] + 0.5 * e * g[i];
    for (int i = 0; i < d; ++i) z1[i] = z[i] + e * q1[i];
    double lp1 = orc_logpost_z(m, z1, g1, NULL);
    for (int i = 0; i < d; ++i) q1[i] += 0.5 * e * g1[i];
    c->leaf++;
    const double H = -lp1 + 0.5 * dot(d, q1, q1);
    if (c->multinomial) {
      /* weight exp(H0 - H); divergent when the energy error exceeds Delta_max */
      out->lw = c->H0 - H;
      out->n = 0.0;
      out->s = (H - c->H0 < NUTS_DELTA_MAX) ? 1 : 0;
      note_margin(&c->margin, H - c->H0 - NUTS_DELTA_MAX);
    } else {
      out->n = (c->log_u <= -H) ? 1.0 : 0.0;
      out->s = (c->log_u < NUTS_DELTA_MAX - H) ? 1 : 0;
      note_margin(&c->margin, c->log_u + H);
      note_margin(&c->margin, c->log_u - NUTS_DELTA_MAX + H);
    }
    if (!out->s) c->diverged = 1;
    c->acc_sum += accept_prob(c->H0 - H);
    memcpy(out->zm, z1, sizeof(double) * (size_t)d);
    memcpy(out->qm, q1, sizeof(double) * (size_t)d);
    memcpy(out->gm, g1, sizeof(double) * (size_t)d);
    memcpy(out->zc, z1, sizeof(double) * (size_t)d);
    memcpy(out->gc, g1, sizeof(double) * (size_t)d);
    out->lpc = lp1;
    return;
  }
  /* first half */
  build_tree(c, z, q, g, v, j - 1, out);
  if (!out->s) return;
  nuts_tree t2;
  tree_alloc(&t2, d);
  if (v == -1)
    build_tree(c, out->zm, out->qm, out->gm, v, j - 1, &t2);
  else
    build_tree(c, out->zp, out->qp, out->gp, v, j - 1, &t2);
  /* the ends move outward in direction v */
  if (v == -1) {
    memcpy(out->zm, t2.zm, sizeof(double) * (size_t)d);
    memcpy(out->qm, t2.qm, sizeof(double) * (size_t)d);
    memcpy(out->gm, t2.gm, sizeof(double) * (size_t)d);
  } else {
    memcpy(out->zp, t2.zp, sizeof(double) * (size_t)d);
    memcpy(out->qp, t2.qp, sizeof(double) * (size_t)d);
    memcpy(out->gp, t2.gp, sizeof(double) * (size_t)d);
  }
  if (t2.s) {
    /* with probability n'' / (n' + n'') (multinomial: w'' / (w' + w'')), take the
     * candidate of the second half */
    const double ntot = out->n + t2.n;
    const double u =
        orc_uniform(c->p->seed, c->chain, c->it, ORC_P_NUTS_SEL, (uint32_t)(8 * (c->leaf - 1) + j));
    int take;
    if (c->multinomial) {
      const double lw_tot = log_add_exp(out->lw, t2.lw);
      take = u < exp(t2.lw - lw_tot);
      note_margin(&c->margin, u - exp(t2.lw - lw_tot));
      out->lw = lw_tot;
    } else {
      take = ntot > 0.0 && u * ntot < t2.n;
      if (ntot > 0.0) note_margin(&c->margin, u - t2.n / ntot);
    }
    if (take) {
      memcpy(out->zc, t2.zc, sizeof(double) * (size_t)d);
      memcpy(out->gc, t2.gc, sizeof(double) * (size_t)d);
      out->lpc = t2.lpc;
    }
    out->s = no_uturn_m(d, out->zm, out->qm, out->zp, out->qp, &c->margin);
    out->n = ntot;
  } else {
    out->s = 0;
  }
  tree_free(&t2);
}

static void nuts_step(const orc_model *m, const orc_step_params *p, uint32_t chain, uint32_t it,
                      double *z, double *lp, double *g, step_out *o, double *acc_stat) {
  const int d = m->d;
  nuts_ctx c;
  c.m = m; c.p = p; c.chain = chain; c.it = it; c.leaf = 0; c.diverged = 0; c.acc_sum = 0.0;
  c.margin = INFINITY;
  c.multinomial = (p->kernel == ORC_NUTS_MULTINOMIAL);
  double *q0 = nalloc(d);
  orc_normals(p->seed, chain, it, ORC_P_XI, d, q0);
  c.H0 = -(*lp) + 0.5 * dot(d, q0, q0);
  /* slice variable u ~ U(0, exp(-H0)) */
  c.log_u = log(orc_uniform(p->seed, chain, it, ORC_P_ACCEPT, 0)) - c.H0;
  /* full trajectory ends */
  double *zm = nalloc(d), *qm = nalloc(d), *gm = nalloc(d);
  double *zp = nalloc(d), *qp = nalloc(d), *gp = nalloc(d);
  double *zs = nalloc(d), *gs = nalloc(d);
  memcpy(zm, z, sizeof(double) * (size_t)d); memcpy(zp, z, sizeof(double) * (size_t)d);
  memcpy(qm, q0, sizeof(double) * (size_t)d); memcpy(qp, q0, sizeof(double) * (size_t)d);
  memcpy(gm, g, sizeof(double) * (size_t)d); memcpy(gp, g, sizeof(double) * (size_t)d);
  memcpy(zs, z, sizeof(double) * (size_t)d); memcpy(gs, g, sizeof(double) * (size_t)d);
  double lps = *lp;
  double n = 1.0;
  double lw = 0.0; /* multinomial: log weight of the trajectory so far (the start: exp(0)) */
  int s = 1, j = 0;
  nuts_tree t;
  tree_alloc(&t, d);
  while (s && j < p->max_depth) {
    double uv = orc_uniform(p->seed, chain, it, ORC_P_NUTS_DIR, (uint32_t)j);
    int v = (uv < 0.5) ? -1 : 1;
    if (v == -1) {
      build_tree(&c, zm, qm, gm, v, j, &t);
      memcpy(zm, t.zm, sizeof(double) * (size_t)d);
      memcpy(qm, t.qm, sizeof(double) * (size_t)d);
      memcpy(gm, t.gm, sizeof(double) * (size_t)d);
    } else {
      build_tree(&c, zp, qp, gp, v, j, &t);
      memcpy(zp, t.zp, sizeof(double) * (size_t)d);
      memcpy(qp, t.qp, sizeof(double) * (size_t)d);
      memcpy(gp, t.gp, sizeof(double) * (size_t)d);
    }
    if (t.s) {
      /* with probability min(1, n'/n) (multinomial: min(1, w'/w)), move to the new
       * subtree's candidate */
      double ut = orc_uniform(p->seed, chain, it, ORC_P_NUTS_TOP, (uint32_t)j);
      note_margin(&c.margin, c.multinomial ? ut - exp(t.lw - lw) : ut - t.n / n);
      if (c.multinomial ? (ut < exp(t.lw - lw)) : (ut * n < t.n)) {
        memcpy(zs, t.zc, sizeof(double) * (size_t)d);
        memcpy(gs, t.gc, sizeof(double) * (size_t)d);
        lps = t.lpc;
      }
    }
    n += t.n;
    if (c.multinomial && t.s) lw = log_add_exp(lw, t.lw);
    s = t.s && no_uturn_m(d, zm, qm, zp, qp, &c.margin);
    j++;
  }
  o->accepted = (memcmp(zs, z, sizeof(double) * (size_t)d) != 0);
  memcpy(z, zs, sizeof(double) * (size_t)d);
  memcpy(g, gs, sizeof(double) * (size_t)d);
  *lp = lps;
  o->depth = j;
  o->nleaf = c.leaf;
  o->diverged = c.diverged;
  o->log_alpha = 0.0;
  o->log_u = c.log_u;
  o->margin = c.margin;
  *acc_stat = c.leaf > 0 ? c.acc_sum / c.leaf : 0.0;
  tree_free(&t);
  free(q0); free(zm); free(qm); free(gm); free(zp); free(qp); free(gp); free(zs); free(gs);
}

static void record(const orc_model *m, const orc_trace *tr, int n_chains, int t, int c,
                   const double *z, const step_out *o) {
  if (!tr) return;
  const size_t k = (size_t)t * (size_t)n_chains + (size_t)c;
  if (tr->samples) to_x(m, z, tr->samples + k * (size_t)m->d);
  if (tr->trace_logalpha) tr->trace_logalpha[k] = o->log_alpha;
  if (tr->trace_logu) tr->trace_logu[k] = o->log_u;
  if (tr->trace_accept) tr->trace_accept[k] = o->accepted;
  if (tr->trace_depth) tr->trace_depth[k] = o->depth;
  if (tr->trace_nleaf) tr->trace_nleaf[k] = o->nleaf;
  /* NUTS takes many decisions per iteration (o->nleaf > 0); the others one Metropolis test */
  if (tr->trace_margin) tr->trace_margin[k] = o->nleaf > 0 ? o->margin : fabs(o->log_alpha - o->log_u);
}

/* AIES stretch move (Sec. 2.3).  Walkers of one ensemble are split into halves S0, S1;
 * S0 moves using partners drawn uniformly from S1, then S1 using the updated S0.
 * y = z_j + Z (z_i - z_j), Z = (u (a - 1) + 1)^2 / a (Eq. (2.15));
 * accept with probability min(1, Z^(d-1) pi(y) / pi(z_i)).  Because x = mu + L z is
 * affine, this is the same move as in x-space.
 * Differential-evolution move (Sec. 2.3, after Eq. (2.15)), same halves and order:
 * y = z_i + gamma (z_j - z_k) with j != k uniform in the other half and
 * gamma = (1 + eta) 2.38 / sqrt(2 d), eta ~ N(0, de_sigma^2); the proposal is symmetric,
 * so accept with probability min(1, pi(y) / pi(z_i)).  j is uniform 0 of the partner
 * stream, k uniform 1 over the other half - 1 walkers (skipping j), eta the first
 * normal of the stretch-factor stream.                                           */
static void aies_run(const orc_model *m, const orc_step_params *p, int n_chains, double *z,
                     double *lp, double *g, uint32_t *iter, double *accept_stat, int64_t *accepts,
                     int64_t *evals, const orc_trace *tr) {
  const int d = m->d, W = p->aies_walkers, half = W / 2, n_ens = n_chains / W;
  const double a = p->aies_a;
  for (int t = 0; t < p->n_steps; ++t) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < n_ens; ++e) {
      double *y = nalloc(d);
      for (int h = 0; h < 2; ++h) {
        const int act = e * W + h * half, oth = e * W + (1 - h) * half;
        /* proposals for the whole active half use the partner positions as they are
         * before this half moves (the other half is not modified in this sweep).   */
        for (int k = 0; k < half; ++k) {
          const int i = act + k;
          const uint32_t it = iter[i];
          double up = orc_uniform(p->seed, (uint32_t)i, it, ORC_P_AIES_PARTNER, 0);
          int jj = (int)(up * half);
          if (jj > half - 1) jj = half - 1;
          const int jw = oth + jj;
          double lpy, la;
          if (p->kernel == ORC_AIES_DE) {
            double uk = orc_uniform(p->seed, (uint32_t)i, it, ORC_P_AIES_PARTNER, 1);
            int kk = (int)(uk * (half - 1));
            if (kk > half - 2) kk = half - 2;
            if (kk >= jj) ++kk;
            const int kw = oth + kk;
            double eta;
            orc_normals(p->seed, (uint32_t)i, it, ORC_P_AIES_Z, 1, &eta);
            const double gamma = (1.0 + p->de_sigma * eta) * 2.38 / sqrt(2.0 * d);
            for (int q = 0; q < d; ++q)
              y[q] = z[(size_t)i * d + q] + gamma * (z[(size_t)jw * d + q] - z[(size_t)kw * d + q]);
            lpy = orc_logpost_z(m, y, NULL, NULL);
            la = lpy - lp[i];
          } else {
            double uz = orc_uniform(p->seed, (uint32_t)i, it, ORC_P_AIES_Z, 0);
            double Z = (uz * (a - 1.0) + 1.0) * (uz * (a - 1.0) + 1.0) / a;
            for (int q = 0; q < d; ++q)
              y[q] = z[(size_t)jw * d + q] + Z * (z[(size_t)i * d + q] - z[(size_t)jw * d + q]);
            lpy = orc_logpost_z(m, y, NULL, NULL);
            la = (d - 1) * log(Z) + lpy - lp[i];
          }
          double u = orc_uniform(p->seed, (uint32_t)i, it, ORC_P_ACCEPT, 0);
          step_out o;
          memset(&o, 0, sizeof(o));
          o.log_alpha = la;
          o.log_u = log(u);
          o.accepted = metropolis(la, u);
          if (o.accepted) {
            memcpy(z + (size_t)i * d, y, sizeof(double) * (size_t)d);
            lp[i] = lpy;
          }
          accept_stat[i] += accept_prob(la);
          accepts[i] += o.accepted;
          evals[i] += 1;
          iter[i] = it + 1;
          record(m, tr, n_chains, t, i, z + (size_t)i * d, &o);
        }
      }
      free(y);
    }
  }
  (void)g;
}

int orc_run(const orc_model *m, const orc_step_params *p, int n_chains, double *z, double *lp,
            double *g, uint32_t *iter, double *accept_stat, int64_t *accepts, int64_t *evals,
            int64_t *divergences, const orc_trace *tr) {
  const int d = m->d;
  if (p->kernel == ORC_AIES || p->kernel == ORC_AIES_DE) {
    if (p->aies_walkers < 2 || p->aies_walkers % 2 || n_chains % p->aies_walkers) return -1;
    if (p->kernel == ORC_AIES_DE && (p->aies_walkers < 4 || !(p->de_sigma >= 0.0))) return -1;
    aies_run(m, p, n_chains, z, lp, g, iter, accept_stat, accepts, evals, tr);
    return 0;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < n_chains; ++c) {
    double *work = nalloc(4 * d);
    double *zc = z + (size_t)c * d, *gc = g + (size_t)c * d;
    for (int t = 0; t < p->n_steps; ++t) {
      const uint32_t it = iter[c];
      step_out o;
      memset(&o, 0, sizeof(o));
      double as = 0.0;
      switch (p->kernel) {
        case ORC_MH:
          mh_step(m, p, (uint32_t)c, it, zc, &lp[c], gc, &o, work);
          evals[c] += 1;
          as = accept_prob(o.log_alpha);
          break;
        case ORC_MALA:
          mala_step(m, p, (uint32_t)c, it, zc, &lp[c], gc, &o, work);
          evals[c] += 1;
          as = accept_prob(o.log_alpha);
          break;
        case ORC_HMC:
          hmc_step(m, p, (uint32_t)c, it, zc, &lp[c], gc, &o, work);
          evals[c] += p->n_leapfrog;
          as = accept_prob(o.log_alpha);
          break;
        case ORC_NUTS:
        case ORC_NUTS_MULTINOMIAL:
          nuts_step(m, p, (uint32_t)c, it, zc, &lp[c], gc, &o, &as);
          evals[c] += o.nleaf;
          divergences[c] += o.diverged;
          break;
        default:
          break;
      }
      accept_stat[c] += as;
      accepts[c] += o.accepted;
      iter[c] = it + 1;
      record(m, tr, n_chains, t, c, zc, &o);
    }
    free(work);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Covariance adaptation (Sec. 3.2)                                         */
/* ------------------------------------------------------------------------ */

/* Pooled mean and unbiased covariance of n samples x[n][d] (two passes). */
void orc_pooled_cov(int n, int d, const double *x, double *mean, double *cov) {
  for (int j = 0; j < d; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += x[(size_t)i * d + j];
    mean[j] = s / n;
  }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double s = 0.0;
      for (int i = 0; i < n; ++i)
        s += (x[(size_t)i * d + a] - mean[a]) * (x[(size_t)i * d + b] - mean[b]);
      cov[a * d + b] = s / (n - 1);
    }
}

/* Chan, Golub & LeVeque pairwise merge of (n, mean, M2) statistics into a. */
void orc_chan_merge(int d, double na, double *mean_a, double *M2_a, double nb, const double *mean_b,
                    const double *M2_b) {
  const double n = na + nb;
  if (nb == 0.0) return;
  double *delta = nalloc(d);
  for (int i = 0; i < d; ++i) delta[i] = mean_b[i] - mean_a[i];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      M2_a[i * d + j] += M2_b[i * d + j] + delta[i] * delta[j] * na * nb / n;
  for (int i = 0; i < d; ++i) mean_a[i] += delta[i] * nb / n;
  free(delta);
}

static int cholesky(int d, const double *S, double *L) {
  memset(L, 0, sizeof(double) * (size_t)d * (size_t)d);
  for (int j = 0; j < d; ++j) {
    double s = S[j * d + j];
    for (int k = 0; k < j; ++k) s -= L[j * d + k] * L[j * d + k];
    if (!(s > 0.0)) return -1;
    L[j * d + j] = sqrt(s);
    for (int i = j + 1; i < d; ++i) {
      double t = S[i * d + j];
      for (int k = 0; k < j; ++k) t -= L[i * d + k] * L[j * d + k];
      L[i * d + j] = t / L[j * d + j];
    }
  }
  return 0;
}

/* Cholesky with diagonal regularisation: plain first; on failure add
 * delta (tr S / d) I with delta = jitter0, x10 per retry, while delta <= 1e-2.
 * Returns 0 on success (used = delta actually added, 0 for none), -1 if not PD. */
int orc_cholesky_jitter(int d, const double *S, double jitter0, double *L, double *used) {
  if (cholesky(d, S, L) == 0) {
    *used = 0.0;
    return 0;
  }
  double tr = 0.0;
  for (int i = 0; i < d; ++i) tr += S[i * d + i];
  double *T = nalloc(d * d);
  for (double delta = jitter0; delta <= 1e-2 * (1.0 + 1e-9); delta *= 10.0) {
    memcpy(T, S, sizeof(double) * (size_t)d * (size_t)d);
    for (int i = 0; i < d; ++i) T[i * d + i] += delta * tr / d;
    if (cholesky(d, T, L) == 0) {
      *used = delta;
      free(T);
      return 0;
    }
  }
  free(T);
  *used = -1.0;
  return -1;
}

/* Keep x fixed across a change of whitening: z_new = L_new^{-1} (mu_old + L_old z_old - mu_new). */
void orc_remap_z(int d, int n, const double *mu_old, const double *L_old, const double *mu_new,
                 const double *L_new, double *z) {
  double *x = nalloc(d);
  for (int c = 0; c < n; ++c) {
    double *zc = z + (size_t)c * d;
    for (int i = 0; i < d; ++i) {
      double s = mu_old[i];
      for (int j = 0; j <= i; ++j) s += L_old[i * d + j] * zc[j];
      x[i] = s - mu_new[i];
    }
    for (int i = 0; i < d; ++i) { /* forward substitution */
      double s = x[i];
      for (int j = 0; j < i; ++j) s -= L_new[i * d + j] * zc[j];
      zc[i] = s / L_new[i * d + i];
    }
  }
  free(x);
}

/* ------------------------------------------------------------------------ */
/* Emulator training                                                        */
/* ------------------------------------------------------------------------ */

/* Loss = mean_i (out_i - y_i)^2 with y_i = (t(chi2_i) - out_m) / out_s (the standardised
 * regression target), t(c) = c for the linear output and log(max(c - out_floor, 1e-30)) for
 * the log output.  grad (same layout as params) = d loss / d params, by reverse-mode
 * differentiation.  bf16 = 1: the operands of the hidden-layer products (layers 2..D) are
 * rounded to bfloat16 -- W_l and h_{l-1} in the forward product, the adjoint delta_l and
 * h_{l-1} in the weight gradient, delta_l and W_l in the adjoint product -- with every sum
 * exact (the mixed-precision training of the tensor-core path); the input layer, the output
 * layer, the biases and the (1 - h^2) factors are exact.                                    */
double orc_train_loss_grad(int d, int D, int w, const double *P, const double *in_m,
                           const double *in_s, double out_m, double out_s, int out_log,
                           double out_floor, int bf16, int mb, const double *X, const double *chi2,
                           double *grad) {
  const int rm = bf16 ? 1 : 0; /* oround mode */
  size_t np = (size_t)d * w + w + (size_t)(D - 1) * ((size_t)w * w + w) + w + 1;
  memset(grad, 0, sizeof(double) * np);
  double loss = 0.0;
  size_t off_W[16], off_b[16];
  size_t o = 0;
  for (int l = 1; l <= D; ++l) {
    int fan_in = (l == 1) ? d : w;
    off_W[l] = o; o += (size_t)w * fan_in;
    off_b[l] = o; o += w;
  }
  const size_t off_wo = o, off_bo = o + w;
  double *h = nalloc((D + 1) * w); /* h[0] holds u (first d entries) */
  double *dl = nalloc(w), *dn = nalloc(w);
  for (int i = 0; i < mb; ++i) {
    const double *x = X + (size_t)i * d;
    for (int j = 0; j < d; ++j) h[j] = (x[j] - in_m[j]) / in_s[j];
    for (int l = 1; l <= D; ++l) {
      int fan_in = (l == 1) ? d : w;
      const double *Wl = P + off_W[l], *bl = P + off_b[l], *hp = h + (size_t)(l - 1) * w;
      double *hl = h + (size_t)l * w;
      for (int k = 0; k < w; ++k) {
        double a = bl[k];
        if (l == 1)
          for (int j = 0; j < fan_in; ++j) a += Wl[(size_t)k * fan_in + j] * hp[j];
        else
          for (int j = 0; j < fan_in; ++j) a += oround(Wl[(size_t)k * fan_in + j], rm) * oround(hp[j], rm);
        hl[k] = tanh(a);
      }
    }
    const double *hD = h + (size_t)D * w;
    double out = P[off_bo];
    for (int k = 0; k < w; ++k) out += P[off_wo + k] * hD[k];
    const double tc = out_log ? log(fmax(chi2[i] - out_floor, 1e-30)) : chi2[i];
    const double y = (tc - out_m) / out_s;
    const double r = out - y;
    loss += r * r;
    const double dout = 2.0 * r / mb;
    grad[off_bo] += dout;
    for (int k = 0; k < w; ++k) {
      grad[off_wo + k] += dout * hD[k];
      dl[k] = dout * P[off_wo + k] * (1.0 - hD[k] * hD[k]);
    }
    for (int l = D; l >= 1; --l) {
      int fan_in = (l == 1) ? d : w;
      const double *Wl = P + off_W[l], *hp = h + (size_t)(l - 1) * w;
      const int r = (l > 1) ? rm : 0;
      for (int k = 0; k < w; ++k) {
        grad[off_b[l] + k] += dl[k];
        for (int j = 0; j < fan_in; ++j) grad[off_W[l] + (size_t)k * fan_in + j] += oround(dl[k], r) * oround(hp[j], r);
      }
      if (l > 1) {
        for (int j = 0; j < w; ++j) {
          double s = 0.0;
          for (int k = 0; k < w; ++k) s += oround(Wl[(size_t)k * w + j], r) * oround(dl[k], r);
          dn[j] = s * (1.0 - hp[j] * hp[j]);
        }
        memcpy(dl, dn, sizeof(double) * (size_t)w);
      }
    }
  }
  free(h); free(dl); free(dn);
  return loss / mb;
}

/* Adam (Kingma & Ba 2015, Algorithm 1), step t >= 1. */
void orc_adam(int n, double *p, const double *g, double *m1, double *m2, int t, double lr,
              double b1, double b2, double eps) {
  const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (int i = 0; i < n; ++i) {
    m1[i] = b1 * m1[i] + (1.0 - b1) * g[i];
    m2[i] = b2 * m2[i] + (1.0 - b2) * g[i] * g[i];
    const double mh = m1[i] / c1, vh = m2[i] / c2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* ------------------------------------------------------------------------ */
/* Multi-chain effective sample size (BDA3 Sec. 11.5, Geyer truncation)     */
/* ------------------------------------------------------------------------ */
void orc_ess(int n_draws, int n_chains, int d, const double *S, double *ess) {
  const int n = n_draws, M = n_chains;
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < d; ++q) {
    double *mean = nalloc(M);
    double gm = 0.0;
    for (int c = 0; c < M; ++c) {
      double s = 0.0;
      for (int t = 0; t < n; ++t) s += S[((size_t)t * M + c) * d + q];
      mean[c] = s / n;
      gm += mean[c];
    }
    gm /= M;
    /* W: mean within-chain variance; B/n: variance of the chain means */
    double Wv = 0.0, Bv = 0.0;
    for (int c = 0; c < M; ++c) {
      double s = 0.0;
      for (int t = 0; t < n; ++t) {
        double e = S[((size_t)t * M + c) * d + q] - mean[c];
        s += e * e;
      }
      Wv += s / (n - 1);
      Bv += (mean[c] - gm) * (mean[c] - gm);
    }
    Wv /= M;
    const double B_over_n = (M > 1) ? Bv / (M - 1) : 0.0;
    const double var_plus = (n - 1.0) / n * Wv + B_over_n;
    /* rho_t = 1 - V_t / (2 var_plus), V_t the variogram at lag t (rho_0 = 1);
     * tau = -1 + 2 sum_k P_k, P_k = rho_2k + rho_2k+1, summed while P_k > 0,
     * each P_k capped by its predecessor (initial monotone sequence).         */
    double sum_P = 0.0, prev_P = INFINITY;
    for (int t = 0; t + 1 < n; t += 2) {
      double rho[2];
      for (int k = 0; k < 2; ++k) {
        const int lag = t + k;
        double v = 0.0;
        for (int c = 0; c < M; ++c)
          for (int i = lag; i < n; ++i) {
            double e = S[((size_t)i * M + c) * d + q] - S[((size_t)(i - lag) * M + c) * d + q];
            v += e * e;
          }
        v /= (double)M * (double)(n - lag);
        rho[k] = 1.0 - v / (2.0 * var_plus);
      }
      double P = rho[0] + rho[1];
      if (!(P > 0.0)) break;
      if (P > prev_P) P = prev_P;
      sum_P += P;
      prev_P = P;
    }
    const double tau = -1.0 + 2.0 * sum_P;
    ess[q] = (double)M * n / tau;
    free(mean);
  }
}
