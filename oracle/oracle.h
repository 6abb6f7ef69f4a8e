/*
 * oracle.h -- plain FP64 CPU oracle for batched emulator posterior sampling.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library under
 * paper_2606_04895_gb300/csrc; both were written separately from the paper
 * ("Posterior sampling in the Age of Emulators", arXiv 2606.04895) and from
 * the published algorithms it cites.
 *
 * Everything is double precision.  Loops are written in the order the paper
 * (or the cited algorithm) states them; OpenMP only parallelises over
 * independent chains.
 */
#ifndef ORC_ORACLE_H
#define ORC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Random-number purposes: the third word of the Philox counter. */
enum {
  ORC_P_XI = 1,          /* proposal noise / momentum normals          */
  ORC_P_ACCEPT = 2,      /* Metropolis uniform, NUTS slice variable     */
  ORC_P_NUTS_DIR = 3,    /* NUTS doubling direction                     */
  ORC_P_NUTS_SEL = 4,    /* NUTS in-subtree candidate selection         */
  ORC_P_NUTS_TOP = 5,    /* NUTS top-level progressive selection        */
  ORC_P_AIES_PARTNER = 6,/* AIES partner walker                         */
  ORC_P_AIES_Z = 7       /* AIES stretch factor                         */
};

enum { ORC_MH = 0, ORC_MALA = 1, ORC_HMC = 2, ORC_NUTS = 3, ORC_AIES = 4, ORC_AIES_DE = 5,
       ORC_NUTS_MULTINOMIAL = 6 };
enum { ORC_LIK_EMULATOR = 0, ORC_LIK_ANALYTIC = 1 };

/* Target model: likelihood + prior + whitening (x = mu + L z). */
typedef struct {
  int lik_kind;       /* ORC_LIK_*                                         */
  int d;              /* parameter dimension                               */
  /* analytic likelihood f(x) = A tanh(B x_c + c) + N x_n                  */
  int d_c;            /* leading dims entering through the tanh map        */
  int n_hidden;       /* rows of B                                         */
  int n_data;         /* rows of A and N                                   */
  int linear;         /* 1: tanh replaced by the identity                  */
  const double *A;    /* [n_data][n_hidden]                                */
  const double *B;    /* [n_hidden][d_c]                                   */
  const double *c;    /* [n_hidden]                                        */
  const double *N;    /* [n_data][d - d_c] (NULL when d == d_c)            */
  const double *data; /* [n_data]                                          */
  double sigma;
  /* emulator: params = W1[w][d] b1[w] (W_l[w][w] b_l[w])_{l=2..D} wo[w] bo */
  int depth, width;
  const double *params;
  const double *in_m, *in_s;  /* input standardisation u = (x - m)/s       */
  double out_m, out_s;        /* chi2_hat = out_s * out + out_m            */
  int bf16;                   /* operand-rounding emulation: 1 BF16, 2 FP16 */
  /* prior: hard box on every dim; N(0,1) on dims with gauss[i] != 0       */
  const double *lower, *upper;
  const int *gauss;           /* [d] or NULL                               */
  /* whitening */
  const double *mu;           /* [d]                                       */
  const double *L;            /* [d][d] lower triangular, row-major        */
  /* emulator output transform: 0 chi2_hat = out_s out + out_m;
   * 1 chi2_hat = out_floor + exp(out_s out + out_m)                       */
  int out_log;
  double out_floor;
  /* smooth bounds penalty (Sec. 3.1): pen_w[i] > 0 replaces the hard box of dim i by
   * log prior -= ((x_i - clamp(x_i, lower_i, upper_i)) / pen_w[i])^2 / 2; NULL = hard box */
  const double *pen_w;
} orc_model;

/* ---- Philox4x32-10 and the draws built on it ---- */
double orc_fp16_round(double v);
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t purpose, uint32_t idx);
void orc_normals(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t purpose, int n, double *out);
double orc_bf16_round(double v);

/* ---- likelihoods and the whitened target ---- */
double orc_loglike(const orc_model *m, const double *x, double *grad_x);
void orc_loglike_batch(const orc_model *m, int n, const double *x, double *logl, double *grad);
double orc_logpost_z(const orc_model *m, const double *z, double *grad_z, double *x_out);
void orc_logpost_batch(const orc_model *m, int n, const double *z, double *lp, double *grad);

/* ---- samplers ---- */
double orc_leapfrog(const orc_model *m, double *z, double *q, double *g, double eps, int n);
typedef struct {
  int kernel;        /* ORC_MH .. ORC_NUTS_MULTINOMIAL         */
  double eps;        /* step size                              */
  int n_leapfrog;    /* HMC L                                  */
  int n_steps;       /* iterations per chain                   */
  int max_depth;     /* NUTS doublings                         */
  double aies_a;     /* stretch parameter a                    */
  int aies_walkers;  /* walkers per ensemble (even)            */
  uint64_t seed;
  double de_sigma;   /* DE move: standard deviation of eta     */
} orc_step_params;

typedef struct {
  double *samples;      /* [n_steps][n][d] x-space, or NULL        */
  double *trace_logalpha;/* [n_steps][n] or NULL                   */
  double *trace_logu;   /* [n_steps][n] or NULL                    */
  int *trace_accept;    /* [n_steps][n] or NULL                    */
  int *trace_depth;     /* [n_steps][n] NUTS doublings, or NULL    */
  int *trace_nleaf;     /* [n_steps][n] NUTS leapfrogs, or NULL    */
  double *trace_margin; /* [n_steps][n] NUTS: the smallest distance of any decision of the
                         * iteration from its threshold (see nuts_step), or NULL           */
} orc_trace;

int orc_run(const orc_model *m, const orc_step_params *p, int n_chains, double *z, double *lp,
            double *g, uint32_t *iter, double *accept_stat, int64_t *accepts, int64_t *evals,
            int64_t *divergences, const orc_trace *tr);

/* ---- covariance adaptation ---- */
void orc_pooled_cov(int n, int d, const double *x, double *mean, double *cov);
void orc_chan_merge(int d, double na, double *mean_a, double *M2_a, double nb, const double *mean_b,
                    const double *M2_b);
int orc_cholesky_jitter(int d, const double *S, double jitter0, double *L, double *used);
void orc_remap_z(int d, int n, const double *mu_old, const double *L_old, const double *mu_new,
                 const double *L_new, double *z);

/* ---- training ---- */
double orc_train_loss_grad(int d, int depth, int width, const double *params, const double *in_m,
                           const double *in_s, double out_m, double out_s, int out_log,
                           double out_floor, int bf16, int m, const double *X, const double *chi2,
                           double *grad);
void orc_adam(int n, double *p, const double *g, double *m1, double *m2, int t, double lr,
              double b1, double b2, double eps);

/* ---- diagnostics ---- */
void orc_ess(int n_draws, int n_chains, int d, const double *samples, double *ess);

#ifdef __cplusplus
}
#endif
#endif
