/*
 * bst.h -- C ABI of the GB300 (sm_103a) batched emulator posterior sampler.
 *
 * The library evaluates a tanh-MLP log-likelihood emulator (or an analytic
 * "theory map" likelihood) and its gradient for thousands of independent
 * chains at once, inside MH / MALA / HMC / NUTS / AIES proposal-and-accept
 * steps, after "Posterior sampling in the Age of Emulators" (arXiv
 * 2606.04895).  The paper's unified interface (Sec. 3.1) is a sampler built
 * from a log-probability and a hyper-rectangle of bounds, run with a method,
 * a number of steps and a number of chains, returning samples, acceptance
 * rates and evaluation counts; the calls below are that interface.
 *
 * Conventions (every entry point):
 *  - Returns a bst_status; nothing throws or aborts across the ABI.  The text
 *    of the last error of the calling thread is bst_last_error().
 *  - Device buffers are owned by the caller, passed as plain device pointers
 *    (``*_dev``), and must stay alive until the work on ``stream`` is done.
 *    Host arrays (``*_host`` or plain ``const double*``) are copied on entry.
 *  - ``stream`` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued asynchronously unless a call says it synchronises.
 *  - Element type of real-valued device buffers ("real"): float for handles of
 *    precision BST_BF16, BST_FP16 and BST_FP32, double for BST_FP64.
 *  - Call order: bst_create -> bst_set_emulator | bst_set_analytic ->
 *    bst_init_chains -> { bst_step, bst_adapt_cov, ... }*.  Out of order ->
 *    BST_ERR_STATE.  The library owns only small persistent state (chain
 *    state, packed weights, Welford accumulators, counters).
 *  - A handle is used by one host thread at a time.
 */
#ifndef BST_H
#define BST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bst_ctx *bst_handle;

typedef enum {
  BST_OK = 0,
  BST_ERR_ARG = 1,         /* invalid argument (NULL, size, range)              */
  BST_ERR_STATE = 2,       /* call out of order                                 */
  BST_ERR_CUDA = 3,        /* CUDA runtime error (message in bst_last_error)     */
  BST_ERR_NOT_PD = 4,      /* covariance not positive definite even with jitter */
  BST_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out                */
  BST_ERR_NONFINITE = 6,   /* non-finite input where a finite one is required   */
  BST_ERR_UNSUPPORTED = 7  /* shape/precision combination not built             */
} bst_status;

typedef enum {
  BST_MH = 0, BST_MALA = 1, BST_HMC = 2, BST_NUTS = 3, BST_AIES = 4, BST_AIES_DE = 5, BST_NUTS_MULTINOMIAL = 6
} bst_kernel;
/* BST_BF16 / BST_FP16: emulator on the tcgen05 tensor cores with BF16 (8 significant bits) or
 * FP16 (11 significant bits, same rate) weights and activations, FP32 accumulation; FP32 chain
 * state.  BST_FP32 / BST_FP64: CUDA-core paths (the plain precisions). */
typedef enum { BST_BF16 = 0, BST_FP32 = 1, BST_FP64 = 2, BST_FP16 = 3 } bst_precision;
typedef enum { BST_LIK_EMULATOR = 0, BST_LIK_ANALYTIC = 1 } bst_lik_kind;

typedef struct {
  int d;              /* parameter dimension, 1..32                                   */
  int n_chains;       /* chains (AIES: a multiple of 4 * aies_walkers)                */
  int precision;      /* bst_precision; BF16 / FP16 require an emulator               */
  int lik_kind;       /* bst_lik_kind                                                 */
  uint64_t seed;      /* Philox4x32-10 key                                            */
  int max_depth;      /* NUTS doublings per iteration (1..10; 0 -> 8)                 */
  int aies_walkers;   /* walkers per AIES ensemble (64; 0 -> 64)                      */
  double aies_a;      /* AIES stretch parameter a > 1 (0 -> 2)                        */
  int thin;           /* record every thin-th step (0 -> 1)                           */
  int device;         /* CUDA device ordinal                                          */
} bst_config;

typedef struct {
  int64_t accepts;        /* accepted moves in this call (NUTS: moved iterations)     */
  int64_t evals;          /* likelihood evaluations in this call (Sec. 3.1 counter)   */
  int64_t divergences;    /* NUTS: iterations stopped by the energy-error bound       */
  double accept_stat;     /* mean Metropolis acceptance statistic over chain-steps    */
  int status;             /* device status word (bst_status)                          */
} bst_step_stats;

/* Version string of the library build. */
const char *bst_version(void);
/* Text of the last error on this host thread ("" if none). */
const char *bst_last_error(void);

/* Create a handle on cfg->device.  Allocates the chain state for n_chains.
 * Errors: BST_ERR_ARG (d outside 1..32, n_chains < 1, AIES shape), BST_ERR_CUDA. */
bst_status bst_create(bst_handle *h, const bst_config *cfg);
/* Release every device and host resource of h (NULL is a no-op). */
void bst_destroy(bst_handle h);

/* Emulator likelihood (stand-in for the CLiENT emulator, paper Sec. 1/4):
 *   u = (x - in_m) / in_s;  h_1 = tanh(W_1 u + b_1);  h_l = tanh(W_l h_{l-1} + b_l);
 *   out = w_o . h_D + b_o;  chi2 = out_s * out + out_m;  logL = -chi2 / 2.
 * params (host, FP64, copied): W_1[width][d] b_1[width] (W_l[width][width] b_l[width])
 * for l = 2..depth, then w_o[width], b_o.  width in {256, 512} for BF16 / FP16, any
 * multiple of 64 up to 1024 for FP32 (up to 512 for FP64); depth 1..8.
 * Errors: BST_ERR_ARG, BST_ERR_UNSUPPORTED, BST_ERR_NONFINITE (non-finite weight). */
bst_status bst_set_emulator(bst_handle h, int depth, int width, const double *params,
                            const double *in_m, const double *in_s, double out_m, double out_s);

/* Read back the current emulator parameters (after training) into params
 * (host, FP64, same layout as bst_set_emulator).  Synchronises. */
bst_status bst_get_emulator(bst_handle h, double *params);

/* Output transform of the emulator (the paper defers the emulator's design to
 * CLiENT, Sec. 4; this is the reading used here).  BST_OUT_LINEAR (the default
 * after bst_set_emulator): chi2 = out_s * out + out_m.  BST_OUT_LOG:
 * chi2 = floor + exp(out_s * out + out_m), i.e. the network predicts the
 * standardised log(chi2 - floor), which resolves the posterior region of a
 * chi2 that spans orders of magnitude over the prior box; the gradient is
 * d logL / dx = -(1/2) exp(out_s * out + out_m) out_s d out / dx.  Applies to
 * every evaluation and to training (bst_train_*: the regression target is
 * (log(chi2 - floor) - out_m) / out_s, with chi2 - floor clamped to >= 1e-30).
 * Call after bst_set_emulator (which resets it to BST_OUT_LINEAR).
 * Errors: BST_ERR_ARG (unknown kind, non-finite floor), BST_ERR_STATE (no emulator). */
typedef enum { BST_OUT_LINEAR = 0, BST_OUT_LOG = 1 } bst_out_kind;
bst_status bst_set_emulator_output(bst_handle h, int kind, double floor);

/* Analytic likelihood: f(x) = A tanh(B x_c + c) + N x_n (tanh -> identity if
 * linear), logL = -|data - f(x)|^2 / (2 sigma^2); x_c = x[0:d_c], x_n = x[d_c:d].
 * A[n_data][n_hidden], B[n_hidden][d_c], c[n_hidden], N[n_data][d - d_c] (NULL
 * when d_c == d), data[n_data]; host FP64, copied.  n_hidden <= 64. */
bst_status bst_set_analytic(bst_handle h, int d_c, int n_hidden, int n_data, const double *A,
                            const double *B, const double *c, const double *N, const double *data,
                            double sigma, int linear);

/* init_chains(theta0, prior box, whitening) -- paper Sec. 2.2 / Algorithm 1 and
 * Sec. 3.1: chains start at theta0[n_chains][d] (host, x-space).  The prior is
 * the box lower <= x <= upper (log prior 0 inside, -inf outside) times N(0,1) on
 * every dim with gauss[i] != 0 (gauss may be NULL).  Sampling runs in whitened
 * coordinates z with x = mu + L z (L[d][d] lower triangular, row-major, positive
 * diagonal); the target is log pi_z(z) = log L(x) + log prior(x) + sum log L_ii
 * (Eq. (2.12)).  Evaluates log pi and its gradient at every start (synchronises).
 * Resets the iteration counters and statistics. */
bst_status bst_init_chains(bst_handle h, const double *theta0, const double *lower,
                           const double *upper, const int *gauss, const double *mu,
                           const double *L);

/* step(kernel, eps, L, n_steps): advance every chain n_steps iterations of
 *   BST_MH   : z' = z + eps xi, Metropolis accept                     (Sec. 2, Sec. 4)
 *   BST_MALA : z' = z + eps grad + sqrt(2 eps) xi, MH-corrected        (Sec. 2.1, Eq. (2.3))
 *   BST_HMC  : n_leapfrog leapfrog steps of H = -log pi + q.q/2        (Sec. 2.1, Eq. (2.1))
 *   BST_NUTS : Hoffman-Gelman NUTS, at most max_depth doublings          (Sec. 2.1)
 *   BST_NUTS_MULTINOMIAL : the same trees, directions and U-turn tests with leaf weights
 *             exp(H0 - H) in place of the slice (Betancourt 2017, Appendix A): in-subtree
 *             merges keep the second half's candidate with probability w'' / (w' + w''),
 *             the top level moves with probability min(1, w_new / w_old), a leaf with
 *             H - H0 > 1000 is divergent
 *   BST_AIES : Goodman-Weare stretch move, ensembles of aies_walkers     (Sec. 2.3)
 *   BST_AIES_DE : differential-evolution move on the same ensembles and halves (Sec. 2.3,
 *             after Eq. (2.15)): y = z_i + gamma (z_j - z_k), j != k uniform in the other
 *             half, gamma = (1 + eps eta) 2.38 / sqrt(2 d), eta ~ N(0, 1): eps is the
 *             standard deviation sigma_gamma of the relative scale (>= 0; the paper gives no
 *             value); symmetric, accepted with min(1, pi(y) / pi(z_i)); aies_walkers >= 4
 * eps is ignored by AIES; n_leapfrog only used by HMC.  If samples_dev is not
 * NULL it receives x-space samples real[n_steps / thin][n_chains][d]: device
 * memory of the handle's device, or page-locked host memory that the device can address
 * (cudaHostAlloc / cudaHostRegister; the kernel then writes the record to host memory
 * directly, with no copy after the call, and the caller reads it once the stream is
 * synchronised).  Any other pointer returns BST_ERR_ARG before anything is launched.
 * If stats is not NULL the call synchronises ``stream`` and fills it with this
 * call's totals; otherwise it only enqueues. */
bst_status bst_step(bst_handle h, int kernel, double eps, int n_leapfrog, int n_steps,
                    void *samples_dev, void *stream, bst_step_stats *stats);

/* loglike(theta): logl_dev[m] = logL(theta_dev[m][d]) (likelihood only, x-space,
 * no prior).  real buffers; m >= 0 (m == 0 is a no-op). */
bst_status bst_loglike(bst_handle h, const void *theta_dev, int m, void *logl_dev, void *stream);

/* grad_loglike(theta): logl_dev[m] = logL, grad_dev[m][d] = d logL / d theta. */
bst_status bst_grad_loglike(bst_handle h, const void *theta_dev, int m, void *logl_dev,
                            void *grad_dev, void *stream);

/* Allocation-free form of bst_grad_loglike.  There is no counterpart in the
 * paper; this entry point exists for callers that must not allocate device
 * memory once they are running -- a program whose device memory is owned by
 * a caching allocator or a fixed budget set at start-up (an outside cudaMalloc
 * there fragments or overcommits the pool), or a service that reserves all
 * its memory before it takes requests.  bst_grad_loglike may allocate: the
 * first call with a larger m than before grows the buffer in which the adjoint
 * keeps the emulator's hidden activations.  This call instead uses one
 * file-scope device array of 16 MiB (g_static_scratch) that every GPU which
 * loads the library holds until the process exits (for the activations), and
 * calls no cudaMalloc, cudaFree or other allocating routine.
 * Arguments and results are those of bst_grad_loglike.  Limit: m times the
 * bytes kept per point, (depth - 1) x width x (2 for BF16 / FP16, 4 for FP32, 8 for
 * FP64), must fit in 16 MiB (for example m <= 5461 for a BF16 8-512x4-1
 * emulator); a larger m returns BST_ERR_ARG and launches nothing.
 * The first call on each device looks the array's device address up with
 * cudaGetSymbolAddress (the device must be current, which the call ensures);
 * make that first call before any stream capture.  The first call after new
 * weights (bst_set_emulator, bst_train_apply) converts them for the device and
 * synchronises the stream, as the first evaluation call of any kind does; make
 * that call outside stream capture too.  Every call on a device
 * shares the one array and overwrites what the previous call left there
 * (nothing in it needs to start at zero), so calls whose work overlaps on the
 * GPU -- on different streams, or from different handles -- race; order them
 * on one stream. */
bst_status bst_grad_loglike_noalloc(bst_handle h, const void *theta_dev, int m, void *logl_dev,
                                    void *grad_dev, void *stream);

/* Covariance adaptation (Sec. 3.2).  bst_welford_reset clears the running
 * statistics and makes every following bst_step add each chain's x after
 * every iteration; bst_welford_add adds external samples x_dev[m][d] (real).
 * bst_adapt_cov merges the statistics in FP64, forms the unbiased covariance,
 * factorises it (plain Cholesky; on failure adds delta (tr S / d) I with
 * delta = jitter0, x10 per retry, up to 1e-2), sets mu = pooled mean and L =
 * the factor as the new whitening, keeps every chain's x fixed (z remapped)
 * and re-evaluates log pi and its gradient.  mu_out[d], L_out[d][d] and
 * jitter_used (host, may be NULL) receive the result.  Synchronises.
 * Errors: BST_ERR_STATE (fewer than 2 samples), BST_ERR_NOT_PD. */
bst_status bst_welford_reset(bst_handle h);
bst_status bst_welford_add(bst_handle h, const void *x_dev, int m, void *stream);
bst_status bst_adapt_cov(bst_handle h, double jitter0, double *mu_out, double *L_out,
                         double *jitter_used);

/* Covariance statistics across processes (one process per GPU, Sec. 3.2 pooled
 * over every rank's chains).  bst_welford_stats returns the statistics this
 * handle has accumulated, merged in FP64: count n, mean[d] and the centred sum
 * of squares M2[d][d] (covariance = M2 / (n - 1)).  bst_welford_merge adds a
 * triple obtained elsewhere (Chan, Golub & LeVeque pairwise merge); reset, then
 * merging every rank's triple in rank order gives bit-identical statistics on
 * every rank, so bst_adapt_cov then returns the same whitening everywhere.
 * Both synchronise. */
bst_status bst_welford_stats(bst_handle h, double *n, double *mean, double *M2);
bst_status bst_welford_merge(bst_handle h, double n, const double *mean, const double *M2);

/* Smooth bounds (Sec. 3.1: outside the box the density is extended by a smooth exponential
 * penalty that keeps it differentiable).  width[d] (host, copied): width_i > 0 replaces
 * dimension i's hard box by the factor exp(-r_i^2 / 2), r_i = (x_i - clamp(x_i, lower_i,
 * upper_i)) / width_i, so log pi gains -r_i^2 / 2 and its gradient -r_i / width_i (both
 * continuous at the bounds; 0 inside); width_i = 0 keeps dimension i's hard box; width = NULL
 * restores hard bounds everywhere.  Applies to every later bst_step; the chains' log pi and
 * gradient are re-evaluated now.  Synchronises.
 * Errors: BST_ERR_STATE (before bst_init_chains), BST_ERR_ARG (negative or non-finite width). */
bst_status bst_set_bounds_penalty(bst_handle h, const double *width);

/* Checkpoint / resume.  Host FP64 copies of the chain state: z[n][d], logp[n],
 * grad[n][d] (whitened), iteration counters iter[n].  Philox draws are keyed by
 * (seed, chain, iter), so a restored state continues bit-identically. */
bst_status bst_get_state(bst_handle h, double *z, double *logp, double *grad, uint32_t *iter);
bst_status bst_set_state(bst_handle h, const double *z, const double *logp, const double *grad,
                         const uint32_t *iter);
/* Current whitening (mu[d], L[d][d]); synchronises. */
bst_status bst_get_whitening(bst_handle h, double *mu, double *L);

/* Initial walker positions by one of the strategies of Sec. 3.1, drawn on the device from
 * this handle's counter-based random streams (stream (chain, 0, 8)), FP64: REPEATED every
 * chain at center; UNIFORM lower + (upper - lower) u (finite bounds, upper > lower);
 * GAUSSIAN center + Lc xi, xi ~ N(0, I) (Lc host double[d][d] row-major).  theta_out: host
 * double[n_chains][d], to pass to bst_init_chains.  A chain's draw depends only on the seed
 * and its index.  Synchronises. */
typedef enum { BST_INIT_REPEATED = 0, BST_INIT_UNIFORM = 1, BST_INIT_GAUSSIAN = 2 } bst_init_strategy;
bst_status bst_draw_positions(bst_handle h, int strategy, const double *center, const double *Lc,
                              const double *lower, const double *upper, double *theta_out);

/* Replace the whitening x = mu + L z (Algorithm 1) of initialised chains: mu host double[d],
 * L host double[d][d] row-major, lower triangular with a positive diagonal (the upper
 * triangle is ignored).  Every chain keeps its x (z is remapped), layer 1 is refolded and
 * log pi and its gradient are recomputed.  Per-dimension step multipliers m (a step of
 * eps m_i along whitened direction i) are the whitening L diag(m).  BST_ERR_ARG for a
 * non-finite mu or an invalid L, BST_ERR_STATE before bst_init_chains.  Synchronises. */
bst_status bst_set_whitening(bst_handle h, const double *mu, const double *L);
/* Per-chain counters since bst_init_chains (host arrays, each n_chains long,
 * any may be NULL).  Synchronises. */
bst_status bst_get_counters(bst_handle h, int64_t *accepts, int64_t *evals, int64_t *divergences,
                            double *accept_stat);

/* Emulator training (the learned part): one Adam step (Kingma & Ba) of the
 * loss mean_i (out_i - (t(chi2_i) - out_m)/out_s)^2 over the batch X_dev[m][d],
 * chi2_dev[m] (float, device), t the output transform (bst_set_emulator_output).
 * FP32 master weights, forward with stored activations, hand-written backward;
 * the sampling weights are re-packed from the master before the next
 * evaluation.  Handles of precision BF16 / FP16 run the hidden-layer products
 * (layers 2..depth: forward, adjoint, weight gradient) on the tcgen05 tensor
 * cores with BF16 operands and FP32 accumulation when m is a multiple of 512
 * and width a multiple of 128 (the input layer, the output head and the bias
 * sums stay FP32); otherwise, and for FP32 / FP64 handles, every product runs
 * in FP32 on the CUDA cores.  loss_dev (float[1], may be NULL) receives the
 * batch loss before the update.  1 <= m <= 65536. */
bst_status bst_train_step(bst_handle h, const float *X_dev, const float *chi2_dev, int m,
                          double lr, double beta1, double beta2, double adam_eps, float *loss_dev,
                          void *stream);
/* Loss and its gradient with respect to every parameter (grad_dev: float, same
 * layout as bst_set_emulator params) without updating; for checks. */
bst_status bst_train_grad(bst_handle h, const float *X_dev, const float *chi2_dev, int m,
                          float *grad_dev, float *loss_dev, void *stream);

/* One Adam step with a gradient supplied by the caller (grad_dev: float, layout
 * of bst_set_emulator params) -- for data-parallel training, where each rank
 * computes bst_train_grad on its batch and the gradients are averaged across
 * ranks before this call. */
bst_status bst_train_apply(bst_handle h, const float *grad_dev, double lr, double beta1, double beta2,
                           double adam_eps, void *stream);

/* Multi-chain effective sample size per dimension (Gelman et al., BDA3
 * Sec. 11.5: variogram autocorrelations, Geyer initial monotone sequence) of
 * samples_dev real[n_draws][n_chains][d] (this handle's n_chains, d and real
 * type).  ess_out: host double[d].  Synchronises. */
bst_status bst_ess(bst_handle h, const void *samples_dev, int n_draws, double *ess_out);

/* Multivariate Gelman-Rubin statistic R - 1 (paper Sec. 4.1) of samples_dev
 * real[n_draws][n_chains][d] (this handle's n_chains, d and real type): B = the
 * covariance of the chain means (n_chains - 1 denominator), W = the mean of the
 * chain covariances (n_draws - 1 denominator), both scaled by D = diag(sqrt(B_ii));
 * *out = the largest |eigenvalue| of W~^-1 B~ (host double).  The cross products run
 * on the device in FP64, the d x d algebra (Cholesky, Jacobi eigenvalues) on the
 * host.  *out is NaN when some B_ii is zero or W is not positive definite (the
 * statistic is undefined).  n_draws >= 2 and n_chains >= 2, else BST_ERR_ARG.
 * Synchronises. */
bst_status bst_r_minus_1(bst_handle h, const void *samples_dev, int n_draws, double *out);

/* The two halves of bst_r_minus_1, for chains spread over several handles (ranks):
 * bst_r_minus_1_parts computes, on the device, every chain's mean (chain_means: host
 * double[n_chains][d]) and the pooled within-chain cross products
 * S = sum_c sum_t (x_tc - m_c)(x_tc - m_c)^T (S: host double[d][d]) of samples_dev
 * (n_draws >= 2; synchronises).  bst_r_minus_1_combine is host-only (no device, no handle):
 * from the means of all n_chains chains and the sum of every part's S it forms
 * W = S / (n_chains (n_draws - 1)), B = the covariance of the chain means, and R - 1 as in
 * bst_r_minus_1 (NaN where that is NaN).  Needs n_chains >= 2, n_draws >= 2, 1 <= d <= 32. */
bst_status bst_r_minus_1_parts(bst_handle h, const void *samples_dev, int n_draws, double *chain_means,
                               double *S);
bst_status bst_r_minus_1_combine(int n_chains, int n_draws, int d, const double *chain_means, const double *S,
                                 double *out);

/* Per-dimension quantiles of the pooled draws samples_dev real[n_draws][n_chains][d]
 * (this handle's n_chains, d and real type) at the levels q[0..nq) in [0, 1], 1 <= nq
 * <= 8: linear interpolation between the order statistics at ranks floor(h) and
 * floor(h) + 1, h = (N - 1) q, N = n_draws n_chains (the order statistics are exact:
 * radix select on the device).  out: host double[d][nq].  Draws must be finite.
 * Synchronises. */
bst_status bst_quantiles(bst_handle h, const void *samples_dev, int n_draws, const double *q, int nq,
                         double *out);

/* Credible metric (paper Sec. 4.1) per dimension at credible level alpha in (0, 1):
 * (|hi - true_hi| + |lo - true_lo|) / (true_hi - true_lo), lo and hi the equal-tailed
 * limits of the pooled draws (quantiles (1 - alpha) / 2 and (1 + alpha) / 2, as in
 * bst_quantiles).  true_lo, true_hi, out: host double[d]; true_hi > true_lo.
 * Synchronises. */
bst_status bst_credible_metric(bst_handle h, const void *samples_dev, int n_draws, double alpha,
                               const double *true_lo, const double *true_hi, double *out);

/* Sliced Wasserstein distance (paper Sec. 4.1) between the pooled draws samples_dev
 * real[n_draws][n_chains][d] and a reference set ref_dev real[n_ref][d] (both device memory,
 * this handle's real type): the mean over n_proj directions u_k of the 1-D Wasserstein-1
 * distance between the projections {x . u_k}, the 1-D distance being the integral of the
 * absolute difference of the two empirical quantile functions (sizes may differ).  Direction
 * k is the normals 0..d-1 of Philox stream (k, 0, 9) under `seed`, normalised, so a fixed
 * seed reuses one set of directions for every comparison.  FP64 arithmetic; *out: host
 * double.  n_draws n_chains + n_ref <= 2^27; draws must be finite.  Synchronises. */
bst_status bst_sliced_wasserstein(bst_handle h, const void *samples_dev, int n_draws, const void *ref_dev,
                                  long long n_ref, int n_proj, unsigned long long seed, double *out);

/* Block until all work of h on ``stream`` is done and check the device status. */
bst_status bst_sync(bst_handle h, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BST_H */
