// api.cu -- the C ABI declared in include/bst.h: handle, validation, device memory of the
// library-owned state, weight preparation and the launches of the sampling kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launch.h"

using namespace bst;

namespace {

thread_local std::string g_err;

bst_status fail(bst_status s, const std::string &m) {
  g_err = m;
  return s;
}

#define BST_CUDA(expr)                                                                            \
  do {                                                                                            \
    cudaError_t e_ = (expr);                                                                      \
    if (e_ != cudaSuccess) return fail(BST_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define BST_TRY(expr)             \
  do {                            \
    bst_status s_ = (expr);       \
    if (s_ != BST_OK) return s_;  \
  } while (0)

int pad16(int d) { return ((d + 15) / 16) * 16; }

// A named range on the calling thread for timeline tools (NVTX; a no-op when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace

struct bst_ctx {
  // configuration
  int d = 0, dp = 0, n = 0, precision = 0, lik = 0, max_depth = 8, walkers = 64, thin = 1, device = 0;
  double aies_a = 2.0;
  uint64_t seed = 0;
  int stage = 0;  // 0 created, 1 likelihood set, 2 chains initialised
  size_t rs = 4;  // bytes per working real
  std::vector<void *> allocs;

  // chain state (working precision, dp-padded rows)
  void *z = nullptr, *g = nullptr, *lp = nullptr, *ze = nullptr, *lle = nullptr, *gle = nullptr, *work = nullptr,
       *xbuf = nullptr;
  uint32_t *iter = nullptr;
  double *acc_stat = nullptr;
  unsigned long long *accepts = nullptr, *evals = nullptr, *divs = nullptr;
  int *steps_done = nullptr, *status = nullptr;
  int work_stride = 0;

  // target: whitening + prior
  std::vector<double> mu, L, lower, upper;
  std::vector<int> gauss;
  double logdet = 0.0;
  int any_gauss = 0;
  std::vector<double> pen_w;  // smooth-bound widths (empty or zeros: hard box)
  double *mu64 = nullptr, *L64 = nullptr, *mu64_new = nullptr, *L64_new = nullptr, *info64 = nullptr;
  double *theta64 = nullptr;  // [n][d] initial positions staged for init_chains
  size_t theta_cap = 0;
  double *stats64 = nullptr;  // [1 + kMaxD + kMaxD^2] Welford triple staging

  // emulator
  int depth = 0, width = 0;
  size_t nparams = 0;
  double *P64 = nullptr, *in_m64 = nullptr, *in_s64 = nullptr;
  double out_m = 0.0, out_s = 1.0, bo = 0.0;
  int out_log = 0;       // bst_out_kind
  double out_floor = 0.0;
  double *W1f[2] = {nullptr, nullptr}, *b1f[2] = {nullptr, nullptr};  // [0] z-space, [1] x-space
  void *sW1T[2] = {nullptr, nullptr}, *sW1[2] = {nullptr, nullptr}, *sb1[2] = {nullptr, nullptr};
  void *sWT = nullptr, *sW = nullptr, *sb = nullptr, *swo = nullptr;
  uint8_t *tl1[2][3] = {}, *tg1[2] = {nullptr, nullptr}, *thid[3] = {};  // [fold][cluster size 1/2/4]
  float *tb1[2] = {nullptr, nullptr}, *tb = nullptr, *two = nullptr;
  int kb1 = 1;
  void *scratch = nullptr;
  size_t scratch_rows = 0, scratch_bytes = 0;

  // analytic likelihood
  int d_c = 0, H = 0, n_data = 0, linear = 0, has_N = 0;
  double sigma = 1.0;
  double *A64 = nullptr, *B64 = nullptr, *c64 = nullptr, *N64 = nullptr, *data64 = nullptr;
  double *fBf = nullptr, *fcf = nullptr, *fAT = nullptr, *fNfT = nullptr, *fdata = nullptr;  // FP64 staging
  void *aBf[2] = {nullptr, nullptr}, *acf[2] = {nullptr, nullptr}, *aAT = nullptr, *aNfT[2] = {nullptr, nullptr},
       *adata[2] = {nullptr, nullptr};

  // training
  float *P32 = nullptr, *G32 = nullptr, *m1 = nullptr, *m2 = nullptr, *in_m32 = nullptr, *in_s32 = nullptr;
  int adam_t = 0;
  int train_cap = 0;
  TrainWork tw{};

  // Welford
  double *wf = nullptr;
  int wf_records = 0;
  bool welford_on = false;

  // flags
  bool weights_dirty = true;  // folds / packs must be rebuilt
  bool p32_newer = false;     // training master newer than the FP64 master
  bool state_stale = true;    // log pi / grad of the chains must be re-evaluated
  bool grad_valid = false;

  // host-side counter snapshot for per-call statistics
  int ess_tmp_cap = 0;
  double *ess_mean = nullptr, *ess_var = nullptr, *ess_V = nullptr;
  double *rhat_part = nullptr;  // [blocks][d (d + 1) / 2] pooled cross products (R - 1)
  double *init_par = nullptr, *init_theta = nullptr;  // initial positions: parameters, [n][d] draws
  void *qsel_prefix = nullptr;    // [d][2 kMaxQuantiles] radix-select prefixes (quantiles)
  unsigned int *qsel_hist = nullptr;  // [d][2 kMaxQuantiles][16]
};

namespace {

bst_status dalloc(bst_ctx *h, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return fail(BST_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(*p);
  cudaMemset(*p, 0, bytes);
  return BST_OK;
}
template <typename T>
bst_status dalloc_t(bst_ctx *h, T **p, size_t count) {
  void *v = nullptr;
  bst_status s = dalloc(h, &v, count * sizeof(T));
  *p = static_cast<T *>(v);
  return s;
}
void dfree(bst_ctx *h, void *p) {
  if (!p) return;
  for (auto &q : h->allocs)
    if (q == p) {
      cudaFree(p);
      q = nullptr;
    }
}

bool all_finite(const double *v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// upload FP64 host values as working-precision device values
bst_status upload_real(bst_ctx *h, void *dst, const double *src, size_t n) {
  if (h->rs == 8) {
    BST_CUDA(cudaMemcpy(dst, src, n * 8, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> t(n);
    for (size_t i = 0; i < n; ++i) t[i] = static_cast<float>(src[i]);
    BST_CUDA(cudaMemcpy(dst, t.data(), n * 4, cudaMemcpyHostToDevice));
  }
  return BST_OK;
}
bst_status download_real(bst_ctx *h, double *dst, const void *src, size_t n) {
  if (h->rs == 8) {
    BST_CUDA(cudaMemcpy(dst, src, n * 8, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> t(n);
    BST_CUDA(cudaMemcpy(t.data(), src, n * 4, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) dst[i] = t[i];
  }
  return BST_OK;
}

// The tensor-core engine serves BF16 and FP16 operands (same kernels, operand type a flag).
bool tc_engine(const bst_ctx *h) { return h->precision == BST_BF16 || h->precision == BST_FP16; }
int is_f16(const bst_ctx *h) { return h->precision == BST_FP16 ? 1 : 0; }

bst_status check_status(bst_ctx *h) {
  int st = 0;
  BST_CUDA(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & kStatusTimeout) {
    cudaMemset(h->status, 0, sizeof(int));
    return fail(BST_ERR_TIMEOUT, "a bounded device-side wait ran out (device status word)");
  }
  return BST_OK;
}

// ------------------------------------------------------------------ argument assembly
size_t act_bytes_for(const bst_ctx *h, size_t rows);
size_t xchg_bytes_for(const bst_ctx *h, size_t rows);
template <typename R>
StepArgs<R> make_args(bst_ctx *h, int mode, double eps, int n_leapfrog, int n_steps, void *samples) {
  StepArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.mode = mode;
  a.n_chains = h->n;
  a.n_rows = is_ensemble_mode(mode) ? h->n / 2 : h->n;
  a.d = h->d;
  a.dp = h->dp;
  a.eps = eps;
  a.n_leapfrog = n_leapfrog;
  a.n_steps = n_steps;
  a.max_depth = h->max_depth;
  a.aies_walkers = h->walkers;
  a.aies_a = h->aies_a;
  a.thin = h->thin;
  a.seed = h->seed;
  a.need_grad = (mode == kModeMALA || mode == kModeHMC || is_nuts_mode(mode) || mode == kModeRefresh) ? 1 : 0;
  a.tgt.d = h->d;
  a.tgt.logdet = h->logdet;
  a.tgt.any_gauss = h->any_gauss;
  {
    // whitening and prior in working precision, into the kernel parameters (entries beyond d
    // stay zero: the device loops run unrolled to 8 or 32 entries)
    const int d = h->d;
    for (int i = 0; i < d; ++i) {
      if (h->mu.size() >= static_cast<size_t>(d)) a.tgt.mu[i] = static_cast<R>(h->mu[i]);
      if (h->L.size() >= static_cast<size_t>(d) * d)
        for (int j = 0; j < d; ++j) a.tgt.L[i * kMaxD + j] = static_cast<R>(h->L[static_cast<size_t>(i) * d + j]);
      if (h->lower.size() >= static_cast<size_t>(d)) a.tgt.lower[i] = static_cast<R>(h->lower[i]);
      if (h->upper.size() >= static_cast<size_t>(d)) a.tgt.upper[i] = static_cast<R>(h->upper[i]);
      if (h->gauss.size() >= static_cast<size_t>(d)) a.tgt.gauss[i] = h->gauss[i];
      if (h->pen_w.size() >= static_cast<size_t>(d) && h->pen_w[i] > 0.0) {
        a.tgt.pen_iw[i] = static_cast<R>(1.0 / h->pen_w[i]);
        a.tgt.any_pen = 1;
      }
    }
  }
  a.st.z = static_cast<R *>(h->z);
  a.st.g = static_cast<R *>(h->g);
  a.st.lp = static_cast<R *>(h->lp);
  a.st.iter = h->iter;
  a.st.acc_stat = h->acc_stat;
  a.st.accepts = h->accepts;
  a.st.evals = h->evals;
  a.st.divs = h->divs;
  a.st.ze = static_cast<R *>(h->ze);
  a.st.lle = static_cast<R *>(h->lle);
  a.st.gle = static_cast<R *>(h->gle);
  // the chains' evaluation rows, gradients and work buffers are chain-blocked (ld 0)
  a.st.ze_ld = 0;
  a.st.gle_ld = 0;
  a.st.work = static_cast<R *>(h->work);
  a.st.dwork = reinterpret_cast<double *>(static_cast<R *>(h->work) +
                                          static_cast<size_t>(kDworkOffsetVecs) * kMaxD * chains_padded(h->n));
  a.st.steps_done = h->steps_done;
  a.samples = static_cast<R *>(samples);
  a.welford_on = (h->welford_on && mode != kModeRefresh && mode != kModeLoglike) ? 1 : 0;
  a.wf = h->wf;
  a.wf_stride = kWfStride;
  a.xbuf = static_cast<R *>(h->xbuf);
  a.status = h->status;
  return a;
}

template <typename R>
EmuWeights<R> emu_weights(bst_ctx *h, int fold) {
  EmuWeights<R> w;
  w.depth = h->depth;
  w.width = h->width;
  w.dp = h->dp;
  w.W1T = static_cast<const R *>(h->sW1T[fold]);
  w.W1 = static_cast<const R *>(h->sW1[fold]);
  w.b1 = static_cast<const R *>(h->sb1[fold]);
  w.WT = static_cast<const R *>(h->sWT);
  w.W = static_cast<const R *>(h->sW);
  w.b = static_cast<const R *>(h->sb);
  w.wo = static_cast<const R *>(h->swo);
  w.bo = static_cast<R>(h->bo);
  w.out_m = static_cast<R>(h->out_m);
  w.out_s = static_cast<R>(h->out_s);
  w.out_log = h->out_log;
  w.out_floor = static_cast<R>(h->out_floor);
  w.scratch = static_cast<R *>(h->scratch);
  return w;
}

int cs_index(int cs) { return cs == 4 ? 2 : (cs == 2 ? 1 : 0); }

Tc2Weights tc2_weights(bst_ctx *h, int fold, int n_rows) {
  Tc2Weights w;
  const int cs = tc2_cluster_size(n_rows, h->width, h->depth), ci = cs_index(cs);
  w.depth = h->depth;
  w.width = h->width;
  w.dp = h->dp;
  w.kb1 = h->kb1;
  w.k16_l1 = 3 * h->dp / 16;
  w.cs = cs;
  const size_t ns = h->width / cs;
  w.l1 = h->tl1[fold][ci];
  w.l1_stride = ns * h->kb1 * 128;
  w.hid = h->thid[ci];
  w.hid_stride = 2 * static_cast<size_t>(h->depth > 1 ? h->depth - 1 : 0) * ns * h->width * 2;
  w.g1 = h->tg1[fold];
  w.b1 = h->tb1[fold];
  w.b = h->tb;
  w.wo = h->two;
  w.bo = static_cast<float>(h->bo);
  w.out_m = static_cast<float>(h->out_m);
  w.out_s = static_cast<float>(h->out_s);
  w.out_log = h->out_log;
  w.out_floor = static_cast<float>(h->out_floor);
  w.f16 = is_f16(h);
  w.scratch = static_cast<__nv_bfloat16 *>(h->scratch);
  {
    // the exchange images follow the stored activations of h->scratch_rows rows
    const size_t ab = act_bytes_for(h, h->scratch_rows);
    w.xchg = h->scratch ? static_cast<uint8_t *>(h->scratch) + ab : nullptr;
    w.xchg_bytes = h->scratch_bytes > ab ? h->scratch_bytes - ab : 0;
  }
  w.n_stages = tc2_stages(h->width, cs, h->depth);
  return w;
}

template <typename R>
AnaWeights<R> ana_weights(bst_ctx *h, int fold) {
  AnaWeights<R> w;
  w.d = h->d;
  w.dp = h->dp;
  w.H = h->H;
  w.n_data = h->n_data;
  w.linear = h->linear;
  w.has_N = (h->d > h->d_c) ? 1 : 0;
  w.Bf = static_cast<const R *>(h->aBf[fold]);
  w.cf = static_cast<const R *>(h->acf[fold]);
  w.AT = static_cast<const R *>(h->aAT);
  w.NfT = static_cast<const R *>(h->aNfT[fold]);
  w.dataf = static_cast<const R *>(h->adata[fold]);
  w.inv_s2 = static_cast<R>(1.0 / (h->sigma * h->sigma));
  return w;
}

// ------------------------------------------------------------------ weight preparation
// Bytes of scratch a launch over `rows` evaluation rows needs: the adjoint's stored
// activations, then (BF16) one slice image per CTA for the cluster exchange through global
// memory (whole 128-row tiles: 128 x width BF16 per tile), 256-byte aligned.
size_t act_bytes_for(const bst_ctx *h, size_t rows) {
  const size_t el = (tc_engine(h)) ? 2 : h->rs;
  const size_t b = rows * static_cast<size_t>(h->depth > 1 ? h->depth - 1 : 1) * h->width * el;
  return (b + 255) / 256 * 256;
}
size_t xchg_bytes_for(const bst_ctx *h, size_t rows) {
  if (!tc_engine(h)) return 0;
  return (rows + kTcRows - 1) / kTcRows * kTcRows * static_cast<size_t>(h->width) * 2;
}
size_t scratch_bytes_for(const bst_ctx *h, size_t rows) { return act_bytes_for(h, rows) + xchg_bytes_for(h, rows); }

bst_status ensure_scratch(bst_ctx *h, size_t rows) {
  if (h->lik != BST_LIK_EMULATOR) return BST_OK;
  if (rows <= h->scratch_rows && h->scratch) return BST_OK;
  dfree(h, h->scratch);
  h->scratch = nullptr;
  h->scratch_rows = 0;
  h->scratch_bytes = 0;
  const size_t bytes = scratch_bytes_for(h, rows);
  BST_TRY(dalloc(h, &h->scratch, bytes));
  h->scratch_rows = rows;
  h->scratch_bytes = bytes;
  return BST_OK;
}

bst_status prepare(bst_ctx *h, cudaStream_t s) {
  if (!h->weights_dirty) return BST_OK;
  if (h->lik == BST_LIK_EMULATOR) {
    if (h->p32_newer) {
      BST_CUDA(launch_cast_f32_to_f64(h->P32, h->P64, h->nparams, s));
      BST_CUDA(cudaMemcpyAsync(&h->bo, h->P64 + h->nparams - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
      BST_CUDA(cudaStreamSynchronize(s));
      h->p32_newer = false;
    }
    const int d = h->d, dp = h->dp, w = h->width, D = h->depth;
    for (int f = 0; f < 2; ++f) {
      BST_CUDA(launch_fold_layer1(h->P64, h->in_m64, h->in_s64, h->mu64, h->L64, d, dp, w, f, h->W1f[f], h->b1f[f], s));
      if (h->precision == BST_FP32)
        BST_CUDA(launch_pack_simt_f32(h->P64, h->W1f[f], h->b1f[f], d, dp, D, w, (float *)h->sW1T[f], (float *)h->sW1[f],
                                      (float *)h->sb1[f], (float *)h->sWT, (float *)h->sW, (float *)h->sb,
                                      (float *)h->swo, s));
      else if (h->precision == BST_FP64)
        BST_CUDA(launch_pack_simt_f64(h->P64, h->W1f[f], h->b1f[f], d, dp, D, w, (double *)h->sW1T[f],
                                      (double *)h->sW1[f], (double *)h->sb1[f], (double *)h->sWT, (double *)h->sW,
                                      (double *)h->sb, (double *)h->swo, s));
      else {
        for (int ci = 0; ci < 3; ++ci) {
          const int cs = 1 << ci, ns = w / cs, tr = ns < 256 ? ns : 256;
          for (int rk = 0; rk < cs; ++rk)
            BST_CUDA(launch_pack_tc2_l1(h->W1f[f], dp, h->kb1, rk, ns, tr, is_f16(h),
                                        h->tl1[f][ci] + static_cast<size_t>(rk) * ns * h->kb1 * 128, s));
        }
        BST_CUDA(launch_pack_tc_g1(h->W1f[f], dp, w, is_f16(h), h->tg1[f], s));
        BST_CUDA(launch_cast_f32(h->b1f[f], h->tb1[f], w, s));
      }
    }
    if (tc_engine(h)) {
      for (int ci = 0; ci < 3; ++ci) {
        const int cs = 1 << ci, ns = w / cs, tr = ns < 256 ? ns : 256;
        const size_t stride = 2 * static_cast<size_t>(D > 1 ? D - 1 : 0) * ns * w * 2;
        for (int rk = 0; rk < cs; ++rk)
          BST_CUDA(launch_pack_tc2_hidden(h->P64, d, D, w, rk, ns, tr, is_f16(h), h->thid[ci] + rk * stride, s));
      }
      for (int l = 2; l <= D; ++l) {
        const size_t ob = static_cast<size_t>(d) * w + w + static_cast<size_t>(l - 2) * (static_cast<size_t>(w) * w + w) +
                          static_cast<size_t>(w) * w;
        BST_CUDA(launch_cast_f32(h->P64 + ob, h->tb + static_cast<size_t>(l - 2) * w, w, s));
      }
      BST_CUDA(launch_cast_f32(h->P64 + h->nparams - 1 - w, h->two, w, s));
    }
  } else {
    for (int f = 0; f < 2; ++f) {
      BST_CUDA(launch_fold_analytic(h->A64, h->B64, h->c64, h->N64, h->data64, h->mu64, h->L64, h->d, h->dp, h->d_c,
                                    h->H, h->n_data, f, h->fBf, h->fcf, h->fAT, h->fNfT, h->fdata, s));
      auto cast = [&](const double *src, void *dst, size_t cnt) -> cudaError_t {
        return (h->rs == 8) ? launch_cast_f64(src, static_cast<double *>(dst), cnt, s)
                            : launch_cast_f32(src, static_cast<float *>(dst), cnt, s);
      };
      BST_CUDA(cast(h->fBf, h->aBf[f], static_cast<size_t>(h->H) * h->dp));
      BST_CUDA(cast(h->fcf, h->acf[f], h->H));
      if (f == 0) BST_CUDA(cast(h->fAT, h->aAT, static_cast<size_t>(h->H) * h->n_data));
      if (h->d > h->d_c) BST_CUDA(cast(h->fNfT, h->aNfT[f], static_cast<size_t>(h->dp) * h->n_data));
      BST_CUDA(cast(h->fdata, h->adata[f], h->n_data));
    }
  }
  h->weights_dirty = false;
  return BST_OK;
}

// one launch of the chain-tile kernel matching the handle's engine
bst_status run(bst_ctx *h, int mode, double eps, int n_leapfrog, int n_steps, void *samples, int fold,
               cudaStream_t s, const void *ext_in = nullptr, void *ext_logl = nullptr, void *ext_grad = nullptr,
               int m = 0, int need_grad = 0) {
  const bool ll = mode == kModeLoglike;
  if (h->precision == BST_FP64) {
    StepArgs<double> a = make_args<double>(h, mode, eps, n_leapfrog, n_steps, samples);
    if (ll) {
      a.n_rows = m;
      a.need_grad = need_grad;
      a.st.ze = (double *)ext_in;
      a.st.ze_ld = h->d;
      a.st.lle = (double *)ext_logl;
      a.st.gle = (double *)ext_grad;
      a.st.gle_ld = h->d;
    }
    if (h->lik == BST_LIK_EMULATOR) BST_CUDA(launch_emu_simt_f64(a, emu_weights<double>(h, fold), s));
    else BST_CUDA(launch_ana_simt_f64(a, ana_weights<double>(h, fold), s));
  } else {
    StepArgs<float> a = make_args<float>(h, mode, eps, n_leapfrog, n_steps, samples);
    if (ll) {
      a.n_rows = m;
      a.need_grad = need_grad;
      a.st.ze = (float *)ext_in;
      a.st.ze_ld = h->d;
      a.st.lle = (float *)ext_logl;
      a.st.gle = (float *)ext_grad;
      a.st.gle_ld = h->d;
    }
    if (h->lik == BST_LIK_ANALYTIC) BST_CUDA(launch_ana_simt_f32(a, ana_weights<float>(h, fold), s));
    else if (tc_engine(h)) BST_CUDA(launch_emu_tc2(a, tc2_weights(h, fold, a.n_rows), s));
    else BST_CUDA(launch_emu_simt_f32(a, emu_weights<float>(h, fold), s));
  }
  return BST_OK;
}

bst_status refresh(bst_ctx *h, cudaStream_t s) {
  BST_TRY(prepare(h, s));
  BST_TRY(ensure_scratch(h, h->n));
  BST_TRY(run(h, kModeRefresh, 0.0, 0, 1, nullptr, 0, s));
  h->state_stale = false;
  h->grad_valid = true;
  return BST_OK;
}

bst_status set_target(bst_ctx *h, const double *mu, const double *L) {
  const int d = h->d;
  // an unchanged whitening (bitwise) keeps the folded layer-1 weights: the chains are refreshed,
  // the weights are repacked only if something else made them dirty
  bool same = static_cast<int>(h->mu.size()) == d && static_cast<int>(h->L.size()) == d * d;
  for (int i = 0; same && i < d; ++i) {
    same = std::memcmp(&h->mu[i], &mu[i], sizeof(double)) == 0;
    for (int j = 0; same && j <= i; ++j) same = std::memcmp(&h->L[i * d + j], &L[i * d + j], sizeof(double)) == 0;
  }
  if (same) {
    h->state_stale = true;
    return BST_OK;
  }
  h->mu.assign(mu, mu + d);
  h->L.assign(d * d, 0.0);
  double ld = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) h->L[i * d + j] = L[i * d + j];
  for (int i = 0; i < d; ++i) ld += std::log(std::fabs(h->L[i * d + i]));
  h->logdet = ld;
  BST_CUDA(cudaMemcpy(h->mu64, h->mu.data(), d * 8, cudaMemcpyHostToDevice));
  BST_CUDA(cudaMemcpy(h->L64, h->L.data(), static_cast<size_t>(d) * d * 8, cudaMemcpyHostToDevice));
  h->weights_dirty = true;
  h->state_stale = true;
  return BST_OK;
}

bst_status sum_counters(bst_ctx *h, double out[4]) {
  const int n = h->n;
  std::vector<unsigned long long> a(n), e(n), dv(n);
  std::vector<double> as(n);
  BST_CUDA(cudaMemcpy(a.data(), h->accepts, n * 8, cudaMemcpyDeviceToHost));
  BST_CUDA(cudaMemcpy(e.data(), h->evals, n * 8, cudaMemcpyDeviceToHost));
  BST_CUDA(cudaMemcpy(dv.data(), h->divs, n * 8, cudaMemcpyDeviceToHost));
  BST_CUDA(cudaMemcpy(as.data(), h->acc_stat, n * 8, cudaMemcpyDeviceToHost));
  out[0] = out[1] = out[2] = out[3] = 0.0;
  for (int i = 0; i < n; ++i) {
    out[0] += static_cast<double>(a[i]);
    out[1] += static_cast<double>(e[i]);
    out[2] += static_cast<double>(dv[i]);
    out[3] += as[i];
  }
  return BST_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

const char *bst_version(void) { return "bst 0.1 (sm_103a)"; }
const char *bst_last_error(void) { return g_err.c_str(); }

bst_status bst_create(bst_handle *out, const bst_config *cfg) {
  if (!out || !cfg) return fail(BST_ERR_ARG, "bst_create: NULL argument");
  *out = nullptr;
  if (cfg->d < 1 || cfg->d > kMaxD) return fail(BST_ERR_ARG, "bst_create: d must be in 1..32");
  if (cfg->n_chains < 1) return fail(BST_ERR_ARG, "bst_create: n_chains must be >= 1");
  if (cfg->precision < BST_BF16 || cfg->precision > BST_FP16) return fail(BST_ERR_ARG, "bst_create: precision");
  if (cfg->lik_kind != BST_LIK_EMULATOR && cfg->lik_kind != BST_LIK_ANALYTIC)
    return fail(BST_ERR_ARG, "bst_create: lik_kind");
  if ((cfg->precision == BST_BF16 || cfg->precision == BST_FP16) && cfg->lik_kind != BST_LIK_EMULATOR)
    return fail(BST_ERR_UNSUPPORTED, "bst_create: BF16 / FP16 precision needs the emulator likelihood");
  const int md = cfg->max_depth ? cfg->max_depth : 8;
  if (md < 1 || md > kMaxDepthNuts) return fail(BST_ERR_ARG, "bst_create: max_depth must be in 1..10");
  const int wk = cfg->aies_walkers ? cfg->aies_walkers : 64;
  if (wk < 2 || wk % 2) return fail(BST_ERR_ARG, "bst_create: aies_walkers must be even and >= 2");
  const double aa = cfg->aies_a != 0.0 ? cfg->aies_a : 2.0;
  if (!(aa > 1.0)) return fail(BST_ERR_ARG, "bst_create: aies_a must be > 1");
  const int th = cfg->thin ? cfg->thin : 1;
  if (th < 1) return fail(BST_ERR_ARG, "bst_create: thin must be >= 1");
  BST_CUDA(cudaSetDevice(cfg->device));
  bst_ctx *h = new bst_ctx();
  h->d = cfg->d;
  h->dp = pad16(cfg->d);
  h->n = cfg->n_chains;
  h->precision = cfg->precision;
  h->lik = cfg->lik_kind;
  h->seed = cfg->seed;
  h->max_depth = md;
  h->walkers = wk;
  h->aies_a = aa;
  h->thin = th;
  h->device = cfg->device;
  h->rs = (cfg->precision == BST_FP64) ? 8 : 4;
  h->kb1 = (3 * h->dp + 63) / 64;
  const size_t n = h->n, dp = h->dp, rs = h->rs;
  // the general sampler code's per-chain buffers are chain-blocked over the padded chain count
  const size_t np = chains_padded(h->n);
  h->work_stride = static_cast<int>(rs == 8 ? work_elems_per_chain<double>() : work_elems_per_chain<float>());
  bst_status st = BST_OK;
  auto A = [&](void **p, size_t b) {
    if (st == BST_OK) st = dalloc(h, p, b);
  };
  A(&h->z, n * dp * rs);
  A(&h->g, n * dp * rs);
  A(&h->lp, n * rs);
  A(&h->ze, np * dp * rs);
  A(&h->lle, n * rs);
  A(&h->gle, np * dp * rs);
  A(&h->work, np * static_cast<size_t>(h->work_stride) * rs);
  A(&h->xbuf, n * dp * rs);
  A((void **)&h->iter, n * 4);
  A((void **)&h->acc_stat, n * 8);
  A((void **)&h->accepts, n * 8);
  A((void **)&h->evals, n * 8);
  A((void **)&h->divs, n * 8);
  A((void **)&h->steps_done, n * 4);
  A((void **)&h->status, 64);
  A((void **)&h->mu64, kMaxD * 8);
  A((void **)&h->L64, kMaxD * kMaxD * 8);
  A((void **)&h->mu64_new, kMaxD * 8);
  A((void **)&h->L64_new, kMaxD * kMaxD * 8);
  A((void **)&h->info64, 8 * 8);
  A((void **)&h->stats64, (1 + kMaxD + kMaxD * kMaxD) * 8);
  h->wf_records = static_cast<int>((n + 15) / 16) + 1;  // one per tile for any tiling + one external
  A((void **)&h->wf, static_cast<size_t>(h->wf_records) * kWfStride * 8);
  if (st != BST_OK) {
    bst_destroy(h);
    return st;
  }
  *out = h;
  return BST_OK;
}

void bst_destroy(bst_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  for (void *p : h->allocs)
    if (p) cudaFree(p);
  delete h;
}

bst_status bst_set_emulator(bst_handle h, int depth, int width, const double *params, const double *in_m,
                            const double *in_s, double out_m, double out_s) {
  NvtxRange nvtx_("bst_set_emulator");
  if (!h || !params || !in_m || !in_s) return fail(BST_ERR_ARG, "bst_set_emulator: NULL argument");
  if (h->lik != BST_LIK_EMULATOR) return fail(BST_ERR_STATE, "bst_set_emulator: handle was created for the analytic likelihood");
  if (depth < 1 || depth > 8) return fail(BST_ERR_ARG, "bst_set_emulator: depth must be in 1..8");
  if (width < 256 || width % 256) return fail(BST_ERR_UNSUPPORTED, "bst_set_emulator: width must be a multiple of 256");
  if (tc_engine(h) && width > 512) return fail(BST_ERR_UNSUPPORTED, "bst_set_emulator: BF16 / FP16 width must be 256 or 512");
  if (h->precision == BST_FP64 && width > 512) return fail(BST_ERR_UNSUPPORTED, "bst_set_emulator: FP64 width must be <= 512");
  if (width > 1024) return fail(BST_ERR_UNSUPPORTED, "bst_set_emulator: width must be <= 1024");
  const int d = h->d;
  const size_t np = static_cast<size_t>(d) * width + width + static_cast<size_t>(depth - 1) * (static_cast<size_t>(width) * width + width) + width + 1;
  if (!all_finite(params, np) || !all_finite(in_m, d) || !all_finite(in_s, d) || !std::isfinite(out_m) || !std::isfinite(out_s))
    return fail(BST_ERR_NONFINITE, "bst_set_emulator: non-finite parameter");
  for (int i = 0; i < d; ++i)
    if (!(in_s[i] > 0.0)) return fail(BST_ERR_ARG, "bst_set_emulator: in_s must be positive");
  BST_CUDA(cudaSetDevice(h->device));
  const bool realloc = !(h->depth == depth && h->width == width && h->P64);
  if (realloc) {
    h->depth = depth;
    h->width = width;
    h->nparams = np;
    const size_t w = width, dp = h->dp, rs = h->rs, nh = static_cast<size_t>(depth - 1);
    BST_TRY(dalloc_t(h, &h->P64, np));
    BST_TRY(dalloc_t(h, &h->in_m64, d));
    BST_TRY(dalloc_t(h, &h->in_s64, d));
    for (int f = 0; f < 2; ++f) {
      BST_TRY(dalloc_t(h, &h->W1f[f], w * dp));
      BST_TRY(dalloc_t(h, &h->b1f[f], w));
    }
    if (tc_engine(h)) {
      for (int f = 0; f < 2; ++f) {
        for (int ci = 0; ci < 3; ++ci) BST_TRY(dalloc(h, (void **)&h->tl1[f][ci], w * h->kb1 * 128));
        BST_TRY(dalloc(h, (void **)&h->tg1[f], (w / 64) * 2 * dp * 128));
        BST_TRY(dalloc_t(h, &h->tb1[f], w));
      }
      for (int ci = 0; ci < 3; ++ci) BST_TRY(dalloc(h, (void **)&h->thid[ci], 2 * nh * w * w * 2 + 16));
      BST_TRY(dalloc_t(h, &h->tb, nh * w + 1));
      BST_TRY(dalloc_t(h, &h->two, w));
    } else {
      for (int f = 0; f < 2; ++f) {
        BST_TRY(dalloc(h, &h->sW1T[f], dp * w * rs));
        BST_TRY(dalloc(h, &h->sW1[f], dp * w * rs));
        BST_TRY(dalloc(h, &h->sb1[f], w * rs));
      }
      BST_TRY(dalloc(h, &h->sWT, nh * w * w * rs + 16));
      BST_TRY(dalloc(h, &h->sW, nh * w * w * rs + 16));
      BST_TRY(dalloc(h, &h->sb, nh * w * rs + 16));
      BST_TRY(dalloc(h, &h->swo, w * rs));
    }
    h->scratch_rows = 0;
    h->scratch_bytes = 0;
    dfree(h, h->scratch);
    h->scratch = nullptr;
    // training state belongs to the old shape
    h->P32 = nullptr;
  }
  BST_CUDA(cudaMemcpy(h->P64, params, np * 8, cudaMemcpyHostToDevice));
  BST_CUDA(cudaMemcpy(h->in_m64, in_m, d * 8, cudaMemcpyHostToDevice));
  BST_CUDA(cudaMemcpy(h->in_s64, in_s, d * 8, cudaMemcpyHostToDevice));
  h->out_m = out_m;
  h->out_s = out_s;
  h->out_log = 0;
  h->out_floor = 0.0;
  h->bo = params[np - 1];
  h->p32_newer = false;
  if (h->P32) {
    BST_CUDA(launch_cast_f32(h->P64, h->P32, np, 0));
    h->adam_t = 0;
    BST_CUDA(cudaMemset(h->m1, 0, np * 4));
    BST_CUDA(cudaMemset(h->m2, 0, np * 4));
  }
  h->weights_dirty = true;
  h->state_stale = true;
  if (h->stage < 1) h->stage = 1;
  if (h->stage < 2) {
    // loglike works before init_chains: identity whitening for the fold buffers
    std::vector<double> mu(d, 0.0), L(static_cast<size_t>(d) * d, 0.0);
    for (int i = 0; i < d; ++i) L[i * d + i] = 1.0;
    if (h->mu.empty()) BST_TRY(set_target(h, mu.data(), L.data()));
  }
  return BST_OK;
}

bst_status bst_get_emulator(bst_handle h, double *params) {
  if (!h || !params) return fail(BST_ERR_ARG, "bst_get_emulator: NULL argument");
  if (h->lik != BST_LIK_EMULATOR || !h->P64) return fail(BST_ERR_STATE, "bst_get_emulator: no emulator set");
  BST_CUDA(cudaSetDevice(h->device));
  if (h->p32_newer) {
    BST_CUDA(launch_cast_f32_to_f64(h->P32, h->P64, h->nparams, 0));
    h->p32_newer = false;
  }
  BST_CUDA(cudaDeviceSynchronize());
  BST_CUDA(cudaMemcpy(params, h->P64, h->nparams * 8, cudaMemcpyDeviceToHost));
  h->bo = params[h->nparams - 1];
  return BST_OK;
}

bst_status bst_set_emulator_output(bst_handle h, int kind, double floor) {
  if (!h) return fail(BST_ERR_ARG, "bst_set_emulator_output: NULL handle");
  if (h->lik != BST_LIK_EMULATOR || !h->P64) return fail(BST_ERR_STATE, "bst_set_emulator_output: no emulator set");
  if (kind != BST_OUT_LINEAR && kind != BST_OUT_LOG) return fail(BST_ERR_ARG, "bst_set_emulator_output: unknown kind");
  if (!std::isfinite(floor)) return fail(BST_ERR_ARG, "bst_set_emulator_output: non-finite floor");
  h->out_log = kind == BST_OUT_LOG ? 1 : 0;
  h->out_floor = floor;
  h->state_stale = true;
  return BST_OK;
}

bst_status bst_set_analytic(bst_handle h, int d_c, int n_hidden, int n_data, const double *A, const double *B,
                            const double *c, const double *N, const double *data, double sigma, int linear) {
  if (!h || !A || !B || !c || !data) return fail(BST_ERR_ARG, "bst_set_analytic: NULL argument");
  if (h->lik != BST_LIK_ANALYTIC) return fail(BST_ERR_STATE, "bst_set_analytic: handle was created for the emulator");
  const int d = h->d;
  if (d_c < 1 || d_c > d) return fail(BST_ERR_ARG, "bst_set_analytic: d_c must be in 1..d");
  if (d_c < d && !N) return fail(BST_ERR_ARG, "bst_set_analytic: N required when d_c < d");
  if (n_hidden < 1 || n_hidden > 64) return fail(BST_ERR_UNSUPPORTED, "bst_set_analytic: n_hidden must be in 1..64");
  if (n_data < 1) return fail(BST_ERR_ARG, "bst_set_analytic: n_data must be >= 1");
  if (!(sigma > 0.0)) return fail(BST_ERR_ARG, "bst_set_analytic: sigma must be positive");
  const size_t nA = static_cast<size_t>(n_data) * n_hidden, nB = static_cast<size_t>(n_hidden) * d_c,
               nN = static_cast<size_t>(n_data) * (d - d_c);
  if (!all_finite(A, nA) || !all_finite(B, nB) || !all_finite(c, n_hidden) || !all_finite(data, n_data) ||
      (nN && !all_finite(N, nN)))
    return fail(BST_ERR_NONFINITE, "bst_set_analytic: non-finite input");
  BST_CUDA(cudaSetDevice(h->device));
  const bool realloc = !(h->H == n_hidden && h->n_data == n_data && h->d_c == d_c && h->A64);
  h->d_c = d_c;
  h->H = n_hidden;
  h->n_data = n_data;
  h->linear = linear ? 1 : 0;
  h->sigma = sigma;
  h->has_N = (d > d_c) ? 1 : 0;
  if (realloc) {
    const size_t dp = h->dp, rs = h->rs;
    BST_TRY(dalloc_t(h, &h->A64, nA));
    BST_TRY(dalloc_t(h, &h->B64, nB));
    BST_TRY(dalloc_t(h, &h->c64, n_hidden));
    BST_TRY(dalloc_t(h, &h->N64, nN + 1));
    BST_TRY(dalloc_t(h, &h->data64, n_data));
    BST_TRY(dalloc_t(h, &h->fBf, n_hidden * dp));
    BST_TRY(dalloc_t(h, &h->fcf, n_hidden));
    BST_TRY(dalloc_t(h, &h->fAT, nA));
    BST_TRY(dalloc_t(h, &h->fNfT, dp * n_data));
    BST_TRY(dalloc_t(h, &h->fdata, n_data));
    BST_TRY(dalloc(h, &h->aAT, nA * rs));
    for (int f = 0; f < 2; ++f) {
      BST_TRY(dalloc(h, &h->aBf[f], n_hidden * dp * rs));
      BST_TRY(dalloc(h, &h->acf[f], n_hidden * rs));
      BST_TRY(dalloc(h, &h->aNfT[f], dp * n_data * rs));
      BST_TRY(dalloc(h, &h->adata[f], n_data * rs));
    }
  }
  BST_CUDA(cudaMemcpy(h->A64, A, nA * 8, cudaMemcpyHostToDevice));
  BST_CUDA(cudaMemcpy(h->B64, B, nB * 8, cudaMemcpyHostToDevice));
  BST_CUDA(cudaMemcpy(h->c64, c, n_hidden * 8, cudaMemcpyHostToDevice));
  if (nN) BST_CUDA(cudaMemcpy(h->N64, N, nN * 8, cudaMemcpyHostToDevice));
  BST_CUDA(cudaMemcpy(h->data64, data, n_data * 8, cudaMemcpyHostToDevice));
  h->weights_dirty = true;
  h->state_stale = true;
  if (h->stage < 1) h->stage = 1;
  if (h->mu.empty()) {
    std::vector<double> mu(d, 0.0), L(static_cast<size_t>(d) * d, 0.0);
    for (int i = 0; i < d; ++i) L[i * d + i] = 1.0;
    BST_TRY(set_target(h, mu.data(), L.data()));
  }
  return BST_OK;
}

bst_status bst_init_chains(bst_handle h, const double *theta0, const double *lower, const double *upper,
                           const int *gauss, const double *mu, const double *L) {
  NvtxRange nvtx_("bst_init_chains");
  if (!h || !theta0 || !lower || !upper || !mu || !L) return fail(BST_ERR_ARG, "bst_init_chains: NULL argument");
  if (h->stage < 1) return fail(BST_ERR_STATE, "bst_init_chains: set a likelihood first");
  const int d = h->d, n = h->n;
  if (!all_finite(theta0, static_cast<size_t>(n) * d) || !all_finite(mu, d))
    return fail(BST_ERR_NONFINITE, "bst_init_chains: non-finite theta0 or mu");
  for (int i = 0; i < d; ++i) {
    if (!(L[i * d + i] > 0.0) || !std::isfinite(L[i * d + i]))
      return fail(BST_ERR_ARG, "bst_init_chains: L must have a positive finite diagonal");
    for (int j = 0; j <= i; ++j)
      if (!std::isfinite(L[i * d + j])) return fail(BST_ERR_NONFINITE, "bst_init_chains: non-finite L");
    if (std::isnan(lower[i]) || std::isnan(upper[i]) || !(lower[i] <= upper[i]))
      return fail(BST_ERR_ARG, "bst_init_chains: need lower <= upper");
  }
  BST_CUDA(cudaSetDevice(h->device));
  BST_TRY(set_target(h, mu, L));
  h->lower.assign(lower, lower + d);
  h->upper.assign(upper, upper + d);
  h->gauss.assign(d, 0);
  h->any_gauss = 0;
  if (gauss)
    for (int i = 0; i < d; ++i) {
      h->gauss[i] = gauss[i] ? 1 : 0;
      h->any_gauss |= h->gauss[i];
    }
  // z0 = L^-1 (theta0 - mu) on the device (FP64 forward substitution): theta0 is copied in once
  // (a DMA when it is page-locked) and the counters are cleared on the same stream
  const size_t nn = n;
  if (h->theta_cap < nn * d) {
    dfree(h, h->theta64);
    h->theta64 = nullptr;
    h->theta_cap = 0;
    BST_TRY(dalloc_t(h, &h->theta64, nn * d));
    h->theta_cap = nn * d;
  }
  BST_CUDA(cudaMemcpyAsync(h->theta64, theta0, nn * d * 8, cudaMemcpyHostToDevice, 0));
  BST_CUDA(launch_init_z(h->rs == 8, h->theta64, h->mu64, h->L64, n, d, h->dp, h->z, 0));
  BST_CUDA(cudaMemsetAsync(h->iter, 0, nn * 4, 0));
  BST_CUDA(cudaMemsetAsync(h->acc_stat, 0, nn * 8, 0));
  BST_CUDA(cudaMemsetAsync(h->accepts, 0, nn * 8, 0));
  BST_CUDA(cudaMemsetAsync(h->evals, 0, nn * 8, 0));
  BST_CUDA(cudaMemsetAsync(h->divs, 0, nn * 8, 0));
  BST_CUDA(cudaMemsetAsync(h->work, 0, chains_padded(h->n) * h->work_stride * h->rs, 0));
  BST_CUDA(cudaMemsetAsync(h->status, 0, 64, 0));
  h->stage = 2;
  BST_TRY(refresh(h, 0));
  BST_CUDA(cudaDeviceSynchronize());
  return check_status(h);
}

bst_status bst_step(bst_handle h, int kernel, double eps, int n_leapfrog, int n_steps, void *samples_dev,
                    void *stream, bst_step_stats *stats) {
  NvtxRange nvtx_("bst_step");
  if (!h) return fail(BST_ERR_ARG, "bst_step: NULL handle");
  if (h->stage < 2) return fail(BST_ERR_STATE, "bst_step: call bst_init_chains first");
  if (kernel < BST_MH || kernel > BST_NUTS_MULTINOMIAL) return fail(BST_ERR_ARG, "bst_step: unknown kernel");
  if (n_steps < 0) return fail(BST_ERR_ARG, "bst_step: n_steps must be >= 0");
  if (kernel != BST_AIES && kernel != BST_AIES_DE && !(eps > 0.0 && std::isfinite(eps)))
    return fail(BST_ERR_ARG, "bst_step: eps must be positive");
  if (kernel == BST_AIES_DE && !(eps >= 0.0 && std::isfinite(eps)))
    return fail(BST_ERR_ARG, "bst_step: the DE move's eps (sigma_gamma) must be finite and >= 0");
  if (kernel == BST_AIES_DE && h->walkers < 4)
    return fail(BST_ERR_ARG, "bst_step: the DE move needs aies_walkers >= 4");
  if (kernel == BST_HMC && n_leapfrog < 1) return fail(BST_ERR_ARG, "bst_step: n_leapfrog must be >= 1");
  if (kernel == BST_AIES || kernel == BST_AIES_DE) {
    const int half = h->walkers / 2;
    const int tile = (tc_engine(h)) ? kTcRows : simt_rows_per_tile(h->precision, h->width, h->lik);  // chains per tile
    if (h->n % h->walkers) return fail(BST_ERR_ARG, "bst_step: AIES needs n_chains to be a multiple of aies_walkers");
    // the tensor-core engine holds whole halves in a tile; the CUDA-core engines spread a half
    // over a cluster of up to 8 tiles
    if (tc_engine(h) ? (tile % half) != 0 : (half % tile != 0 && tile % half != 0) || half / tile > 8)
      return fail(BST_ERR_UNSUPPORTED, "bst_step: AIES ensemble halves do not fit the chain tiles");
  }
  BST_CUDA(cudaSetDevice(h->device));
  // the sample record: device memory of this device, or page-locked host memory mapped into
  // the device's address space (written by the kernel directly, over the host link)
  void *samples_ptr = samples_dev;
  if (samples_dev) {
    cudaPointerAttributes at = {};
    if (cudaPointerGetAttributes(&at, samples_dev) != cudaSuccess) {
      cudaGetLastError();
      return fail(BST_ERR_ARG, "bst_step: samples is neither device memory nor page-locked host memory");
    }
    if (at.type == cudaMemoryTypeHost) {
      if (!at.devicePointer) return fail(BST_ERR_ARG, "bst_step: page-locked samples buffer not mapped for the device");
      samples_ptr = at.devicePointer;
    } else if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
      if (at.type == cudaMemoryTypeDevice && at.device != h->device)
        return fail(BST_ERR_ARG, "bst_step: samples buffer on another device");
    } else {
      return fail(BST_ERR_ARG, "bst_step: samples must be device memory or page-locked host memory");
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_steps == 0) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    return BST_OK;
  }
  BST_TRY(prepare(h, s));
  BST_TRY(ensure_scratch(h, h->n));
  const bool needs_grad = kernel == BST_MALA || kernel == BST_HMC || kernel == BST_NUTS || kernel == BST_NUTS_MULTINOMIAL;
  if (h->state_stale || (needs_grad && !h->grad_valid)) BST_TRY(refresh(h, s));
  double before[4] = {0, 0, 0, 0}, after[4];
  if (stats) {
    BST_CUDA(cudaStreamSynchronize(s));
    BST_TRY(sum_counters(h, before));
  }
  BST_TRY(run(h, kernel, eps, n_leapfrog, n_steps, samples_ptr, 0, s));
  if (!needs_grad) h->grad_valid = false;
  if (stats) {
    BST_CUDA(cudaStreamSynchronize(s));
    BST_TRY(sum_counters(h, after));
    stats->accepts = static_cast<int64_t>(after[0] - before[0]);
    stats->evals = static_cast<int64_t>(after[1] - before[1]);
    stats->divergences = static_cast<int64_t>(after[2] - before[2]);
    stats->accept_stat = (after[3] - before[3]) / (static_cast<double>(h->n) * n_steps);
    bst_status st = check_status(h);
    stats->status = st;
    return st;
  }
  return BST_OK;
}

static bst_status loglike_impl(bst_handle h, const void *theta, int m, void *logl, void *grad, void *stream,
                               int need_grad) {
  NvtxRange nvtx_(need_grad ? "bst_grad_loglike" : "bst_loglike");
  const std::string fn = need_grad ? "bst_grad_loglike" : "bst_loglike";
  if (!h || (m > 0 && (!theta || !logl || (need_grad && !grad)))) return fail(BST_ERR_ARG, fn + ": NULL argument");
  if (h->stage < 1) return fail(BST_ERR_STATE, fn + ": set a likelihood first");
  if (m < 0) return fail(BST_ERR_ARG, fn + ": m must be >= 0");
  if (m == 0) return BST_OK;
  BST_CUDA(cudaSetDevice(h->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BST_TRY(prepare(h, s));
  const int chunk = h->n > 65536 ? h->n : 65536;
  // (the BF16 engine also needs the scratch for the cluster exchange of forward-only runs)
  if (need_grad || tc_engine(h)) BST_TRY(ensure_scratch(h, chunk < m ? chunk : m));
  const size_t rs = h->rs;
  for (int r0 = 0; r0 < m; r0 += chunk) {
    const int rows = (m - r0) < chunk ? (m - r0) : chunk;
    const char *ti = static_cast<const char *>(theta) + static_cast<size_t>(r0) * h->d * rs;
    char *lo = static_cast<char *>(logl) + static_cast<size_t>(r0) * rs;
    char *go = need_grad ? static_cast<char *>(grad) + static_cast<size_t>(r0) * h->d * rs : nullptr;
    BST_TRY(run(h, kModeLoglike, 0.0, 0, 1, nullptr, 1, s, ti, lo, go, rows, need_grad));
  }
  return BST_OK;
}

bst_status bst_loglike(bst_handle h, const void *theta_dev, int m, void *logl_dev, void *stream) {
  return loglike_impl(h, theta_dev, m, logl_dev, nullptr, stream, 0);
}
bst_status bst_grad_loglike(bst_handle h, const void *theta_dev, int m, void *logl_dev, void *grad_dev,
                            void *stream) {
  return loglike_impl(h, theta_dev, m, logl_dev, grad_dev, stream, 1);
}

bst_status bst_welford_reset(bst_handle h) {
  if (!h) return fail(BST_ERR_ARG, "bst_welford_reset: NULL handle");
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(launch_welford_clear(h->wf, h->wf_records, kWfStride, 0));
  h->welford_on = true;
  return BST_OK;
}

bst_status bst_welford_add(bst_handle h, const void *x_dev, int m, void *stream) {
  NvtxRange nvtx_("bst_welford_add");
  if (!h || (m > 0 && !x_dev)) return fail(BST_ERR_ARG, "bst_welford_add: NULL argument");
  if (m < 0) return fail(BST_ERR_ARG, "bst_welford_add: m must be >= 0");
  if (m == 0) return BST_OK;
  BST_CUDA(cudaSetDevice(h->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *rec = h->wf + static_cast<size_t>(h->wf_records - 1) * kWfStride;
  if (h->rs == 8) BST_CUDA(launch_welford_add_f64(static_cast<const double *>(x_dev), m, h->d, rec, kWfStride, s));
  else BST_CUDA(launch_welford_add_f32(static_cast<const float *>(x_dev), m, h->d, rec, kWfStride, s));
  return BST_OK;
}

bst_status bst_welford_stats(bst_handle h, double *n, double *mean, double *M2) {
  if (!h || !n || !mean || !M2) return fail(BST_ERR_ARG, "bst_welford_stats: NULL argument");
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(cudaDeviceSynchronize());
  const int d = h->d;
  std::vector<double> host(1 + d + static_cast<size_t>(d) * d);
  BST_CUDA(launch_welford_stats(h->wf, h->wf_records, kWfStride, d, h->stats64, 0));
  BST_CUDA(cudaMemcpy(host.data(), h->stats64, host.size() * 8, cudaMemcpyDeviceToHost));
  *n = host[0];
  std::memcpy(mean, host.data() + 1, d * 8);
  std::memcpy(M2, host.data() + 1 + d, static_cast<size_t>(d) * d * 8);
  return BST_OK;
}

bst_status bst_welford_merge(bst_handle h, double n, const double *mean, const double *M2) {
  if (!h || !mean || !M2) return fail(BST_ERR_ARG, "bst_welford_merge: NULL argument");
  if (!(n >= 0.0)) return fail(BST_ERR_ARG, "bst_welford_merge: n must be >= 0");
  const int d = h->d;
  std::vector<double> host(1 + d + static_cast<size_t>(d) * d);
  host[0] = n;
  std::memcpy(host.data() + 1, mean, d * 8);
  std::memcpy(host.data() + 1 + d, M2, static_cast<size_t>(d) * d * 8);
  if (!all_finite(host.data(), host.size())) return fail(BST_ERR_NONFINITE, "bst_welford_merge: non-finite input");
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(cudaDeviceSynchronize());
  BST_CUDA(cudaMemcpy(h->stats64, host.data(), host.size() * 8, cudaMemcpyHostToDevice));
  double *rec = h->wf + static_cast<size_t>(h->wf_records - 1) * kWfStride;
  BST_CUDA(launch_welford_merge(rec, d, h->stats64, 0));
  BST_CUDA(cudaDeviceSynchronize());
  return BST_OK;
}

bst_status bst_adapt_cov(bst_handle h, double jitter0, double *mu_out, double *L_out, double *jitter_used) {
  NvtxRange nvtx_("bst_adapt_cov");
  if (!h) return fail(BST_ERR_ARG, "bst_adapt_cov: NULL handle");
  if (h->stage < 2) return fail(BST_ERR_STATE, "bst_adapt_cov: call bst_init_chains first");
  if (!(jitter0 > 0.0)) return fail(BST_ERR_ARG, "bst_adapt_cov: jitter0 must be positive");
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(cudaDeviceSynchronize());
  BST_TRY(check_status(h));
  const int d = h->d;
  BST_CUDA(launch_adapt_finalize(h->wf, h->wf_records, kWfStride, d, jitter0, h->mu64_new, h->L64_new, h->info64, 0));
  double info[3];
  BST_CUDA(cudaMemcpy(info, h->info64, 3 * 8, cudaMemcpyDeviceToHost));
  if (info[2] == 1.0) return fail(BST_ERR_STATE, "bst_adapt_cov: fewer than 2 samples accumulated");
  if (info[2] == 2.0) return fail(BST_ERR_NOT_PD, "bst_adapt_cov: covariance not positive definite up to jitter 1e-2");
  std::vector<double> mu(d), L(static_cast<size_t>(d) * d);
  BST_CUDA(cudaMemcpy(mu.data(), h->mu64_new, d * 8, cudaMemcpyDeviceToHost));
  BST_CUDA(cudaMemcpy(L.data(), h->L64_new, static_cast<size_t>(d) * d * 8, cudaMemcpyDeviceToHost));
  // keep x fixed: z_new = L_new^-1 (mu_old + L_old z_old - mu_new)
  if (h->rs == 8) BST_CUDA(launch_remap_f64((double *)h->z, h->n, d, h->dp, h->mu64, h->L64, h->mu64_new, h->L64_new, 0));
  else BST_CUDA(launch_remap_f32((float *)h->z, h->n, d, h->dp, h->mu64, h->L64, h->mu64_new, h->L64_new, 0));
  BST_CUDA(cudaDeviceSynchronize());
  BST_TRY(set_target(h, mu.data(), L.data()));
  h->welford_on = false;
  BST_TRY(refresh(h, 0));
  BST_CUDA(cudaDeviceSynchronize());
  if (mu_out) std::memcpy(mu_out, mu.data(), d * 8);
  if (L_out) std::memcpy(L_out, L.data(), static_cast<size_t>(d) * d * 8);
  if (jitter_used) *jitter_used = info[1];
  return check_status(h);
}

bst_status bst_draw_positions(bst_handle h, int strategy, const double *center, const double *Lc, const double *lower,
                              const double *upper, double *theta_out) {
  NvtxRange nvtx_("bst_draw_positions");
  if (!h || !theta_out) return fail(BST_ERR_ARG, "bst_draw_positions: NULL argument");
  const int n = h->n, d = h->d;
  std::vector<double> par(static_cast<size_t>(3 + kMaxD) * kMaxD, 0.0);
  if (strategy == BST_INIT_REPEATED || strategy == BST_INIT_GAUSSIAN) {
    if (!center) return fail(BST_ERR_ARG, "bst_draw_positions: center required");
    for (int i = 0; i < d; ++i) {
      if (!std::isfinite(center[i])) return fail(BST_ERR_ARG, "bst_draw_positions: center not finite");
      par[i] = center[i];
    }
  }
  if (strategy == BST_INIT_UNIFORM) {
    if (!lower || !upper) return fail(BST_ERR_ARG, "bst_draw_positions: bounds required");
    for (int i = 0; i < d; ++i) {
      if (!std::isfinite(lower[i]) || !std::isfinite(upper[i]) || !(upper[i] > lower[i]))
        return fail(BST_ERR_ARG, "bst_draw_positions: need finite bounds with upper > lower");
      par[kMaxD + i] = lower[i];
      par[2 * kMaxD + i] = upper[i];
    }
  }
  if (strategy == BST_INIT_GAUSSIAN) {
    if (!Lc) return fail(BST_ERR_ARG, "bst_draw_positions: Lc required");
    for (int i = 0; i < d * d; ++i) {
      if (!std::isfinite(Lc[i])) return fail(BST_ERR_ARG, "bst_draw_positions: Lc not finite");
      par[3 * kMaxD + i] = Lc[i];
    }
  }
  if (strategy < BST_INIT_REPEATED || strategy > BST_INIT_GAUSSIAN) return fail(BST_ERR_ARG, "bst_draw_positions: unknown strategy");
  BST_CUDA(cudaSetDevice(h->device));
  if (!h->init_par) {
    BST_TRY(dalloc_t(h, &h->init_par, par.size()));
    BST_TRY(dalloc_t(h, &h->init_theta, static_cast<size_t>(n) * d));
  }
  BST_CUDA(cudaMemcpy(h->init_par, par.data(), par.size() * 8, cudaMemcpyHostToDevice));
  BST_CUDA(launch_init_positions(strategy, h->seed, n, d, h->init_par, h->init_theta, 0));
  BST_CUDA(cudaMemcpy(theta_out, h->init_theta, static_cast<size_t>(n) * d * 8, cudaMemcpyDeviceToHost));
  return BST_OK;
}

bst_status bst_set_whitening(bst_handle h, const double *mu, const double *L) {
  NvtxRange nvtx_("bst_set_whitening");
  if (!h || !mu || !L) return fail(BST_ERR_ARG, "bst_set_whitening: NULL argument");
  if (h->stage < 2) return fail(BST_ERR_STATE, "bst_set_whitening: call bst_init_chains first");
  const int d = h->d;
  for (int i = 0; i < d; ++i) {
    if (!std::isfinite(mu[i]) || !(L[i * d + i] > 0.0) || !std::isfinite(L[i * d + i]))
      return fail(BST_ERR_ARG, "bst_set_whitening: mu must be finite and L lower triangular with positive diagonal");
    for (int j = 0; j < i; ++j)
      if (!std::isfinite(L[i * d + j])) return fail(BST_ERR_ARG, "bst_set_whitening: L not finite");
  }
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(cudaDeviceSynchronize());
  BST_TRY(check_status(h));
  std::vector<double> Ll(static_cast<size_t>(d) * d, 0.0);  // lower triangle only
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) Ll[i * d + j] = L[i * d + j];
  BST_CUDA(cudaMemcpy(h->mu64_new, mu, d * 8, cudaMemcpyHostToDevice));
  BST_CUDA(cudaMemcpy(h->L64_new, Ll.data(), static_cast<size_t>(d) * d * 8, cudaMemcpyHostToDevice));
  // keep x fixed: z_new = L_new^-1 (mu_old + L_old z_old - mu_new), as after adaptation
  if (h->rs == 8) BST_CUDA(launch_remap_f64((double *)h->z, h->n, d, h->dp, h->mu64, h->L64, h->mu64_new, h->L64_new, 0));
  else BST_CUDA(launch_remap_f32((float *)h->z, h->n, d, h->dp, h->mu64, h->L64, h->mu64_new, h->L64_new, 0));
  BST_CUDA(cudaDeviceSynchronize());
  BST_TRY(set_target(h, mu, Ll.data()));
  BST_TRY(refresh(h, 0));
  BST_CUDA(cudaDeviceSynchronize());
  return check_status(h);
}

bst_status bst_set_bounds_penalty(bst_handle h, const double *width) {
  NvtxRange nvtx_("bst_set_bounds_penalty");
  if (!h) return fail(BST_ERR_ARG, "bst_set_bounds_penalty: NULL handle");
  if (h->stage < 2) return fail(BST_ERR_STATE, "bst_set_bounds_penalty: call bst_init_chains first");
  const int d = h->d;
  if (width)
    for (int i = 0; i < d; ++i)
      if (!std::isfinite(width[i]) || width[i] < 0.0)
        return fail(BST_ERR_ARG, "bst_set_bounds_penalty: widths must be finite and >= 0");
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(cudaDeviceSynchronize());
  BST_TRY(check_status(h));
  if (width) h->pen_w.assign(width, width + d);
  else h->pen_w.clear();
  BST_TRY(refresh(h, 0));
  BST_CUDA(cudaDeviceSynchronize());
  return check_status(h);
}

bst_status bst_get_state(bst_handle h, double *z, double *logp, double *grad, uint32_t *iter) {
  if (!h) return fail(BST_ERR_ARG, "bst_get_state: NULL handle");
  if (h->stage < 2) return fail(BST_ERR_STATE, "bst_get_state: no chain state");
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(cudaDeviceSynchronize());
  const int n = h->n, d = h->d, dp = h->dp;
  std::vector<double> t(static_cast<size_t>(n) * dp);
  if (z) {
    BST_TRY(download_real(h, t.data(), h->z, t.size()));
    for (int c = 0; c < n; ++c)
      for (int i = 0; i < d; ++i) z[static_cast<size_t>(c) * d + i] = t[static_cast<size_t>(c) * dp + i];
  }
  if (grad) {
    BST_TRY(download_real(h, t.data(), h->g, t.size()));
    for (int c = 0; c < n; ++c)
      for (int i = 0; i < d; ++i) grad[static_cast<size_t>(c) * d + i] = t[static_cast<size_t>(c) * dp + i];
  }
  if (logp) BST_TRY(download_real(h, logp, h->lp, n));
  if (iter) BST_CUDA(cudaMemcpy(iter, h->iter, n * 4, cudaMemcpyDeviceToHost));
  return BST_OK;
}

bst_status bst_set_state(bst_handle h, const double *z, const double *logp, const double *grad,
                         const uint32_t *iter) {
  if (!h || !z || !logp || !grad || !iter) return fail(BST_ERR_ARG, "bst_set_state: NULL argument");
  if (h->stage < 2) return fail(BST_ERR_STATE, "bst_set_state: call bst_init_chains first");
  const int n = h->n, d = h->d, dp = h->dp;
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(cudaDeviceSynchronize());
  std::vector<double> t(static_cast<size_t>(n) * dp, 0.0);
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < d; ++i) t[static_cast<size_t>(c) * dp + i] = z[static_cast<size_t>(c) * d + i];
  BST_TRY(upload_real(h, h->z, t.data(), t.size()));
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < d; ++i) t[static_cast<size_t>(c) * dp + i] = grad[static_cast<size_t>(c) * d + i];
  BST_TRY(upload_real(h, h->g, t.data(), t.size()));
  BST_TRY(upload_real(h, h->lp, logp, n));
  BST_CUDA(cudaMemcpy(h->iter, iter, n * 4, cudaMemcpyHostToDevice));
  h->grad_valid = true;
  h->state_stale = false;
  return BST_OK;
}

bst_status bst_get_whitening(bst_handle h, double *mu, double *L) {
  if (!h || !mu || !L) return fail(BST_ERR_ARG, "bst_get_whitening: NULL argument");
  if (h->mu.empty()) return fail(BST_ERR_STATE, "bst_get_whitening: no whitening set");
  std::memcpy(mu, h->mu.data(), h->d * 8);
  std::memcpy(L, h->L.data(), static_cast<size_t>(h->d) * h->d * 8);
  return BST_OK;
}

bst_status bst_get_counters(bst_handle h, int64_t *accepts, int64_t *evals, int64_t *divergences,
                            double *accept_stat) {
  if (!h) return fail(BST_ERR_ARG, "bst_get_counters: NULL handle");
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(cudaDeviceSynchronize());
  const size_t n = h->n;
  if (accepts) BST_CUDA(cudaMemcpy(accepts, h->accepts, n * 8, cudaMemcpyDeviceToHost));
  if (evals) BST_CUDA(cudaMemcpy(evals, h->evals, n * 8, cudaMemcpyDeviceToHost));
  if (divergences) BST_CUDA(cudaMemcpy(divergences, h->divs, n * 8, cudaMemcpyDeviceToHost));
  if (accept_stat) BST_CUDA(cudaMemcpy(accept_stat, h->acc_stat, n * 8, cudaMemcpyDeviceToHost));
  return BST_OK;
}

static bst_status train_setup(bst_handle h, int m) {
  if (h->lik != BST_LIK_EMULATOR || !h->P64) return fail(BST_ERR_STATE, "bst_train: no emulator set");
  if (m < 1 || m > 65536) return fail(BST_ERR_ARG, "bst_train: batch size must be in 1..65536");
  const size_t np = h->nparams;
  if (!h->P32) {
    BST_TRY(dalloc_t(h, &h->P32, np));
    BST_TRY(dalloc_t(h, &h->G32, np));
    BST_TRY(dalloc_t(h, &h->m1, np));
    BST_TRY(dalloc_t(h, &h->m2, np));
    BST_TRY(dalloc_t(h, &h->in_m32, h->d));
    BST_TRY(dalloc_t(h, &h->in_s32, h->d));
    if (h->p32_newer) h->p32_newer = false;
    BST_CUDA(launch_cast_f32(h->P64, h->P32, np, 0));
    BST_CUDA(launch_cast_f32(h->in_m64, h->in_m32, h->d, 0));
    BST_CUDA(launch_cast_f32(h->in_s64, h->in_s32, h->d, 0));
    h->adam_t = 0;
    h->train_cap = 0;
  }
  if (m > h->train_cap) {
    const size_t mm = m, w = h->width, D = h->depth;
    BST_TRY(dalloc_t(h, &h->tw.U, mm * h->d));
    BST_TRY(dalloc_t(h, &h->tw.H, D * mm * w));
    BST_TRY(dalloc_t(h, &h->tw.Dl, mm * w));
    BST_TRY(dalloc_t(h, &h->tw.Dn, mm * w));
    BST_TRY(dalloc_t(h, &h->tw.dout, mm));
    BST_TRY(dalloc_t(h, &h->tw.loss, 4));
    const size_t fmax = w > static_cast<size_t>(h->d) ? w : static_cast<size_t>(h->d);
    // split weight-gradient partials, or the slices of the batch-sliced column sums
    const size_t ws_gemm = static_cast<size_t>(kTrainSplits) * w * fmax;
    const size_t ws_sum = static_cast<size_t>(kWsumSlices) * w * static_cast<size_t>(h->d > 1 ? h->d : 1);
    BST_TRY(dalloc_t(h, &h->tw.ws, ws_gemm > ws_sum ? ws_gemm : ws_sum));
    h->tw.Hb = h->tw.HbT = h->tw.Db = h->tw.DbT = h->tw.Wb = h->tw.WbT = nullptr;
    h->tw.wsg = nullptr;
    if (tc_engine(h) && D >= 2) {
      // BF16 operands of the tensor-core training GEMMs
      const size_t nh = D - 1;
      BST_TRY(dalloc(h, reinterpret_cast<void **>(&h->tw.Hb), nh * mm * w * 2));
      BST_TRY(dalloc(h, reinterpret_cast<void **>(&h->tw.HbT), nh * mm * w * 2));
      BST_TRY(dalloc(h, reinterpret_cast<void **>(&h->tw.Db), 2 * mm * w * 2));
      BST_TRY(dalloc(h, reinterpret_cast<void **>(&h->tw.DbT), 2 * mm * w * 2));
      BST_TRY(dalloc(h, reinterpret_cast<void **>(&h->tw.Wb), nh * w * w * 2));
      BST_TRY(dalloc(h, reinterpret_cast<void **>(&h->tw.WbT), nh * w * w * 2));
      BST_TRY(dalloc_t(h, &h->tw.wsg, static_cast<size_t>(kTcTrainSplits) * w * w));
    }
    h->train_cap = m;
  }
  return BST_OK;
}

// The training gradient: on the tensor cores (BF16 operands, FP32 accumulation) for handles of a
// tensor-core precision whose shapes fit its tiles, else on the CUDA cores in FP32.
static bst_status train_grad_impl(bst_handle h, const float *X_dev, const float *chi2_dev, int m, float *grad_dev,
                                  cudaStream_t s) {
  const float om = static_cast<float>(h->out_m), os = static_cast<float>(h->out_s), of = static_cast<float>(h->out_floor);
  if (h->tw.Hb && tc_train_shape_ok(h->d, h->depth, h->width, m)) {
    BST_CUDA(launch_train_grad_tc(h->P32, h->in_m32, h->in_s32, om, os, h->out_log, of, h->d, h->depth, h->width, m,
                                  X_dev, chi2_dev, grad_dev, h->tw, h->status, s));
  } else {
    BST_CUDA(launch_train_grad(h->P32, h->in_m32, h->in_s32, om, os, h->out_log, of, h->d, h->depth, h->width, m, X_dev,
                               chi2_dev, grad_dev, h->tw, s));
  }
  return BST_OK;
}

bst_status bst_train_grad(bst_handle h, const float *X_dev, const float *chi2_dev, int m, float *grad_dev,
                          float *loss_dev, void *stream) {
  NvtxRange nvtx_("bst_train_grad");
  if (!h || !X_dev || !chi2_dev || !grad_dev) return fail(BST_ERR_ARG, "bst_train_grad: NULL argument");
  BST_CUDA(cudaSetDevice(h->device));
  BST_TRY(train_setup(h, m));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BST_TRY(train_grad_impl(h, X_dev, chi2_dev, m, grad_dev, s));
  if (loss_dev) BST_CUDA(cudaMemcpyAsync(loss_dev, h->tw.loss, 4, cudaMemcpyDeviceToDevice, s));
  return BST_OK;
}

bst_status bst_train_step(bst_handle h, const float *X_dev, const float *chi2_dev, int m, double lr, double beta1,
                          double beta2, double adam_eps, float *loss_dev, void *stream) {
  NvtxRange nvtx_("bst_train_step");
  if (!h || !X_dev || !chi2_dev) return fail(BST_ERR_ARG, "bst_train_step: NULL argument");
  if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(adam_eps > 0.0))
    return fail(BST_ERR_ARG, "bst_train_step: bad Adam hyper-parameters");
  BST_CUDA(cudaSetDevice(h->device));
  BST_TRY(train_setup(h, m));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BST_TRY(train_grad_impl(h, X_dev, chi2_dev, m, h->G32, s));
  if (loss_dev) BST_CUDA(cudaMemcpyAsync(loss_dev, h->tw.loss, 4, cudaMemcpyDeviceToDevice, s));
  h->adam_t += 1;
  BST_CUDA(launch_adam(h->P32, h->G32, h->m1, h->m2, h->nparams, h->adam_t, static_cast<float>(lr),
                       static_cast<float>(beta1), static_cast<float>(beta2), static_cast<float>(adam_eps), s));
  h->p32_newer = true;
  h->weights_dirty = true;
  h->state_stale = true;
  return BST_OK;
}

bst_status bst_train_apply(bst_handle h, const float *grad_dev, double lr, double beta1, double beta2,
                           double adam_eps, void *stream) {
  NvtxRange nvtx_("bst_train_apply");
  if (!h || !grad_dev) return fail(BST_ERR_ARG, "bst_train_apply: NULL argument");
  if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(adam_eps > 0.0))
    return fail(BST_ERR_ARG, "bst_train_apply: bad Adam hyper-parameters");
  BST_CUDA(cudaSetDevice(h->device));
  BST_TRY(train_setup(h, 1));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->adam_t += 1;
  BST_CUDA(launch_adam(h->P32, grad_dev, h->m1, h->m2, h->nparams, h->adam_t, static_cast<float>(lr),
                       static_cast<float>(beta1), static_cast<float>(beta2), static_cast<float>(adam_eps), s));
  h->p32_newer = true;
  h->weights_dirty = true;
  h->state_stale = true;
  return BST_OK;
}

// Eigenvalues of the symmetric d x d matrix A (row-major; destroyed) by cyclic Jacobi
// rotations (Golub & Van Loan, Matrix Computations, Sec. 8.5): each rotation zeroes one
// off-diagonal pair; sweeps repeat until the off-diagonal mass is negligible.
static void jacobi_eigenvalues(std::vector<double> &A, int d, std::vector<double> &ev) {
  auto at = [&](int r, int c) -> double & { return A[static_cast<size_t>(r) * d + c]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        tot += at(r, c) * at(r, c);
        if (r != c) off += at(r, c) * at(r, c);
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < d - 1; ++p)
      for (int q = p + 1; q < d; ++q) {
        const double apq = at(p, q);
        if (apq == 0.0) continue;
        const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < d; ++k) {  // columns p, q
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < d; ++k) {  // rows p, q
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
      }
  }
  ev.resize(d);
  for (int r = 0; r < d; ++r) ev[r] = at(r, r);
}

// R - 1 in two parts, so that ranks holding different chains can pool it: the device part
// gives every chain's mean and the pooled within-chain cross products
// S = sum_c sum_t (x_tc - m_c)(x_tc - m_c)^T (per-block partials summed in block order); the
// host part forms W = S / (M (n - 1)), B from the chain means, and the eigenvalue problem.
bst_status bst_r_minus_1_parts(bst_handle h, const void *samples_dev, int n_draws, double *chain_means,
                               double *S_out) {
  NvtxRange nvtx_("bst_r_minus_1_parts");
  if (!h || !samples_dev || !chain_means || !S_out) return fail(BST_ERR_ARG, "bst_r_minus_1_parts: NULL argument");
  if (n_draws < 2) return fail(BST_ERR_ARG, "bst_r_minus_1_parts: need at least 2 draws");
  BST_CUDA(cudaSetDevice(h->device));
  const int M = h->n, d = h->d, n = n_draws;
  const size_t md = static_cast<size_t>(M) * d;
  const int nb = rhat_blocks(M), np = d * (d + 1) / 2;
  if (!h->ess_mean) {
    BST_TRY(dalloc_t(h, &h->ess_mean, md));
    BST_TRY(dalloc_t(h, &h->ess_var, md));
    BST_TRY(dalloc_t(h, &h->ess_V, static_cast<size_t>(d) * 32));
  }
  if (!h->rhat_part) BST_TRY(dalloc_t(h, &h->rhat_part, static_cast<size_t>(nb) * np));
  // per-chain means, then the pooled within-chain cross products about them
  if (h->rs == 8) {
    BST_CUDA(launch_ess_moments_f64((const double *)samples_dev, n, M, d, h->ess_mean, h->ess_var, 0));
    BST_CUDA(launch_rhat_cross_f64((const double *)samples_dev, n, M, d, h->ess_mean, h->rhat_part, 0));
  } else {
    BST_CUDA(launch_ess_moments_f32((const float *)samples_dev, n, M, d, h->ess_mean, h->ess_var, 0));
    BST_CUDA(launch_rhat_cross_f32((const float *)samples_dev, n, M, d, h->ess_mean, h->rhat_part, 0));
  }
  std::vector<double> part(static_cast<size_t>(nb) * np);
  BST_CUDA(cudaMemcpy(chain_means, h->ess_mean, md * 8, cudaMemcpyDeviceToHost));
  BST_CUDA(cudaMemcpy(part.data(), h->rhat_part, part.size() * 8, cudaMemcpyDeviceToHost));
  for (int i = 0, p = 0; i < d; ++i)
    for (int j = i; j < d; ++j, ++p) {
      double sum = 0.0;
      for (int b = 0; b < nb; ++b) sum += part[static_cast<size_t>(b) * np + p];
      S_out[i * d + j] = S_out[j * d + i] = sum;
    }
  return BST_OK;
}

bst_status bst_r_minus_1_combine(int n_chains, int n_draws, int d, const double *chain_means, const double *S,
                                 double *out) {
  if (!chain_means || !S || !out) return fail(BST_ERR_ARG, "bst_r_minus_1_combine: NULL argument");
  if (n_chains < 2 || n_draws < 2 || d < 1 || d > kMaxD)
    return fail(BST_ERR_ARG, "bst_r_minus_1_combine: need n_chains >= 2, n_draws >= 2 and 1 <= d <= 32");
  const int M = n_chains, n = n_draws;
  const double *mean = chain_means;
  // W and B
  std::vector<double> W(static_cast<size_t>(d) * d), B(static_cast<size_t>(d) * d, 0.0), gm(d, 0.0);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) W[i * d + j] = S[i * d + j] / (static_cast<double>(M) * (n - 1));
  for (int c = 0; c < M; ++c)
    for (int i = 0; i < d; ++i) gm[i] += mean[static_cast<size_t>(c) * d + i];
  for (int i = 0; i < d; ++i) gm[i] /= M;
  for (int c = 0; c < M; ++c)
    for (int i = 0; i < d; ++i) {
      const double ei = mean[static_cast<size_t>(c) * d + i] - gm[i];
      for (int j = 0; j < d; ++j) B[i * d + j] += ei * (mean[static_cast<size_t>(c) * d + j] - gm[j]);
    }
  for (auto &v : B) v /= (M - 1);
  // scaling by D = diag(sqrt(B_ii)), then eig(W~^-1 B~) = eig(L^-1 B~ L^-T) with W~ = L L^T
  std::vector<double> dB(d);
  for (int i = 0; i < d; ++i) {
    dB[i] = std::sqrt(B[i * d + i]);
    if (!(dB[i] > 0.0)) {
      *out = NAN;
      return BST_OK;
    }
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      B[i * d + j] /= dB[i] * dB[j];
      W[i * d + j] /= dB[i] * dB[j];
    }
  std::vector<double> Lc(static_cast<size_t>(d) * d, 0.0);
  for (int j = 0; j < d; ++j) {
    double s = W[j * d + j];
    for (int k = 0; k < j; ++k) s -= Lc[j * d + k] * Lc[j * d + k];
    if (!(s > 0.0)) {
      *out = NAN;
      return BST_OK;
    }
    Lc[j * d + j] = std::sqrt(s);
    for (int i = j + 1; i < d; ++i) {
      double t = W[i * d + j];
      for (int k = 0; k < j; ++k) t -= Lc[i * d + k] * Lc[j * d + k];
      Lc[i * d + j] = t / Lc[j * d + j];
    }
  }
  auto lsolve = [&](const std::vector<double> &Rhs, std::vector<double> &X) {  // X = L^-1 Rhs
    X = Rhs;
    for (int col = 0; col < d; ++col)
      for (int i = 0; i < d; ++i) {
        double s = X[i * d + col];
        for (int k = 0; k < i; ++k) s -= Lc[i * d + k] * X[k * d + col];
        X[i * d + col] = s / Lc[i * d + i];
      }
  };
  std::vector<double> Y, Yt(static_cast<size_t>(d) * d), Cm;
  lsolve(B, Y);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Yt[i * d + j] = Y[j * d + i];
  lsolve(Yt, Cm);
  for (int i = 0; i < d; ++i)  // symmetric up to rounding: use the symmetric part
    for (int j = i + 1; j < d; ++j) Cm[i * d + j] = Cm[j * d + i] = 0.5 * (Cm[i * d + j] + Cm[j * d + i]);
  std::vector<double> ev;
  jacobi_eigenvalues(Cm, d, ev);
  double r = 0.0;
  for (double v : ev) r = std::fmax(r, std::fabs(v));
  *out = r;
  return BST_OK;
}

bst_status bst_r_minus_1(bst_handle h, const void *samples_dev, int n_draws, double *out) {
  if (!h || !samples_dev || !out) return fail(BST_ERR_ARG, "bst_r_minus_1: NULL argument");
  if (n_draws < 2 || h->n < 2) return fail(BST_ERR_ARG, "bst_r_minus_1: need at least 2 draws and 2 chains");
  std::vector<double> means(static_cast<size_t>(h->n) * h->d), S(static_cast<size_t>(h->d) * h->d);
  BST_TRY(bst_r_minus_1_parts(h, samples_dev, n_draws, means.data(), S.data()));
  return bst_r_minus_1_combine(h->n, n_draws, h->d, means.data(), S.data(), out);
}

// Quantiles of the pooled draws per dimension: order statistics by radix select on the
// device (qsel_hist_kernel), the key of each rank fixed 4 bits per pass from the most
// significant digit; then linear interpolation between ranks floor(h) and floor(h) + 1,
// h = (N - 1) q, in FP64.
constexpr int kMaxQuantiles = 8;
extern "C++" {
template <typename R, typename K>
static bst_status quantiles_impl(bst_ctx *h, const R *x, int n_draws, const double *q, int nq, double *out) {
  const int d = h->d, M = h->n;
  const size_t N = static_cast<size_t>(n_draws) * M;
  const int jpd = 2 * nq, nj = d * jpd;
  if (!h->qsel_prefix) {
    BST_TRY(dalloc(h, &h->qsel_prefix, static_cast<size_t>(kMaxD) * 2 * kMaxQuantiles * 8));
    BST_TRY(dalloc(h, reinterpret_cast<void **>(&h->qsel_hist), static_cast<size_t>(kMaxD) * 2 * kMaxQuantiles * 16 * 4));
  }
  std::vector<K> prefix(nj, K(0));
  std::vector<unsigned long long> rank(nj);
  std::vector<double> frac(static_cast<size_t>(d) * nq);
  for (int qd = 0; qd < d; ++qd)
    for (int k = 0; k < nq; ++k) {
      const double hpos = (static_cast<double>(N) - 1.0) * q[k];
      unsigned long long lo = static_cast<unsigned long long>(std::floor(hpos));
      if (lo > N - 1) lo = N - 1;
      const unsigned long long hi = lo + 1 < N ? lo + 1 : N - 1;
      rank[qd * jpd + 2 * k] = lo;
      rank[qd * jpd + 2 * k + 1] = hi;
      frac[static_cast<size_t>(qd) * nq + k] = hpos - static_cast<double>(lo);
    }
  std::vector<unsigned int> hist(static_cast<size_t>(nj) * 16);
  const int bits = 8 * static_cast<int>(sizeof(K));
  for (int shift = bits - 4; shift >= 0; shift -= 4) {
    BST_CUDA(cudaMemcpy(h->qsel_prefix, prefix.data(), nj * sizeof(K), cudaMemcpyHostToDevice));
    BST_CUDA(cudaMemset(h->qsel_hist, 0, static_cast<size_t>(nj) * 16 * 4));
    if (sizeof(R) == 8)
      BST_CUDA(launch_qsel_hist_f64(reinterpret_cast<const double *>(x), N * d, d, jpd,
                                    static_cast<const unsigned long long *>(h->qsel_prefix), shift, h->qsel_hist, 0));
    else
      BST_CUDA(launch_qsel_hist_f32(reinterpret_cast<const float *>(x), N * d, d, jpd,
                                    static_cast<const uint32_t *>(h->qsel_prefix), shift, h->qsel_hist, 0));
    BST_CUDA(cudaMemcpy(hist.data(), h->qsel_hist, hist.size() * 4, cudaMemcpyDeviceToHost));
    for (int j = 0; j < nj; ++j) {  // the digit whose bin holds the job's remaining rank
      unsigned long long below = 0;
      int b = 0;
      for (; b < 15; ++b) {
        const unsigned long long cnt = hist[static_cast<size_t>(j) * 16 + b];
        if (rank[j] < below + cnt) break;
        below += cnt;
      }
      rank[j] -= below;
      prefix[j] |= static_cast<K>(b) << shift;
    }
  }
  for (int qd = 0; qd < d; ++qd)
    for (int k = 0; k < nq; ++k) {
      double v[2];
      for (int e = 0; e < 2; ++e) {  // key -> value
        const K key = prefix[qd * jpd + 2 * k + e];
        const K top = K(1) << (8 * sizeof(K) - 1);
        const K b = (key & top) ? (key & ~top) : ~key;
        if (sizeof(K) == 8) {
          double dv;
          std::memcpy(&dv, &b, 8);
          v[e] = dv;
        } else {
          float fv;
          std::memcpy(&fv, &b, 4);
          v[e] = fv;
        }
      }
      out[static_cast<size_t>(qd) * nq + k] = v[0] + frac[static_cast<size_t>(qd) * nq + k] * (v[1] - v[0]);
    }
  return BST_OK;
}
}  // extern "C++"

bst_status bst_quantiles(bst_handle h, const void *samples_dev, int n_draws, const double *q, int nq, double *out) {
  NvtxRange nvtx_("bst_quantiles");
  if (!h || !samples_dev || !q || !out) return fail(BST_ERR_ARG, "bst_quantiles: NULL argument");
  if (n_draws < 1 || nq < 1 || nq > kMaxQuantiles) return fail(BST_ERR_ARG, "bst_quantiles: need n_draws >= 1 and 1 <= nq <= 8");
  for (int k = 0; k < nq; ++k)
    if (!(q[k] >= 0.0 && q[k] <= 1.0)) return fail(BST_ERR_ARG, "bst_quantiles: levels must lie in [0, 1]");
  BST_CUDA(cudaSetDevice(h->device));
  if (h->rs == 8) return quantiles_impl<double, unsigned long long>(h, static_cast<const double *>(samples_dev), n_draws, q, nq, out);
  return quantiles_impl<float, uint32_t>(h, static_cast<const float *>(samples_dev), n_draws, q, nq, out);
}

bst_status bst_credible_metric(bst_handle h, const void *samples_dev, int n_draws, double alpha, const double *true_lo,
                               const double *true_hi, double *out) {
  if (!h || !samples_dev || !true_lo || !true_hi || !out) return fail(BST_ERR_ARG, "bst_credible_metric: NULL argument");
  if (!(alpha > 0.0 && alpha < 1.0)) return fail(BST_ERR_ARG, "bst_credible_metric: alpha must lie in (0, 1)");
  const int d = h->d;
  for (int i = 0; i < d; ++i)
    if (!(true_hi[i] > true_lo[i])) return fail(BST_ERR_ARG, "bst_credible_metric: need true_hi > true_lo");
  const double q[2] = {(1.0 - alpha) / 2.0, (1.0 + alpha) / 2.0};
  std::vector<double> lim(static_cast<size_t>(d) * 2);
  BST_TRY(bst_quantiles(h, samples_dev, n_draws, q, 2, lim.data()));
  for (int i = 0; i < d; ++i)
    out[i] = (std::fabs(lim[2 * i + 1] - true_hi[i]) + std::fabs(lim[2 * i] - true_lo[i])) / (true_hi[i] - true_lo[i]);
  return BST_OK;
}

// Sliced Wasserstein distance: directions, then per chunk of directions the projections of the
// draws and the reference set side by side (segment 2k: draws, 2k + 1: reference), a
// segmented sort and the per-direction 1-D distances; the mean over directions on the host.
constexpr long long kSwdChunkElems = 1LL << 27;  // projected values per chunk (1 GiB in FP64)
extern "C++" {
namespace {
struct DevScratch {  // call-local device buffer, freed on every return path
  void *p = nullptr;
  DevScratch() = default;
  DevScratch(const DevScratch &) = delete;
  DevScratch &operator=(const DevScratch &) = delete;
  ~DevScratch() {
    if (p) cudaFree(p);
  }
  template <typename T>
  T *as() const {
    return static_cast<T *>(p);
  }
};
}  // namespace
}  // extern "C++"

bst_status bst_sliced_wasserstein(bst_handle h, const void *samples_dev, int n_draws, const void *ref_dev,
                                  long long n_ref, int n_proj, unsigned long long seed, double *out) {
  NvtxRange nvtx_("bst_sliced_wasserstein");
  if (!h || !samples_dev || !ref_dev || !out) return fail(BST_ERR_ARG, "bst_sliced_wasserstein: NULL argument");
  if (n_draws < 1 || n_ref < 1 || n_proj < 1)
    return fail(BST_ERR_ARG, "bst_sliced_wasserstein: need n_draws, n_ref and n_proj >= 1");
  const long long n = static_cast<long long>(n_draws) * h->n, m = n_ref, nm = n + m;
  if (nm > kSwdChunkElems) return fail(BST_ERR_ARG, "bst_sliced_wasserstein: at most 2^27 draws and reference points");
  BST_CUDA(cudaSetDevice(h->device));
  const int d = h->d;
  const int kc = static_cast<int>(std::min<long long>(n_proj, kSwdChunkElems / nm));
  DevScratch U, proj, sorted, offs, w1, temp;
  BST_CUDA(cudaMalloc(&U.p, static_cast<size_t>(n_proj) * d * 8));
  BST_CUDA(cudaMalloc(&proj.p, static_cast<size_t>(kc) * nm * 8));
  BST_CUDA(cudaMalloc(&sorted.p, static_cast<size_t>(kc) * nm * 8));
  BST_CUDA(cudaMalloc(&offs.p, (2 * static_cast<size_t>(kc) + 1) * sizeof(int)));
  BST_CUDA(cudaMalloc(&w1.p, static_cast<size_t>(n_proj) * 8));
  std::vector<int> o(2 * static_cast<size_t>(kc) + 1);
  for (int k = 0; k < kc; ++k) {
    o[2 * k] = static_cast<int>(k * nm);
    o[2 * k + 1] = static_cast<int>(k * nm + n);
  }
  o[2 * kc] = static_cast<int>(kc * nm);
  BST_CUDA(cudaMemcpy(offs.p, o.data(), o.size() * sizeof(int), cudaMemcpyHostToDevice));
  size_t temp_bytes = 0;
  BST_CUDA(swd_sort_segments(nullptr, temp_bytes, proj.as<double>(), sorted.as<double>(), static_cast<int>(kc * nm),
                             2 * kc, offs.as<int>(), 0));
  BST_CUDA(cudaMalloc(&temp.p, temp_bytes > 0 ? temp_bytes : 1));
  BST_CUDA(launch_swd_directions(seed, n_proj, d, U.as<double>(), 0));
  for (int k0 = 0; k0 < n_proj; k0 += kc) {
    const int nk = std::min(kc, n_proj - k0);
    const double *Uk = U.as<double>() + static_cast<size_t>(k0) * d;
    if (h->rs == 8) {
      BST_CUDA(launch_swd_project_f64(static_cast<const double *>(samples_dev), n, d, Uk, nk, proj.as<double>(), nm, 0));
      BST_CUDA(launch_swd_project_f64(static_cast<const double *>(ref_dev), m, d, Uk, nk, proj.as<double>() + n, nm, 0));
    } else {
      BST_CUDA(launch_swd_project_f32(static_cast<const float *>(samples_dev), n, d, Uk, nk, proj.as<double>(), nm, 0));
      BST_CUDA(launch_swd_project_f32(static_cast<const float *>(ref_dev), m, d, Uk, nk, proj.as<double>() + n, nm, 0));
    }
    size_t tb = temp_bytes;
    BST_CUDA(swd_sort_segments(temp.p, tb, proj.as<double>(), sorted.as<double>(), static_cast<int>(nk * nm), 2 * nk,
                               offs.as<int>(), 0));
    BST_CUDA(launch_swd_w1(sorted.as<double>(), n, m, nk, w1.as<double>() + k0, 0));
  }
  std::vector<double> w(n_proj);
  BST_CUDA(cudaMemcpy(w.data(), w1.p, static_cast<size_t>(n_proj) * 8, cudaMemcpyDeviceToHost));
  double sum = 0.0;
  for (double v : w) sum += v;
  *out = sum / n_proj;
  return BST_OK;
}

bst_status bst_ess(bst_handle h, const void *samples_dev, int n_draws, double *ess_out) {
  NvtxRange nvtx_("bst_ess");
  if (!h || !samples_dev || !ess_out) return fail(BST_ERR_ARG, "bst_ess: NULL argument");
  if (n_draws < 4) return fail(BST_ERR_ARG, "bst_ess: need at least 4 draws");
  BST_CUDA(cudaSetDevice(h->device));
  const int M = h->n, d = h->d, n = n_draws;
  const size_t md = static_cast<size_t>(M) * d;
  if (!h->ess_mean) {
    BST_TRY(dalloc_t(h, &h->ess_mean, md));
    BST_TRY(dalloc_t(h, &h->ess_var, md));
    BST_TRY(dalloc_t(h, &h->ess_V, static_cast<size_t>(d) * 32));
  }
  if (h->rs == 8) BST_CUDA(launch_ess_moments_f64((const double *)samples_dev, n, M, d, h->ess_mean, h->ess_var, 0));
  else BST_CUDA(launch_ess_moments_f32((const float *)samples_dev, n, M, d, h->ess_mean, h->ess_var, 0));
  std::vector<double> mean(md), var(md);
  BST_CUDA(cudaMemcpy(mean.data(), h->ess_mean, md * 8, cudaMemcpyDeviceToHost));
  BST_CUDA(cudaMemcpy(var.data(), h->ess_var, md * 8, cudaMemcpyDeviceToHost));
  std::vector<double> var_plus(d), sumP(d, 0.0), prevP(d, INFINITY);
  std::vector<int> active(d, 1);
  for (int q = 0; q < d; ++q) {
    double gm = 0.0, Wv = 0.0, Bv = 0.0;
    for (int c = 0; c < M; ++c) gm += mean[static_cast<size_t>(c) * d + q];
    gm /= M;
    for (int c = 0; c < M; ++c) {
      Wv += var[static_cast<size_t>(c) * d + q];
      const double e = mean[static_cast<size_t>(c) * d + q] - gm;
      Bv += e * e;
    }
    Wv /= M;
    const double Bn = (M > 1) ? Bv / (M - 1) : 0.0;
    var_plus[q] = (n - 1.0) / n * Wv + Bn;
  }
  std::vector<double> V(static_cast<size_t>(d) * 32);
  int n_active = d;
  for (int t0 = 0; t0 + 1 < n && n_active > 0; t0 += 32) {
    const int nt = (n - t0) < 32 ? (n - t0) : 32;
    BST_CUDA(cudaMemset(h->ess_V, 0, static_cast<size_t>(d) * 32 * 8));
    if (h->rs == 8) BST_CUDA(launch_ess_variogram_f64((const double *)samples_dev, n, M, d, t0, nt, h->ess_V, 0));
    else BST_CUDA(launch_ess_variogram_f32((const float *)samples_dev, n, M, d, t0, nt, h->ess_V, 0));
    BST_CUDA(cudaMemcpy(V.data(), h->ess_V, static_cast<size_t>(d) * 32 * 8, cudaMemcpyDeviceToHost));
    for (int q = 0; q < d; ++q) {
      if (!active[q]) continue;
      for (int k = 0; k + 1 < nt; k += 2) {
        const int t = t0 + k;
        if (t + 1 >= n) {
          active[q] = 0;
          break;
        }
        const double r0 = 1.0 - V[q * nt + k] / (static_cast<double>(M) * (n - t)) / (2.0 * var_plus[q]);
        const double r1 = 1.0 - V[q * nt + k + 1] / (static_cast<double>(M) * (n - t - 1)) / (2.0 * var_plus[q]);
        double P = r0 + r1;
        if (!(P > 0.0)) {
          active[q] = 0;
          break;
        }
        if (P > prevP[q]) P = prevP[q];
        sumP[q] += P;
        prevP[q] = P;
      }
      if (nt % 2 && active[q] && t0 + nt >= n) active[q] = 0;
      if (!active[q]) --n_active;
    }
  }
  for (int q = 0; q < d; ++q) ess_out[q] = static_cast<double>(M) * n / (-1.0 + 2.0 * sumP[q]);
  return BST_OK;
}

bst_status bst_sync(bst_handle h, void *stream) {
  if (!h) return fail(BST_ERR_ARG, "bst_sync: NULL handle");
  BST_CUDA(cudaSetDevice(h->device));
  BST_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  return check_status(h);
}

}  // extern "C"

// ============================================================================ allocation-free gradient
// bst_grad_loglike_noalloc keeps the emulator activations that its adjoint needs in one
// fixed device array instead of library-allocated memory, so the call itself never allocates.
namespace {
constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB, held by every GPU that loads the library
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on `dev` (the current device), looked up once per device.
bst_status static_scratch_address(int dev, void **out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (dev < 0 || dev >= kMaxDevices) return fail(BST_ERR_ARG, "bst_grad_loglike_noalloc: device ordinal out of range");
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(BST_ERR_CUDA, std::string("bst_grad_loglike_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return BST_OK;
}
}  // namespace

extern "C" bst_status bst_grad_loglike_noalloc(bst_handle h, const void *theta_dev, int m, void *logl_dev,
                                               void *grad_dev, void *stream) {
  NvtxRange nvtx_("bst_grad_loglike_noalloc");
  if (!h || (m > 0 && (!theta_dev || !logl_dev || !grad_dev)))
    return fail(BST_ERR_ARG, "bst_grad_loglike_noalloc: NULL argument");
  if (h->stage < 1) return fail(BST_ERR_STATE, "bst_grad_loglike_noalloc: set a likelihood first");
  if (m < 0) return fail(BST_ERR_ARG, "bst_grad_loglike_noalloc: m must be >= 0");
  if (m == 0) return BST_OK;
  size_t row_bytes = 0;  // activation bytes the adjoint keeps per evaluated point
  if (h->lik == BST_LIK_EMULATOR) {
    const size_t el = (tc_engine(h)) ? 2 : h->rs;
    row_bytes = static_cast<size_t>(h->depth > 1 ? h->depth - 1 : 1) * h->width * el;
    const size_t max_rows = kStaticScratchBytes / row_bytes;
    if (static_cast<size_t>(m) > max_rows)
      return fail(BST_ERR_ARG, "bst_grad_loglike_noalloc: m = " + std::to_string(m) + " exceeds the " +
                                   std::to_string(max_rows) + " points the 16 MiB static scratch holds for this emulator");
  }
  BST_CUDA(cudaSetDevice(h->device));
  void *scratch = nullptr;
  BST_TRY(static_scratch_address(h->device, &scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BST_TRY(prepare(h, s));
  if (h->precision == BST_FP64) {
    StepArgs<double> a = make_args<double>(h, kModeLoglike, 0.0, 0, 1, nullptr);
    a.n_rows = m;
    a.need_grad = 1;
    a.st.ze = (double *)theta_dev;
    a.st.ze_ld = h->d;
    a.st.lle = (double *)logl_dev;
    a.st.gle = (double *)grad_dev;
    a.st.gle_ld = h->d;
    if (h->lik == BST_LIK_EMULATOR) {
      EmuWeights<double> w = emu_weights<double>(h, 1);
      w.scratch = static_cast<double *>(scratch);
      BST_CUDA(launch_emu_simt_f64(a, w, s));
    } else {
      BST_CUDA(launch_ana_simt_f64(a, ana_weights<double>(h, 1), s));
    }
  } else {
    StepArgs<float> a = make_args<float>(h, kModeLoglike, 0.0, 0, 1, nullptr);
    a.n_rows = m;
    a.need_grad = 1;
    a.st.ze = (float *)theta_dev;
    a.st.ze_ld = h->d;
    a.st.lle = (float *)logl_dev;
    a.st.gle = (float *)grad_dev;
    a.st.gle_ld = h->d;
    if (h->lik == BST_LIK_ANALYTIC) {
      BST_CUDA(launch_ana_simt_f32(a, ana_weights<float>(h, 1), s));
    } else if (tc_engine(h)) {
      Tc2Weights w = tc2_weights(h, 1, m);
      w.scratch = static_cast<__nv_bfloat16 *>(scratch);
      // exchange images after the activations if they fit, else the shared->shared exchange
      w.xchg = nullptr;
      w.xchg_bytes = 0;
      if (scratch_bytes_for(h, static_cast<size_t>(m)) <= kStaticScratchBytes) {
        w.xchg = static_cast<uint8_t *>(scratch) + act_bytes_for(h, static_cast<size_t>(m));
        w.xchg_bytes = kStaticScratchBytes - act_bytes_for(h, static_cast<size_t>(m));
      }
      BST_CUDA(launch_emu_tc2(a, w, s));
    } else {
      EmuWeights<float> w = emu_weights<float>(h, 1);
      w.scratch = static_cast<float *>(scratch);
      BST_CUDA(launch_emu_simt_f32(a, w, s));
    }
  }
  return BST_OK;
}
