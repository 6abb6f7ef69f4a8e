// launch.h -- host-side launch wrappers between the C-ABI runtime (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "engine_simt.cuh"
#include "engine_tc.cuh"
#include "engine_tc2.cuh"

namespace bst {

// Chain-tile step / evaluation launches (k_simt.cu, k_tc2.cu).
cudaError_t launch_emu_simt_f32(const StepArgs<float> &a, const EmuWeights<float> &w, cudaStream_t s);
cudaError_t launch_emu_simt_f64(const StepArgs<double> &a, const EmuWeights<double> &w, cudaStream_t s);
cudaError_t launch_ana_simt_f32(const StepArgs<float> &a, const AnaWeights<float> &w, cudaStream_t s);
cudaError_t launch_ana_simt_f64(const StepArgs<double> &a, const AnaWeights<double> &w, cudaStream_t s);
int simt_rows_per_tile(int precision, int width, int lik_kind);
// cluster tcgen05 kernel: cs in {1, 2, 4}
cudaError_t launch_emu_tc2(const StepArgs<float> &a, const Tc2Weights &w, cudaStream_t s);
int tc2_stages(int width, int cs, int depth);
int tc2_cluster_size(int n_rows, int width, int depth);

// Weight preparation (k_aux.cu).
// Fold whitening / standardisation into layer 1 (FP64 out): z-space (mode 0) or x-space (mode 1).
cudaError_t launch_fold_layer1(const double *P, const double *in_m, const double *in_s, const double *mu,
                               const double *L, int d, int dp, int w, int mode, double *W1f, double *b1f,
                               cudaStream_t s);
// Emulator SIMT weights in working precision from the FP64 master + fold.
cudaError_t launch_pack_simt_f32(const double *P, const double *W1f, const double *b1f, int d, int dp, int D,
                                 int w, float *W1T, float *W1, float *b1, float *WT, float *W, float *b, float *wo,
                                 cudaStream_t s);
cudaError_t launch_pack_simt_f64(const double *P, const double *W1f, const double *b1f, int d, int dp, int D,
                                 int w, double *W1T, double *W1, double *b1, double *WT, double *W, double *b,
                                 double *wo, cudaStream_t s);
// BF16 tensor-core tiles (pre-swizzled): layer-1 split tiles, hidden fwd + adjoint tiles,
// input-gradient split tiles; FP32 biases.
cudaError_t launch_pack_tc2_l1(const double *W1f, int dp, int kb1, int rank, int NS, int TR, int f16, uint8_t *out,
                               cudaStream_t s);
cudaError_t launch_pack_tc2_hidden(const double *P, int d, int D, int w, int rank, int NS, int TR, int f16,
                                   uint8_t *out, cudaStream_t s);
cudaError_t launch_pack_tc_g1(const double *W1f, int dp, int w, int f16, uint8_t *out, cudaStream_t s);
cudaError_t launch_cast_f32(const double *src, float *dst, size_t n, cudaStream_t s);
// Initial whitened positions z0 = L^-1 (theta0 - mu) (FP64 forward substitution; z in FP64 or FP32).
cudaError_t launch_init_z(bool f64, const double *theta, const double *mu, const double *L, int n, int d, int dp,
                          void *z, cudaStream_t s);
cudaError_t launch_cast_f64(const double *src, double *dst, size_t n, cudaStream_t s);
cudaError_t launch_cast_f32_to_f64(const float *src, double *dst, size_t n, cudaStream_t s);
// Analytic fold: Bf = B L_c, cf = B mu_c + c, Nf = N L_n, dataf = data - N mu_n (mode 0) or
// the x-space embedding (mode 1); outputs in working precision via a FP64 staging buffer.
cudaError_t launch_fold_analytic(const double *A, const double *B, const double *c, const double *N,
                                 const double *data, const double *mu, const double *L, int d, int dp, int d_c,
                                 int H, int n_data, int mode, double *Bf, double *cf, double *AT, double *NfT,
                                 double *dataf, cudaStream_t s);

// Covariance adaptation (k_aux.cu): merge n_tiles FP64 Welford tile records, factorise.
// out: mu[d], L[d*d], info[0] = n, info[1] = jitter used (or -1 if not PD), info[2] = status.
cudaError_t launch_adapt_finalize(const double *wf, int n_tiles, int stride, int d, double jitter0, double *mu,
                                  double *L, double *info, cudaStream_t s);
cudaError_t launch_welford_clear(double *wf, int n_tiles, int stride, cudaStream_t s);
// out = [n, mean[d], M2[d][d]] of all records merged; merge of such a triple into one record.
cudaError_t launch_welford_stats(const double *wf, int n_tiles, int stride, int d, double *out, cudaStream_t s);
cudaError_t launch_welford_merge(double *W, int d, const double *in, cudaStream_t s);
cudaError_t launch_welford_add_f32(const float *x, int m, int d, double *wf, int stride, cudaStream_t s);
cudaError_t launch_welford_add_f64(const double *x, int m, int d, double *wf, int stride, cudaStream_t s);
// z_new = L_new^-1 (mu_old + L_old z_old - mu_new), FP64 arithmetic.
cudaError_t launch_remap_f32(float *z, int n, int d, int dp, const double *mu_o, const double *L_o,
                             const double *mu_n, const double *L_n, cudaStream_t s);
cudaError_t launch_remap_f64(double *z, int n, int d, int dp, const double *mu_o, const double *L_o,
                             const double *mu_n, const double *L_n, cudaStream_t s);

// ESS (k_aux.cu): per-(chain, dim) means and variances, then variograms per lag block.
cudaError_t launch_ess_moments_f32(const float *x, int n, int M, int d, double *mean, double *var, cudaStream_t s);
cudaError_t launch_rhat_cross_f32(const float *x, int n, int M, int d, const double *mean, double *partial,
                                  cudaStream_t s);
cudaError_t launch_rhat_cross_f64(const double *x, int n, int M, int d, const double *mean, double *partial,
                                  cudaStream_t s);
int rhat_blocks(int M);
cudaError_t launch_init_positions(int strategy, uint64_t seed, int n, int d, const double *par, double *theta,
                                  cudaStream_t s);
cudaError_t launch_qsel_hist_f32(const float *x, size_t n_elems, int d, int jpd, const uint32_t *prefix, int shift,
                                 unsigned int *hist, cudaStream_t s);
cudaError_t launch_qsel_hist_f64(const double *x, size_t n_elems, int d, int jpd, const unsigned long long *prefix,
                                 int shift, unsigned int *hist, cudaStream_t s);
cudaError_t launch_ess_moments_f64(const double *x, int n, int M, int d, double *mean, double *var, cudaStream_t s);

// Sliced Wasserstein distance (k_swd.cu), FP64: directions U[n_proj][d]; projections
// out[kk * ld + i] = X_i . U_kk; per-segment sorting (offsets[n_segments + 1], temp_bytes
// queried with temp = nullptr); per-direction 1-D W1 of the sorted pair (a: n values, then b: m).
cudaError_t launch_swd_directions(uint64_t seed, int n_proj, int d, double *U, cudaStream_t s);
cudaError_t launch_swd_project_f32(const float *X, long long n_rows, int d, const double *U, int nk, double *out,
                                   long long ld, cudaStream_t s);
cudaError_t launch_swd_project_f64(const double *X, long long n_rows, int d, const double *U, int nk, double *out,
                                   long long ld, cudaStream_t s);
cudaError_t swd_sort_segments(void *temp, size_t &temp_bytes, const double *in, double *out, int n_items,
                              int n_segments, const int *offsets, cudaStream_t s);
cudaError_t launch_swd_w1(const double *sorted, long long n, long long m, int nk, double *w1, cudaStream_t s);
cudaError_t launch_ess_variogram_f32(const float *x, int n, int M, int d, int t0, int nt, double *V, cudaStream_t s);
cudaError_t launch_ess_variogram_f64(const double *x, int n, int M, int d, int t0, int nt, double *V, cudaStream_t s);

// Training (k_aux.cu), FP32.
struct TrainWork {
  float *U;     // [m][d] standardised inputs
  float *H;     // [D][m][w] activations
  float *Dl;    // [m][w] adjoint buffer
  float *Dn;    // [m][w] adjoint buffer
  float *dout;  // [m]
  float *loss;  // [1]
  float *ws;    // [kTrainSplits][w][w] partial weight gradients (split over the batch), or the
                //   [kWsumSlices][w][d] slices of the batch-sliced column sums
  // tensor-core training (BF16 operands): null when the handle trains on the CUDA cores
  __nv_bfloat16 *Hb, *HbT;   // [D-1][m][w] / [D-1][w][m] hidden activations h_1..h_{D-1}
  __nv_bfloat16 *Db, *DbT;   // [2][m][w] / [2][w][m] adjoints (double-buffered)
  __nv_bfloat16 *Wb, *WbT;   // [D-1][w][w] W_l and W_l^T, l = 2..D
  float *wsg;                // [kTcTrainSplits][w][w] partial weight gradients of the tensor-core GEMM
};
constexpr int kTcTrainSplits = 8;

// BF16 tcgen05 GEMM C[M][N] = A[M][K] . B[N][K]^T (k_train_tc.cu), K-major BF16 operands, FP32
// accumulation; fused epilogues (C FP32, optional BF16 copies Cb [M][N] and CbT [N][M]):
enum { kTcEpiStore = 0, kTcEpiTanh = 1, kTcEpiDtanh = 2 };
struct TcGemmArgs {
  int M, N, K;
  int k_chunk;          // set by the launcher: K / splits (grid.z slices, C + z M N each)
  int epi;              // kTcEpiStore: C = acc; kTcEpiTanh: tanh(acc + bias); kTcEpiDtanh: acc (1 - H^2)
  float *C;
  const float *bias;    // [N]
  const float *H;       // [M][N]
  __nv_bfloat16 *Cb;
  __nv_bfloat16 *CbT;
  int *status;
};
bool tc_gemm_shape_ok(int M, int N, int K, int splits);
cudaError_t launch_tc_gemm(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int splits, const TcGemmArgs &args,
                           cudaStream_t s);
cudaError_t launch_cast_transpose_bf16(const float *X, int rows, int cols, __nv_bfloat16 *Xb, __nv_bfloat16 *XbT,
                                       cudaStream_t s);
bool tc_train_shape_ok(int d, int D, int w, int m);
cudaError_t launch_train_grad_tc(const float *P, const float *in_m, const float *in_s, float out_m, float out_s,
                                 int out_log, float out_floor, int d, int D, int w, int m, const float *X,
                                 const float *chi2, float *G, TrainWork &tw, int *status, cudaStream_t s);
constexpr int kTrainSplits = 4;
// Batch-sliced column sums of the training gradient (bias and head gradients, the fan-in-d layer):
// at most kWsumSlices slices of the batch, at most kWsumMaxU weights per row.
constexpr int kWsumSlices = 32;
constexpr int kWsumMaxU = 32;
cudaError_t launch_train_grad(const float *P, const float *in_m, const float *in_s, float out_m, float out_s,
                              int out_log, float out_floor, int d, int D, int w, int m, const float *X,
                              const float *chi2, float *G, TrainWork &tw, cudaStream_t s);
cudaError_t launch_adam(float *P, const float *G, float *m1, float *m2, size_t n, int t, float lr, float b1,
                        float b2, float eps, cudaStream_t s);
cudaError_t launch_zero(void *p, size_t bytes, cudaStream_t s);

}  // namespace bst
