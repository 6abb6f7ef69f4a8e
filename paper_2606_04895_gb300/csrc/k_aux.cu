// k_aux.cu -- weight preparation, covariance adaptation, ESS and training kernels.
#include <cuda_bf16.h>

#include "launch.h"

namespace bst {

namespace {
inline int blocks_for(size_t n, int t) { return static_cast<int>((n + t - 1) / t); }

// Offsets of the flat emulator parameter vector:
// W1[w][d] b1[w] (W_l[w][w] b_l[w])_{l=2..D} wo[w] bo.
__host__ __device__ inline size_t off_W(int l, int d, int w) {
  return l == 1 ? 0 : static_cast<size_t>(d) * w + w + static_cast<size_t>(l - 2) * (static_cast<size_t>(w) * w + w);
}
__host__ __device__ inline size_t off_b(int l, int d, int w) {
  return off_W(l, d, w) + static_cast<size_t>(w) * (l == 1 ? d : w);
}
__host__ __device__ inline size_t off_wo(int d, int D, int w) { return off_W(D + 1, d, w); }
}  // namespace

// ------------------------------------------------------------------------------------------
// Layer-1 fold.  mode 0 (sampling, z-space): W1f = W1 diag(1/s) L, b1f = b1 + W1 (mu - m)/s.
//              mode 1 (loglike, x-space):   W1f = W1 diag(1/s),   b1f = b1 - W1 m/s.
__global__ void fold_layer1_kernel(const double *P, const double *in_m, const double *in_s, const double *mu,
                                   const double *L, int d, int dp, int w, int mode, double *W1f, double *b1f) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= w) return;
  const double *W1 = P + static_cast<size_t>(k) * d;
  double bb = P[off_b(1, d, w) + k];
  for (int i = 0; i < d; ++i) {
    const double wi = W1[i] / in_s[i];
    bb += (mode == 0) ? wi * (mu[i] - in_m[i]) : -wi * in_m[i];
  }
  b1f[k] = bb;
  for (int j = 0; j < dp; ++j) {
    double s = 0.0;
    if (j < d) {
      if (mode == 0)
        for (int i = j; i < d; ++i) s += W1[i] / in_s[i] * L[i * d + j];
      else
        s = W1[j] / in_s[j];
    }
    W1f[static_cast<size_t>(k) * dp + j] = s;
  }
}

cudaError_t launch_fold_layer1(const double *P, const double *in_m, const double *in_s, const double *mu,
                               const double *L, int d, int dp, int w, int mode, double *W1f, double *b1f,
                               cudaStream_t s) {
  fold_layer1_kernel<<<blocks_for(w, 128), 128, 0, s>>>(P, in_m, in_s, mu, L, d, dp, w, mode, W1f, b1f);
  return cudaGetLastError();
}

template <typename R>
__global__ void pack_simt_kernel(const double *P, const double *W1f, const double *b1f, int d, int dp, int D, int w,
                                 R *W1T, R *W1, R *b1, R *WT, R *W, R *b, R *wo) {
  const size_t tid = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  const size_t n1 = static_cast<size_t>(w) * dp;
  const size_t nh = static_cast<size_t>(D - 1) * w * w;
  if (tid < n1) {
    const int k = static_cast<int>(tid / dp), j = static_cast<int>(tid % dp);
    W1[tid] = static_cast<R>(W1f[tid]);
    W1T[static_cast<size_t>(j) * w + k] = static_cast<R>(W1f[tid]);
  }
  if (tid < static_cast<size_t>(w)) {
    b1[tid] = static_cast<R>(b1f[tid]);
    wo[tid] = static_cast<R>(P[off_wo(d, D, w) + tid]);
  }
  if (tid < nh) {
    const int l = static_cast<int>(tid / (static_cast<size_t>(w) * w)) + 2;
    const size_t e = tid % (static_cast<size_t>(w) * w);
    const int r = static_cast<int>(e / w), c = static_cast<int>(e % w);
    const double v = P[off_W(l, d, w) + e];
    W[tid] = static_cast<R>(v);
    WT[static_cast<size_t>(l - 2) * w * w + static_cast<size_t>(c) * w + r] = static_cast<R>(v);
  }
  if (tid < static_cast<size_t>(D - 1) * w) {
    const int l = static_cast<int>(tid / w) + 2, k = static_cast<int>(tid % w);
    b[tid] = static_cast<R>(P[off_b(l, d, w) + k]);
  }
}

template <typename R>
static cudaError_t pack_simt(const double *P, const double *W1f, const double *b1f, int d, int dp, int D, int w,
                             R *W1T, R *W1, R *b1, R *WT, R *W, R *b, R *wo, cudaStream_t s) {
  size_t n = static_cast<size_t>(w) * dp;
  n = n > static_cast<size_t>(D - 1) * w * w ? n : static_cast<size_t>(D - 1) * w * w;
  n = n > static_cast<size_t>(w) ? n : static_cast<size_t>(w);
  pack_simt_kernel<R><<<blocks_for(n, 256), 256, 0, s>>>(P, W1f, b1f, d, dp, D, w, W1T, W1, b1, WT, W, b, wo);
  return cudaGetLastError();
}
cudaError_t launch_pack_simt_f32(const double *P, const double *W1f, const double *b1f, int d, int dp, int D, int w,
                                 float *W1T, float *W1, float *b1, float *WT, float *W, float *b, float *wo,
                                 cudaStream_t s) {
  return pack_simt<float>(P, W1f, b1f, d, dp, D, w, W1T, W1, b1, WT, W, b, wo, s);
}
cudaError_t launch_pack_simt_f64(const double *P, const double *W1f, const double *b1f, int d, int dp, int D, int w,
                                 double *W1T, double *W1, double *b1, double *WT, double *W, double *b, double *wo,
                                 cudaStream_t s) {
  return pack_simt<double>(P, W1f, b1f, d, dp, D, w, W1T, W1, b1, WT, W, b, wo, s);
}

// ------------------------------------------------------------------------------------------
// BF16 tile packing.  A tile is rows x 64 BF16 (128 bytes per row) in the 128-byte-swizzled
// K-major layout the tcgen05 shared-memory descriptors expect: the 16-byte chunk j of row r sits
// at r * 128 + ((j ^ (r % 8)) * 16).  Each thread writes one 16-byte chunk.
__device__ __forceinline__ void put_chunk(uint8_t *tile, int r, int j, const float v[8], int f16) {
  uint16_t h[8];
#pragma unroll
  for (int e = 0; e < 8; ++e)
    h[e] = f16 ? __half_as_ushort(__float2half_rn(v[e])) : __bfloat16_as_ushort(__float2bfloat16_rn(v[e]));
  *reinterpret_cast<uint4 *>(tile + r * 128 + ((j ^ (r & 7)) << 4)) = *reinterpret_cast<uint4 *>(h);
}
// FP64 -> operand type (BF16, or FP16 when f16), round to nearest even, back as float
__device__ __forceinline__ float bf16_hi(double v, int f16) {
  return f16 ? __half2float(__double2half(v)) : __bfloat162float(__double2bfloat16(v));
}

// Input-gradient split tiles: rows [W1f^T hi (dp rows); W1f^T lo (dp rows)], cols = hidden
// units, one tile of 2 dp rows per 64-column k-block.
__global__ void pack_tc_g1_kernel(const double *W1f, int dp, int w, int f16, uint8_t *out) {
  const int rows = 2 * dp, kbw = w / 64;
  const size_t chunks = static_cast<size_t>(kbw) * rows * 8;
  const size_t id = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (id >= chunks) return;
  const int j = static_cast<int>(id % 8), r = static_cast<int>((id / 8) % rows);
  const int kb = static_cast<int>(id / (8 * rows));
  const int i = r % dp;
  float v[8];
  for (int e = 0; e < 8; ++e) {
    const int k = kb * 64 + j * 8 + e;
    const double wv = W1f[static_cast<size_t>(k) * dp + i];
    const float hi = bf16_hi(wv, f16);
    v[e] = (r < dp) ? hi : static_cast<float>(wv - static_cast<double>(hi));
  }
  put_chunk(out + static_cast<size_t>(kb) * rows * 128, r, j, v, f16);
}
cudaError_t launch_pack_tc_g1(const double *W1f, int dp, int w, int f16, uint8_t *out, cudaStream_t s) {
  const size_t chunks = static_cast<size_t>(w / 64) * 2 * dp * 8;
  pack_tc_g1_kernel<<<blocks_for(chunks, 256), 256, 0, s>>>(W1f, dp, w, f16, out);
  return cudaGetLastError();
}

// Per-rank streams for the cluster kernel: rank r owns output rows [r NS, (r + 1) NS) of
// every layer, packed as tiles of TR rows x 64 columns (same swizzle as above).
__global__ void pack_tc2_l1_kernel(const double *W1f, int dp, int kb1, int rank, int NS, int TR, int f16,
                                   uint8_t *out) {
  const int nsub = NS / TR;
  const size_t chunks = static_cast<size_t>(nsub) * kb1 * TR * 8;
  const size_t id = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (id >= chunks) return;
  const int j = static_cast<int>(id % 8), r = static_cast<int>((id / 8) % TR);
  const int tile = static_cast<int>(id / (8 * static_cast<size_t>(TR)));
  const int sub = tile / kb1, kb = tile % kb1;
  const int k = rank * NS + sub * TR + r;
  float v[8];
  for (int e = 0; e < 8; ++e) {
    const int kk = kb * 64 + j * 8 + e;
    const int seg = kk / dp, i = kk % dp;
    float x = 0.f;
    if (seg < 3) {
      const double wv = W1f[static_cast<size_t>(k) * dp + i];
      const float hi = bf16_hi(wv, f16);
      x = (seg == 2) ? static_cast<float>(wv - static_cast<double>(hi)) : hi;
    }
    v[e] = x;
  }
  put_chunk(out + static_cast<size_t>(tile) * TR * 128, r, j, v, f16);
}
cudaError_t launch_pack_tc2_l1(const double *W1f, int dp, int kb1, int rank, int NS, int TR, int f16, uint8_t *out,
                               cudaStream_t s) {
  const size_t chunks = static_cast<size_t>(NS / TR) * kb1 * TR * 8;
  pack_tc2_l1_kernel<<<blocks_for(chunks, 256), 256, 0, s>>>(W1f, dp, kb1, rank, NS, TR, f16, out);
  return cudaGetLastError();
}

__global__ void pack_tc2_hidden_kernel(const double *P, int d, int D, int w, int rank, int NS, int TR, int f16,
                                       uint8_t *out) {
  const int nsub = NS / TR, kbw = w / 64;
  const size_t per_layer = static_cast<size_t>(nsub) * kbw;
  const size_t chunks = 2 * static_cast<size_t>(D - 1) * per_layer * TR * 8;
  const size_t id = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (id >= chunks) return;
  const int j = static_cast<int>(id % 8), r = static_cast<int>((id / 8) % TR);
  const size_t tile = id / (8 * static_cast<size_t>(TR));
  const size_t seg = tile / per_layer;
  const int within = static_cast<int>(tile % per_layer);
  const int sub = within / kbw, kb = within % kbw;
  const bool adj = seg >= static_cast<size_t>(D - 1);
  const int l = adj ? D - static_cast<int>(seg - (D - 1)) : static_cast<int>(seg) + 2;
  const double *Wl = P + off_W(l, d, w);
  const int row = rank * NS + sub * TR + r;
  uint16_t hb[8];
  for (int e = 0; e < 8; ++e) {
    const int col = kb * 64 + j * 8 + e;
    const double x = adj ? Wl[static_cast<size_t>(col) * w + row] : Wl[static_cast<size_t>(row) * w + col];
    hb[e] = f16 ? __half_as_ushort(__double2half(x)) : __bfloat16_as_ushort(__double2bfloat16(x));
  }
  *reinterpret_cast<uint4 *>(out + tile * TR * 128 + r * 128 + ((j ^ (r & 7)) << 4)) = *reinterpret_cast<uint4 *>(hb);
}
cudaError_t launch_pack_tc2_hidden(const double *P, int d, int D, int w, int rank, int NS, int TR, int f16,
                                   uint8_t *out, cudaStream_t s) {
  if (D < 2) return cudaSuccess;
  const size_t chunks = 2 * static_cast<size_t>(D - 1) * (NS / TR) * (w / 64) * TR * 8;
  pack_tc2_hidden_kernel<<<blocks_for(chunks, 256), 256, 0, s>>>(P, d, D, w, rank, NS, TR, f16, out);
  return cudaGetLastError();
}

template <typename S, typename D_>
__global__ void cast_kernel(const S *src, D_ *dst, size_t n) {
  const size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (i < n) dst[i] = static_cast<D_>(src[i]);
}
cudaError_t launch_cast_f32(const double *src, float *dst, size_t n, cudaStream_t s) {
  if (n) cast_kernel<<<blocks_for(n, 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}
cudaError_t launch_cast_f64(const double *src, double *dst, size_t n, cudaStream_t s) {
  if (n) cast_kernel<<<blocks_for(n, 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}
cudaError_t launch_cast_f32_to_f64(const float *src, double *dst, size_t n, cudaStream_t s) {
  if (n) cast_kernel<<<blocks_for(n, 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Analytic fold (FP64): z-space t = tanh(B (mu_c + L_c z) + c), f = A t + N (mu_n + L_n z).
__global__ void fold_analytic_kernel(const double *A, const double *B, const double *c, const double *N,
                                     const double *data, const double *mu, const double *L, int d, int dp, int d_c,
                                     int H, int n_data, int mode, double *Bf, double *cf, double *AT, double *NfT,
                                     double *dataf) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int dn = d - d_c;
  if (tid < H) {
    const int k = tid;
    double cc = c[k];
    for (int j = 0; j < dp; ++j) {
      double s = 0.0;
      if (j < d) {
        if (mode == 0) {
          for (int i = j; i < d_c; ++i) s += B[k * d_c + i] * L[i * d + j];
        } else if (j < d_c) {
          s = B[k * d_c + j];
        }
      }
      Bf[k * dp + j] = s;
    }
    if (mode == 0)
      for (int i = 0; i < d_c; ++i) cc += B[k * d_c + i] * mu[i];
    cf[k] = cc;
  }
  if (tid < n_data) {
    const int i = tid;
    for (int k = 0; k < H; ++k) AT[static_cast<size_t>(k) * n_data + i] = A[static_cast<size_t>(i) * H + k];
    double dd = data[i];
    if (dn > 0) {
      for (int j = 0; j < dp; ++j) {
        double s = 0.0;
        if (j < d) {
          if (mode == 0) {
            for (int q = (j > d_c ? j : d_c); q < d; ++q) s += N[static_cast<size_t>(i) * dn + (q - d_c)] * L[q * d + j];
          } else if (j >= d_c) {
            s = N[static_cast<size_t>(i) * dn + (j - d_c)];
          }
        }
        NfT[static_cast<size_t>(j) * n_data + i] = s;
      }
      if (mode == 0)
        for (int q = d_c; q < d; ++q) dd -= N[static_cast<size_t>(i) * dn + (q - d_c)] * mu[q];
    }
    dataf[i] = dd;
  }
}
cudaError_t launch_fold_analytic(const double *A, const double *B, const double *c, const double *N,
                                 const double *data, const double *mu, const double *L, int d, int dp, int d_c, int H,
                                 int n_data, int mode, double *Bf, double *cf, double *AT, double *NfT, double *dataf,
                                 cudaStream_t s) {
  const int n = H > n_data ? H : n_data;
  fold_analytic_kernel<<<blocks_for(n, 128), 128, 0, s>>>(A, B, c, N, data, mu, L, d, dp, d_c, H, n_data, mode, Bf,
                                                          cf, AT, NfT, dataf);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Covariance adaptation.  One thread merges the FP64 tile records (Chan et al.), forms the
// unbiased covariance and factorises it; jitter delta (tr S / d) I, delta = jitter0 x 10^k, is
// added only if the plain factorisation fails.
__global__ void adapt_finalize_kernel(const double *wf, int n_tiles, int stride, int d, double jitter0, double *mu,
                                      double *Lout, double *info) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double n = 0.0, mean[kMaxD], M2[kMaxD * kMaxD], S[kMaxD * kMaxD];
  for (int i = 0; i < d; ++i) mean[i] = 0.0;
  for (int i = 0; i < d * d; ++i) M2[i] = 0.0;
  for (int t = 0; t < n_tiles; ++t) {
    const double *W = wf + static_cast<size_t>(t) * stride;
    const double nb = W[kWfN];
    if (nb <= 0.0) continue;
    const double nn = n + nb;
    for (int i = 0; i < d; ++i)
      for (int j = i; j < d; ++j) {
        const double di = W[kWfMean + i] - mean[i], dj = W[kWfMean + j] - mean[j];
        M2[i * d + j] += W[kWfM2 + i * kMaxD + j] + di * dj * n * nb / nn;
      }
    for (int i = 0; i < d; ++i) mean[i] += (W[kWfMean + i] - mean[i]) * nb / nn;
    n = nn;
  }
  info[0] = n;
  info[1] = -1.0;
  info[2] = 0.0;
  for (int i = 0; i < d; ++i) mu[i] = mean[i];
  if (n < 2.0) {
    info[2] = 1.0;
    return;
  }
  double tr = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = i; j < d; ++j) {
      S[i * d + j] = S[j * d + i] = M2[i * d + j] / (n - 1.0);
      if (i == j) tr += S[i * d + i];
    }
  double delta = 0.0;
  for (int attempt = 0; attempt < 12; ++attempt) {
    // attempt 0: plain; then delta = jitter0, 10 jitter0, ... while <= 1e-2
    if (attempt > 0) {
      delta = (attempt == 1) ? jitter0 : delta * 10.0;
      if (delta > 1e-2 * (1.0 + 1e-9)) break;
    }
    bool ok = true;
    for (int i = 0; i < d * d; ++i) Lout[i] = 0.0;
    for (int j = 0; j < d && ok; ++j) {
      double s = S[j * d + j] + delta * tr / d;
      for (int k = 0; k < j; ++k) s -= Lout[j * d + k] * Lout[j * d + k];
      if (!(s > 0.0)) {
        ok = false;
        break;
      }
      const double ljj = sqrt(s);
      Lout[j * d + j] = ljj;
      for (int i = j + 1; i < d; ++i) {
        double t = S[i * d + j];
        for (int k = 0; k < j; ++k) t -= Lout[i * d + k] * Lout[j * d + k];
        Lout[i * d + j] = t / ljj;
      }
    }
    if (ok) {
      info[1] = delta;
      return;
    }
  }
  info[2] = 2.0;
}
cudaError_t launch_adapt_finalize(const double *wf, int n_tiles, int stride, int d, double jitter0, double *mu,
                                  double *L, double *info, cudaStream_t s) {
  adapt_finalize_kernel<<<1, 32, 0, s>>>(wf, n_tiles, stride, d, jitter0, mu, L, info);
  return cudaGetLastError();
}

// Merged statistics of every record (n, mean, M2 upper triangle mirrored), no factorisation.
__global__ void welford_stats_kernel(const double *wf, int n_tiles, int stride, int d, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double n = 0.0, mean[kMaxD], M2[kMaxD * kMaxD];
  for (int i = 0; i < d; ++i) mean[i] = 0.0;
  for (int i = 0; i < d * d; ++i) M2[i] = 0.0;
  for (int t = 0; t < n_tiles; ++t) {
    const double *W = wf + static_cast<size_t>(t) * stride;
    const double nb = W[kWfN];
    if (nb <= 0.0) continue;
    const double nn = n + nb;
    for (int i = 0; i < d; ++i)
      for (int j = i; j < d; ++j) {
        const double di = W[kWfMean + i] - mean[i], dj = W[kWfMean + j] - mean[j];
        M2[i * d + j] += W[kWfM2 + i * kMaxD + j] + di * dj * n * nb / nn;
      }
    for (int i = 0; i < d; ++i) mean[i] += (W[kWfMean + i] - mean[i]) * nb / nn;
    n = nn;
  }
  out[0] = n;
  for (int i = 0; i < d; ++i) out[1 + i] = mean[i];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) out[1 + d + i * d + j] = (j >= i) ? M2[i * d + j] : M2[j * d + i];
}
cudaError_t launch_welford_stats(const double *wf, int n_tiles, int stride, int d, double *out, cudaStream_t s) {
  welford_stats_kernel<<<1, 32, 0, s>>>(wf, n_tiles, stride, d, out);
  return cudaGetLastError();
}

// Chan merge of one (n, mean, M2) triple (device copy of host values) into record W.
__global__ void welford_merge_kernel(double *W, int d, const double *in) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double na = W[kWfN], nb = in[0];
  if (nb <= 0.0) return;
  const double n = na + nb;
  for (int i = 0; i < d; ++i)
    for (int j = i; j < d; ++j) {
      const double di = in[1 + i] - W[kWfMean + i], dj = in[1 + j] - W[kWfMean + j];
      W[kWfM2 + i * kMaxD + j] += in[1 + d + i * d + j] + di * dj * na * nb / n;
    }
  for (int i = 0; i < d; ++i) W[kWfMean + i] += (in[1 + i] - W[kWfMean + i]) * nb / n;
  W[kWfN] = n;
}
cudaError_t launch_welford_merge(double *W, int d, const double *in, cudaStream_t s) {
  welford_merge_kernel<<<1, 32, 0, s>>>(W, d, in);
  return cudaGetLastError();
}

__global__ void welford_clear_kernel(double *wf, size_t n) {
  const size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (i < n) wf[i] = 0.0;
}
cudaError_t launch_welford_clear(double *wf, int n_tiles, int stride, cudaStream_t s) {
  const size_t n = static_cast<size_t>(n_tiles) * stride;
  welford_clear_kernel<<<blocks_for(n, 256), 256, 0, s>>>(wf, n);
  return cudaGetLastError();
}

// External samples into tile record 0: batch of m rows, FP64 two-pass batch statistics
// merged into the record.
template <typename R>
__global__ void welford_add_kernel(const R *x, int m, int d, double *W) {
  __shared__ double bmean[kMaxD];
  const int t = threadIdx.x;
  for (int i = t; i < d; i += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < m; ++r) s += static_cast<double>(x[static_cast<size_t>(r) * d + i]);
    bmean[i] = s / m;
  }
  __syncthreads();
  const double na = W[kWfN], nb = m, n = na + nb;
  for (int p = t; p < d * d; p += blockDim.x) {
    const int i = p / d, j = p % d;
    if (j < i) continue;
    double s = 0.0;
    for (int r = 0; r < m; ++r)
      s += (static_cast<double>(x[static_cast<size_t>(r) * d + i]) - bmean[i]) *
           (static_cast<double>(x[static_cast<size_t>(r) * d + j]) - bmean[j]);
    const double di = bmean[i] - W[kWfMean + i], dj = bmean[j] - W[kWfMean + j];
    W[kWfM2 + i * kMaxD + j] += s + di * dj * na * nb / n;
  }
  __syncthreads();
  for (int i = t; i < d; i += blockDim.x) W[kWfMean + i] += (bmean[i] - W[kWfMean + i]) * nb / n;
  if (t == 0) W[kWfN] = n;
}
cudaError_t launch_welford_add_f32(const float *x, int m, int d, double *wf, int, cudaStream_t s) {
  welford_add_kernel<float><<<1, 256, 0, s>>>(x, m, d, wf);
  return cudaGetLastError();
}
cudaError_t launch_welford_add_f64(const double *x, int m, int d, double *wf, int, cudaStream_t s) {
  welford_add_kernel<double><<<1, 256, 0, s>>>(x, m, d, wf);
  return cudaGetLastError();
}

template <typename R>
__global__ void remap_kernel(R *z, int n, int d, int dp, const double *mu_o, const double *L_o, const double *mu_n,
                             const double *L_n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  R *zc = z + static_cast<size_t>(c) * dp;
  double x[kMaxD], zn[kMaxD];
  for (int i = 0; i < d; ++i) {
    double s = mu_o[i];
    for (int j = 0; j <= i; ++j) s += L_o[i * d + j] * static_cast<double>(zc[j]);
    x[i] = s - mu_n[i];
  }
  for (int i = 0; i < d; ++i) {
    double s = x[i];
    for (int j = 0; j < i; ++j) s -= L_n[i * d + j] * zn[j];
    zn[i] = s / L_n[i * d + i];
  }
  for (int i = 0; i < d; ++i) zc[i] = static_cast<R>(zn[i]);
}
cudaError_t launch_remap_f32(float *z, int n, int d, int dp, const double *mu_o, const double *L_o, const double *mu_n,
                             const double *L_n, cudaStream_t s) {
  remap_kernel<float><<<blocks_for(n, 128), 128, 0, s>>>(z, n, d, dp, mu_o, L_o, mu_n, L_n);
  return cudaGetLastError();
}
cudaError_t launch_remap_f64(double *z, int n, int d, int dp, const double *mu_o, const double *L_o,
                             const double *mu_n, const double *L_n, cudaStream_t s) {
  remap_kernel<double><<<blocks_for(n, 128), 128, 0, s>>>(z, n, d, dp, mu_o, L_o, mu_n, L_n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// ESS: samples x[n][M][d].  (1) per series (chain c, dim q): mean and variance (n - 1 denominator).
template <typename R>
__global__ void ess_moments_kernel(const R *x, int n, int M, int d, double *mean, double *var) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;  // series index c * d + q
  if (s >= M * d) return;
  const size_t st = static_cast<size_t>(M) * d;
  double sum = 0.0;
  for (int t = 0; t < n; ++t) sum += static_cast<double>(x[t * st + s]);
  const double m = sum / n;
  double ss = 0.0;
  for (int t = 0; t < n; ++t) {
    const double e = static_cast<double>(x[t * st + s]) - m;
    ss += e * e;
  }
  mean[s] = m;
  var[s] = ss / (n - 1);
}
// ------------------------------------------------------------------------------------------
// Initial walker positions (the initialisation strategies of Sec. 3.1), one thread per chain, in
// FP64 from stream (chain, 0, kInit): 0 every chain at `center`; 1 lower + (upper - lower) u with
// the uniforms 0..d-1; 2 center + Lc xi with the normals 0..d-1 (Lc row-major d x d).  par holds
// center, lower, upper (kMaxD each) and Lc (kMaxD x kMaxD).
constexpr uint32_t kInit = 8;  // Philox purpose of the initial positions (after those of common.cuh)
__global__ void init_positions_kernel(int strategy, uint64_t seed, int n, int d, const double *par, double *theta) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double *center = par, *lower = par + kMaxD, *upper = par + 2 * kMaxD, *Lc = par + 3 * kMaxD;
  double *out = theta + static_cast<size_t>(c) * d;
  if (strategy == 1) {
    for (int i = 0; i < d; ++i)
      out[i] = lower[i] + (upper[i] - lower[i]) * draw_uniform<double>(seed, static_cast<uint32_t>(c), 0u, kInit,
                                                                      static_cast<uint32_t>(i));
  } else if (strategy == 2) {
    double xi[kMaxD];
    draw_normals<double>(seed, static_cast<uint32_t>(c), 0u, kInit, d, xi);
    for (int i = 0; i < d; ++i) {
      double s = center[i];
      for (int j = 0; j < d; ++j) s += Lc[i * d + j] * xi[j];
      out[i] = s;
    }
  } else {
    for (int i = 0; i < d; ++i) out[i] = center[i];
  }
}
cudaError_t launch_init_positions(int strategy, uint64_t seed, int n, int d, const double *par, double *theta,
                                  cudaStream_t s) {
  init_positions_kernel<<<blocks_for(static_cast<size_t>(n), 128), 128, 0, s>>>(strategy, seed, n, d, par, theta);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// R - 1 (Sec. 4.1): pooled within-chain cross products S_ij = sum_c sum_t (x_tci - m_ci)(x_tcj - m_cj)
// for the chains of one block (kRhatChains of them), FP64; one partial per block and pair
// i <= j (pair p = i * d - i (i - 1) / 2 + j - i), summed over blocks in order on the host.
constexpr int kRhatChains = 32;
template <typename R>
__global__ void __launch_bounds__(256) rhat_cross_kernel(const R *x, int n, int M, int d, const double *mean,
                                                         double *partial) {
  __shared__ double y[kRhatChains * kMaxD];
  const int c0 = blockIdx.x * kRhatChains;
  const int nc = min(kRhatChains, M - c0);
  const int npairs = d * (d + 1) / 2;
  double acc[3] = {0.0, 0.0, 0.0};  // pairs threadIdx.x + 256 k, k < 3 (npairs <= 528)
  int pi[3], pj[3];
  for (int k = 0; k < 3; ++k) {
    int p = threadIdx.x + 256 * k, i = 0;
    pi[k] = pj[k] = -1;
    if (p < npairs) {
      while (p >= d - i) {
        p -= d - i;
        ++i;
      }
      pi[k] = i;
      pj[k] = i + p;
    }
  }
  const size_t st = static_cast<size_t>(M) * d;
  for (int t = 0; t < n; ++t) {
    __syncthreads();
    for (int e = threadIdx.x; e < nc * d; e += blockDim.x)
      y[e] = static_cast<double>(x[t * st + static_cast<size_t>(c0) * d + e]) - mean[static_cast<size_t>(c0) * d + e];
    __syncthreads();
    for (int k = 0; k < 3; ++k)
      if (pi[k] >= 0)
        for (int c = 0; c < nc; ++c) acc[k] += y[c * d + pi[k]] * y[c * d + pj[k]];
  }
  for (int k = 0; k < 3; ++k)
    if (pi[k] >= 0) partial[static_cast<size_t>(blockIdx.x) * npairs + threadIdx.x + 256 * k] = acc[k];
}
cudaError_t launch_rhat_cross_f32(const float *x, int n, int M, int d, const double *mean, double *partial,
                                  cudaStream_t s) {
  rhat_cross_kernel<float><<<(M + kRhatChains - 1) / kRhatChains, 256, 0, s>>>(x, n, M, d, mean, partial);
  return cudaGetLastError();
}
cudaError_t launch_rhat_cross_f64(const double *x, int n, int M, int d, const double *mean, double *partial,
                                  cudaStream_t s) {
  rhat_cross_kernel<double><<<(M + kRhatChains - 1) / kRhatChains, 256, 0, s>>>(x, n, M, d, mean, partial);
  return cudaGetLastError();
}
int rhat_blocks(int M) { return (M + kRhatChains - 1) / kRhatChains; }

// ------------------------------------------------------------------------------------------
// Quantiles of the pooled draws per dimension by radix select (exact order statistics).  A
// value's key is its order-preserving unsigned image; pass by pass (4-bit digits, most
// significant first) every job (one rank of one dimension; the jobs of dimension q are
// q * jpd .. q * jpd + jpd - 1) histograms the next digit of the keys that match its prefix.
template <typename R>
struct SelKey;
template <>
struct SelKey<float> {
  using K = uint32_t;
  static __device__ __forceinline__ K of(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  }
};
template <>
struct SelKey<double> {
  using K = unsigned long long;
  static __device__ __forceinline__ K of(double v) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
  }
};
template <typename R>
__global__ void qsel_hist_kernel(const R *x, size_t n_elems, int d, int jpd, const typename SelKey<R>::K *prefix,
                                 int shift, unsigned int *hist) {
  using K = typename SelKey<R>::K;
  extern __shared__ unsigned int qh[];  // [d * jpd][16]
  const int njobs = d * jpd;
  for (int i = threadIdx.x; i < njobs * 16; i += blockDim.x) qh[i] = 0u;
  __syncthreads();
  const int top = shift + 4;  // bits at and above `top` are fixed by the prefix
  const K hi_mask = top >= static_cast<int>(8 * sizeof(K)) ? K(0) : (~K(0) << top);
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n_elems;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(e % static_cast<size_t>(d));
    const K key = SelKey<R>::of(x[e]);
    const unsigned digit = static_cast<unsigned>((key >> shift) & K(15));
    for (int j = q * jpd; j < (q + 1) * jpd; ++j)
      if ((key & hi_mask) == prefix[j]) atomicAdd(&qh[j * 16 + digit], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < njobs * 16; i += blockDim.x)
    if (qh[i]) atomicAdd(&hist[i], qh[i]);
}
cudaError_t launch_qsel_hist_f32(const float *x, size_t n_elems, int d, int jpd, const uint32_t *prefix, int shift,
                                 unsigned int *hist, cudaStream_t s) {
  const size_t smem = static_cast<size_t>(d) * jpd * 16 * sizeof(unsigned int);
  qsel_hist_kernel<float><<<1216, 256, smem, s>>>(x, n_elems, d, jpd, prefix, shift, hist);
  return cudaGetLastError();
}
cudaError_t launch_qsel_hist_f64(const double *x, size_t n_elems, int d, int jpd, const unsigned long long *prefix,
                                 int shift, unsigned int *hist, cudaStream_t s) {
  const size_t smem = static_cast<size_t>(d) * jpd * 16 * sizeof(unsigned int);
  qsel_hist_kernel<double><<<1216, 256, smem, s>>>(x, n_elems, d, jpd, prefix, shift, hist);
  return cudaGetLastError();
}
cudaError_t launch_ess_moments_f32(const float *x, int n, int M, int d, double *mean, double *var, cudaStream_t s) {
  ess_moments_kernel<float><<<blocks_for(static_cast<size_t>(M) * d, 128), 128, 0, s>>>(x, n, M, d, mean, var);
  return cudaGetLastError();
}
cudaError_t launch_ess_moments_f64(const double *x, int n, int M, int d, double *mean, double *var, cudaStream_t s) {
  ess_moments_kernel<double><<<blocks_for(static_cast<size_t>(M) * d, 128), 128, 0, s>>>(x, n, M, d, mean, var);
  return cudaGetLastError();
}

// (2) variogram sums V[q][t - t0] += sum_c sum_{i >= t} (x_i - x_{i-t})^2 for lags t0..t0+nt-1.
// Block = 32 series (threadIdx.x, coalesced) x 32 lags (threadIdx.y, sharing the series' draws
// through L1).
constexpr int kVgLags = 32;
template <typename R>
__global__ void ess_variogram_kernel(const R *x, int n, int M, int d, int t0, int nt, double *V) {
  const int s = blockIdx.x * 32 + threadIdx.x;
  const int lag = threadIdx.y, t = t0 + lag;
  if (lag >= nt || s >= M * d) return;
  const size_t st = static_cast<size_t>(M) * d;
  double acc = 0.0;
  for (int i = t; i < n; ++i) {
    const double e = static_cast<double>(x[i * st + s]) - static_cast<double>(x[(i - t) * st + s]);
    acc += e * e;
  }
  atomicAdd(&V[(s % d) * nt + lag], acc);
}
cudaError_t launch_ess_variogram_f32(const float *x, int n, int M, int d, int t0, int nt, double *V, cudaStream_t s) {
  dim3 blk(32, kVgLags);
  ess_variogram_kernel<float><<<blocks_for(static_cast<size_t>(M) * d, 32), blk, 0, s>>>(x, n, M, d, t0, nt, V);
  return cudaGetLastError();
}
cudaError_t launch_ess_variogram_f64(const double *x, int n, int M, int d, int t0, int nt, double *V, cudaStream_t s) {
  dim3 blk(32, kVgLags);
  ess_variogram_kernel<double><<<blocks_for(static_cast<size_t>(M) * d, 32), blk, 0, s>>>(x, n, M, d, t0, nt, V);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Training (FP32).  Generic tiled GEMM C[M][N] = sum_k A(i,k) B(k,j) with strided operands
// and a fused epilogue:
//   EPI_STORE : C = acc
//   EPI_TANH  : C = tanh(acc + bias[j])
//   EPI_DTANH : C = acc * (1 - H[i][j]^2)
enum { EPI_STORE = 0, EPI_TANH = 1, EPI_DTANH = 2 };
// Split over K (gridDim.z slices of k_chunk, a multiple of kGK): slice z accumulates its
// k range into its own output C + z * M * ldc (EPI_STORE only); sum_slices adds the slices in
// slice order, so the result does not depend on scheduling.
constexpr int kGT = 64, kGK = 16;
__global__ void __launch_bounds__(256) gemm_f32_kernel(int M, int N, int K, const float *A, long long a_i,
                                                       long long a_k, const float *B, long long b_k, long long b_j,
                                                       float *C, int ldc, int epi, const float *bias, const float *H,
                                                       int ldh, int k_chunk) {
  __shared__ __align__(16) float As[kGK][kGT + 4];
  __shared__ __align__(16) float Bs[kGK][kGT + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * kGT, j0 = blockIdx.x * kGT;
  const int kbeg = blockIdx.z * k_chunk, kend = min(K, kbeg + k_chunk);
  C += static_cast<size_t>(blockIdx.z) * M * ldc;
  float acc[4][4] = {};
  (void)acc;
  // staging loads run along whichever index of an operand is contiguous in memory
  const bool a_kc = (a_k == 1), b_kc = (b_k == 1);
  for (int k0 = kbeg; k0 < kend; k0 += kGK) {
    for (int e = threadIdx.x; e < kGK * kGT; e += 256) {
      {
        const int kk = a_kc ? e % kGK : e / kGT, ii = a_kc ? e / kGK : e % kGT;
        const int i = i0 + ii, k = k0 + kk;
        As[kk][ii] = (i < M && k < kend) ? A[i * a_i + k * a_k] : 0.f;
      }
      {
        const int kk = b_kc ? e % kGK : e / kGT, jj = b_kc ? e / kGK : e % kGT;
        const int j = j0 + jj, k = k0 + kk;
        Bs[kk][jj] = (j < N && k < kend) ? B[k * b_k + j * b_j] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
      const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i >= M || j >= N) continue;
      float r = acc[u][v];
      if (epi == EPI_TANH) r = tanhf(r + bias[j]);
      else if (epi == EPI_DTANH) {
        const float h = H[static_cast<size_t>(i) * ldh + j];
        r = r * (1.f - h * h);
      }
      C[static_cast<size_t>(i) * ldc + j] = r;
    }
}
static void gemm_f32(int M, int N, int K, const float *A, long long a_i, long long a_k, const float *B, long long b_k,
                     long long b_j, float *C, int ldc, int epi, const float *bias, const float *H, int ldh,
                     cudaStream_t s, int splits = 1) {
  const int k_chunk = ((K + splits - 1) / splits + kGK - 1) / kGK * kGK;
  dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT, splits);
  gemm_f32_kernel<<<grid, 256, 0, s>>>(M, N, K, A, a_i, a_k, B, b_k, b_j, C, ldc, epi, bias, H, ldh, k_chunk);
}
__global__ void sum_slices_kernel(const float *ws, int splits, size_t n, float *out) {
  const size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  float r = ws[i];
  for (int z = 1; z < splits; ++z) r += ws[static_cast<size_t>(z) * n + i];
  out[i] = r;
}

__global__ void standardise_kernel(const float *X, const float *m, const float *sd, int rows, int d, float *U) {
  const size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<size_t>(rows) * d) return;
  const int j = static_cast<int>(i % d);
  U[i] = (X[i] - m[j]) / sd[j];
}

// out = wo . h_D + bo;  r = out - (t(chi2) - out_m)/out_s;  loss += r^2 / m;  dout = 2 r / m;
// delta_D = dout wo (1 - h_D^2).  t(chi2) = chi2 (linear output) or log(max(chi2 - floor, 1e-30))
// (log output).  One warp per row.
__global__ void train_head_kernel(const float *HD, const float *wo, const float *bo_ptr, const float *chi2, float out_m,
                                  float out_s, int out_log, float out_floor, int m, int w, float *dout, float *delta,
                                  float *loss) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= m) return;
  const float *h = HD + static_cast<size_t>(warp) * w;
  float s = 0.f;
  for (int k = lane; k < w; k += 32) s += wo[k] * h[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const float tc = out_log ? logf(fmaxf(chi2[warp] - out_floor, 1e-30f)) : chi2[warp];
  const float y = (tc - out_m) / out_s;
  const float r = s + *bo_ptr - y;
  const float g = 2.f * r / m;
  if (lane == 0) {
    dout[warp] = g;
    atomicAdd(loss, r * r / m);
  }
  for (int k = lane; k < w; k += 32) delta[static_cast<size_t>(warp) * w + k] = g * wo[k] * (1.f - h[k] * h[k]);
}

// column sums: out[j] = sum_i X[i][j] (bias gradients).  A block of 256 threads takes 32
// columns; its 8 row groups sum interleaved rows (i = g, g + 8, ...) and the 8 partial sums
// are added in group order, so the result does not depend on scheduling.
// Column sums over the batch, optionally weighted: out[j du + k] = sum_i X[i][j] U[i][k] (U null: du = 1,
// plain sums) -- the bias and output-head gradients and the layer-1 weight gradient (fan-in d).  The
// batch is split in `slices` runs of consecutive rows; one block per 32 columns and slice sums its
// rows in a fixed order (8 row groups, combined in order), and sum_slices_kernel adds the slices in
// order: deterministic, with enough blocks to fill the GPU (a product with so few output columns
// leaves a tiled GEMM with a handful of blocks).
__global__ void __launch_bounds__(256) wsum_kernel(const float *X, int rows, int cols, const float *U, int du,
                                                   int slices, float *ws) {
  __shared__ float part[8][32][kWsumMaxU + 1];
  const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + c, sl = blockIdx.y;
  const int r0 = static_cast<int>(static_cast<long long>(rows) * sl / slices);
  const int r1 = static_cast<int>(static_cast<long long>(rows) * (sl + 1) / slices);
  float acc[kWsumMaxU];
#pragma unroll
  for (int k = 0; k < kWsumMaxU; ++k) acc[k] = 0.f;
  if (j < cols) {
    for (int i = r0 + g; i < r1; i += 8) {
      const float x = X[static_cast<size_t>(i) * cols + j];
      if (U == nullptr) {
        acc[0] += x;
      } else {
        const float *u = U + static_cast<size_t>(i) * du;
#pragma unroll
        for (int k = 0; k < kWsumMaxU; ++k)
          if (k < du) acc[k] = fmaf(x, u[k], acc[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kWsumMaxU; ++k)
    if (k < du) part[g][c][k] = acc[k];
  __syncthreads();
  if (j < cols)
    for (int k = g; k < du; k += 8) {
      float t = part[0][c][k];
      for (int q = 1; q < 8; ++q) t += part[q][c][k];
      ws[(static_cast<size_t>(sl) * cols + j) * du + k] = t;
    }
}

cudaError_t launch_wsum(const float *X, int rows, int cols, const float *U, int du, float *ws, float *out,
                        cudaStream_t s) {
  if (du < 1 || du > kWsumMaxU || (U == nullptr && du != 1) || rows < 1 || cols < 1) return cudaErrorInvalidValue;
  const int slices = rows / 64 < 1 ? 1 : (rows / 64 < kWsumSlices ? rows / 64 : kWsumSlices);
  wsum_kernel<<<dim3((cols + 31) / 32, slices), 256, 0, s>>>(X, rows, cols, U, du, slices, ws);
  const size_t n = static_cast<size_t>(cols) * du;
  sum_slices_kernel<<<blocks_for(n, 256), 256, 0, s>>>(ws, slices, n, out);
  return cudaGetLastError();
}

// Initial whitened positions z0 = L^-1 (theta0 - mu) (Algorithm 1's map inverted), one chain per
// thread, forward substitution in FP64, rows padded to dp with zeros, stored in the working type.
template <typename R>
__global__ void init_z_kernel(const double *theta, const double *mu, const double *L, int n, int d, int dp, R *z) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double zz[kMaxD];
  for (int i = 0; i < d; ++i) {
    double s = theta[static_cast<size_t>(c) * d + i] - mu[i];
    for (int j = 0; j < i; ++j) s -= L[i * d + j] * zz[j];
    zz[i] = s / L[i * d + i];
  }
  for (int i = 0; i < dp; ++i) z[static_cast<size_t>(c) * dp + i] = static_cast<R>(i < d ? zz[i] : 0.0);
}

cudaError_t launch_init_z(bool f64, const double *theta, const double *mu, const double *L, int n, int d, int dp,
                          void *z, cudaStream_t s) {
  if (n < 1 || d < 1 || d > kMaxD || dp < d) return cudaErrorInvalidValue;
  if (f64)
    init_z_kernel<double><<<blocks_for(n, 128), 128, 0, s>>>(theta, mu, L, n, d, dp, static_cast<double *>(z));
  else
    init_z_kernel<float><<<blocks_for(n, 128), 128, 0, s>>>(theta, mu, L, n, d, dp, static_cast<float *>(z));
  return cudaGetLastError();
}

cudaError_t launch_train_grad(const float *P, const float *in_m, const float *in_s, float out_m, float out_s,
                              int out_log, float out_floor, int d, int D, int w, int m, const float *X,
                              const float *chi2, float *G, TrainWork &tw, cudaStream_t s) {
  cudaMemsetAsync(tw.loss, 0, sizeof(float), s);
  standardise_kernel<<<blocks_for(static_cast<size_t>(m) * d, 256), 256, 0, s>>>(X, in_m, in_s, m, d, tw.U);
  // forward: H_l = tanh(H_{l-1} W_l^T + b_l)
  for (int l = 1; l <= D; ++l) {
    const int fan = (l == 1) ? d : w;
    const float *Ain = (l == 1) ? tw.U : tw.H + static_cast<size_t>(l - 2) * m * w;
    const float *Wl = P + off_W(l, d, w);
    float *Hl = tw.H + static_cast<size_t>(l - 1) * m * w;
    gemm_f32(m, w, fan, Ain, fan, 1, Wl, 1, fan, Hl, w, EPI_TANH, P + off_b(l, d, w), nullptr, 0, s);
  }
  const float *HD = tw.H + static_cast<size_t>(D - 1) * m * w;
  const size_t owo = off_wo(d, D, w);
  train_head_kernel<<<blocks_for(static_cast<size_t>(m) * 32, 256), 256, 0, s>>>(HD, P + owo, P + owo + w, chi2, out_m,
                                                                               out_s, out_log, out_floor, m, w,
                                                                               tw.dout, tw.Dl, tw.loss);
  // g_wo[j] = sum_i dout_i H_D[i][j] ; g_bo = sum_i dout_i
  cudaError_t e = launch_wsum(HD, m, w, tw.dout, 1, tw.ws, G + owo, s);
  if (e != cudaSuccess) return e;
  e = launch_wsum(tw.dout, m, 1, nullptr, 1, tw.ws, G + owo + w, s);
  if (e != cudaSuccess) return e;
  float *dl = tw.Dl, *dn = tw.Dn;
  for (int l = D; l >= 1; --l) {
    const int fan = (l == 1) ? d : w;
    const float *Hprev = (l == 1) ? tw.U : tw.H + static_cast<size_t>(l - 2) * m * w;
    // g_W_l[k][j] = sum_i delta_l[i][k] Hprev[i][j]  (the batch split in kTrainSplits slices: a
    // w x fan product has too few output tiles to fill the GPU; fan-in d: weighted column sums)
    if (l == 1) {
      e = launch_wsum(dl, m, w, tw.U, d, tw.ws, G + off_W(1, d, w), s);
      if (e != cudaSuccess) return e;
    } else {
      gemm_f32(w, fan, m, dl, 1, w, Hprev, fan, 1, tw.ws, fan, EPI_STORE, nullptr, nullptr, 0, s, kTrainSplits);
      sum_slices_kernel<<<blocks_for(static_cast<size_t>(w) * fan, 256), 256, 0, s>>>(
          tw.ws, kTrainSplits, static_cast<size_t>(w) * fan, G + off_W(l, d, w));
    }
    e = launch_wsum(dl, m, w, nullptr, 1, tw.ws, G + off_b(l, d, w), s);
    if (e != cudaSuccess) return e;
    if (l > 1) {
      // delta_{l-1} = (delta_l W_l) (1 - H_{l-1}^2)
      gemm_f32(m, w, w, dl, w, 1, P + off_W(l, d, w), w, 1, dn, w, EPI_DTANH, nullptr, Hprev, w, s);
      float *t = dl;
      dl = dn;
      dn = t;
    }
  }
  return cudaGetLastError();
}

// The same gradient with the hidden-layer products on the tensor cores (BF16 operands, FP32
// accumulation; k_train_tc.cu).  The input layer (K = d), the output head, the bias sums and
// the (1 - h^2) factors stay FP32 on the CUDA cores.  Needs m % 512 == 0, w % 128 == 0, D >= 2
// (tc_train_shape_ok) and the BF16 buffers of tw.
bool tc_train_shape_ok(int d, int D, int w, int m) {
  (void)d;
  return D >= 2 && tc_gemm_shape_ok(m, w, w, 1) && tc_gemm_shape_ok(w, w, m, kTcTrainSplits);
}
cudaError_t launch_train_grad_tc(const float *P, const float *in_m, const float *in_s, float out_m, float out_s,
                                 int out_log, float out_floor, int d, int D, int w, int m, const float *X,
                                 const float *chi2, float *G, TrainWork &tw, int *status, cudaStream_t s) {
  if (!tc_train_shape_ok(d, D, w, m)) return cudaErrorInvalidValue;
  const size_t mw = static_cast<size_t>(m) * w, ww = static_cast<size_t>(w) * w;
  cudaMemsetAsync(tw.loss, 0, sizeof(float), s);
  standardise_kernel<<<blocks_for(static_cast<size_t>(m) * d, 256), 256, 0, s>>>(X, in_m, in_s, m, d, tw.U);
  cudaError_t e;
  // BF16 copies of W_l and W_l^T (l = 2..D) from the FP32 masters
  for (int l = 2; l <= D; ++l) {
    e = launch_cast_transpose_bf16(P + off_W(l, d, w), w, w, tw.Wb + (l - 2) * ww, tw.WbT + (l - 2) * ww, s);
    if (e != cudaSuccess) return e;
  }
  // forward: layer 1 on the CUDA cores (K = d), then H_l = tanh(H_{l-1} W_l^T + b_l) on the tensor cores
  gemm_f32(m, w, d, tw.U, d, 1, P + off_W(1, d, w), 1, d, tw.H, w, EPI_TANH, P + off_b(1, d, w), nullptr, 0, s);
  e = launch_cast_transpose_bf16(tw.H, m, w, tw.Hb, tw.HbT, s);
  if (e != cudaSuccess) return e;
  for (int l = 2; l <= D; ++l) {
    TcGemmArgs a = {};
    a.M = m;
    a.N = w;
    a.K = w;
    a.epi = kTcEpiTanh;
    a.C = tw.H + static_cast<size_t>(l - 1) * mw;
    a.bias = P + off_b(l, d, w);
    a.Cb = l < D ? tw.Hb + (l - 1) * mw : nullptr;
    a.CbT = l < D ? tw.HbT + (l - 1) * mw : nullptr;
    a.status = status;
    e = launch_tc_gemm(tw.Hb + (l - 2) * mw, tw.Wb + (l - 2) * ww, 1, a, s);
    if (e != cudaSuccess) return e;
  }
  const float *HD = tw.H + static_cast<size_t>(D - 1) * mw;
  const size_t owo = off_wo(d, D, w);
  train_head_kernel<<<blocks_for(static_cast<size_t>(m) * 32, 256), 256, 0, s>>>(HD, P + owo, P + owo + w, chi2, out_m,
                                                                               out_s, out_log, out_floor, m, w,
                                                                               tw.dout, tw.Dl, tw.loss);
  e = launch_wsum(HD, m, w, tw.dout, 1, tw.ws, G + owo, s);
  if (e != cudaSuccess) return e;
  e = launch_wsum(tw.dout, m, 1, nullptr, 1, tw.ws, G + owo + w, s);
  if (e != cudaSuccess) return e;
  int cur = 0;
  e = launch_cast_transpose_bf16(tw.Dl, m, w, tw.Db, tw.DbT, s);
  if (e != cudaSuccess) return e;
  float *dl = tw.Dl, *dn = tw.Dn;
  for (int l = D; l >= 2; --l) {
    // G_l = delta_l^T H_{l-1} over the batch (split in kTcTrainSplits slices summed in order)
    TcGemmArgs gw = {};
    gw.M = w;
    gw.N = w;
    gw.K = m;
    gw.epi = kTcEpiStore;
    gw.C = tw.wsg;
    gw.status = status;
    e = launch_tc_gemm(tw.DbT + cur * mw, tw.HbT + (l - 2) * mw, kTcTrainSplits, gw, s);
    if (e != cudaSuccess) return e;
    sum_slices_kernel<<<blocks_for(ww, 256), 256, 0, s>>>(tw.wsg, kTcTrainSplits, ww, G + off_W(l, d, w));
    e = launch_wsum(dl, m, w, nullptr, 1, tw.ws, G + off_b(l, d, w), s);
    if (e != cudaSuccess) return e;
    // delta_{l-1} = (delta_l W_l) (1 - H_{l-1}^2), FP32 and its BF16 copies
    TcGemmArgs gd = {};
    gd.M = m;
    gd.N = w;
    gd.K = w;
    gd.epi = kTcEpiDtanh;
    gd.C = dn;
    gd.H = tw.H + static_cast<size_t>(l - 2) * mw;
    gd.Cb = l > 2 ? tw.Db + (1 - cur) * mw : nullptr;
    gd.CbT = l > 2 ? tw.DbT + (1 - cur) * mw : nullptr;
    gd.status = status;
    e = launch_tc_gemm(tw.Db + cur * mw, tw.WbT + (l - 2) * ww, 1, gd, s);
    if (e != cudaSuccess) return e;
    float *t = dl;
    dl = dn;
    dn = t;
    cur = 1 - cur;
  }
  // layer 1 (fan-in d) on the CUDA cores
  e = launch_wsum(dl, m, w, tw.U, d, tw.ws, G + off_W(1, d, w), s);
  if (e != cudaSuccess) return e;
  e = launch_wsum(dl, m, w, nullptr, 1, tw.ws, G + off_b(1, d, w), s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

__global__ void adam_kernel(float *P, const float *G, float *m1, float *m2, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float a = b1 * m1[i] + (1.f - b1) * g;
  const float v = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = a;
  m2[i] = v;
  P[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}
cudaError_t launch_adam(float *P, const float *G, float *m1, float *m2, size_t n, int t, float lr, float b1, float b2,
                        float eps, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, static_cast<float>(t)), c2 = 1.f - powf(b2, static_cast<float>(t));
  adam_kernel<<<blocks_for(n, 256), 256, 0, s>>>(P, G, m1, m2, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_zero(void *p, size_t bytes, cudaStream_t s) { return cudaMemsetAsync(p, 0, bytes, s); }

}  // namespace bst
