// engine_simt.cuh -- CUDA-core (FP32 / FP64) likelihood engines and the chain-tile kernel.
//
// These are the "plain" precision paths: the emulator forward + adjoint as
// register-tiled SIMT GEMMs over a tile of T chains held in shared memory, and
// the analytic theory-map likelihood one warp per chain.  The BF16 tensor-core
// engine lives in engine_tc.cuh and shares the sampler state machines.
#pragma once

#include "common.cuh"
#include "sampler.cuh"

namespace bst {

// ------------------------------------------------------------------------------------------
// Emulator weights for the SIMT engines (working precision R).
//   layer 1 acts on the evaluated point directly: the whitening x = mu + L z and the input
//   standardisation are folded in (W1f = W1 diag(1/s) L, b1f = b1 + W1 (mu - m)/s), so the
//   returned gradient is already d logL / dz.
template <typename R>
struct EmuWeights {
  int depth, width, dp;
  const R *W1T;  // [dp][w]     folded layer-1, transposed (forward operand)
  const R *W1;   // [w][dp]     folded layer-1 (input-gradient operand)
  const R *b1;   // [w]
  const R *WT;   // [D-1][w][w] W_l^T, l = 2..D (forward operand)
  const R *W;    // [D-1][w][w] W_l             (adjoint operand)
  const R *b;    // [D-1][w]
  const R *wo;   // [w]
  R bo, out_m, out_s;
  int out_log;   // chi2 = out_floor + exp(out_s out + out_m) instead of out_s out + out_m
  R out_floor;
  R *scratch;    // [rows][D-1][w] hidden activations h_1..h_{D-1} kept for the adjoint
};

// Analytic theory map in evaluation coordinates (folded like the emulator):
//   t = tanh(Bf z + cf), r = dataf - A t - Nf z, logL = -|r|^2 / (2 sigma^2).
template <typename R>
struct AnaWeights {
  int d, dp, H, n_data, linear, has_N;
  const R *Bf;     // [H][dp]
  const R *cf;     // [H]
  const R *AT;     // [H][n_data]  (A transposed)
  const R *NfT;    // [dp][n_data] (Nf transposed) or nullptr
  const R *dataf;  // [n_data]
  R inv_s2;
};

template <typename R>
struct SimtCfg;
template <>
struct SimtCfg<float> {
  static constexpr int KC = 16;  // K rows per staged B chunk
};
template <>
struct SimtCfg<double> {
  static constexpr int KC = 8;
};

constexpr int kSimtThreads = 256;
constexpr int kSimtNB = 256;  // output columns per pass (8 warps x 32)

// Register-tiled C[T][N] = A[T][K] (smem, lda) * B[K][N] (global, row-major), followed by an
// element-wise epilogue epi(row, col, acc).  256 threads; each warp owns 32 columns of a
// 256-column pass; each thread owns 8 rows x CPT consecutive columns.
template <typename R, int T, class Epi>
__device__ __forceinline__ void simt_gemm(const R *__restrict__ A, int lda, int K,
                                          const R *__restrict__ B, int N, R *stage, Epi epi) {
  constexpr int KC = SimtCfg<R>::KC;
  constexpr int LY = T / 8;          // lanes along rows
  constexpr int LX = 32 / LY;        // lanes along columns
  constexpr int CPT = 32 / LX;       // consecutive columns per thread
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ly = lane / LX, lx = lane % LX;
  const int nk = (K + KC - 1) / KC;
  constexpr int CH_PER_ROW = kSimtNB * static_cast<int>(sizeof(R)) / 16;  // 16-byte chunks
  for (int n0 = 0; n0 < N; n0 += kSimtNB) {
    R acc[8][CPT];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int q = 0; q < CPT; ++q) acc[i][q] = R(0);
    auto load_chunk = [&](int kc, int buf) {
      R *dst = stage + buf * KC * kSimtNB;
      const int k0 = kc * KC;
      for (int ch = tid; ch < KC * CH_PER_ROW; ch += kSimtThreads) {
        const int r = ch / CH_PER_ROW, cc = ch % CH_PER_ROW;
        const int k = k0 + r;
        R *dptr = dst + r * kSimtNB + cc * (16 / sizeof(R));
        const unsigned saddr = static_cast<unsigned>(__cvta_generic_to_shared(dptr));
        if (k < K) {
          const R *src = B + static_cast<size_t>(k) * N + n0 + cc * (16 / sizeof(R));
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(src));
        } else {
          *reinterpret_cast<float4 *>(dptr) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      asm volatile("cp.async.commit_group;\n" ::);
    };
    load_chunk(0, 0);
    for (int kc = 0; kc < nk; ++kc) {
      if (kc + 1 < nk) {
        load_chunk(kc + 1, (kc + 1) & 1);
        asm volatile("cp.async.wait_group 1;\n" ::);
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::);
      }
      __syncthreads();
      const R *Bs = stage + (kc & 1) * KC * kSimtNB + warp * 32 + lx * CPT;
      const int kmax = min(KC, K - kc * KC);
      const R *Ak = A + kc * KC;
      for (int kk = 0; kk < kmax; ++kk) {
        R av[8], bv[CPT];
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] = Ak[(ly + LY * i) * lda + kk];
#pragma unroll
        for (int q = 0; q < CPT; ++q) bv[q] = Bs[kk * kSimtNB + q];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int q = 0; q < CPT; ++q) acc[i][q] = fma(av[i], bv[q], acc[i][q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int q = 0; q < CPT; ++q) epi(ly + LY * i, n0 + warp * 32 + lx * CPT + q, acc[i][q]);
  }
}

__device__ __forceinline__ float tanh_r(float v) { return tanhf(v); }
__device__ __forceinline__ double tanh_r(double v) { return tanh(v); }

// ------------------------------------------------------------------------------------------
// SIMT emulator engine: forward (and adjoint) of the MLP for the T rows of this CTA.
template <typename R, int T>
struct EmuSimt {
  static constexpr int kThreads = kSimtThreads;
  static size_t smem_bytes(int width) {
    const int lda = width + (sizeof(R) == 4 ? 4 : 2);
    return sizeof(R) * (2 * static_cast<size_t>(T) * lda + 2 * SimtCfg<R>::KC * kSimtNB + T);
  }

  // Evaluate rows [row0, row0 + T) of ze into lle / gle.
  static __device__ void eval(const EmuWeights<R> &E, const StepArgs<R> &a, int row0,
                              bool need_grad, char *smem_raw) {
    const int w = E.width, D = E.depth, dp = E.dp;
    const int lda = w + (sizeof(R) == 4 ? 4 : 2);
    R *bufA = reinterpret_cast<R *>(smem_raw);
    R *bufB = bufA + T * lda;
    R *stage = bufB + T * lda;
    R *outv = stage + 2 * SimtCfg<R>::KC * kSimtNB;
    const int tid = threadIdx.x;
    const int lda1 = dp + (sizeof(R) == 4 ? 4 : 2);
    // layer-1 input rows (zero for rows past the end)
    for (int idx = tid; idx < T * dp; idx += kThreads) {
      const int r = idx / dp, i = idx % dp;
      const int row = row0 + r;
      bufB[r * lda1 + i] = (row < a.n_rows && i < a.d) ? a.st.ze[row_off(a.st.ze_ld, row, a.dp) + i * row_es(a.st.ze_ld)] : R(0);
    }
    __syncthreads();
    R *cur = bufA, *nxt = bufB;
    const size_t sstride = static_cast<size_t>(D > 1 ? D - 1 : 1) * w;
    // layer 1
    {
      const bool keep = need_grad && D > 1;
      simt_gemm<R, T>(bufB, lda1, dp, E.W1T, w, stage, [&](int r, int n, R acc) {
        const R h = tanh_r(acc + E.b1[n]);
        cur[r * lda + n] = h;
        const int row = row0 + r;
        if (keep && row < a.n_rows) E.scratch[row * sstride + n] = h;
      });
      __syncthreads();
    }
    for (int l = 2; l <= D; ++l) {
      const R *WT = E.WT + static_cast<size_t>(l - 2) * w * w;
      const R *bl = E.b + static_cast<size_t>(l - 2) * w;
      const bool keep = need_grad && l < D;
      simt_gemm<R, T>(cur, lda, w, WT, w, stage, [&](int r, int n, R acc) {
        const R h = tanh_r(acc + bl[n]);
        nxt[r * lda + n] = h;
        const int row = row0 + r;
        if (keep && row < a.n_rows) E.scratch[row * sstride + static_cast<size_t>(l - 1) * w + n] = h;
      });
      __syncthreads();
      R *t = cur;
      cur = nxt;
      nxt = t;
    }
    // output: out = wo . h_D + bo; logL = -chi2 / 2 with chi2 = out_s out + out_m (linear output)
    // or out_floor + exp(out_s out + out_m) (log output), one warp per row; outv[r] keeps
    // d chi2 / d(out_s out + out_m) (1, or the exponential) for the adjoint's seed
    const int warp = tid >> 5, lane = tid & 31;
    for (int r = warp; r < T; r += kThreads / 32) {
      R s = 0;
      for (int n = lane; n < w; n += 32) s += E.wo[n] * cur[r * lda + n];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const R arg = E.out_s * (s + E.bo) + E.out_m;
        const R t = E.out_log ? exp(arg) : R(1);
        outv[r] = t;
        const int row = row0 + r;
        if (row < a.n_rows) a.st.lle[row] = R(-0.5) * (E.out_log ? E.out_floor + t : arg);
      }
    }
    if (!need_grad) {
      __syncthreads();
      return;
    }
    // delta_D = (-out_s / 2) t_r wo (1 - h_D^2), in place
    const R c0 = R(-0.5) * E.out_s;
    __syncthreads();
    for (int idx = tid; idx < T * w; idx += kThreads) {
      const int r = idx / w, n = idx % w;
      const R h = cur[r * lda + n];
      cur[r * lda + n] = (c0 * outv[r]) * E.wo[n] * (R(1) - h * h);
    }
    __syncthreads();
    // delta_{l-1} = (W_l^T delta_l) (1 - h_{l-1}^2), l = D..2
    for (int l = D; l >= 2; --l) {
      const R *Wl = E.W + static_cast<size_t>(l - 2) * w * w;
      simt_gemm<R, T>(cur, lda, w, Wl, w, stage, [&](int r, int n, R acc) {
        const int row = row0 + r;
        const R h = (row < a.n_rows) ? E.scratch[row * sstride + static_cast<size_t>(l - 2) * w + n] : R(0);
        nxt[r * lda + n] = acc * (R(1) - h * h);
      });
      __syncthreads();
      R *t = cur;
      cur = nxt;
      nxt = t;
    }
    // d logL / dz_i = sum_k delta_1[k] W1f[k][i]
    for (int idx = tid; idx < T * dp; idx += kThreads) {
      const int r = idx / dp, i = idx % dp;
      const int row = row0 + r;
      if (i >= a.d || row >= a.n_rows) continue;
      R s = 0;
      for (int k = 0; k < w; ++k) s += cur[r * lda + k] * E.W1[k * dp + i];
      a.st.gle[row_off(a.st.gle_ld, row, a.dp) + i * row_es(a.st.gle_ld)] = s;
    }
    __syncthreads();
  }
};

// ------------------------------------------------------------------------------------------
// SIMT analytic engine: one warp per row; data rows strided over lanes.
template <typename R, int T>
struct AnaSimt {
  static constexpr int kThreads = kSimtThreads;
  static size_t smem_bytes(int) { return sizeof(R) * (kThreads / 32) * (64 + 64 + kMaxD); }

  static __device__ void eval(const AnaWeights<R> &P, const StepArgs<R> &a, int row0,
                              bool need_grad, char *smem_raw) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    R *tsh = reinterpret_cast<R *>(smem_raw) + warp * (64 + 64 + kMaxD);
    R *ssh = tsh + 64;
    R *zsh = ssh + 64;
    const int H = P.H, nd = P.n_data, dp = P.dp;
    for (int r = warp; r < T; r += kThreads / 32) {
      const int row = row0 + r;
      if (row >= a.n_rows) continue;
      const R *zr = a.st.ze + row_off(a.st.ze_ld, row, a.dp);
      for (int i = lane; i < dp; i += 32) zsh[i] = (i < P.d) ? zr[i * row_es(a.st.ze_ld)] : R(0);
      __syncwarp();
      for (int k = lane; k < H; k += 32) {
        R s = P.cf[k];
        for (int i = 0; i < P.d; ++i) s += P.Bf[k * dp + i] * zsh[i];
        tsh[k] = P.linear ? s : tanh_r(s);
      }
      __syncwarp();
      R chi2 = 0;
      R sk[2] = {R(0), R(0)};  // partial A^T r for k = lane, lane + 32
      R sn = 0;                // partial Nf^T r for i = lane (d <= 32)
      for (int i0 = 0; i0 < nd; i0 += 32) {
        const int i = i0 + lane;
        R rv = 0;
        if (i < nd) {
          R f = 0;
          for (int k = 0; k < H; ++k) f += P.AT[static_cast<size_t>(k) * nd + i] * tsh[k];
          if (P.has_N)
            for (int j = 0; j < P.d; ++j) f += P.NfT[static_cast<size_t>(j) * nd + i] * zsh[j];
          rv = P.dataf[i] - f;
        }
        chi2 += rv * rv;
        if (need_grad) {
          // s_k += sum_i A[i][k] r_i over this chunk (lanes hold r_i)
          for (int k = 0; k < H; ++k) {
            R v = (i < nd) ? P.AT[static_cast<size_t>(k) * nd + i] * rv : R(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((k & 31) == lane) sk[k >> 5] += v;
          }
          if (P.has_N)
            for (int j = 0; j < P.d; ++j) {
              R v = (i < nd) ? P.NfT[static_cast<size_t>(j) * nd + i] * rv : R(0);
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
              if (j == lane) sn += v;
            }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) chi2 += __shfl_xor_sync(0xffffffffu, chi2, o);
      if (lane == 0) a.st.lle[row] = R(-0.5) * chi2 * P.inv_s2;
      if (need_grad) {
        for (int k = lane; k < H; k += 32) {
          const R t = tsh[k];
          ssh[k] = sk[k >> 5] * (P.linear ? R(1) : (R(1) - t * t));
        }
        __syncwarp();
        if (lane < P.d) {
          R gsum = 0;
          for (int k = 0; k < H; ++k) gsum += P.Bf[k * dp + lane] * ssh[k];
          if (P.has_N) gsum += sn;
          a.st.gle[row_off(a.st.gle_ld, row, a.dp) + lane * row_es(a.st.gle_ld)] = gsum * P.inv_s2;
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
};

// ------------------------------------------------------------------------------------------
// Welford tile update (covariance adaptation, Sec. 3.2): rows of this tile that finished an
// iteration contributed x to xbuf; their batch mean / M2 (working precision, two passes) is
// merged into the tile's FP64 running statistics (Chan, Golub & LeVeque).  Called by all
// `nthr` threads of the owner group with a group barrier `sync`.
template <typename R, class Sync>
__device__ void welford_tile(const StepArgs<R> &a, int row0, int nrows, const int *mask, int t,
                             int nthr, Sync sync, int tile) {
  double *W = a.wf + static_cast<size_t>(tile) * a.wf_stride;
  const int d = a.d;
  const R *xb = a.xbuf;
  if (t == 0) {
    int cnt = 0;
    for (int r = 0; r < nrows; ++r) cnt += mask[r];
    W[kWfBn] = cnt;
  }
  sync();
  const double cnt = W[kWfBn];
  if (cnt > 0.0) {
    for (int i = t; i < d; i += nthr) {
      R s = 0;
      for (int r = 0; r < nrows; ++r)
        if (mask[r]) s += xb[static_cast<size_t>(row0 + r) * a.dp + i];
      W[kWfBMean + i] = static_cast<double>(s) / cnt;
    }
    sync();
    for (int p = t; p < d * d; p += nthr) {
      const int i = p / d, j = p % d;
      if (j < i) continue;
      const R mi = static_cast<R>(W[kWfBMean + i]), mj = static_cast<R>(W[kWfBMean + j]);
      R s = 0;
      for (int r = 0; r < nrows; ++r)
        if (mask[r]) {
          const R *x = xb + static_cast<size_t>(row0 + r) * a.dp;
          s += (x[i] - mi) * (x[j] - mj);
        }
      W[kWfBM2 + i * kMaxD + j] = s;
    }
    sync();
    const double na = W[kWfN], nb = cnt, n = na + nb;
    for (int p = t; p < d * d; p += nthr) {
      const int i = p / d, j = p % d;
      if (j < i) continue;
      const double di = W[kWfBMean + i] - W[kWfMean + i];
      const double dj = W[kWfBMean + j] - W[kWfMean + j];
      W[kWfM2 + i * kMaxD + j] += W[kWfBM2 + i * kMaxD + j] + di * dj * na * nb / n;
    }
    sync();
    for (int i = t; i < d; i += nthr) W[kWfMean + i] += (W[kWfBMean + i] - W[kWfMean + i]) * nb / n;
    if (t == 0) W[kWfN] = n;
  }
  sync();
}

// ------------------------------------------------------------------------------------------
// Chain-tile kernel: T rows per CTA, thread t < T owns row row0 + t.
// The per-chain sampler code as separate functions: inlined, its registers raised the
// kernel's allocation (255 with spills) and slowed the emulator GEMM loop by ~15 %.
template <typename R>
__device__ __noinline__ bool simt_chain_pre(const StepArgs<R> &a, int row, int h) {
  return Chain<R, false>(a).pre(row, h);
}
template <typename R>
__device__ __noinline__ bool simt_chain_post(const StepArgs<R> &a, int row, int h) {
  return Chain<R, false>(a).post(row, h);
}

// Tiles per ensemble half (the cluster size of an ensemble-move launch), 1 otherwise.
template <int T, typename R>
__host__ __device__ inline int simt_ensemble_cluster(const StepArgs<R> &a) {
  return (is_ensemble_mode(a.mode) && a.aies_walkers / 2 > T) ? a.aies_walkers / 2 / T : 1;
}

// Launched with kSimtThreads threads.  Registers capped at 128: the emulator GEMM loop ran
// fastest there (FP32 MALA, 4096 chains, 8-512x4-1: 711 us per round at 128, 739 at 168,
// 898 at the 255 the compiler picks by itself).
template <typename R, int T, class Engine, class Weights>
__global__ void __maxnreg__(128)
simt_chain_kernel(const __grid_constant__ StepArgs<R> a, const __grid_constant__ Weights W) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int mask[T];
  const int row0 = blockIdx.x * T;
  const int tid = threadIdx.x;
  const bool owner = tid < T && row0 + tid < a.n_rows;
  Chain<R, false> ch(a);
  const int row = row0 + tid;
  if (a.mode == kModeLoglike) {
    // ze / lle / gle point at the caller's theta, logL and gradient rows
    Engine::eval(W, a, row0, a.need_grad != 0, smem);
    return;
  }
  // per-launch chain bookkeeping
  if (owner) {
    if (is_ensemble_mode(a.mode)) {
      for (int h = 0; h < 2; ++h) a.st.steps_done[ch.aies_walker(row, h)] = 0;
    } else {
      a.st.steps_done[row] = 0;
      if (a.mode == kModeHMC) ch.dw(row)[0] = 0.0;
      if (is_nuts_mode(a.mode)) ch.dw(row)[0] = 1.0;
    }
  }
  __syncthreads();
  for (int ev = 0;; ++ev) {
    const int h = ev & 1;
    const bool need = owner && simt_chain_pre(a, row, h);
    if (!__syncthreads_or(need)) break;
    Engine::eval(W, a, row0, a.need_grad != 0, smem);
    bool done = false;
    if (need) done = simt_chain_post(a, row, h);
    if (tid < T) mask[tid] = done ? 1 : 0;
    __syncthreads();
    if (a.welford_on && __syncthreads_or(done)) {
      welford_tile(a, row0, min(T, a.n_rows - row0), mask, tid, kSimtThreads, [] { __syncthreads(); },
                   static_cast<int>(blockIdx.x));
    }
    // ensemble halves spread over the tiles of a cluster: every tile has finished this half-step
    // (its walkers' positions written) before any proposes the other half, whose partners are
    // these walkers.  All tiles of a cluster run the same number of half-steps.
    if (simt_ensemble_cluster<T>(a) > 1)
      asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  }
}

}  // namespace bst
