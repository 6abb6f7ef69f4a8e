// engine_tc.cuh -- BF16 tensor-core (tcgen05 / TMEM) emulator engine for sm_103a.
//
// One CTA owns a tile of 128 chains (one TMEM lane per chain) for a whole
// bst_step call and keeps its activations in shared memory:
//
//   warp 0     producer: streams pre-swizzled BF16 weight tiles (256 x 64) from
//              global/L2 into a ring of shared-memory stages with cp.async.bulk,
//              completion tracked by mbarrier transaction counts;
//   warp 1     MMA issuer: one thread issues tcgen05.mma (M=128, N=256, K=16,
//              BF16 x BF16 -> FP32 in TMEM) per 16-wide K slice and releases
//              each stage with tcgen05.commit;
//   warps 2-5  sampler + epilogue: one thread per chain.  They run the
//              proposal / accept state machines, write the layer-1 operand, and
//              after each layer read the accumulator row with tcgen05.ld, apply
//              bias + tanh (forward) or the (1 - h^2) factor (adjoint), round to
//              BF16 and write the next layer's operand back into shared memory.
//
// Per evaluation: layer 1 (the whitening-folded input layer, with the input and
// the weights split into BF16 hi + lo parts so it is accurate to ~2^-16), the
// hidden layers 2..D, the FP32 output dot on CUDA cores, then (for gradient
// samplers) the adjoint layers D..2 with W_l^T and the input-gradient product,
// again with hi + lo weights.  Every wait is bounded by a time limit; a timeout
// sets a status bit and all roles leave their loops.
#pragma once

#include "common.cuh"
#include "engine_simt.cuh"
#include "sampler.cuh"

namespace bst {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 192;
constexpr int kTcStageBytes = 256 * 128;  // one 256-row x 64-col BF16 tile
constexpr int kTcMaxStages = 6;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

struct TcWeights {
  int depth, width, dp, kb1, k16_l1;
  const uint8_t *l1;   // layer-1 tiles of this launch's fold set
  const uint8_t *hid;  // hidden forward tiles then adjoint tiles
  const uint8_t *g1;   // input-gradient tiles of this launch's fold set
  const float *b1;     // [w] folded layer-1 bias
  const float *b;      // [D-1][w]
  const float *wo;     // [w]
  float bo, out_m, out_s;
  __nv_bfloat16 *scratch;  // [rows][D-1][w]
  int n_stages;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and a status bit) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *status) {
  for (int i = 0; i < 256; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kWaitLimitNs) {
      set_status(status, kStatusTimeout);
      return false;
    }
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// Named barrier among the 128 sampler threads (id 1); returns the OR of pred.
__device__ __forceinline__ bool group_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred ? 1u : 0u)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void group_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;            // leading byte offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;    // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;            // descriptor version
  d |= static_cast<uint64_t>(2) << 61;            // 128-byte swizzle
  return d;
}
// Instruction descriptor: kind::f16, A = B = BF16, D = FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of 16-byte chunk j (8 BF16 values) of row r inside a 128-byte-swizzled K block.
__device__ __forceinline__ uint32_t sw128_off(int r, int j) {
  return static_cast<uint32_t>(r * 128 + ((j ^ (r & 7)) << 4));
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

// Evaluation phases: 0 = layer 1; 1..D-1 = hidden layers 2..D; then (gradient) D..2D-2 =
// adjoint layers D..2 and 2D-1 = input gradient.
__device__ __forceinline__ int tc_num_phases(int D, bool grad) { return grad ? 2 * D : D; }

// ---------------------------------------------------------------- the kernel
template <int W>
__global__ void __launch_bounds__(kTcThreads, 1) tc_chain_kernel(const StepArgs<float> a, const TcWeights E) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  constexpr int KBW = W / 64;   // K blocks of the hidden width
  constexpr int NH = W / 256;   // 256-wide N halves
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *act = base;                              // KBW x 16 KB activation operand
  uint8_t *stages = act + KBW * 16384;              // n_stages x 32 KB weight tiles
  uint64_t *bars = reinterpret_cast<uint64_t *>(stages + E.n_stages * kTcStageBytes);
  // bars: full[S], empty[S], go, act, acc, fin
  const int S = E.n_stages;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
  const uint32_t go_bar = smem_u32(bars + 2 * S), act_bar = smem_u32(bars + 2 * S + 1);
  const uint32_t acc_bar = smem_u32(bars + 2 * S + 2), fin_bar = smem_u32(bars + 2 * S + 3);
  volatile int *cmd = reinterpret_cast<volatile int *>(bars + 2 * S + 4);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 5);
  int *mask = reinterpret_cast<int *>(bars + 2 * S + 6);  // [128]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int D = E.depth, dp = E.dp;
  const bool grad = a.need_grad != 0;
  const int nph = tc_num_phases(D, grad);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(go_bar, 1);
    mbar_init(act_bar, 1);
    mbar_init(acc_bar, 1);
    mbar_init(fin_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(static_cast<uint32_t>(W))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t fills[kTcMaxStages] = {0, 0, 0, 0, 0, 0};
      int s = 0;
      uint32_t go_par = 0;
      bool ok = true;
      while (ok) {
        if (!mbar_wait(go_bar, go_par, a.status)) break;
        go_par ^= 1;
        const int c = *cmd;
        if (c == 0) break;
        const bool g = c == 2;
        const int n_l1 = NH * E.kb1, n_h = (D - 1) * NH * KBW;
        const int n_tiles = n_l1 + n_h + (g ? n_h + KBW : 0);
        for (int t = 0; t < n_tiles && ok; ++t) {
          const uint8_t *src;
          uint32_t bytes = kTcStageBytes;
          if (t < n_l1) {
            src = E.l1 + static_cast<size_t>(t) * kTcStageBytes;
          } else if (t < n_l1 + (g ? 2 : 1) * n_h) {
            src = E.hid + static_cast<size_t>(t - n_l1) * kTcStageBytes;
          } else {
            bytes = 2 * dp * 128;
            src = E.g1 + static_cast<size_t>(t - n_l1 - 2 * n_h) * bytes;
          }
          if (!mbar_wait(empty0 + 8 * s, (fills[s] & 1) ^ 1, a.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full0 + 8 * s, bytes);
          bulk_g2s(smem_u32(stages + s * kTcStageBytes), src, bytes, full0 + 8 * s);
          fills[s]++;
          s = (s + 1 == S) ? 0 : s + 1;
        }
      }
      // drain: every issued copy must land before the CTA can exit
      for (int q = 0; q < S; ++q)
        if (fills[q]) mbar_wait(full0 + 8 * q, (fills[q] - 1) & 1, a.status);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t uses[kTcMaxStages] = {0, 0, 0, 0, 0, 0};
      int s = 0;
      uint32_t go_par = 0, act_par = 0;
      bool ok = true;
      const uint32_t id256 = idesc_bf16(128, 256), idg = idesc_bf16(128, 2 * dp);
      const uint32_t act_addr = smem_u32(act);
      while (ok) {
        if (!mbar_wait(go_bar, go_par, a.status)) break;
        go_par ^= 1;
        const int c = *cmd;
        if (c == 0) break;
        const int phases = tc_num_phases(D, c == 2);
        for (int p = 0; p < phases && ok; ++p) {
          if (p > 0) {
            if (!mbar_wait(act_bar, act_par, a.status)) {
              ok = false;
              break;
            }
            act_par ^= 1;
          }
          tc_fence_after();
          const bool last = (p == 2 * D - 1);
          const int nh_n = last ? 1 : NH;
          const int nkb = (p == 0) ? E.kb1 : KBW;
          for (int nh = 0; nh < nh_n && ok; ++nh) {
            for (int kb = 0; kb < nkb; ++kb) {
              if (!mbar_wait(full0 + 8 * s, uses[s] & 1, a.status)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t b_addr = smem_u32(stages + s * kTcStageBytes);
              const int k16 = (p == 0) ? min(4, E.k16_l1 - 4 * kb) : 4;
              for (int k = 0; k < k16; ++k) {
                const uint64_t ad = sw128_desc(act_addr + kb * 16384 + k * 32);
                const uint64_t bd = sw128_desc(b_addr + k * 32);
                mma_bf16(tmem + nh * 256, ad, bd, last ? idg : id256, (kb > 0 || k > 0) ? 1u : 0u);
              }
              mma_commit(empty0 + 8 * s);
              uses[s]++;
              s = (s + 1 == S) ? 0 : s + 1;
            }
          }
          if (ok) mma_commit(acc_bar);
        }
      }
      // make sure no MMA is in flight before TMEM is released
      mma_commit(fin_bar);
      mbar_wait(fin_bar, 0, a.status);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ sampler + epilogue
    const int q = warp & 3;              // TMEM lane quadrant of this warp
    const int r = q * 32 + lane;         // tile row == TMEM lane
    const int row = blockIdx.x * kTcRows + r;
    const bool valid = row < a.n_rows;
    const int t = (warp - 2) * 32 + lane;  // 0..127 within the group
    const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16);
    const uint32_t act_addr = smem_u32(act);
    Chain<float> ch(a);
    const bool loglike = a.mode == kModeLoglike;
    if (valid && !loglike) {
      if (a.mode == kModeAIES) {
        for (int h = 0; h < 2; ++h) a.st.steps_done[ch.aies_walker(row, h)] = 0;
      } else {
        a.st.steps_done[row] = 0;
        if (a.mode == kModeHMC) ch.dwork_ptr(row)[0] = 0.0;
        if (a.mode == kModeNUTS) ch.dwork_ptr(row)[0] = 1.0;
      }
    }
    group_sync();
    uint32_t acc_par = 0;
    const size_t sstride = static_cast<size_t>(D > 1 ? D - 1 : 1) * W;
    for (int ev = 0;; ++ev) {
      const int h = ev & 1;
      bool need;
      if (loglike) need = valid && ev == 0;
      else need = valid && ch.pre(row, h);
      if (!group_or(need)) {
        if (t == 0) {
          *cmd = 0;
          mbar_arrive(go_bar);
        }
        break;
      }
      // layer-1 operand: [z_hi | z_lo | z_hi | 0] per row, BF16, swizzled
      {
        float zv[kMaxD];
        const float *zr = a.st.ze + static_cast<size_t>(row) * a.st.ze_ld;
        for (int i = 0; i < dp; ++i) zv[i] = (valid && i < a.d) ? zr[i] : 0.f;
        const int k1 = E.kb1 * 64;
        for (int j = 0; j < k1 / 8; ++j) {
          uint32_t w4[4];
          for (int e2 = 0; e2 < 4; ++e2) {
            float v2[2];
            for (int u = 0; u < 2; ++u) {
              const int kk = j * 8 + e2 * 2 + u;
              const int seg = kk / dp, i = kk % dp;
              float v = 0.f;
              if (seg < 3) {
                const float hi = __bfloat162float(__float2bfloat16_rn(zv[i]));
                v = (seg == 1) ? (zv[i] - hi) : hi;
              }
              v2[u] = v;
            }
            w4[e2] = pack_bf16x2(v2[0], v2[1]);
          }
          const int kb = j / 8, jj = j % 8;
          st_shared_v4(act_addr + kb * 16384 + sw128_off(r, jj), w4[0], w4[1], w4[2], w4[3]);
        }
      }
      fence_proxy_async();
      group_sync();
      if (t == 0) {
        *cmd = grad ? 2 : 1;
        mbar_arrive(go_bar);
      }
      bool ok = true;
      float outacc = 0.f;
      for (int p = 0; p < nph; ++p) {
        const bool waited = mbar_wait(acc_bar, acc_par, a.status);
        acc_par ^= 1;
        if (group_or(!waited)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const bool fwd = p < D;
        const bool last_fwd = p == D - 1;
        if (p == 2 * D - 1) {
          // input gradient: g_i = acc[i] + acc[dp + i]
          float v[64];
          tmem_ld32(trow, v);
          if (dp > 16) tmem_ld32(trow + 32, v + 32);
          if (valid)
            for (int i = 0; i < a.d; ++i) a.st.gle[static_cast<size_t>(row) * a.st.gle_ld + i] = v[i] + v[dp + i];
        } else {
          const int l = fwd ? p + 1 : (2 * D - 1 - p) + 1;  // layer index (adjoint: the layer of W^T)
          const float *bias = fwd ? (l == 1 ? E.b1 : E.b + static_cast<size_t>(l - 2) * W) : nullptr;
          const __nv_bfloat16 *hprev =
              (!fwd && valid) ? E.scratch + static_cast<size_t>(row) * sstride + static_cast<size_t>(l - 2) * W : nullptr;
          __nv_bfloat16 *hkeep = (fwd && grad && !last_fwd && valid)
                                     ? E.scratch + static_cast<size_t>(row) * sstride + static_cast<size_t>(l - 1) * W
                                     : nullptr;
          const float c0 = -0.5f * E.out_s;
          for (int c32 = 0; c32 < W / 32; ++c32) {
            float v[32];
            tmem_ld32(trow + c32 * 32, v);
            if (fwd) {
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const int col = c32 * 32 + i;
                const float hv = tanhf(v[i] + bias[col]);
                if (last_fwd) {
                  const float wo = E.wo[col];
                  outacc = fmaf(wo, hv, outacc);
                  v[i] = c0 * wo * (1.f - hv * hv);
                } else {
                  v[i] = hv;
                }
              }
            } else {
              uint4 hb[4];
              if (hprev) {
                const uint4 *hp = reinterpret_cast<const uint4 *>(hprev + c32 * 32);
#pragma unroll
                for (int u = 0; u < 4; ++u) hb[u] = hp[u];
              } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) hb[u] = make_uint4(0, 0, 0, 0);
              }
              const __nv_bfloat16 *hh = reinterpret_cast<const __nv_bfloat16 *>(hb);
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const float hv = __bfloat162float(hh[i]);
                v[i] = v[i] * (1.f - hv * hv);
              }
            }
            // round to BF16, write the next operand (and keep h for the adjoint)
            if (!(last_fwd && !grad)) {
              uint32_t pk[16];
#pragma unroll
              for (int i = 0; i < 16; ++i) pk[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
              const int kb = c32 >> 1;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int jj = (c32 & 1) * 4 + u;
                st_shared_v4(act_addr + kb * 16384 + sw128_off(r, jj), pk[4 * u], pk[4 * u + 1], pk[4 * u + 2],
                             pk[4 * u + 3]);
              }
              if (hkeep) {
                uint4 *dst = reinterpret_cast<uint4 *>(hkeep + c32 * 32);
#pragma unroll
                for (int u = 0; u < 4; ++u) dst[u] = make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
              }
            }
          }
          if (last_fwd && valid) a.st.lle[row] = -0.5f * (E.out_s * (outacc + E.bo) + E.out_m);
        }
        fence_proxy_async();
        tc_fence_before();
        group_sync();
        if (t == 0 && p + 1 < nph) mbar_arrive(act_bar);
      }
      if (!ok) {
        // the MMA / producer roles time out on their own waits
        if (t == 0) {
          *cmd = 0;
          mbar_arrive(go_bar);
        }
        break;
      }
      bool done = false;
      if (need && !loglike) done = ch.post(row, h);
      if (!loglike && a.welford_on) {
        mask[r] = done ? 1 : 0;
        group_sync();
        if (group_or(done))
          welford_tile(a, blockIdx.x * kTcRows, min(kTcRows, a.n_rows - blockIdx.x * kTcRows), mask, t, 128,
                       [] { group_sync(); });
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(static_cast<uint32_t>(W))
                 : "memory");
  }
}

// Shared memory a launch needs (bytes) and the number of weight stages that fit.
inline int tc_stages_for(int width, int smem_cap) {
  const int act = (width / 64) * 16384;
  const int ctrl = 8 * (2 * kTcMaxStages + 6) + 4 * kTcRows + 64;
  int s = (smem_cap - 1024 - ctrl - act) / kTcStageBytes;
  if (s > kTcMaxStages) s = kTcMaxStages;
  return s;
}
inline size_t tc_smem_bytes(int width, int stages) {
  return 1024 + static_cast<size_t>(width / 64) * 16384 + static_cast<size_t>(stages) * kTcStageBytes +
         8 * (2 * stages + 6) + 4 * kTcRows + 64;
}

}  // namespace bst
