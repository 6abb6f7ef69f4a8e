// engine_tc2.cuh -- BF16 tcgen05 engine with the layer width split across a thread-block cluster.
//
// A tile of 128 chains is owned by a cluster of CS CTAs (CS = 1, 2 or 4).  CTA rank r of the
// cluster computes output columns [r NS, (r + 1) NS) of every layer (NS = W / CS):
//
//   warp 0      producer: streams this rank's pre-swizzled BF16 weight tiles (TR rows x 64)
//               into a ring of shared-memory stages with cp.async.bulk;
//   warp 1      MMA issuer: tcgen05.mma M=128, N=TR, K=16, BF16 -> FP32 accumulators in TMEM;
//   warps 2-9   epilogue: two warps per TMEM lane quadrant, each on half of the slice's
//               columns.  Warps 2-5 of rank 0 also run the per-chain samplers (one thread
//               per chain).
//
// Per layer every CTA holds the whole input activation (128 x W BF16, 128-byte-swizzled
// K-major) in shared memory, multiplies it by its slice of the weights (its own K blocks
// first), runs the epilogue on its NS columns, writes the BF16 result into its own
// activation buffer and copies that slice into every peer's buffer: in clusters of 4 through
// a global image of the slice and one global->shared bulk copy per peer and 4 KB piece,
// otherwise with shared->shared bulk copies (completion counted on the peer's mbarrier).  A
// peer's buffer is written only after the peer's MMAs of the layer have finished reading it
// ("free" arrivals).  The output dot w_o . h_D is reduced across the cluster in a fixed
// order on rank 0.  All waits are bounded by a time limit; a timeout sets a status bit and
// every role leaves its loop; a cluster barrier precedes exit so no CTA leaves while a peer
// may still touch its shared memory.
#pragma once

#include "common.cuh"
#include "engine_simt.cuh"
#include "engine_tc.cuh"
#include "sampler.cuh"

namespace bst {

constexpr int kTc2EQ = 2;                       // epilogue warps per TMEM lane quadrant
constexpr int kTc2EpiThreads = 128 * kTc2EQ;    // 256
constexpr int kTc2Threads = 64 + kTc2EpiThreads;  // producer warp, MMA warp, epilogue warps

// Configurations whose stored activations h_1..h_{D-1} live in tensor memory (after the
// accumulator columns, this rank's NS columns as BF16 pairs) instead of global scratch, and the
// deepest network that fits there.
__host__ __device__ constexpr bool tc2_h_in_tmem(int W, int CS) { return (W == 512 && CS == 4) || (W == 256 && CS >= 2); }
__host__ __device__ constexpr int tc2_tcols(int W, int CS) { return W / CS < 64 ? 64 : W / CS; }
__host__ __device__ constexpr int tc2_tmem_max_depth(int W, int CS) {
  return tc2_h_in_tmem(W, CS) ? (512 - tc2_tcols(W, CS)) / (W / CS / 2) + 1 : 1 << 20;
}
// K blocks per weight stage: with 128-column slices (16 KB per K block) two consecutive K
// blocks, which are contiguous in the weight streams, share one copy and one barrier, so the
// MMA thread waits once per eight MMAs instead of once per four.
__host__ __device__ constexpr int tc2_stage_kblocks(int W, int CS) { return (W == 512 && CS == 4) ? 2 : 1; }

struct Tc2Weights {
  int depth, width, dp, kb1, k16_l1;
  int cs;             // cluster size
  const uint8_t *l1;  // [cs] streams of layer-1 tiles (this launch's fold set)
  size_t l1_stride;   // bytes per rank
  const uint8_t *hid; // [cs] streams: hidden forward tiles then adjoint tiles
  size_t hid_stride;
  const uint8_t *g1;  // input-gradient tiles (shared by all ranks)
  const float *b1;    // [w]
  const float *b;     // [D-1][w]
  const float *wo;    // [w]
  float bo, out_m, out_s;
  int out_log;        // chi2 = out_floor + exp(out_s out + out_m) instead of out_s out + out_m
  float out_floor;
  int f16;            // operands FP16 instead of BF16; the adjoint is then seeded with
                      // -w_o (1 - h_D^2) / 2 and the input gradient scaled by out_s
  __nv_bfloat16 *scratch;  // [rows][D-1][w] stored activations (unless in tensor memory)
  uint8_t *xchg;           // [CTAs][128 x NS BF16] slice images of the cluster exchange
  size_t xchg_bytes;
  int n_stages;
};

// ---------------------------------------------------------------- cluster helpers
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(d) : "r"(saddr), "r"(rank));
  return d;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];\n" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, int *status) {
  for (int i = 0; i < 256; ++i)
    if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kWaitLimitNs) {
      set_status(status, kStatusTimeout);
      return false;
    }
  }
}
// Bounded wait that backs off between polls: for threads that wait while the tensor pipe
// runs, whose shared-memory operand reads would otherwise compete with every poll.
__device__ __forceinline__ bool mbar_wait_backoff(uint32_t bar, uint32_t parity, int *status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    __nanosleep(128);
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kWaitLimitNs) {
      set_status(status, kStatusTimeout);
      return false;
    }
  }
}
__device__ __forceinline__ void bulk_s2cluster(uint32_t dst_cluster, uint32_t src_cta, uint32_t bytes,
                                               uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          dst_cluster),
      "r"(src_cta), "r"(bytes), "r"(bar_cluster)
      : "memory");
}
// Arrive on the barrier at `bar`'s offset in every CTA of `mask` once this thread's
// tcgen05 operations issued so far have completed.
__device__ __forceinline__ void mma_commit_multicast(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n" ::"r"(bar),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;\n" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
}
__device__ __forceinline__ void st_cluster_v4f(uint32_t addr, float x, float y, float z, float w) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(x), "f"(y), "f"(z), "f"(w)
               : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;\n" ::: "memory"); }
__device__ __forceinline__ bool epi_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 256, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred ? 1u : 0u)
      : "memory");
  return r != 0;
}
// sampler subgroup (warps 2-5): named barrier 2
__device__ __forceinline__ void smp_sync() { asm volatile("bar.sync 2, 128;\n" ::: "memory"); }
__device__ __forceinline__ bool smp_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 2, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred ? 1u : 0u)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;\n" : "=f"(y) : "f"(x));
  return y;
}
// tanh for the last hidden layer, which feeds the FP32 output dot: the identity
// tanh x = 1 - 2 / (exp(2x) + 1) with the hardware exponential and a fast division.  The
// absolute error stays at a few 1e-7 over the whole range (the relative error of exp(2x) is
// at most about 2e-6 for |x| <= 15 and enters as at most half of it); |x| > 15 rounds to +-1.
__device__ __forceinline__ float tanh_out(float x) {
  const float xc = fminf(fmaxf(x, -15.f), 15.f);
  const float e = __expf(2.f * xc);
  return 1.f - __fdividef(2.f, e + 1.f);
}
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Makes r depend on a preceding tcgen05.wait::ld (both statements are volatile, so they stay
// in order and later reads of r see the loaded values).
__device__ __forceinline__ void tmem_after_wait16(uint32_t *r) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
// Wait for outstanding tcgen05.ld and make the destination registers depend on the wait, so
// the compiler cannot read them before the data has arrived.
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t *r) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;\n"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
        "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
        "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
        "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
      :
      : "memory");
}

// ---------------------------------------------------------------- the kernel
// L2X: cluster exchange through global slice images and global->shared copies into each peer
// (clusters of 4 with room for the images), else direct shared->shared copies.  RC: MALA / MH / HMC with d <= 8
// (padded to 16), whose chains live in the sampler threads' registers (RegChain8); else the
// general per-chain code (Chain) or loglike mode.
template <int W, int CS, bool L2X, bool RC>
__global__ void __launch_bounds__(kTc2Threads, 1) tc2_chain_kernel(const __grid_constant__ StepArgs<float> a,
                                                                   const __grid_constant__ Tc2Weights E) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  constexpr int KBW = W / 64;           // K blocks of the hidden width
  constexpr int NS = W / CS;            // output columns of this rank
  constexpr int TR = NS < 256 ? NS : 256;  // rows of a weight tile == MMA N
  constexpr int NSUB = NS / TR;
  constexpr int KT = TR * 128;                  // bytes of a weight tile (one K block)
  constexpr int G = tc2_stage_kblocks(W, CS);   // K blocks per stage
  constexpr int STAGE = G * KT;
  constexpr int SLICE_BYTES = 128 * NS * 2;  // one rank's slice of an activation
  constexpr int TCOLS = NS < 64 ? 64 : NS;   // TMEM columns (>= 2 dp for the input gradient)
  constexpr int CW = NS / kTc2EQ;            // slice columns per epilogue warp
  constexpr int CPW = CW / 32;               // 32-column chunks per epilogue warp
  constexpr int NOWN = NS / 64;              // K blocks of a layer input this rank computed itself
  // each epilogue warp sends its own rows x columns to the peers as soon as they are written
  // (whole 64-column K blocks: 32 rows of a K block are 4 KB contiguous in the swizzled layout)
  constexpr bool kWarpSend = CS > 1 && CW % 64 == 0;
  // One CTA per tile with the layer in two MMA halves (N = TR = NS / 2): the epilogue warps
  // take the columns in quarters (each warp its share of a quarter, two chunks) and signal a
  // barrier after the first half and one after the third quarter, so the next layer's MMAs on
  // K blocks 0 .. KBW / 2 - 1, then on the third quarter's K blocks, run while the epilogue
  // works on the rest (the MMAs of the first N half overwrite only tensor-memory columns of the
  // first half, read by then).
  constexpr bool kHalfFirst = (CS == 1) && (NSUB == 2);
  constexpr int kQC = CPW >= 4 ? CPW / 4 : 1;  // chunks of a warp per quarter (kHalfFirst)
  static_assert(!kHalfFirst || (CPW % 4 == 0 && kQC * 32 * kTc2EQ == TR / 2), "quarter chunk order");
  // the barrier checks of the MMA thread (own K blocks, quarters) fall on stage boundaries
  static_assert(G == 1 || (!kHalfFirst && NOWN % G == 0 && KBW % G == 0), "K blocks per stage");

  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *act = base;
  uint8_t *stages = act + KBW * 16384;
  const int S = E.n_stages;
  uint64_t *bars = reinterpret_cast<uint64_t *>(stages + S * STAGE);
  // bars: full[S] empty[S] go act_full acc fin peer_free part peer_free_last (cmd tmem) own own_h0
  //       own_q2
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
  const uint32_t go_bar = smem_u32(bars + 2 * S), actf_bar = smem_u32(bars + 2 * S + 1);
  const uint32_t acc_bar = smem_u32(bars + 2 * S + 2), fin_bar = smem_u32(bars + 2 * S + 3);
  const uint32_t free_bar = smem_u32(bars + 2 * S + 4), part_bar = smem_u32(bars + 2 * S + 5);
  const uint32_t free2_bar = smem_u32(bars + 2 * S + 6);
  volatile int *cmd = reinterpret_cast<volatile int *>(bars + 2 * S + 7);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 8);
  // own slice of the next layer input written (the peers' slices complete act_full)
  const uint32_t own_bar = smem_u32(bars + 2 * S + 9);
  // first half / first three quarters of the columns written (kHalfFirst)
  const uint32_t own_h0_bar = smem_u32(bars + 2 * S + 10);
  const uint32_t own_q2_bar = smem_u32(bars + 2 * S + 11);
  // everything from `partial` on is 16-byte aligned for vector access
  float *partial = reinterpret_cast<float *>(bars + 2 * S + 12);  // [CS][128] (rank 0 gathers)
  float *red = partial + CS * 128;                                // [EQ-1][128] column-group combine
  int *mask = reinterpret_cast<int *>(red + (kTc2EQ - 1) * 128);  // [128]
  float *sbias = reinterpret_cast<float *>(mask + 128);           // [D + 1][NS]: b_1..b_D, w_o slices
  // register-resident chains (rank 0 writes them): [128][8] proposals (every rank), then on
  // rank 0 [128][8] grad logL at the proposals and [128][8] the next proposal's noise
  float *zbuf = sbias + (E.depth + 1) * NS;
  float *gbuf = zbuf + 128 * 8;
  float *xibuf = gbuf + 128 * 8;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = (CS > 1) ? cluster_rank() : 0u;
  const int tile = blockIdx.x / CS;
  const int D = E.depth, dp = E.dp;
  const bool grad = a.need_grad != 0;
  const int nph = tc_num_phases(D, grad);
  // The activations h_1..h_{D-1} that the adjoint pass needs stay in tensor memory after the
  // accumulator columns (this rank's NS columns, BF16 pairs) in the configurations of
  // tc2_h_in_tmem (the launch keeps the depth within tc2_tmem_max_depth), else in global
  // scratch.
  constexpr bool h_tmem = tc2_h_in_tmem(W, CS);
  // In clusters of 4, given room for them (E.xchg), each CTA also writes its slice of a layer
  // output to global memory (a byte image of its shared-memory slice, which stays in L2) and
  // every epilogue warp sends its part to each of the three peers with a global->shared bulk
  // copy instead of a shared->shared copy (with a single peer the direct copy is faster).
  constexpr bool l2x = L2X && kWarpSend && CS == 4;
  const uint32_t tcols_alloc = h_tmem ? 512u : static_cast<uint32_t>(TCOLS);
  // the launch picks a cluster size whose stored activations fit, and sizes the scratch for
  // the exchange images; never taken
  if (D > tc2_tmem_max_depth(W, CS) ||
      (l2x && (E.xchg == nullptr || static_cast<size_t>(gridDim.x) * SLICE_BYTES > E.xchg_bytes))) {
    if (threadIdx.x == 0) set_status(a.status, kStatusBadArg);
    return;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(go_bar, 1);
    mbar_init(actf_bar, 1);
    mbar_init(acc_bar, 1);
    mbar_init(fin_bar, 1);
    mbar_init(free_bar, CS > 1 ? CS - 1 : 1);
    mbar_init(part_bar, CS);
    mbar_init(free2_bar, CS > 1 ? CS - 1 : 1);
    mbar_init(own_bar, kTc2EpiThreads / 32);  // one arrive per epilogue warp
    mbar_init(own_h0_bar, kTc2EpiThreads / 32);
    mbar_init(own_q2_bar, kTc2EpiThreads / 32);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(tcols_alloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  {
    const int c0g = static_cast<int>(rank) * NS;
    for (int i = threadIdx.x; i < (D + 1) * NS; i += kTc2Threads) {
      const int l = i / NS, j = c0g + i % NS;  // l = 0..D-1: bias of layer l+1; l = D: w_o
      sbias[i] = (l == 0) ? E.b1[j] : (l < D ? E.b[static_cast<size_t>(l - 1) * W + j] : E.wo[j]);
    }
    for (int i = threadIdx.x; i < 3 * 128 * 8; i += kTc2Threads) zbuf[i] = 0.f;
  }
  tc_fence_before();
  __syncthreads();
  if (CS > 1) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      // bit s of fpar: parity of the fills of stage s so far; bit s of used: stage s filled
      uint32_t fpar = 0, used = 0, go_par = 0;
      int s = 0;
      bool ok = true;
      const uint8_t *l1 = E.l1 + rank * E.l1_stride;
      const uint8_t *hid = E.hid + rank * E.hid_stride;
      // layers after the first start at this rank's own K blocks (ready before the peers')
      const int rot = static_cast<int>(rank) * NOWN;
      while (ok) {
        if (!mbar_wait_cluster(go_bar, go_par, a.status)) break;
        go_par ^= 1;
        const int c = *cmd;
        if (c == 0) break;
        const int phases = tc_num_phases(D, c == 2);
        for (int p = 0; p < phases && ok; ++p) {
          const bool last = (p == 2 * D - 1);
          const int nsub = last ? 1 : NSUB;
          const int nkb = (p == 0) ? E.kb1 : KBW;
          const uint32_t bytes = last ? 2 * dp * 128 : KT;  // per K block
          for (int sb = 0; sb < nsub && ok; ++sb) {
            int kb = (p == 0) ? 0 : rot;
            for (int j = 0; j < nkb;) {
              // K blocks kb .. kb + g - 1 in one stage (the rotation never splits a stage)
              const int g = min(G, min(nkb - j, nkb - kb));
              const uint8_t *src;
              if (p == 0) src = l1 + static_cast<size_t>(sb * nkb + kb) * KT;
              else if (!last) src = hid + (static_cast<size_t>(p - 1) * NSUB * KBW + sb * KBW + kb) * KT;
              else src = E.g1 + static_cast<size_t>(kb) * bytes;
              if (!mbar_wait(empty0 + 8 * s, ((fpar >> s) & 1u) ^ 1u, a.status)) {
                ok = false;
                break;
              }
              mbar_expect_tx(full0 + 8 * s, g * bytes);
              bulk_g2s(smem_u32(stages + s * STAGE), src, g * bytes, full0 + 8 * s);
              fpar ^= 1u << s;
              used |= 1u << s;
              s = (s + 1 == S) ? 0 : s + 1;
              j += g;
              kb = (kb + g == nkb) ? 0 : kb + g;
            }
          }
        }
      }
      for (int q2 = 0; q2 < S; ++q2)
        if ((used >> q2) & 1u) mbar_wait(full0 + 8 * q2, ((fpar >> q2) & 1u) ^ 1u, a.status);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t upar = 0;  // bit s: parity of the next wait on stage s
      int s = 0;
      uint32_t go_par = 0, act_par = 0, own_par = 0, own_h0_par = 0, own_q2_par = 0;
      bool ok = true;
      const uint32_t idn = idesc_bf16(128, TR, E.f16 != 0), idg = idesc_bf16(128, 2 * dp, E.f16 != 0);
      // descriptors of K block 0 of the activation and of stage 0; K block kb / stage s / its
      // i-th K block / the k-th 16-wide step are offsets of kb * 16384, s * STAGE, i * kbytes
      // and k * 32 bytes (address >> 4)
      const uint64_t adesc0 = sw128_desc(smem_u32(act)), bdesc0 = sw128_desc(smem_u32(stages));
      const int rot = static_cast<int>(rank) * NOWN;  // own K blocks first (as the producer)
      const uint16_t peer_mask = static_cast<uint16_t>(((1u << CS) - 1u) & ~(1u << rank));
      while (ok) {
        if (!mbar_wait_cluster(go_bar, go_par, a.status)) break;
        go_par ^= 1;
        const int c = *cmd;
        if (c == 0) break;
        const int phases = tc_num_phases(D, c == 2);
        for (int p = 0; p < phases && ok; ++p) {
          // the whole layer input (layer 1), or its first half of the columns (kHalfFirst)
          const bool split = kHalfFirst && p > 0;
          if (!mbar_wait(split ? own_h0_bar : own_bar, split ? own_h0_par : own_par, a.status)) {
            ok = false;
            break;
          }
          if (split)
            own_h0_par ^= 1;
          else
            own_par ^= 1;
          tc_fence_after();
          const bool last = (p == 2 * D - 1);
          const int nsub = last ? 1 : NSUB;
          const int nkb = (p == 0) ? E.kb1 : KBW;
          const uint32_t id = last ? idg : idn;
          const int kbytes = last ? 2 * dp * 128 : KT;  // bytes of one K block in a stage
          for (int sb = 0; sb < nsub && ok; ++sb) {
            int kb = (p == 0) ? 0 : rot;
            const uint32_t dcol = tmem + sb * TR;
            for (int j = 0; j < nkb;) {
              // the producer's stage split: K blocks kb .. kb + g - 1 in stage s
              const int g = min(G, min(nkb - j, nkb - kb));
              if (split && sb == 0 && j == KBW / 2) {
                // the third quarter of the layer input
                if (!mbar_wait(own_q2_bar, own_q2_par, a.status)) {
                  ok = false;
                  break;
                }
                own_q2_par ^= 1;
                tc_fence_after();
              }
              if (split && sb == 0 && j == 3 * KBW / 4) {
                // the last quarter
                if (!mbar_wait(own_bar, own_par, a.status)) {
                  ok = false;
                  break;
                }
                own_par ^= 1;
                tc_fence_after();
              }
              if (CS > 1 && p > 0 && j == NOWN) {
                // the peers' slices of this layer input have landed
                if (!mbar_wait_cluster(actf_bar, act_par, a.status)) {
                  ok = false;
                  break;
                }
                act_par ^= 1;
                tc_fence_after();
              }
              if (!mbar_wait(full0 + 8 * s, (upar >> s) & 1u, a.status)) {
                ok = false;
                break;
              }
              upar ^= 1u << s;
              tc_fence_after();
              for (int i = 0; i < g; ++i) {
                const uint64_t ad = adesc0 + static_cast<uint64_t>((kb + i) * (16384 >> 4));
                const uint64_t bd = bdesc0 + static_cast<uint64_t>((s * STAGE + i * kbytes) >> 4);
                const int k16 = (p == 0) ? min(4, E.k16_l1 - 4 * (kb + i)) : 4;
                for (int k = 0; k < k16; ++k)
                  mma_bf16(dcol, ad + 2 * k, bd + 2 * k, id, (j + i > 0 || k > 0) ? 1u : 0u);
              }
              mma_commit(empty0 + 8 * s);
              s = (s + 1 == S) ? 0 : s + 1;
              j += g;
              kb = (kb + g == nkb) ? 0 : kb + g;
            }
          }
          if (ok) {
            mma_commit(acc_bar);
            // once these MMAs are done our activation buffer may be overwritten by the peers,
            // and every slice they sent us for this phase has landed (the last phase of an
            // evaluation signals a barrier of its own, so neither barrier runs two phases ahead)
            if (CS > 1) mma_commit_multicast(p + 1 < phases ? free_bar : free2_bar, peer_mask);
          }
        }
      }
      mma_commit(fin_bar);
      mbar_wait(fin_bar, 0, a.status);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (+ samplers on rank 0)
    const int e = warp - 2;              // 0..4 EQ - 1
    const int q = warp & 3;              // TMEM lane quadrant
    const int ch = e >> 2;               // column group of the slice
    const int r = q * 32 + lane;         // tile row == TMEM lane
    const int row = tile * kTcRows + r;
    const bool valid = row < a.n_rows;
    const int t = e * 32 + lane;         // index within the epilogue group
    const bool sampler = (rank == 0) && (ch == 0);
    const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16);
    const uint32_t act_addr = smem_u32(act);
    const int col0 = static_cast<int>(rank) * NS + ch * CW;  // first global column of this warp
    // column of chunk cc of this warp within the rank's slice: CW consecutive columns, or
    // (kHalfFirst) its share of each quarter of the columns in turn
    auto chunk_col = [&](int cc) -> int {
      if constexpr (kHalfFirst) return (cc / kQC) * (TR / 2) + ch * (TR / 2 / kTc2EQ) + (cc % kQC) * 32;
      else return ch * CW + cc * 32;
    };
    Chain<float> chn(a);
    const bool loglike = a.mode == kModeLoglike;
    // this CTA's global image of its slice (l2x)
    uint8_t *ximg = E.xchg + static_cast<size_t>(blockIdx.x) * SLICE_BYTES;
    const bool mala = a.mode == kModeMALA, hmc = a.mode == kModeHMC;
    // MALA / MH / HMC with d <= 8 (padded to 16) keep the chain in the sampler thread's registers
    constexpr bool fast = RC;
    RegChain8<float> rc;
    if (fast && sampler && valid) rc.load(a, row, zbuf + r * 8, gbuf + r * 8, xibuf + r * 8);
    if (sampler && valid && !loglike) {
      if (is_ensemble_mode(a.mode)) {
        for (int h = 0; h < 2; ++h) a.st.steps_done[chn.aies_walker(row, h)] = 0;
      } else {
        a.st.steps_done[row] = 0;
        if (a.mode == kModeHMC) chn.dw(row)[0] = 0.0;
        if (is_nuts_mode(a.mode)) chn.dw(row)[0] = 1.0;
      }
    }
    epi_sync();
    uint32_t acc_par = 0, go_par = 0, free_par = 0, free2_par = 0, part_par = 0;
    // The peers' MMAs of a phase release our activation buffer (free_bar).  The epilogue of a
    // distributing phase waits for that before writing the buffer; the release of an
    // evaluation's last phase (free2_bar) is taken before the next layer-1 operand is written
    // (or at exit).
    bool free_pending = false;
    auto wait_free = [&](uint32_t bar, uint32_t &par) -> bool {
      int got = 1;
      if (lane == 0) got = mbar_wait_cluster(bar, par, a.status) ? 1 : 0;
      par ^= 1;
      return __shfl_sync(0xffffffffu, got, 0) != 0;
    };
    const size_t sstride = static_cast<size_t>(D > 1 ? D - 1 : 1) * W;
    const bool f16 = E.f16 != 0;
    // adjoint seed scale (FP16: without out_s, applied to the input gradient instead, so the
    // adjoint vectors stay far from the FP16 range limit whatever the output scale)
    const float c0 = f16 ? -0.5f : -0.5f * E.out_s;
    for (int ev = 0;; ++ev) {
      const int h = ev & 1;
      bool need = false;
      // ---- proposal (rank 0) and the go signal to every CTA of the cluster
      if (rank == 0) {
        if (ev > 0) epi_sync();  // a proposal may read positions other threads just accepted (AIES)
        if (sampler) {
          if (loglike) need = valid && ev == 0;
          else need = valid && (fast ? (hmc ? rc.hmc_pre(a, row) : rc.pre(a, row, mala)) : chn.pre(row, h));
          if (fast && need && CS > 1) {
            // the proposal (already in this rank's staging buffer) goes straight into every
            // peer's operand staging buffer
            const uint32_t zb = smem_u32(zbuf + r * 8);
            const float4 z0 = *reinterpret_cast<const float4 *>(zbuf + r * 8);
            const float4 z1 = *reinterpret_cast<const float4 *>(zbuf + r * 8 + 4);
            for (int pr = 1; pr < CS; ++pr) {
              const uint32_t dst = mapa(zb, static_cast<uint32_t>(pr));
              st_cluster_v4f(dst, z0.x, z0.y, z0.z, z0.w);
              st_cluster_v4f(dst + 16, z1.x, z1.y, z1.z, z1.w);
            }
          }
        }
        const bool any = epi_or(need);
        if (t < CS) {  // thread t signals rank t (the release arrives run in parallel)
          const int c = any ? (grad ? 2 : 1) : 0;
          st_cluster_u32(mapa(smem_u32(const_cast<int *>(cmd)), t), static_cast<uint32_t>(c));
          mbar_arrive_cluster(mapa(go_bar, t));
        }
      }
      if (!mbar_wait_cluster(go_bar, go_par, a.status)) break;
      go_par ^= 1;
      const int c = *cmd;
      if (c == 0) break;
      if (free_pending) {
        wait_free(free2_bar, free2_par);  // a timeout is recorded in the status word
        free_pending = false;
      }
      // ---- layer-1 operand [z_hi | z_lo | z_hi | 0] from ze (written by rank 0's samplers)
      if (fast && E.kb1 == 1) {
        // dp == 16, d <= 8: chunks of 8 values are hi(z), 0, lo(z), 0 (this thread, ch 0) or
        // hi(z), 0, 0, 0 (ch 1); z beyond d is zero in the staging buffer
        const float4 za = *reinterpret_cast<const float4 *>(zbuf + r * 8);
        const float4 zb = *reinterpret_cast<const float4 *>(zbuf + r * 8 + 4);
        const float zv[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
        uint32_t hi2[4], lo2[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float h0 = op_round(zv[2 * u], f16);
          const float h1 = op_round(zv[2 * u + 1], f16);
          hi2[u] = pack_op2(h0, h1, f16);
          lo2[u] = pack_op2(zv[2 * u] - h0, zv[2 * u + 1] - h1, f16);
        }
        const int j0 = 4 * ch;
        st_shared_v4(act_addr + sw128_off(r, j0), hi2[0], hi2[1], hi2[2], hi2[3]);
        st_shared_v4(act_addr + sw128_off(r, j0 + 1), 0u, 0u, 0u, 0u);
        if (ch == 0) st_shared_v4(act_addr + sw128_off(r, j0 + 2), lo2[0], lo2[1], lo2[2], lo2[3]);
        else st_shared_v4(act_addr + sw128_off(r, j0 + 2), 0u, 0u, 0u, 0u);
        st_shared_v4(act_addr + sw128_off(r, j0 + 3), 0u, 0u, 0u, 0u);
      } else {
        const float *zr = fast ? zbuf + r * 8 : a.st.ze + row_off(a.st.ze_ld, row, a.dp);
        const int zes = fast ? 1 : row_es(a.st.ze_ld);
        const int nch = E.kb1 * 8;  // 16-byte chunks in the row; dp is a multiple of 16, so a
                                    // chunk (8 values) lies inside one segment
        for (int j = ch * (nch / kTc2EQ); j < (ch + 1) * (nch / kTc2EQ); ++j) {
          const int seg = (j * 8) / dp, i0 = j * 8 - seg * dp;
          float v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = i0 + u;
            const float zval = (valid && seg < 3 && i < a.d) ? zr[i * zes] : 0.f;
            const float hi = op_round(zval, f16);
            v[u] = (seg == 1) ? (zval - hi) : hi;
          }
          st_shared_v4(act_addr + (j >> 3) * 16384 + sw128_off(r, j & 7), pack_op2(v[0], v[1], f16),
                       pack_op2(v[2], v[3], f16), pack_op2(v[4], v[5], f16), pack_op2(v[6], v[7], f16));
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(own_bar);  // the whole layer-1 operand is local
      bool ok = true;
      for (int p = 0; p < nph; ++p) {
        // while the second layer is in flight the chain does the evaluation-independent part
        // of its accept step and draws the next proposal's noise
        if (p == 1 && fast && sampler && valid) {
          rc.record(a, row, row);  // the previous iteration's memory side, if still pending
          if (need) {
            rc.prep(a, row);
            rc.prep_next(a, row);
          }
        }
        // adjoint phases read the stored activation h_{l-1}: start loading its first chunk now
        const bool adj_phase = (p >= D) && (p != 2 * D - 1);
        const __nv_bfloat16 *hprev =
            (adj_phase && valid && !h_tmem)
                ? E.scratch + static_cast<size_t>(row) * sstride + static_cast<size_t>(2 * D - p - 2) * W
                : nullptr;
        uint4 hcur[4];
        {
          const uint4 *hp =
              hprev ? reinterpret_cast<const uint4 *>(hprev + static_cast<int>(rank) * NS + chunk_col(0)) : nullptr;
#pragma unroll
          for (int u = 0; u < 4; ++u) hcur[u] = hp ? __ldcs(hp + u) : make_uint4(0, 0, 0, 0);
        }
        // one poller per warp, backing off, while the MMAs of the phase run
        int wok = 1;
        if (lane == 0) wok = mbar_wait_backoff(acc_bar, acc_par, a.status) ? 1 : 0;
        const bool waited = __shfl_sync(0xffffffffu, wok, 0) != 0;
        acc_par ^= 1;
        if (epi_or(!waited)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const bool fwd = p < D;
        const bool last_fwd = p == D - 1;
        const bool distribute = (p + 1 < nph);  // this phase's output feeds another phase
        if (p == 2 * D - 1) {
          // input gradient: g_i = acc[i] + acc[dp + i] (every rank computes it, rank 0 writes)
          if (ch == 0) {
            uint32_t v0[32], v1[32];
            tmem_ld32_nowait(trow, v0);
            if (dp > 16) tmem_ld32_nowait(trow + 32, v1);
            tmem_wait_ld();
            if (rank == 0 && valid && fast) {
              // (the register-resident chain takes the gradient from shared memory only)
#pragma unroll
              for (int i = 0; i < RegChain8<float>::DB; ++i)
                if (i < a.d) rc.gp[i] = __uint_as_float(v0[i]) + __uint_as_float(v0[16 + i]);  // dp == 16
            } else if (rank == 0 && valid) {
              float *gout = a.st.gle + row_off(a.st.gle_ld, row, a.dp);
              const int ges = row_es(a.st.gle_ld);
              for (int i = 0; i < a.d; ++i) {
                const int j2 = dp + i;
                const float hi = __uint_as_float(v0[i]);
                const float lo = __uint_as_float(j2 < 32 ? v0[j2] : v1[j2 - 32]);
                gout[i * ges] = hi + lo;
              }
            }
          }
        } else {
          const int l = fwd ? p + 1 : 2 * D - p;  // layer index (adjoint: layer whose W^T is applied)
          const float *bias = fwd ? sbias + (l - 1) * NS : nullptr;  // this rank's columns
          const float *wos = sbias + D * NS;
          __nv_bfloat16 *hkeep = (fwd && grad && !last_fwd && valid)
                                     ? E.scratch + static_cast<size_t>(row) * sstride + static_cast<size_t>(l - 1) * W
                                     : nullptr;
          float part = 0.f;
#pragma unroll 1
          for (int cc = 0; cc < CPW; ++cc) {
            const int tcol = chunk_col(cc);                         // TMEM column
            const int gcol = static_cast<int>(rank) * NS + tcol;    // global column of the chunk
            uint32_t raw[32];
            tmem_ld32_nowait(trow + tcol, raw);
            // stored activation h_{l-1} of these columns (tensor-memory copy)
            uint32_t hv16[16];
            const bool ht = adj_phase && h_tmem;
            if (ht) tmem_ld16_nowait(trow + TCOLS + (2 * D - p - 2) * (NS / 2) + (tcol >> 1), hv16);
            tmem_wait_ld_regs(raw);
            if (ht) tmem_after_wait16(hv16);
            float aux[32];
            uint4 hnext[4];
            if (fwd) {
              const float4 *bp = reinterpret_cast<const float4 *>(bias + tcol);
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const float4 b4 = bp[u];
                aux[4 * u] = b4.x;
                aux[4 * u + 1] = b4.y;
                aux[4 * u + 2] = b4.z;
                aux[4 * u + 3] = b4.w;
              }
            } else if (ht) {
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                aux[2 * i] = op_lo(hv16[i], f16);      // low half: even column
                aux[2 * i + 1] = op_hi(hv16[i], f16);  // high half: odd column
              }
            } else {
              // stored activations of this chunk were loaded one chunk ahead; start the next one
              const bool more = hprev && cc + 1 < CPW;
              const uint4 *hp =
                  more ? reinterpret_cast<const uint4 *>(hprev + static_cast<int>(rank) * NS + chunk_col(cc + 1)) : nullptr;
#pragma unroll
              for (int u = 0; u < 4; ++u) hnext[u] = more ? __ldcs(hp + u) : make_uint4(0, 0, 0, 0);
              const uint32_t *hh = reinterpret_cast<const uint32_t *>(hcur);
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                aux[2 * i] = op_lo(hh[i], f16);
                aux[2 * i + 1] = op_hi(hh[i], f16);
              }
            }
            if (!fwd) {
#pragma unroll
              for (int u = 0; u < 4; ++u) hcur[u] = hnext[u];
            }
            float v[32];
            if (fwd) {
              if (last_fwd) {
                const float4 *wp = reinterpret_cast<const float4 *>(wos + tcol);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  const float4 w4 = wp[u];
                  const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                  for (int k = 0; k < 4; ++k) {
                    const int i = 4 * u + k;
                    // the last hidden layer feeds the FP32 output dot: accurate tanh
                    const float hv = tanh_out(__uint_as_float(raw[i]) + aux[i]);
                    part = fmaf(wv[k], hv, part);
                    v[i] = c0 * wv[k] * (1.f - hv * hv);
                  }
                }
              } else if (f16) {
                // FP16 keeps 11 significant bits: tanh.approx (about 2^-11 relative error) would
                // dominate its rounding, so the accurate form is used
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = tanh_out(__uint_as_float(raw[i]) + aux[i]);
              } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = tanh_fast(__uint_as_float(raw[i]) + aux[i]);
              }
            } else {
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(raw[i]) * (1.f - aux[i] * aux[i]);
            }
            if (distribute) {
              uint32_t pk[16];
#pragma unroll
              for (int i = 0; i < 16; ++i) pk[i] = pack_op2(v[2 * i], v[2 * i + 1], f16);
              // before the first write into the activation buffer: the peers' MMAs of this
              // phase are done with it (the first chunk's math overlaps the wait)
              if (CS > 1 && cc == 0 && !wait_free(free_bar, free_par)) ok = false;
              const int kb = gcol >> 6;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int jj = ((gcol & 63) >> 3) + u;
                st_shared_v4(act_addr + kb * 16384 + sw128_off(r, jj), pk[4 * u], pk[4 * u + 1], pk[4 * u + 2],
                             pk[4 * u + 3]);
                if (l2x)
                  *reinterpret_cast<uint4 *>(ximg + (kb - static_cast<int>(rank) * NOWN) * 16384 + sw128_off(r, jj)) =
                      make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
              }
              if (fwd && grad && !last_fwd && h_tmem) {
                tmem_st16(trow + TCOLS + p * (NS / 2) + (tcol >> 1), pk);
              } else if (hkeep) {
                // streaming accesses: the stored activations are read once, by the adjoint
                // pass, and should not displace the samplers' working set from L1
                uint4 *dst = reinterpret_cast<uint4 *>(hkeep + gcol);
#pragma unroll
                for (int u = 0; u < 4; ++u) __stcs(dst + u, make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]));
              }
            }
            if (kHalfFirst && distribute && (cc == 2 * kQC - 1 || cc == 3 * kQC - 1)) {
              // this warp's chunks of the first half (then of the third quarter) are read from
              // tensor memory and written to the next layer's operand: the MMAs on those K
              // blocks may start
              fence_proxy_async();
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(cc == 2 * kQC - 1 ? own_h0_bar : own_q2_bar);
            }
          }
          if (fwd && grad && !last_fwd && h_tmem) tmem_wait_st();
          if (last_fwd) {
            // per-row partial of w_o . h_D over this rank's columns, gathered on rank 0
            if (ch > 0) red[(ch - 1) * 128 + r] = part;
            epi_sync();
            if (ch == 0) {
              float tot = part;
              for (int g2 = 1; g2 < kTc2EQ; ++g2) tot += red[(g2 - 1) * 128 + r];
              st_cluster_f32(mapa(smem_u32(partial + rank * 128 + r), 0), tot);
            }
            epi_sync();
            if (t == 0) mbar_arrive_cluster(mapa(part_bar, 0));
          }
        }
        if (distribute) {
          // this warp's part of the own slice is written: the next layer's MMAs on the own K
          // blocks may start (one arrive per warp)
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(own_bar);
          if (CS > 1 && t == 0) mbar_expect_tx(actf_bar, (CS - 1) * SLICE_BYTES);  // the peers' slices
          if (l2x) {
            // this warp's rows (32 q ..) of its K blocks, from the global image into every
            // peer's buffer at the same place (one copy per peer and 4 KB, read from L2)
            fence_proxy_async_global();
            __syncwarp();
            if (lane == 0 && ok)
              for (int kb2 = 0; kb2 < CW / 64; ++kb2) {
                const int kbl = col0 / 64 + kb2;
                const uint32_t dst = act_addr + static_cast<uint32_t>(kbl) * 16384 + q * 4096;
                const uint8_t *src = ximg + (kbl - static_cast<int>(rank) * NOWN) * 16384 + q * 4096;
                for (int pr = 0; pr < CS; ++pr)
                  if (pr != static_cast<int>(rank)) bulk_g2s(mapa(dst, pr), src, 4096, mapa(actf_bar, pr));
              }
          } else if (kWarpSend) {
            // this warp's rows (32 q ..) of its K blocks, to every peer's buffer at the same place
            if (lane == 0 && ok)
              for (int kb2 = 0; kb2 < CW / 64; ++kb2) {
                const uint32_t src = act_addr + static_cast<uint32_t>(col0 / 64 + kb2) * 16384 + q * 4096;
                for (int pr = 0; pr < CS; ++pr)
                  if (pr != static_cast<int>(rank))
                    bulk_s2cluster(mapa(src, pr), src, 4096, mapa(actf_bar, pr));
              }
          } else if (CS > 1) {
            epi_sync();
            if (t == 0 && ok) {
              const uint32_t off = static_cast<uint32_t>(rank) * SLICE_BYTES;  // slice = NS/64 K blocks
              for (int pr = 0; pr < CS; ++pr)
                if (pr != static_cast<int>(rank))
                  bulk_s2cluster(mapa(act_addr + off, pr), act_addr + off, SLICE_BYTES, mapa(actf_bar, pr));
            }
          }
        }
        tc_fence_before();
        if (epi_or(!ok)) {
          ok = false;
          break;
        }
      }
      if (!ok) {
        if (rank == 0 && t == 0)
          for (int pr = 0; pr < CS; ++pr) {
            st_cluster_u32(mapa(smem_u32(const_cast<int *>(cmd)), pr), 0u);
            mbar_arrive_cluster(mapa(go_bar, pr));
          }
        break;
      }
      free_pending = CS > 1;
      // ---- accept (rank 0): logL from the cluster-reduced output dot, then the samplers
      if (rank == 0) {
        const bool got = mbar_wait_cluster(part_bar, part_par, a.status);
        part_par ^= 1;
        float lle_v = 0.f;
        if (sampler && valid && got) {
          float s_out = 0.f;
          for (int pr = 0; pr < CS; ++pr) s_out += partial[pr * 128 + r];
          const float arg = E.out_s * (s_out + E.bo) + E.out_m;
          // log output: chi2 = floor + t, t = exp(arg); the adjoint ran with the linear output's
          // seed, so the gradient takes the factor t (d chi2 / d arg); with FP16 operands also
          // out_s (see c0)
          const float tx = E.out_log ? expf(arg) : 1.f;
          lle_v = -0.5f * (E.out_log ? E.out_floor + tx : arg);
          const float gfac = tx * (f16 ? E.out_s : 1.f);
          {
            if (grad && (E.out_log || f16)) {
              if (fast) {
#pragma unroll
                for (int i = 0; i < RegChain8<float>::DB; ++i) rc.gp[i] *= gfac;
              } else {
                float *gout = a.st.gle + row_off(a.st.gle_ld, row, a.dp);
                const int ges = row_es(a.st.gle_ld);
                for (int i = 0; i < a.d; ++i) gout[i * ges] *= gfac;
              }
            }
          }
          a.st.lle[row] = lle_v;
        }
        epi_sync();
        bool done = false;
        // the register-resident chains write their record while the next evaluation runs,
        // unless the covariance accumulator reads it right away
        const bool defer = !a.welford_on;
        if (sampler && need && !loglike)
          done = fast ? (hmc ? rc.hmc_post(a, row, row, lle_v, defer) : rc.post(a, row, row, lle_v, mala, defer))
                      : chn.post(row, h);
        if (sampler && !loglike && a.welford_on) {
          mask[r] = done ? 1 : 0;
          smp_sync();
          if (smp_or(done))
            welford_tile(a, tile * kTcRows, min(kTcRows, a.n_rows - tile * kTcRows), mask, t, 128,
                         [] { smp_sync(); }, tile);
        }
      }
    }
    if (fast && sampler && valid) rc.record(a, row, row);
    // the peers' release of the last phase: no copy or MMA arrive may still target this CTA
    if (free_pending) wait_free(free2_bar, free2_par);
  }
  tc_fence_before();
  __syncthreads();
  if (CS > 1) cluster_sync_all();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tcols_alloc)
                 : "memory");
  }
}

inline size_t tc2_smem_bytes(int width, int cs, int stages, int depth) {
  const int ns = width / cs, tr = ns < 256 ? ns : 256;
  return 1024 + static_cast<size_t>(width / 64) * 16384 +
         static_cast<size_t>(stages) * tc2_stage_kblocks(width, cs) * tr * 128 +
         8 * (2 * stages + 12) + 4 * (cs * 128 + kTc2EQ * 128) + 4 * static_cast<size_t>(depth + 1) * ns +
         3 * 4 * 128 * 8 + 64;
}
inline int tc2_stages_for(int width, int cs, int depth, int smem_cap) {
  for (int s = kTcMaxStages + 2; s >= 2; --s)
    if (tc2_smem_bytes(width, cs, s, depth) <= static_cast<size_t>(smem_cap)) return s;
  return 2;
}

}  // namespace bst
