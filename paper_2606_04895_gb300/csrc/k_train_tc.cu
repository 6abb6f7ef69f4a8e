// k_train_tc.cu -- BF16 tensor-core (tcgen05) GEMMs of emulator training.
//
// The learned part of the method (Sec. 1, Sec. 4: a neural-network likelihood fitted to
// likelihood evaluations) is trained with minibatch Adam; its hidden-layer products are dense
// contractions of a batch of activations with the weights, run here on the 5th-generation tensor
// cores: BF16 operands, FP32 accumulation in tensor memory.  One GEMM kernel
//   C[M][N] = sum_k A[m][k] B[n][k]   (A, B row-major BF16, k contiguous: "K-major")
// with a fused epilogue covers the three products of a layer:
//   forward          H_l   = tanh(H_{l-1} W_l^T + b_l)      A = H_{l-1},   B = W_l
//   input adjoint    D_l-1 = (D_l W_l) (1 - H_{l-1}^2)       A = D_l,       B = W_l^T
//   weight gradient  G_l   = D_l^T H_{l-1}                   A = D_l^T,     B = H_{l-1}^T
// (the epilogues also write the BF16 copies, row-major and transposed, that the next products take
// as operands).  Operand tiles (128 rows x 64 k) are loaded by TMA (cp.async.bulk.tensor) into
// 128-byte-swizzled K-major shared-memory stages (mbarrier ring); one thread issues
// tcgen05.mma (M = 128, N = 128, K = 16); four warps read the accumulator back with tcgen05.ld.
// The weight gradient splits the batch (k) over grid.z slices whose FP32 partials are summed in
// slice order by the caller, so results do not depend on scheduling.
#include <cuda.h>

#include "launch.h"

namespace bst {

namespace {

constexpr int kTgBM = 128, kTgBN = 128, kTgBK = 64;
constexpr int kTgStages = 4;
constexpr int kTgThreads = 192;  // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr uint32_t kTgTileBytes = kTgBM * kTgBK * 2;  // 16 KB (A and B tiles alike)

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(kTgThreads, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                                const __grid_constant__ CUtensorMap tb,
                                                                const __grid_constant__ TcGemmArgs g) {
  extern __shared__ __align__(1024) uint8_t tg_smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tg_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sa = base;                               // [stages][128 x 64] A tiles
  uint8_t *sb = base + kTgStages * kTgTileBytes;    // [stages][128 x 64] B tiles
  uint64_t *bars = reinterpret_cast<uint64_t *>(sb + kTgStages * kTgTileBytes);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kTgStages), acc_bar = smem_u32(bars + 2 * kTgStages);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kTgStages + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTgBM, n0 = blockIdx.x * kTgBN;
  const int kbeg = blockIdx.z * g.k_chunk;
  const int kend = min(g.K, kbeg + g.k_chunk);
  const int nkb = (kend - kbeg) / kTgBK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTgStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(acc_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(static_cast<uint32_t>(kTgBN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
      asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
      uint32_t fpar = 0, used = 0;
      int s = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait(empty0 + 8 * s, ((fpar >> s) & 1u) ^ 1u, g.status)) break;
        mbar_expect_tx(full0 + 8 * s, 2 * kTgTileBytes);
        const int kx = kbeg + kb * kTgBK;  // a multiple of 64 elements: 128-byte aligned x coordinate
        tma_load_2d(smem_u32(sa + s * kTgTileBytes), &ta, kx, m0, full0 + 8 * s);
        tma_load_2d(smem_u32(sb + s * kTgTileBytes), &tb, kx, n0, full0 + 8 * s);
        fpar ^= 1u << s;
        used |= 1u << s;
        s = (s + 1 == kTgStages) ? 0 : s + 1;
      }
      // every load issued has landed before the CTA may exit
      for (int q = 0; q < kTgStages; ++q)
        if ((used >> q) & 1u) mbar_wait(full0 + 8 * q, ((fpar >> q) & 1u) ^ 1u, g.status);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id = idesc_bf16(kTgBM, kTgBN);
      const uint64_t ad0 = sw128_desc(smem_u32(sa)), bd0 = sw128_desc(smem_u32(sb));
      uint32_t upar = 0;
      int s = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait(full0 + 8 * s, (upar >> s) & 1u, g.status)) break;
        upar ^= 1u << s;
        tc_fence_after();
        const uint64_t ad = ad0 + static_cast<uint64_t>(s * (kTgTileBytes >> 4));
        const uint64_t bd = bd0 + static_cast<uint64_t>(s * (kTgTileBytes >> 4));
#pragma unroll
        for (int k = 0; k < kTgBK / 16; ++k) mma_bf16(tmem, ad + 2 * k, bd + 2 * k, id, (kb > 0 || k > 0) ? 1u : 0u);
        mma_commit(empty0 + 8 * s);
        s = (s + 1 == kTgStages) ? 0 : s + 1;
      }
      mma_commit(acc_bar);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue: row = TMEM lane
    const int q = warp & 3;
    const int row = m0 + q * 32 + lane;
    const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16);
    bool ok = true;
    if (lane == 0) ok = mbar_wait(acc_bar, 0, g.status);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    tc_fence_after();
    if (ok && nkb > 0) {
#pragma unroll 1
      for (int c = 0; c < kTgBN / 32; ++c) {
        uint32_t raw[32];
        tmem_ld32_nowait(trow + c * 32, raw);
        tmem_wait_ld_regs(raw);
        const int col0 = n0 + c * 32;
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(raw[i]);
        if (g.epi == kTcEpiTanh) {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = tanhf(v[i] + g.bias[col0 + i]);
        } else if (g.epi == kTcEpiDtanh) {
          const float *hr = g.H + static_cast<size_t>(row) * g.N + col0;
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] *= 1.f - hr[i] * hr[i];
        }
        float *cr = g.C + (static_cast<size_t>(blockIdx.z) * g.M + row) * g.N + col0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          reinterpret_cast<float4 *>(cr)[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        if (g.Cb) {
          uint32_t pk[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) pk[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
          uint4 *br = reinterpret_cast<uint4 *>(g.Cb + static_cast<size_t>(row) * g.N + col0);
#pragma unroll
          for (int u = 0; u < 4; ++u) br[u] = make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
        }
        if (g.CbT) {
          // transposed copy: for each column the warp's 32 rows are 64 contiguous bytes
#pragma unroll
          for (int i = 0; i < 32; ++i) g.CbT[static_cast<size_t>(col0 + i) * g.M + row] = __float2bfloat16_rn(v[i]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(static_cast<uint32_t>(kTgBN))
                 : "memory");
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link-time
// dependency on libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<EncodeTiledFn>(nullptr);
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Map of a row-major BF16 matrix [rows][cols] (cols contiguous) read in 128 x 64 boxes with the
// 128-byte swizzle of the MMA's shared-memory descriptors.
bool make_map(CUtensorMap *m, const __nv_bfloat16 *ptr, int rows, int cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * 2};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(kTgBK), static_cast<cuuint32_t>(kTgBM)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tg_smem_bytes() { return 1024 + 2 * kTgStages * kTgTileBytes + 8 * (2 * kTgStages + 1) + 16; }

}  // namespace

bool tc_gemm_shape_ok(int M, int N, int K, int splits) {
  return M > 0 && N > 0 && K > 0 && splits > 0 && M % kTgBM == 0 && N % kTgBN == 0 && K % (kTgBK * splits) == 0;
}

cudaError_t launch_tc_gemm(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int splits, const TcGemmArgs &args,
                           cudaStream_t s) {
  TcGemmArgs g = args;
  if (!tc_gemm_shape_ok(g.M, g.N, g.K, splits)) return cudaErrorInvalidValue;
  g.k_chunk = g.K / splits;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, g.M, g.K) || !make_map(&tb, B, g.N, g.K)) return cudaErrorInvalidValue;
  const size_t smem = tg_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  dim3 grid(g.N / kTgBN, g.M / kTgBM, splits);
  tc_gemm_kernel<<<grid, kTgThreads, smem, s>>>(ta, tb, g);
  return cudaGetLastError();
}

// FP32 [rows][cols] -> BF16 row-major copy and BF16 transposed copy [cols][rows] (either may be
// null).  32 x 32 tiles through shared memory so that both writes are coalesced.
__global__ void cast_transpose_bf16_kernel(const float *X, int rows, int cols, __nv_bfloat16 *Xb,
                                           __nv_bfloat16 *XbT) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    const float v = (r < rows && c < cols) ? X[static_cast<size_t>(r) * cols + c] : 0.f;
    t[i][threadIdx.x] = v;
    if (Xb && r < rows && c < cols) Xb[static_cast<size_t>(r) * cols + c] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  if (!XbT) return;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) XbT[static_cast<size_t>(c) * rows + r] = __float2bfloat16_rn(t[threadIdx.x][i]);
  }
}
cudaError_t launch_cast_transpose_bf16(const float *X, int rows, int cols, __nv_bfloat16 *Xb, __nv_bfloat16 *XbT,
                                       cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), blk(32, 8);
  cast_transpose_bf16_kernel<<<grid, blk, 0, s>>>(X, rows, cols, Xb, XbT);
  return cudaGetLastError();
}

}  // namespace bst
