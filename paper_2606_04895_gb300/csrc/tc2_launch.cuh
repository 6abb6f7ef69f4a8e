// tc2_launch.cuh -- launch of one instantiation of the cluster tcgen05 chain-tile kernel.  Each
// instantiation (width W, cluster size CS, exchange through global images L2X) is compiled in a
// translation unit of its own (k_tc2_w*.cu), so the builds run in parallel.
#pragma once

#include "launch.h"

namespace bst {

template <int W, int CS, bool L2X, bool RC>
cudaError_t tc2_launch(const StepArgs<float> &a, const Tc2Weights &w, cudaStream_t s) {
  const int tiles = (a.n_rows + kTcRows - 1) / kTcRows;
  if (tiles == 0) return cudaSuccess;
  const size_t smem = tc2_smem_bytes(W, CS, w.n_stages, w.depth);
  auto k = tc2_chain_kernel<W, CS, L2X, RC>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (CS > 1) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles * CS, 1, 1);
  cfg.blockDim = dim3(kTc2Threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k, a, w);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Launcher and kernel address of one (W, CS, L2X), both chain flavours, as plain functions:
// rc selects the register-resident chains (MALA / MH / HMC, d <= 8, d padded to 16).
#define BST_TC2_VARIANT(NAME, W, CS, L2X)                                                                   \
  cudaError_t tc2_launch_##NAME(const StepArgs<float> &a, const Tc2Weights &w, bool rc, cudaStream_t s) { \
    return rc ? tc2_launch<W, CS, L2X, true>(a, w, s) : tc2_launch<W, CS, L2X, false>(a, w, s);            \
  }                                                                                                        \
  const void *tc2_kernel_##NAME(bool rc) {                                                                 \
    return rc ? reinterpret_cast<const void *>(tc2_chain_kernel<W, CS, L2X, true>)                         \
              : reinterpret_cast<const void *>(tc2_chain_kernel<W, CS, L2X, false>);                       \
  }

#define BST_TC2_DECLARE(NAME)                                                                               \
  cudaError_t tc2_launch_##NAME(const StepArgs<float> &a, const Tc2Weights &w, bool rc, cudaStream_t s); \
  const void *tc2_kernel_##NAME(bool rc);

}  // namespace bst
