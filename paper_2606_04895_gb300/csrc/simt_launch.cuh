// simt_launch.cuh -- launch of one instantiation of the CUDA-core chain-tile kernel.  The
// instantiations are spread over k_simt*.cu so that they compile in parallel.
#pragma once

#include "launch.h"

namespace bst {

template <typename R, int T, class Engine, class Weights>
cudaError_t launch_simt(const StepArgs<R> &a, const Weights &w, size_t smem, cudaStream_t s) {
  auto k = simt_chain_kernel<R, T, Engine, Weights>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int grid = (a.n_rows + T - 1) / T;
  if (grid == 0) return cudaSuccess;
  const int cl = simt_ensemble_cluster<T>(a);
  if (cl == 1) {
    k<<<grid, kSimtThreads, smem, s>>>(a, w);
    return cudaGetLastError();
  }
  // ensemble halves wider than a tile: the tiles of a half form a cluster (the kernel
  // synchronises the cluster between half-steps); n_rows is a multiple of the half
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kSimtThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k, a, w);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace bst
