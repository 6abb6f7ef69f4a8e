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
  k<<<grid, kSimtThreads, smem, s>>>(a, w);
  return cudaGetLastError();
}

}  // namespace bst
