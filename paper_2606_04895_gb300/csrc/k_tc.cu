// k_tc.cu -- instantiations and launch wrappers of the tcgen05 chain-tile kernels.
#include "launch.h"

namespace bst {

namespace {
constexpr int kSmemCap = 232448;  // opt-in dynamic shared memory per block
}  // namespace

int tc_stages(int width) { return tc_stages_for(width, kSmemCap); }
size_t tc_smem_for(int width) { return tc_smem_bytes(width, tc_stages(width)); }

cudaError_t launch_emu_tc(const StepArgs<float> &a, const TcWeights &w, cudaStream_t s) {
  const size_t smem = tc_smem_for(w.width);
  const int grid = (a.n_rows + kTcRows - 1) / kTcRows;
  if (grid == 0) return cudaSuccess;
  cudaError_t e;
  if (w.width == 512) {
    e = cudaFuncSetAttribute(tc_chain_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    tc_chain_kernel<512><<<grid, kTcThreads, smem, s>>>(a, w);
  } else if (w.width == 256) {
    e = cudaFuncSetAttribute(tc_chain_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    tc_chain_kernel<256><<<grid, kTcThreads, smem, s>>>(a, w);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace bst
