// k_simt.cu -- instantiations and launch wrappers of the CUDA-core chain-tile kernels.
#include "launch.h"

namespace bst {

namespace {
constexpr int kSmemCap = 232448;  // opt-in dynamic shared memory per block on sm_100-class parts

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
}  // namespace

int simt_rows_per_tile(int precision, int width, int lik_kind) {
  if (lik_kind == BST_LIK_ANALYTIC) return 32;
  if (precision == BST_FP64) return 16;
  return width > 512 ? 16 : 32;
}

cudaError_t launch_emu_simt_f32(const StepArgs<float> &a, const EmuWeights<float> &w, cudaStream_t s) {
  if (w.width > 512)
    return launch_simt<float, 16, EmuSimt<float, 16>>(a, w, EmuSimt<float, 16>::smem_bytes(w.width), s);
  return launch_simt<float, 32, EmuSimt<float, 32>>(a, w, EmuSimt<float, 32>::smem_bytes(w.width), s);
}
cudaError_t launch_emu_simt_f64(const StepArgs<double> &a, const EmuWeights<double> &w, cudaStream_t s) {
  return launch_simt<double, 16, EmuSimt<double, 16>>(a, w, EmuSimt<double, 16>::smem_bytes(w.width), s);
}
cudaError_t launch_ana_simt_f32(const StepArgs<float> &a, const AnaWeights<float> &w, cudaStream_t s) {
  return launch_simt<float, 32, AnaSimt<float, 32>>(a, w, AnaSimt<float, 32>::smem_bytes(0), s);
}
cudaError_t launch_ana_simt_f64(const StepArgs<double> &a, const AnaWeights<double> &w, cudaStream_t s) {
  return launch_simt<double, 32, AnaSimt<double, 32>>(a, w, AnaSimt<double, 32>::smem_bytes(0), s);
}

}  // namespace bst
