// k_simt_ana.cu -- the CUDA-core chain-tile kernel, FP32 analytic-likelihood instantiation.
#include "simt_launch.cuh"

namespace bst {

cudaError_t launch_ana_simt_f32(const StepArgs<float> &a, const AnaWeights<float> &w, cudaStream_t s) {
  return launch_simt<float, 32, AnaSimt<float, 32>>(a, w, AnaSimt<float, 32>::smem_bytes(0), s);
}

}  // namespace bst
