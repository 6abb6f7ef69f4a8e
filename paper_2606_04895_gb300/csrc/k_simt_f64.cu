// k_simt_f64.cu -- the CUDA-core chain-tile kernel, FP64 instantiations (emulator, analytic).
#include "simt_launch.cuh"

namespace bst {

cudaError_t launch_emu_simt_f64(const StepArgs<double> &a, const EmuWeights<double> &w, cudaStream_t s) {
  return launch_simt<double, 16, EmuSimt<double, 16>>(a, w, EmuSimt<double, 16>::smem_bytes(w.width), s);
}
cudaError_t launch_ana_simt_f64(const StepArgs<double> &a, const AnaWeights<double> &w, cudaStream_t s) {
  return launch_simt<double, 32, AnaSimt<double, 32>>(a, w, AnaSimt<double, 32>::smem_bytes(0), s);
}

}  // namespace bst
