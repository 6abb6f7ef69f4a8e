// k_simt.cu -- the CUDA-core chain-tile kernel, FP32 emulator instantiations, and the tile size.
#include "simt_launch.cuh"

namespace bst {

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

}  // namespace bst
