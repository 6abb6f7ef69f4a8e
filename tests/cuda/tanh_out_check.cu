// Error of the engine's last-layer tanh (tanh x = 1 - 2 / (exp(2x) + 1), hardware exp and
// fast division) against double-precision tanh and against CUDA's tanhf on a dense grid of
// [-20, 20].  Prints "max_abs_err <ours> <tanhf>" and exits non-zero on a CUDA error.
#include <cmath>
#include <cstdio>
#include <vector>

#include "engine_tc2.cuh"

__global__ void eval_tanh(const float *x, float *ours, float *ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    ours[i] = bst::tanh_out(x[i]);
    ref[i] = tanhf(x[i]);
  }
}

int main() {
  const int n = 1 << 22;
  std::vector<float> hx(n), ha(n), hb(n);
  for (int i = 0; i < n; ++i) hx[i] = -20.f + 40.f * (static_cast<float>(i) + 0.5f) / n;
  float *dx = nullptr, *da = nullptr, *db = nullptr;
  if (cudaMalloc(&dx, n * 4) || cudaMalloc(&da, n * 4) || cudaMalloc(&db, n * 4)) return 2;
  cudaMemcpy(dx, hx.data(), n * 4, cudaMemcpyHostToDevice);
  eval_tanh<<<(n + 255) / 256, 256>>>(dx, da, db, n);
  if (cudaDeviceSynchronize() != cudaSuccess) return 3;
  cudaMemcpy(ha.data(), da, n * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(hb.data(), db, n * 4, cudaMemcpyDeviceToHost);
  double ea = 0.0, eb = 0.0;
  for (int i = 0; i < n; ++i) {
    const double t = std::tanh(static_cast<double>(hx[i]));
    ea = std::fmax(ea, std::fabs(ha[i] - t));
    eb = std::fmax(eb, std::fabs(hb[i] - t));
  }
  std::printf("max_abs_err %.6g %.6g\n", ea, eb);
  cudaFree(dx);
  cudaFree(da);
  cudaFree(db);
  return 0;
}
