// The library's device Philox4x32-10 (bst::Philox::block) against cuRAND's
// curand_Philox4x32_10 (a separate implementation of the same published generator, called
// from the toolkit header) on the known-answer counters and keys and on 2^20 random
// (counter, key) pairs drawn on the host.  Prints "kat <12 hex words>" and
// "mismatches <count> of <n>"; exits non-zero on a CUDA error.
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include <curand_philox4x32_x.h>

#include "common.cuh"

__global__ void compare(const uint32_t *ctr, const uint32_t *key, uint32_t *ours, uint32_t *ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t *c = ctr + 4 * i;
  const uint64_t seed = static_cast<uint64_t>(key[2 * i]) | (static_cast<uint64_t>(key[2 * i + 1]) << 32);
  uint32_t w[4];
  bst::Philox::block(seed, c[0], c[1], c[2], c[3], w);
  const uint4 r = curand_Philox4x32_10(make_uint4(c[0], c[1], c[2], c[3]), make_uint2(key[2 * i], key[2 * i + 1]));
  for (int j = 0; j < 4; ++j) ours[4 * i + j] = w[j];
  ref[4 * i + 0] = r.x;
  ref[4 * i + 1] = r.y;
  ref[4 * i + 2] = r.z;
  ref[4 * i + 3] = r.w;
}

int main() {
  const int n = 1 << 20;
  std::vector<uint32_t> ctr(4 * n), key(2 * n), ours(4 * n), ref(4 * n);
  const uint32_t kat_c[3][4] = {{0, 0, 0, 0},
                                {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu},
                                {0x243f6a88u, 0x85a308d3u, 0x13198a2eu, 0x03707344u}};
  const uint32_t kat_k[3][2] = {{0, 0}, {0xffffffffu, 0xffffffffu}, {0xa4093822u, 0x299f31d0u}};
  std::mt19937_64 gen(12345);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < 4; ++j) ctr[4 * i + j] = static_cast<uint32_t>(gen());
    for (int j = 0; j < 2; ++j) key[2 * i + j] = static_cast<uint32_t>(gen());
  }
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 4; ++j) ctr[4 * i + j] = kat_c[i][j];
    for (int j = 0; j < 2; ++j) key[2 * i + j] = kat_k[i][j];
  }
  uint32_t *dc = nullptr, *dk = nullptr, *d_ours = nullptr, *d_ref = nullptr;
  if (cudaMalloc(&dc, 16ull * n) || cudaMalloc(&dk, 8ull * n) || cudaMalloc(&d_ours, 16ull * n) ||
      cudaMalloc(&d_ref, 16ull * n))
    return 2;
  cudaMemcpy(dc, ctr.data(), 16ull * n, cudaMemcpyHostToDevice);
  cudaMemcpy(dk, key.data(), 8ull * n, cudaMemcpyHostToDevice);
  compare<<<(n + 255) / 256, 256>>>(dc, dk, d_ours, d_ref, n);
  if (cudaDeviceSynchronize() != cudaSuccess) return 3;
  cudaMemcpy(ours.data(), d_ours, 16ull * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(ref.data(), d_ref, 16ull * n, cudaMemcpyDeviceToHost);
  long bad = 0;
  for (long i = 0; i < 4l * n; ++i) bad += ours[i] != ref[i];
  std::printf("kat");
  for (int i = 0; i < 12; ++i) std::printf(" %08x", ours[i]);
  std::printf("\nmismatches %ld of %ld\n", bad, 4l * n);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(d_ours);
  cudaFree(d_ref);
  return 0;
}
