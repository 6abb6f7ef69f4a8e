// k_tc2.cu -- launch wrappers and configuration of the cluster tcgen05 chain-tile kernel.
#include <cstdlib>

#include "tc2_launch.cuh"

namespace bst {

int tc2_cluster_size_for(int n_rows, int width);

namespace {
constexpr int kSmemCap = 232448;
constexpr int kNumSMs = 152;
}  // namespace

// one translation unit per instantiation (k_tc2_w*.cu)
BST_TC2_DECLARE(w512_c4x)
BST_TC2_DECLARE(w512_c4)
BST_TC2_DECLARE(w512_c2)
BST_TC2_DECLARE(w512_c1)
BST_TC2_DECLARE(w256_c4)
BST_TC2_DECLARE(w256_c2)
BST_TC2_DECLARE(w256_c1)

int tc2_stages(int width, int cs, int depth) { return tc2_stages_for(width, cs, depth, kSmemCap); }

// Clusters of this configuration that can be co-resident (diagnostic).
int tc2_max_active_clusters(int width, int cs, int depth) {
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kTc2Threads, 1, 1);
  cfg.gridDim = dim3(cs * 64, 1, 1);
  cfg.dynamicSmemBytes = tc2_smem_bytes(width, cs, tc2_stages(width, cs, depth), depth);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = -1;
  const void *k = nullptr;
  if (width == 512)
    k = cs == 4 ? tc2_kernel_w512_c4x(true) : cs == 2 ? tc2_kernel_w512_c2(true) : tc2_kernel_w512_c1(true);
  else
    k = cs == 4 ? tc2_kernel_w256_c4(true) : cs == 2 ? tc2_kernel_w256_c2(true) : tc2_kernel_w256_c1(true);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(cfg.dynamicSmemBytes));
  if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) return -1;
  return n;
}

// Split a layer across more CTAs while there are fewer 128-chain tiles than SMs.  The
// environment variable BST_TC_CLUSTER (1, 2 or 4) overrides the choice (tuning).
int tc2_cluster_size(int n_rows, int width, int depth) {
  int cs = tc2_cluster_size_for(n_rows, width);
  // a smaller cluster keeps the stored activations in global scratch when they do not fit in
  // tensor memory
  while (cs > 1 && depth > tc2_tmem_max_depth(width, cs)) cs /= 2;
  return cs;
}

int tc2_cluster_size_for(int n_rows, int width) {
  // every epilogue warp needs at least one 32-column chunk of its rank's slice
  const int cs_max = width / (32 * kTc2EQ);
  static const int forced = [] {
    const char *v = getenv("BST_TC_CLUSTER");
    const int c = v ? atoi(v) : 0;
    return (c == 1 || c == 2 || c == 4) ? c : 0;
  }();
  if (forced) return forced <= cs_max ? forced : cs_max;
  const int tiles = (n_rows + kTcRows - 1) / kTcRows;
  if (4 * tiles <= kNumSMs && cs_max >= 4) return 4;
  if (2 * tiles <= kNumSMs && cs_max >= 2) return 2;
  return 1;
}

cudaError_t launch_emu_tc2(const StepArgs<float> &a, const Tc2Weights &w, cudaStream_t s) {
  // register-resident chains: MALA / MH / HMC with d <= 8 (padded to 16)
  const bool rc = (a.mode == kModeMALA || a.mode == kModeMH || a.mode == kModeHMC) && a.d <= RegChain8<float>::DB &&
                  a.dp == 16;
  if (w.width == 512) {
    if (w.cs == 4) return w.xchg ? tc2_launch_w512_c4x(a, w, rc, s) : tc2_launch_w512_c4(a, w, rc, s);
    if (w.cs == 2) return tc2_launch_w512_c2(a, w, rc, s);
    return tc2_launch_w512_c1(a, w, rc, s);
  }
  if (w.width == 256) {
    if (w.cs == 4) return tc2_launch_w256_c4(a, w, rc, s);
    if (w.cs == 2) return tc2_launch_w256_c2(a, w, rc, s);
    return tc2_launch_w256_c1(a, w, rc, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace bst
