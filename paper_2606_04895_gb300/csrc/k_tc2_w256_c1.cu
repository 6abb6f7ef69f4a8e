// k_tc2_w256_c1.cu -- the cluster tcgen05 chain-tile kernel for width 256, clusters of 1 CTA.
#include "tc2_launch.cuh"

namespace bst {
BST_TC2_VARIANT(w256_c1, 256, 1, false)
}  // namespace bst
