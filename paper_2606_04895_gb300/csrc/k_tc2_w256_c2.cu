// k_tc2_w256_c2.cu -- the cluster tcgen05 chain-tile kernel for width 256, clusters of 2 CTAs.
#include "tc2_launch.cuh"

namespace bst {
BST_TC2_VARIANT(w256_c2, 256, 2, false)
}  // namespace bst
