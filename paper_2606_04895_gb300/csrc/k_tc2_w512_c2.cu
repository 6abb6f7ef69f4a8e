// k_tc2_w512_c2.cu -- the cluster tcgen05 chain-tile kernel for width 512, clusters of 2 CTAs.
#include "tc2_launch.cuh"

namespace bst {
BST_TC2_VARIANT(w512_c2, 512, 2, false)
}  // namespace bst
