// k_tc2_w512_c1.cu -- the cluster tcgen05 chain-tile kernel for width 512, clusters of 1 CTA.
#include "tc2_launch.cuh"

namespace bst {
BST_TC2_VARIANT(w512_c1, 512, 1, false)
}  // namespace bst
