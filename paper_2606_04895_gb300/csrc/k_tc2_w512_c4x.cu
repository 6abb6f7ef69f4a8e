// k_tc2_w512_c4x.cu -- the cluster tcgen05 chain-tile kernel for width 512, clusters of 4 CTAs, exchange through global slice images (one copy per peer).
#include "tc2_launch.cuh"

namespace bst {
BST_TC2_VARIANT(w512_c4x, 512, 4, true)
}  // namespace bst
