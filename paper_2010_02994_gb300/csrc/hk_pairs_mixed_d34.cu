// Mixed pair kernels for D = 3, 4.
#include "hk_pairs_mixed_launch.cuh"

namespace hk {
HK_INSTANTIATE_MIXED(3)
HK_INSTANTIATE_MIXED(4)
}  // namespace hk
