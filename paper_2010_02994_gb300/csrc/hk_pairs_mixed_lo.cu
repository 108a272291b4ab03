// Mixed pair kernels for D = 1..4.
#include "hk_pairs_mixed_launch.cuh"

namespace hk {
HK_INSTANTIATE_MIXED(1)
HK_INSTANTIATE_MIXED(2)
HK_INSTANTIATE_MIXED(3)
HK_INSTANTIATE_MIXED(4)
}  // namespace hk
