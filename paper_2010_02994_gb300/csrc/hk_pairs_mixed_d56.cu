// Mixed pair kernels for D = 5, 6.
#include "hk_pairs_mixed_launch.cuh"

namespace hk {
HK_INSTANTIATE_MIXED(5)
HK_INSTANTIATE_MIXED(6)
}  // namespace hk
