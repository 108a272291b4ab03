// Mixed pair kernels for D = 1, 2 (the instantiations are split over four
// translation units so that they compile in parallel).
#include "hk_pairs_mixed_launch.cuh"

namespace hk {
HK_INSTANTIATE_MIXED(1)
HK_INSTANTIATE_MIXED(2)
}  // namespace hk
