// Mixed pair kernels for D = 7, 8, and the dispatch on D.
#include "hk_pairs_mixed_launch.cuh"

namespace hk {
HK_INSTANTIATE_MIXED(7)
HK_INSTANTIATE_MIXED(8)

#define HK_EXTERN_MIXED(D)                                                                                      \
    extern template cudaError_t launch_pass_t<D>(int, const Work &, const Sched &, int, int, int,      \
                                                 cudaStream_t);                                                \
    extern template size_t smem_t<D>(int, int, int);                                                            \
    extern template int occupancy_t<D>(int, int, int);
HK_EXTERN_MIXED(1)
HK_EXTERN_MIXED(2)
HK_EXTERN_MIXED(3)
HK_EXTERN_MIXED(4)
HK_EXTERN_MIXED(5)
HK_EXTERN_MIXED(6)

#define HK_SWITCH_D(d, EXPR)                                                                                   \
    switch (d) {                                                                                               \
    case 1: { constexpr int D = 1; return EXPR; }                                                             \
    case 2: { constexpr int D = 2; return EXPR; }                                                             \
    case 3: { constexpr int D = 3; return EXPR; }                                                             \
    case 4: { constexpr int D = 4; return EXPR; }                                                             \
    case 5: { constexpr int D = 5; return EXPR; }                                                             \
    case 6: { constexpr int D = 6; return EXPR; }                                                             \
    case 7: { constexpr int D = 7; return EXPR; }                                                             \
    case 8: { constexpr int D = 8; return EXPR; }                                                             \
    default: break;                                                                                            \
    }

cudaError_t launch_pair_pass_mixed(int pass, int d, const Work &w, const Sched &sc, int grid,
                                   int wr, int wc, cudaStream_t s)
{
    HK_SWITCH_D(d, launch_pass_t<D>(pass, w, sc, grid, wr, wc, s))
    return cudaErrorInvalidValue;
}

size_t pass_smem_bytes(int d, int pass, int wr, int wc)
{
    HK_SWITCH_D(d, smem_t<D>(pass, wr, wc))
    return 0;
}

int pass_max_ctas_per_sm(int d, int pass, int wr, int wc)
{
    HK_SWITCH_D(d, occupancy_t<D>(pass, wr, wc))
    return 0;
}

}  // namespace hk
