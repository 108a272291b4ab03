// BMDS FP32 pair kernels for D = 1..4 (the kernel is in hk_bmds.cuh).
#include "hk_bmds.cuh"

namespace hk {

namespace {

template <int D, int W>
void launch_f32(const bmds::Args<float> &a, bool y_f32, bool value, int64_t pairs, cudaStream_t s)
{
    if (y_f32 && value)
        bmds::pairs_kernel<float, float, D, W, true><<<(unsigned)pairs, 32 * W, 0, s>>>(a);
    else if (y_f32)
        bmds::pairs_kernel<float, float, D, W, false><<<(unsigned)pairs, 32 * W, 0, s>>>(a);
    else if (value)
        bmds::pairs_kernel<float, double, D, W, true><<<(unsigned)pairs, 32 * W, 0, s>>>(a);
    else
        bmds::pairs_kernel<float, double, D, W, false><<<(unsigned)pairs, 32 * W, 0, s>>>(a);
}

}  // namespace

cudaError_t launch_bmds_pairs_f32_lo(const bmds::Args<float> &a, bool y_f32, bool value, int W, int64_t pairs,
                                     cudaStream_t s)
{
#define HK_BMDS_CASE(D)                       \
    case D:                                   \
        if (W == 4)                           \
            launch_f32<D, 4>(a, y_f32, value, pairs, s); \
        else                                  \
            launch_f32<D, 2>(a, y_f32, value, pairs, s); \
        break;
    switch (a.d) {
        HK_BMDS_CASE(1)
        HK_BMDS_CASE(2)
        HK_BMDS_CASE(3)
        HK_BMDS_CASE(4)
    default:
        return cudaErrorInvalidValue;
    }
#undef HK_BMDS_CASE
    return cudaGetLastError();
}

}  // namespace hk
