// Launch helpers of the mixed pair kernels, instantiated per dimension by
// hk_pairs_mixed_lo.cu (D = 1..4) and hk_pairs_mixed_hi.cu (D = 5..8).
#pragma once

#include "hk_pairs_mixed.cuh"

namespace hk {

template <int D>
cudaError_t launch_pass1_t(const Work &w, const WorkItem *items, int nitems, int grid, int warps, cudaStream_t s)
{
    const size_t smem = pass_smem_bytes_t<D>(1, false, warps);
    pass1_mixed_kernel<D><<<grid, warps * 32, smem, s>>>(w, items, nitems);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_pass1_theta_t(const Work &w, const WorkItem *items, int nitems, int grid, int warps,
                                 cudaStream_t s)
{
    const size_t smem = pass_smem_bytes_t<D>(1, true, warps);
    pass1_theta_kernel<D><<<grid, warps * 32, smem, s>>>(w, items, nitems);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_pass2_t(const Work &w, const WorkItem *items, int nitems, int grid, int warps, cudaStream_t s)
{
    const size_t smem = pass_smem_bytes_t<D>(2, false, warps);
    pass2_mixed_kernel<D><<<grid, warps * 32, smem, s>>>(w, items, nitems);
    return cudaGetLastError();
}

// Allow the largest dynamic shared memory any warp count needs, and return
// how many CTAs of `warps` warps fit on one SM.
// pass: 1 rates, 2 gradient, 3 rates with Theta sums.
template <int D>
int occupancy_t(int pass, int warps)
{
    const bool theta = pass == 3;
    const int p = theta ? 1 : pass;
    const size_t smem = pass_smem_bytes_t<D>(p, theta, warps);
    const size_t smem_max = pass_smem_bytes_t<D>(p, theta, 8);
    int nb = 0;
    if (theta) {
        cudaFuncSetAttribute(pass1_theta_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass1_theta_kernel<D>, warps * 32, smem);
    } else if (pass == 1) {
        cudaFuncSetAttribute(pass1_mixed_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass1_mixed_kernel<D>, warps * 32, smem);
    } else {
        cudaFuncSetAttribute(pass2_mixed_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass2_mixed_kernel<D>, warps * 32, smem);
    }
    return nb;
}

#define HK_INSTANTIATE_MIXED(D)                                                                              \
    template cudaError_t launch_pass1_t<D>(const Work &, const WorkItem *, int, int, int, cudaStream_t);      \
    template cudaError_t launch_pass2_t<D>(const Work &, const WorkItem *, int, int, int, cudaStream_t);      \
    template cudaError_t launch_pass1_theta_t<D>(const Work &, const WorkItem *, int, int, int, cudaStream_t);\
    template int occupancy_t<D>(int, int);                                                                     \
    template size_t pass_smem_bytes_t<D>(int, bool, int);

}  // namespace hk
