// Launch helpers of the mixed pair kernels, instantiated per dimension by
// hk_pairs_mixed_lo.cu (D = 1..4) and hk_pairs_mixed_hi.cu (D = 5..8).
// pass: 1 rates, 2 gradient, 3 rates with Theta sums, 4 rates with the
// self-excitation sums apart.
#pragma once

#include <algorithm>

#include "hk_pairs_mixed.cuh"

namespace hk {

template <int KIND, int D>
cudaError_t launch_kind_t(const Work &w, const WorkItem *items, int nitems, int grid, int warps, cudaStream_t s)
{
    constexpr int R = rows_per_lane(D);
    const size_t smem = pair_smem_bytes<KIND, D, R>(warps);
    pair_kernel<KIND, D, R><<<grid, warps * 32, smem, s>>>(w, items, nitems);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_pass_t(int pass, const Work &w, const WorkItem *items, int nitems, int grid, int warps,
                          cudaStream_t s)
{
    if (pass == 1)
        return launch_kind_t<kRate, D>(w, items, nitems, grid, warps, s);
    if (pass == 2)
        return launch_kind_t<kGrad, D>(w, items, nitems, grid, warps, s);
    if (pass == 4)
        return launch_kind_t<kRateXi, D>(w, items, nitems, grid, warps, s);
    return launch_kind_t<kRateTheta, D>(w, items, nitems, grid, warps, s);
}

template <int D>
size_t smem_t(int pass, int warps)
{
    constexpr int R = rows_per_lane(D);
    if (pass == 1)
        return pair_smem_bytes<kRate, D, R>(warps);
    if (pass == 2)
        return pair_smem_bytes<kGrad, D, R>(warps);
    if (pass == 4)
        return pair_smem_bytes<kRateXi, D, R>(warps);
    return pair_smem_bytes<kRateTheta, D, R>(warps);
}

template <int KIND, int D>
int occupancy_kind(int warps)
{
    constexpr int R = rows_per_lane(D);
    const size_t smem = pair_smem_bytes<KIND, D, R>(warps);
    // the largest any warp count needs, capped at the per-CTA maximum (some
    // 8-warp shapes exceed it; the shape choice never selects those)
    // (static shared memory counts against the same per-CTA maximum)
    int dev = 0, cap = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, pair_kernel<KIND, D, R>);
    const size_t smem_max = std::min<size_t>(pair_smem_bytes<KIND, D, R>(8), (size_t)cap - fa.sharedSizeBytes);
    if (smem > smem_max)
        return 0;
    cudaFuncSetAttribute(pair_kernel<KIND, D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_kernel<KIND, D, R>, warps * 32, smem);
    return nb;
}

// Allow the largest dynamic shared memory any warp count needs, and return
// how many CTAs of `warps` warps fit on one SM.
template <int D>
int occupancy_t(int pass, int warps)
{
    if (pass == 1)
        return occupancy_kind<kRate, D>(warps);
    if (pass == 2)
        return occupancy_kind<kGrad, D>(warps);
    if (pass == 4)
        return occupancy_kind<kRateXi, D>(warps);
    return occupancy_kind<kRateTheta, D>(warps);
}

#define HK_INSTANTIATE_MIXED(D)                                                                               \
    template cudaError_t launch_pass_t<D>(int, const Work &, const WorkItem *, int, int, int, cudaStream_t);  \
    template size_t smem_t<D>(int, int);                                                                        \
    template int occupancy_t<D>(int, int);

}  // namespace hk
