// Launch helpers of the mixed pair kernels, instantiated per dimension by
// hk_pairs_mixed_lo.cu (D = 1..4) and hk_pairs_mixed_hi.cu (D = 5..8).
// pass: 1 rates, 2 gradient, 3 rates with Theta sums, 4 rates with the
// self-excitation sums apart, 5 gradient with the BMDS term.  A shape is (wr, wc): wr row groups of 32 R
// rows (block size B = 32 R wr) and wc column groups, wr * wc <= 8 warps.
#pragma once

#include <algorithm>

#include "hk_pairs_mixed.cuh"

namespace hk {

// Column groups are a template parameter (1, 2 or 4; a runtime count costs
// the hot loop about twenty registers); only the rate and gradient passes
// split columns, the passes with extra row sums run one column group.
template <int KIND>
constexpr bool kind_splits_columns()
{
    return KIND == kRate || KIND == kGrad;
}

template <int KIND, int D, int WC>
cudaError_t launch_wc_t(const Work &w, const Sched &sc, int grid, int wr, cudaStream_t s)
{
    constexpr int R = rows_per_lane(D);
    const size_t smem = pair_smem_bytes<KIND, D, R>(wr * WC, WC);
    pair_kernel<KIND, D, R, WC><<<grid, wr * WC * 32, smem, s>>>(w, sc);
    return cudaGetLastError();
}

template <int KIND, int D>
cudaError_t launch_kind_t(const Work &w, const Sched &sc, int grid, int wr, int wc,
                          cudaStream_t s)
{
    if (!kind_splits_columns<KIND>() || wc == 1)
        return launch_wc_t<KIND, D, 1>(w, sc, grid, wr, s);
    if (wc == 2)
        return launch_wc_t<KIND, D, kind_splits_columns<KIND>() ? 2 : 1>(w, sc, grid, wr, s);
    if (wc == 4)
        return launch_wc_t<KIND, D, kind_splits_columns<KIND>() ? 4 : 1>(w, sc, grid, wr, s);
    return cudaErrorInvalidValue;
}

template <int D>
cudaError_t launch_pass_t(int pass, const Work &w, const Sched &sc, int grid, int wr, int wc,
                          cudaStream_t s)
{
    if (pass == 1)
        return launch_kind_t<kRate, D>(w, sc, grid, wr, wc, s);
    if (pass == 2)
        return launch_kind_t<kGrad, D>(w, sc, grid, wr, wc, s);
    if (pass == 4)
        return launch_kind_t<kRateXi, D>(w, sc, grid, wr, 1, s);
    if (pass == 5)
        return launch_kind_t<kGradB, D>(w, sc, grid, wr, 1, s);
    return launch_kind_t<kRateTheta, D>(w, sc, grid, wr, 1, s);
}

template <int D>
size_t smem_t(int pass, int wr, int wc)
{
    constexpr int R = rows_per_lane(D);
    if (pass == 1)
        return pair_smem_bytes<kRate, D, R>(wr * wc, wc);
    if (pass == 2)
        return pair_smem_bytes<kGrad, D, R>(wr * wc, wc);
    if (pass == 4)
        return pair_smem_bytes<kRateXi, D, R>(wr, 1);
    if (pass == 5)
        return pair_smem_bytes<kGradB, D, R>(wr, 1);
    return pair_smem_bytes<kRateTheta, D, R>(wr, 1);
}

// Allow the largest dynamic shared memory any shape of this kernel needs
// (capped at the per-CTA maximum; static shared memory counts against the
// same maximum), and return how many CTAs of wr row groups fit on one SM.
template <int KIND, int D, int WC>
int occupancy_wc(int wr)
{
    constexpr int R = rows_per_lane(D);
    const size_t smem = pair_smem_bytes<KIND, D, R>(wr * WC, WC);
    int dev = 0, cap = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, pair_kernel<KIND, D, R, WC>);
    size_t largest = 0;
    for (int a = 1; a * WC <= 8; a *= 2)
        largest = std::max(largest, pair_smem_bytes<KIND, D, R>(a * WC, WC));
    const size_t smem_max = std::min<size_t>(largest, (size_t)cap - fa.sharedSizeBytes);
    if (smem > smem_max)
        return 0;
    cudaFuncSetAttribute(pair_kernel<KIND, D, R, WC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_kernel<KIND, D, R, WC>, wr * WC * 32, smem);
    return nb;
}

template <int KIND, int D>
int occupancy_kind(int wr, int wc)
{
    if (!kind_splits_columns<KIND>() || wc == 1)
        return occupancy_wc<KIND, D, 1>(wr);
    if (wc == 2)
        return occupancy_wc<KIND, D, kind_splits_columns<KIND>() ? 2 : 1>(wr);
    if (wc == 4)
        return occupancy_wc<KIND, D, kind_splits_columns<KIND>() ? 4 : 1>(wr);
    return 0;
}

// CTAs of shape (wr, wc) that fit on one SM (the passes with extra row sums
// always run one column group).
template <int D>
int occupancy_t(int pass, int wr, int wc)
{
    if (pass == 1)
        return occupancy_kind<kRate, D>(wr, wc);
    if (pass == 2)
        return occupancy_kind<kGrad, D>(wr, wc);
    if (pass == 4)
        return occupancy_kind<kRateXi, D>(wr, 1);
    if (pass == 5)
        return occupancy_kind<kGradB, D>(wr, 1);
    return occupancy_kind<kRateTheta, D>(wr, 1);
}

#define HK_INSTANTIATE_MIXED(D)                                                                                \
    template cudaError_t launch_pass_t<D>(int, const Work &, const Sched &, int, int, int, cudaStream_t); \
    template size_t smem_t<D>(int, int, int);                                                                    \
    template int occupancy_t<D>(int, int, int);

}  // namespace hk
