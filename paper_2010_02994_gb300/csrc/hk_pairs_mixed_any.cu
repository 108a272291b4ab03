// The rate and gradient passes over a batch of several dimensions in one
// persistent launch (pair_kernel_any_d): every dimension's pair blocks in
// one work list, each item dispatched on its set's dimension.
#include <algorithm>

#include "hk_pairs_mixed.cuh"

namespace hk {

namespace {

// The largest dynamic shared memory any dimension's block of `warps` row
// groups (one column group) needs in pass KIND.
template <int KIND>
size_t any_smem(int warps)
{
    size_t m = 0;
    m = std::max(m, pair_smem_bytes<KIND, 1, rows_per_lane(1)>(warps, 1));
    m = std::max(m, pair_smem_bytes<KIND, 2, rows_per_lane(2)>(warps, 1));
    m = std::max(m, pair_smem_bytes<KIND, 3, rows_per_lane(3)>(warps, 1));
    m = std::max(m, pair_smem_bytes<KIND, 4, rows_per_lane(4)>(warps, 1));
    m = std::max(m, pair_smem_bytes<KIND, 5, rows_per_lane(5)>(warps, 1));
    m = std::max(m, pair_smem_bytes<KIND, 6, rows_per_lane(6)>(warps, 1));
    m = std::max(m, pair_smem_bytes<KIND, 7, rows_per_lane(7)>(warps, 1));
    m = std::max(m, pair_smem_bytes<KIND, 8, rows_per_lane(8)>(warps, 1));
    return m;
}

template <int KIND>
int any_occupancy(int warps)
{
    int dev = 0, cap = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, pair_kernel_any_d<KIND>);
    const size_t smem_max = std::min<size_t>(any_smem<KIND>(8), (size_t)cap - fa.sharedSizeBytes);
    const size_t smem = any_smem<KIND>(warps);
    if (smem > smem_max)
        return 0;
    cudaFuncSetAttribute(pair_kernel_any_d<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_kernel_any_d<KIND>, warps * 32, smem);
    return nb;
}

}  // namespace

cudaError_t launch_pair_pass_any_d(int pass, const Work &w, const Sched &sc, int grid,
                                   int warps, cudaStream_t s)
{
    if (pass == 1) {
        pair_kernel_any_d<kRate><<<grid, warps * 32, any_smem<kRate>(warps), s>>>(w, sc);
        return cudaGetLastError();
    }
    if (pass == 2) {
        pair_kernel_any_d<kGrad><<<grid, warps * 32, any_smem<kGrad>(warps), s>>>(w, sc);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

int pass_any_d_max_ctas_per_sm(int pass, int warps)
{
    if (pass == 1)
        return any_occupancy<kRate>(warps);
    if (pass == 2)
        return any_occupancy<kGrad>(warps);
    return 0;
}

}  // namespace hk
