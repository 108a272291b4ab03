// Input validation, time sort and packing of the per-row arrays.
//
// The pair kernels visit events in time order: the self-excitation indicator
// I[t_n' < t_n] of Section 2.1 then says that, of an unordered pair, only the
// later event is excited, and exactly tied times form contiguous runs that
// the kernels mask by index.  Coordinates and times are scaled so that the
// background kernel's exponent is a plain sum of squares in base 2, and split
// into an FP32 hi/lo pair so that differences of nearby events keep their
// full relative accuracy in FP32.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>

#include "hk_internal.cuh"

namespace hk {

namespace {

__device__ __forceinline__ int find_set_by(const int64_t *starts, int nsets, int64_t idx)
{
    // largest s with starts[s] <= idx (starts ascending, nsets >= 1)
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= idx)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void validate_keys_kernel(const double *__restrict__ t, const double *__restrict__ X, int64_t n_total,
                                     int64_t x_total, double *__restrict__ keys, int32_t *__restrict__ vals,
                                     const int64_t *__restrict__ set_ev0, int32_t nsets, unsigned *status)
{
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_total; e += stride) {
        double v = t[e];
        if (!(v >= 0.0) || !isfinite(v))
            bad = true;
        keys[e] = v;
        int s = find_set_by(set_ev0, nsets, e);
        vals[e] = (int32_t)(e - set_ev0[s]);
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < x_total; e += stride) {
        if (!isfinite(X[e]))
            bad = true;
    }
    if (bad)
        atomicOr(status, kStInvalidData);
}

__global__ void identity_order_kernel(const double *__restrict__ t, double *__restrict__ keys,
                                      int32_t *__restrict__ vals, int64_t n_total,
                                      const int64_t *__restrict__ set_ev0, int32_t nsets, unsigned *status)
{
    bool unsorted = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_total; e += stride) {
        int s = find_set_by(set_ev0, nsets, e);
        keys[e] = t[e];
        vals[e] = (int32_t)(e - set_ev0[s]);
        if (e + 1 < set_ev0[s + 1] && t[e + 1] < t[e])
            unsorted = true;
    }
    if (unsorted)
        atomicOr(status, kStNotSorted | kStInvalidData);
}

// FP32 hi/lo split: hi = fl(v), lo = fl(v - hi).  For two events the
// difference (hi_a - hi_b) + (lo_a - lo_b) then has a relative error of a
// few FP32 units of the difference itself, not of the coordinates.
__device__ __forceinline__ void split_hilo(double v, float &hi, float &lo)
{
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

// One thread per row of every set.
__global__ void pack_kernel(Work w, const double *__restrict__ X, const double *__restrict__ keys_sorted,
                            const int32_t *__restrict__ vals_sorted, int64_t total_rows,
                            const int64_t *__restrict__ set_row0)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total_rows; r += stride) {
        const int s = find_set_by(set_row0, w.nsets, r);
        const SetDesc &S = w.sets[s];
        const int64_t i = r - S.row0;
        const int d = S.d;
        const int np = nrec(d);
        float f[4 * nrec(kMaxD)];
#pragma unroll
        for (int k = 0; k < 4 * nrec(kMaxD); ++k)
            f[k] = 0.0f;
        if (i < S.n) {
            const int32_t src = vals_sorted[S.ev0 + i];
            const double tv = keys_sorted[S.ev0 + i];
            w.perm[r] = src;
            w.t64[r] = tv;
            for (int k = 0; k < d; ++k) {
                double xv = X[S.x0 + (int64_t)src * d + k];
                w.x64[r * kMaxD + k] = xv;
                split_hilo(xv * S.kx, f[2 * k], f[2 * k + 1]);
            }
            split_hilo(tv * S.kt, f[2 * d], f[2 * d + 1]);
            // Lambda_n, Section 2.1 (T = the set's largest time)
            const double T = keys_sorted[S.ev0 + S.n - 1];
            const double a = T - tv;
            w.Lam64[r] = S.mu0 * (normcdf(a / S.tau_t) - normcdf(-tv / S.tau_t)) - S.theta * expm1(-S.omega * a);
            // first row of a strictly later time (upper bound of tv); most
            // times are unique, so look at the next row before searching
            int64_t lo = i + 1, hi = S.n;
            if (lo < hi && keys_sorted[S.ev0 + lo] > tv)
                hi = lo;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (keys_sorted[S.ev0 + mid] > tv)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            w.tie_end[r] = (int32_t)lo;
        } else {
            w.perm[r] = -1;
            w.t64[r] = 0.0;
            for (int k = 0; k < d; ++k)
                w.x64[r * kMaxD + k] = 0.0;
            f[2 * d] = kPadTime;
            w.Lam64[r] = 0.0;
            w.tie_end[r] = (int32_t)(i + 1);
        }
        w.w32[r] = 0.0f;
        w.cm32[r] = -INFINITY;
        for (int p = 0; p < np; ++p)
            w.rec[S.rec0 + (int64_t)p * S.npad + i] = make_float4(f[4 * p], f[4 * p + 1], f[4 * p + 2], f[4 * p + 3]);
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1)
        g = 1;
    if (g > 4096)
        g = 4096;
    return (int)g;
}

}  // namespace

cudaError_t launch_validate_keys(const double *t, const double *X, int64_t n_total, int64_t x_total, double *keys,
                                 int32_t *vals, const int64_t *set_ev0, int32_t nsets, unsigned *status,
                                 cudaStream_t s)
{
    validate_keys_kernel<<<grid_for(x_total > n_total ? x_total : n_total, 256), 256, 0, s>>>(
        t, X, n_total, x_total, keys, vals, set_ev0, nsets, status);
    return cudaGetLastError();
}

cudaError_t launch_identity_order(const double *t, double *keys_out, int32_t *vals_out, int64_t n_total,
                                  const int64_t *set_ev0, int32_t nsets, unsigned *status, cudaStream_t s)
{
    identity_order_kernel<<<grid_for(n_total, 256), 256, 0, s>>>(t, keys_out, vals_out, n_total, set_ev0, nsets,
                                                                    status);
    return cudaGetLastError();
}

// Batches are sorted by two stable radix sorts instead of a segmented one:
// every event by its full FP64 time (value: its global index), then that
// order by set index (a few key bits).  The result is exact -- grouped by
// set, in time order within a set, ties in the caller's order -- and costs
// a handful of full-width passes instead of one small sort per set.
namespace {

// Sort of one set of at most kCountSortMax events by rank counting (about
// ten instructions per comparison, N^2 comparisons spread over every SM).  The key
// of an event is the bit pattern of its time with the sign cleared: times are
// validated non-negative, non-negative doubles order like their bit patterns,
// and -0 then equals +0.  Event i's rank is the number of events j with
// key_j < key_i, or key_j == key_i and j < i (the caller's order among equal
// times, as a stable sort keeps it).  Each thread counts for kCountPer events
// over one slice of the keys, staged in shared memory; the slices' counts
// are added with integer atomics, exact in any order.
constexpr int kCountSortMax = 12288;  // N^2 comparisons: beyond this the radix sort is faster on GB300
constexpr int kCountThreads = 256, kCountPer = 4, kCountPerCta = kCountThreads * kCountPer;
constexpr int kCountTile = 1024, kCountSplitsMax = 64, kCountCtas = 608;  // 4 CTAs per SM

__device__ __forceinline__ unsigned long long time_key(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

__global__ void __launch_bounds__(kCountThreads) count_rank_kernel(const double *__restrict__ keys, int n, int splits,
                                                                   int32_t *rank)
{
    __shared__ unsigned long long sk[kCountTile];
    int idx[kCountPer];
    unsigned long long key[kCountPer];
    int cnt[kCountPer];
#pragma unroll
    for (int k = 0; k < kCountPer; ++k) {
        idx[k] = blockIdx.x * kCountPerCta + k * kCountThreads + threadIdx.x;
        key[k] = idx[k] < n ? time_key(keys[idx[k]]) : 0ull;
        cnt[k] = 0;
    }
    const int per = (n + splits - 1) / splits;
    const int lo = min((int)blockIdx.y * per, n), hi = min(lo + per, n);
    for (int j0 = lo; j0 < hi; j0 += kCountTile) {
        const int m = min(kCountTile, hi - j0);
        __syncthreads();
        for (int u = threadIdx.x; u < m; u += kCountThreads)
            sk[u] = time_key(keys[j0 + u]);
        __syncthreads();
        for (int u = 0; u < m; ++u) {
            const unsigned long long kj = sk[u];
            const int j = j0 + u;
#pragma unroll
            for (int k = 0; k < kCountPer; ++k)
                cnt[k] += (kj < key[k] || (kj == key[k] && j < idx[k])) ? 1 : 0;
        }
    }
#pragma unroll
    for (int k = 0; k < kCountPer; ++k)
        if (idx[k] < n && cnt[k])
            atomicAdd(rank + idx[k], cnt[k]);
}

__global__ void scatter_rank_kernel(const double *__restrict__ keys_in, const int32_t *__restrict__ vals_in,
                                    const int32_t *__restrict__ rank, int n, double *keys_out, int32_t *vals_out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = rank[i];
        keys_out[r] = __longlong_as_double((long long)time_key(keys_in[i]));
        vals_out[r] = vals_in[i];
    }
}

}  // namespace

namespace {

int set_bits(int32_t nsets)
{
    int b = 1;
    while ((1 << b) < nsets)
        ++b;
    return b;
}

__global__ void iota_kernel(int32_t *v, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (int32_t)i;
}

__global__ void set_key_kernel(const int32_t *__restrict__ gidx, int32_t *__restrict__ key, int64_t n,
                               const int64_t *__restrict__ set_ev0, int32_t nsets)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        key[i] = find_set_by(set_ev0, nsets, gidx[i]);
}

// final order: times and set-relative indices, as the segmented sort gave
__global__ void batch_order_kernel(const double *__restrict__ t, const int32_t *__restrict__ gidx,
                                   double *__restrict__ keys_out, int32_t *__restrict__ vals_out, int64_t n,
                                   const int64_t *__restrict__ set_ev0, int32_t nsets)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = gidx[i];
        keys_out[i] = t[g];
        vals_out[i] = (int32_t)(g - set_ev0[find_set_by(set_ev0, nsets, g)]);
    }
}

}  // namespace

size_t sort_temp_bytes(int64_t n_total, int32_t nsets)
{
    size_t bytes = 0, b2 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, bytes, (const double *)nullptr, (double *)nullptr,
                                    (const int32_t *)nullptr, (int32_t *)nullptr, (int)n_total);
    if (nsets > 1)
        cub::DeviceRadixSort::SortPairs(nullptr, b2, (const int32_t *)nullptr, (int32_t *)nullptr,
                                        (const int32_t *)nullptr, (int32_t *)nullptr, (int)n_total, 0,
                                        set_bits(nsets));
    return bytes > b2 ? bytes : b2;
}

cudaError_t launch_sort(void *temp, size_t temp_bytes, const double *t, double *keys_in, double *keys_out,
                        int32_t *vals_in, int32_t *vals_out, int64_t n_total, int32_t nsets,
                        const int64_t *d_set_ev0, cudaStream_t s, int64_t *launches, int64_t *lib_launches)
{
    // Both sorts are stable: events with equal times keep the caller's order.
    if (nsets <= 1 && n_total <= kCountSortMax && temp_bytes >= sizeof(int32_t) * (size_t)n_total) {
        // one set of at most 12288 events: ranks by counting, which takes a
        // few microseconds where the eight radix passes take tens
        int32_t *rank = static_cast<int32_t *>(temp);
        cudaError_t e = cudaMemsetAsync(rank, 0, sizeof(int32_t) * n_total, s);
        if (e != cudaSuccess)
            return e;
        const int n = (int)n_total;
        const int gx = (n + kCountPerCta - 1) / kCountPerCta;
        const int splits = std::max(1, std::min({kCountSplitsMax, kCountCtas / gx, n / 64}));
        const dim3 grid((unsigned)gx, (unsigned)splits);
        count_rank_kernel<<<grid, kCountThreads, 0, s>>>(keys_in, n, splits, rank);
        scatter_rank_kernel<<<grid_for(n_total, 256), 256, 0, s>>>(keys_in, vals_in, rank, n, keys_out, vals_out);
        if (launches)
            *launches += 2;
        return cudaGetLastError();
    }
    if (lib_launches)
        *lib_launches += nsets <= 1 ? 1 : 2;
    if (nsets <= 1)
        return cub::DeviceRadixSort::SortPairs(temp, temp_bytes, keys_in, keys_out, vals_in, vals_out, (int)n_total,
                                               0, 64, s);
    const int g = grid_for(n_total, 256);
    iota_kernel<<<g, 256, 0, s>>>(vals_in, n_total);
    cudaError_t e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, keys_in, keys_out, vals_in, vals_out,
                                                    (int)n_total, 0, 64, s);
    if (e != cudaSuccess)
        return e;
    // keys_in is free now: its 8-byte slots hold two int32 key arrays
    int32_t *sk_in = reinterpret_cast<int32_t *>(keys_in), *sk_out = sk_in + n_total;
    set_key_kernel<<<g, 256, 0, s>>>(vals_out, sk_in, n_total, d_set_ev0, nsets);
    e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, sk_in, sk_out, vals_out, vals_in, (int)n_total, 0,
                                        set_bits(nsets), s);
    if (e != cudaSuccess)
        return e;
    batch_order_kernel<<<g, 256, 0, s>>>(t, vals_in, keys_out, vals_out, n_total, d_set_ev0, nsets);
    if (launches)
        *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_pack_rows(const Work &w, const double *X, const double *keys_sorted, const int32_t *vals_sorted,
                             int64_t total_rows, const int64_t *set_row0, cudaStream_t s)
{
    // 64-thread CTAs: the FP64 work per row (Lambda, the hi/lo splits) spreads
    // over four times as many SMs at the sizes of the paper's data sets
    pack_kernel<<<grid_for(total_rows, 64), 64, 0, s>>>(w, X, keys_sorted, vals_sorted, total_rows, set_row0);
    return cudaGetLastError();
}

}  // namespace hk
