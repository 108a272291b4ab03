// BMDS likelihood and gradients (Section 2.2.3, Eq. (4)): FP32 pair kernels
// for D = 5..8, the FP64 pair kernel, the finalize kernels and the launcher.
// The pair kernels and their tiling are described in hk_bmds.cuh.
#include "hk_bmds.cuh"

namespace hk {
namespace bmds {

// Row totals, the gradient, and the two scalars.  A CTA owns 32 consecutive
// rows (never straddling a tile) and splits each row's T slots -- row-side
// slots J = 0..K, then column-side slots I = K+1..T-1, K the row's tile --
// over 8 thread groups, so a warp reads one slot for 32 consecutive rows
// (coalesced).  Groups and rows are combined in a fixed order; the last CTA
// to finish (ticket counter, reset by that CTA) adds the per-CTA value and
// sigma2 sums in CTA order and writes ell_B and d ell_B / d sigma2.  A set
// invalid-data bit in the status word makes every output NaN.
constexpr int kFinRows = 16, kFinGroups = 16, kFinThreads = kFinRows * kFinGroups;

// Compensated (Kahan) sum in the partials' own type: the FP32 partials of the
// mixed precision are added on the FP32 units (FP64 is scarce on this GPU),
// with an error of a few FP32 ulps of the sum of magnitudes.
template <typename F>
struct KSum {
    F s = F(0), c = F(0);
    __device__ __forceinline__ void add(F x)
    {
        const F y = x - c;
        const F t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename F>
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(Args<F> a, int KT, double sigma2, double *out_grad,
                                                               double *blockpart, unsigned *ticket,
                                                               double *out_loglik, double *out_grad_sigma2)
{
    // the per-group sums, later reused for the last CTA's reduction
    static_assert(sizeof(F) * kFinGroups * (kMaxD + 2) * kFinRows >= sizeof(double) * 2 * kFinThreads, "");
    static_assert(kFinThreads >= (kMaxD + 2) * kFinRows, "one thread per value and row combines the groups");
    __shared__ __align__(16) F sh_s[kFinGroups][kMaxD + 2][kFinRows];
    __shared__ F sh_c[kFinGroups][kMaxD + 2][kFinRows];
    __shared__ double sh_tot[kMaxD + 2][kFinRows];
    __shared__ bool last;
    double(*red)[kFinThreads] = reinterpret_cast<double(*)[kFinThreads]>(&sh_s[0][0][0]);
    const int d = a.d;
    const int r = threadIdx.x % kFinRows, gi = threadIdx.x / kFinRows;
    const int64_t i = (int64_t)blockIdx.x * kFinRows + r;
    KSum<F> acc[kMaxD + 2];
    if (i < a.n) {
        const int K = (int)(blockIdx.x * kFinRows / KT), rr = (int)(i - (int64_t)K * KT);
        // slots q = gi, gi + G, ...; four slots' loads are issued before
        // their adds, so each batch of four costs one memory round trip
        // (missing slots add zeros, which leaves a compensated sum exact)
        for (int q0 = gi; q0 < a.T; q0 += 4 * kFinGroups) {
            F v[4][kMaxD + 2];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + u * kFinGroups;
                const bool rowside = q <= K;
                const int nv = q < a.T ? (rowside ? d + 2 : d) : 0;
                const F *P = rowside ? a.rowpart + pair_index(K, q) * (d + 2) * KT + rr
                                     : a.colpart + pair_index(q, K) * d * KT + rr;
#pragma unroll
                for (int c = 0; c < kMaxD + 2; ++c)
                    v[u][c] = c < nv ? P[c * KT] : F(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < kMaxD + 2; ++c)
                    if (c < d + 2)
                        acc[c].add(v[u][c]);
        }
    }
#pragma unroll
    for (int c = 0; c < kMaxD + 2; ++c)
        if (c < d + 2) {
            sh_s[gi][c][r] = acc[c].s;
            sh_c[gi][c][r] = acc[c].c;
        }
    __syncthreads();
    const bool bad = (*(volatile unsigned *)a.status & kStInvalidData) != 0;
    {
        // one thread per (value, row) adds the groups in order
        const int c = threadIdx.x / kFinRows, rr2 = threadIdx.x % kFinRows;
        if (c < d + 2) {
            KSum<F> t;
            for (int g = 0; g < kFinGroups; ++g) {
                t.add(sh_s[g][c][rr2]);
                t.add(-sh_c[g][c][rr2]);
            }
            sh_tot[c][rr2] = t.value();
        }
    }
    __syncthreads();
    if (i < a.n && out_grad && gi < d)
        out_grad[i * d + gi] = bad ? nan("") : sh_tot[gi][r];
    if (threadIdx.x < 32) {
        const bool mine = threadIdx.x < kFinRows && (int64_t)blockIdx.x * kFinRows + threadIdx.x < a.n;
        double v = mine ? sh_tot[d][threadIdx.x] : 0.0, s = mine ? sh_tot[d + 1][threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        if (threadIdx.x == 0) {
            blockpart[2 * blockIdx.x] = v;
            blockpart[2 * blockIdx.x + 1] = s;
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    double v = 0.0, s = 0.0;
    const volatile double *bp = blockpart;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kFinThreads) {
        v += bp[2 * b];
        s += bp[2 * b + 1];
    }
    red[0][threadIdx.x] = v;
    red[1][threadIdx.x] = s;
    __syncthreads();
    for (int o = kFinThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            red[0][threadIdx.x] += red[0][threadIdx.x + o];
            red[1][threadIdx.x] += red[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double c = (double)a.n * (1.0 - (double)a.n) / 4.0;
        *out_loglik = bad ? nan("") : c * log(sigma2) - red[0][0];
        if (out_grad_sigma2)
            *out_grad_sigma2 = bad ? nan("") : c / sigma2 + red[1][0];
        *ticket = 0u;
    }
}

template <typename F>
Consts<F> make_consts(double sigma2)
{
    const double sigma = std::sqrt(sigma2);
    Consts<F> k;
    k.inv_sigma = (F)(1.0 / sigma);
    k.inv_s2 = (F)(1.0 / sigma2);
    k.h2 = (F)(0.5 / sigma2);
    k.h4 = (F)(0.5 / (sigma2 * sigma2));
    k.h3 = (F)(0.5 / (sigma2 * sigma));
    return k;
}

}  // namespace bmds

// FP32 pair kernels for D = 1..4 live in hk_bmds_lo.cu.
cudaError_t launch_bmds_pairs_f32_lo(const bmds::Args<float> &a, bool y_f32, bool value, int W, int64_t pairs,
                                     cudaStream_t s);

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

cudaError_t launch_f32_hi(const bmds::Args<float> &a, bool y_f32, bool value, int W, int64_t pairs, cudaStream_t s)
{
#define HK_BMDS_CASE(D)                       \
    case D:                                   \
        if (W == 4)                           \
            launch_f32<D, 4>(a, y_f32, value, pairs, s); \
        else                                  \
            launch_f32<D, 2>(a, y_f32, value, pairs, s); \
        break;
    switch (a.d) {
        HK_BMDS_CASE(5)
        HK_BMDS_CASE(6)
        HK_BMDS_CASE(7)
        HK_BMDS_CASE(8)
    default:
        return cudaErrorInvalidValue;
    }
#undef HK_BMDS_CASE
    return cudaGetLastError();
}

constexpr int kFp64Warps = 2;

// 128-row tiles from 8192 events (at least 2080 tile pairs); 64-row tiles
// below. On one GB300 the two sizes break even near 8300 events; the smaller
// tile is 2% faster at 4733 events and 15% faster at 6000 (two dimensions),
// the larger one 5-7% faster from 12000 events on.
int choose_warps(int64_t n, bool fp64) { return fp64 ? kFp64Warps : (n >= 8192 ? 4 : 2); }

struct Layout {
    int W, KT, T;
    int64_t pairs;
    size_t off_ticket, off_row, off_col, off_blk, bytes;
    int nblocks;
};

// Workspace: the finalize ticket counter in the first 256 bytes (zeroed when
// the workspace is allocated, reset by the finalize kernel after each use,
// so it stays zero whatever n the next call has), then the row and column
// partial slots and the per-CTA sums.
Layout layout(int64_t n, int d, bool fp64)
{
    Layout L;
    L.W = choose_warps(n, fp64);
    L.KT = 32 * L.W;
    L.T = (int)((n + L.KT - 1) / L.KT);
    L.pairs = bmds::pair_index(L.T, 0);
    const size_t elem = fp64 ? sizeof(double) : sizeof(float);
    const size_t row_bytes = (size_t)L.pairs * (d + 2) * L.KT * elem;
    const size_t col_bytes = (size_t)L.pairs * d * L.KT * elem;
    L.nblocks = (int)((n + bmds::kFinRows - 1) / bmds::kFinRows);
    L.off_ticket = 0;
    L.off_row = 256;
    L.off_col = (L.off_row + row_bytes + 255) & ~size_t(255);
    L.off_blk = (L.off_col + col_bytes + 255) & ~size_t(255);
    L.bytes = L.off_blk + (size_t)L.nblocks * 2 * sizeof(double);
    return L;
}

}  // namespace

namespace {

__global__ void sort_y_kernel(const void *__restrict__ Y, int y_f32, const int32_t *__restrict__ perm, int64_t n,
                              int64_t npad, float *__restrict__ Ys)
{
    const int64_t i = blockIdx.x;
    const int64_t a = i < n ? perm[i] : -1;
    for (int64_t j = threadIdx.x; j < npad; j += blockDim.x) {
        float v = 0.0f;
        if (a >= 0 && j < n && j != i) {
            const int64_t b = perm[j];
            const int64_t hi = a > b ? a : b, lo = a > b ? b : a;
            v = y_f32 ? static_cast<const float *>(Y)[hi * n + lo]
                      : __double2float_rn(static_cast<const double *>(Y)[hi * n + lo]);
        }
        Ys[i * npad + j] = v;
    }
}

}  // namespace

cudaError_t launch_bmds_sort_y(const void *Y, bool y_f32, const int32_t *perm, int64_t n, int64_t npad, float *Ys,
                               cudaStream_t s)
{
    if (npad <= 0)
        return cudaSuccess;
    sort_y_kernel<<<(unsigned)npad, 256, 0, s>>>(Y, y_f32 ? 1 : 0, perm, n, npad, Ys);
    return cudaGetLastError();
}

size_t bmds_workspace_bytes(int64_t n, int d, bool fp64) { return layout(n, d, fp64).bytes; }


cudaError_t launch_bmds(const void *Y, bool y_f32, const double *X, int64_t n, int d, double sigma2, bool fp64, void *ws,
                        unsigned *status, double *out_loglik, double *out_grad, double *out_grad_sigma2,
                        cudaStream_t s, int64_t *launches, bool value)
{
    const Layout L = layout(n, d, fp64);
    char *base = static_cast<char *>(ws);
    double *blockpart = reinterpret_cast<double *>(base + L.off_blk);
    unsigned *ticket = reinterpret_cast<unsigned *>(base + L.off_ticket);
    cudaError_t e;
    if (fp64) {
        bmds::Args<double> a{Y, X, n, d, L.T, bmds::make_consts<double>(sigma2),
                             reinterpret_cast<double *>(base + L.off_row), reinterpret_cast<double *>(base + L.off_col),
                             status};
        if (y_f32)
            bmds::pairs_kernel<double, float, 0, kFp64Warps><<<(unsigned)L.pairs, 32 * kFp64Warps, 0, s>>>(a);
        else
            bmds::pairs_kernel<double, double, 0, kFp64Warps><<<(unsigned)L.pairs, 32 * kFp64Warps, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        bmds::finalize_kernel<double><<<L.nblocks, bmds::kFinThreads, 0, s>>>(a, L.KT, sigma2, out_grad, blockpart,
                                                                             ticket, out_loglik, out_grad_sigma2);
    } else {
        bmds::Args<float> a{Y, X, n, d, L.T, bmds::make_consts<float>(sigma2),
                            reinterpret_cast<float *>(base + L.off_row), reinterpret_cast<float *>(base + L.off_col),
                            status};
        e = d <= 4 ? launch_bmds_pairs_f32_lo(a, y_f32, value, L.W, L.pairs, s)
                   : launch_f32_hi(a, y_f32, value, L.W, L.pairs, s);
        if (e != cudaSuccess)
            return e;
        bmds::finalize_kernel<float><<<L.nblocks, bmds::kFinThreads, 0, s>>>(a, L.KT, sigma2, out_grad, blockpart,
                                                                            ticket, out_loglik, out_grad_sigma2);
    }
    if (launches)
        *launches += 2;
    return cudaGetLastError();
}

}  // namespace hk
