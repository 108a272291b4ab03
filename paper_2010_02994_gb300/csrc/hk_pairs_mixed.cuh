// Mixed-precision pair kernels: the two O(N^2) passes of the log-likelihood
// (Eq. (1)) and of its location gradient (Appendix A).
//
// Formulation.  Rows are events in time order, so for an unordered pair
// (n, m) with n < m and t_n < t_m only the later event m is self-excited by
// n (the indicator I[t_n' < t_n] of Section 2.1), while the background term
// is symmetric: mu_nm = mu_mn.  With coordinates scaled by
// kx = sqrt(log2(e)/2)/tau_x and times by kt = sqrt(log2(e)/2)/tau_t,
//   q   = |x~_m - x~_n|^2,   dt = t~_m - t~_n >= 0
//   mu' = 2^(-q - dt^2)                      = mu_nm / P_mu
//   xi''= 2^(c_xi1 - rho q - kappa dt)       = xi_mn / P_mu
// with rho = tau_x^2/h^2, kappa = omega log2(e)/kt,
// c_xi1 = log2(theta omega tau_x^D tau_t sqrt(2 pi) / (mu0 h^D)) and
// P_mu = mu0 / (tau_x^D tau_t (2 pi)^((D+1)/2)).  Each kernel value is one
// MUFU ex2.
//   The self-excitation exponent is not formed as c_xi1 - kappa dt - rho q
//   with c_xi1 and kappa rounded to FP32 once per set: that rounding would
//   bias every xi'' of the set the same way (a relative error of a few
//   1e-7 shared by all terms, which the sum over N rows does not average
//   out).  Instead each row carries a = c_xi1 + kappa (t~_n - o) and each
//   staged column b = kappa (t~_m - o), both relative to the block's time
//   origin o and formed with a two-word kappa and c_xi1, so the exponent is
//   fmaf(-rho, q, a - b): the same two operations, with rounding errors
//   that differ from row to row and column to column.
//   Rate pass: S_n += mu' for the earlier event, S_m += mu' + xi'' for the
//     later one; lambda_n = P_mu S_n.
//   Gradient pass: with w = 1/S, c = mu' (w_n + w_m) + 2^(C_m - rho q - kappa dt),
//     C_m = c_xi1 + log2(rho) + log2(w_m) (per column, from the finalize step;
//     the row carries a = kappa (t~_n - o), the staged column
//     b = kappa (t~_m - o) - C_m):
//     g~_n += c (x~_m - x~_n),  g~_m -= c (x~_m - x~_n);
//     d ell/d x_n = g~_n / (tau_x^2 kx).
//   Rate pass with Theta sums: also mu' q, mu' dt^2 (both events) and
//     xi'' dt, xi'' q (later event) for the parameter gradient.
//
// Tiling.  A CTA of W warps processes one pair block (I, J), I <= J, of
// B = 32 R W rows (block I) by B columns (block J) at a time, taking blocks
// from a persistent work list.  Each lane keeps R rows in registers for the
// whole block.  Each warp sweeps block J in chunks of 32 columns, read from
// L2 one chunk ahead; a chunk is staged in a warp-private shared buffer with
// every record written twice (entries L and L + 32), so that at step j lane L
// reads entry L + j -- column (L + j) mod 32 -- at a compile-time offset.
// The lane adds that column's share into an accumulator that then moves to
// lane L - 1 by one shuffle; after 32 steps every column's total over the
// warp's rows sits in one lane, with no transpose and no atomics.  Row sums
// are compensated (Kahan) once per chunk.  Per-warp column totals are summed
// over the warps at the end of the block, and the block's row and column
// totals go to one partial slot each (see hk_internal.cuh).  Pairs that must
// not count (m <= n in a diagonal block, exactly tied times) are removed by an
// index test only in the chunks that can contain them.
#pragma once

#include "hk_bmds.cuh"
#include "hk_internal.cuh"

namespace hk {

// kRateXi: the rate pass that also keeps the self-excitation sum of each row
// apart (plane 0: background terms, plane 1: self-excitation terms).
// kGradB: the gradient pass that also carries the BMDS term of Eq. (4) (the
// BMDS-Hawkes potential of Section 3): every unordered pair of distinct
// events adds coef_B (x_m - x_n) to g_n (and the opposite to g_m) beside its
// Hawkes term, with the observed distance y from a time-ordered copy of Y.
enum PairKind : int { kRate = 0, kRateTheta = 1, kGrad = 2, kRateXi = 3, kGradB = 4 };

template <int KIND>
__host__ __device__ constexpr bool grad_kind()
{
    return KIND == kGrad || KIND == kGradB;
}

template <int KIND, int D>
struct KindTraits {
    static constexpr int VR = grad_kind<KIND>() ? D : (KIND == kRateTheta ? 3 : 1);   // values per row
    static constexpr int VC = grad_kind<KIND>() ? D : (KIND == kRateTheta ? 6 : (KIND == kRateXi ? 2 : 1));  // per column
    // staged fields: coordinates (hi, lo), time, then b (rate kinds) or
    // w_m and b (gradient)
    static constexpr int NF = grad_kind<KIND>() ? 2 * D + 3 : 2 * D + 2;
    static constexpr int NPP = (NF + 3) / 4;                                       // staged float4 planes
};

// Which partial plane a row value goes to (the Theta pass's rows carry
// planes 0, 2, 3 of the six).
template <int KIND>
__device__ __forceinline__ int row_plane(int v)
{
    return KIND == kRateTheta ? (v == 0 ? 0 : v + 1) : v;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int D>
__device__ __forceinline__ void load_rec(const float4 *__restrict__ planes, int64_t stride, int64_t i,
                                         float (&f)[4 * nrec(D)])
{
#pragma unroll
    for (int p = 0; p < nrec(D); ++p) {
        const float4 v = planes[(int64_t)p * stride + i];
        f[4 * p + 0] = v.x;
        f[4 * p + 1] = v.y;
        f[4 * p + 2] = v.z;
        f[4 * p + 3] = v.w;
    }
}

struct PairConsts {
    float rho, kappa, cxi;
};

// The BMDS term of kGradB: q scale 1/kx^2 (scaled q -> delta^2), coefficient
// scale tau_x^2 (a BMDS coefficient in the scaled gradient's units),
// 1/sigma and 1/sigma2; ys: this lane's row of the chunk's Y in shared
// memory (row r of the lane at ys[1024 r]), row0: the warp's first row, n:
// events of the set.
struct BmdsIn {
    float qscale, cscale, inv_sigma, inv_s2;
    const float *ys;
    int row0, n;
};

// c + k t for the two-word constant k = k_hi + k_lo (and c = c_hi + c_lo),
// with the error of one FP32 rounding of the result: the product's rounding
// error is recovered exactly by an FMA and added back with the low words.
__device__ __forceinline__ float kt_plus_c(float k_hi, float k_lo, float t, float c_hi, float c_lo)
{
    const float p = k_hi * t;
    const float e = fmaf(k_hi, t, -p);
    return (c_hi + p) + fmaf(k_lo, t, e + c_lo);
}

// Asynchronous global -> shared copies (16 bytes each, bypassing L1) for the
// Y tiles of kGradB: a warp's 32 R rows x 32 columns, row stride ld floats
// in global memory, 32 in shared memory; lanes 8k .. 8k + 7 copy one row.
__device__ __forceinline__ void cp_async16(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int R>
__device__ __forceinline__ void stage_y_async(float *dst, const float *src, int64_t ld, int lane)
{
#pragma unroll 4
    for (int k = 0; k < R * 8; ++k) {
        const int v = 32 * k + lane, row = v >> 3, seg = v & 7;
        cp_async16(dst + 32 * row + 4 * seg, src + (int64_t)row * ld + 4 * seg);
    }
}

// One pair: its contributions to the row's values (part) and to the
// travelling column accumulator (acc).  cf holds the staged column fields.
template <int KIND, int D>
__device__ __forceinline__ void pair_update(const float *cf, const float *rx, float rt, float rw, float ra,
                                            const PairConsts &k, bool valid, float *part, float *acc,
                                            const BmdsIn &kb, float y, bool valid_b)
{
    float dx[D], q;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        dx[d] = (cf[2 * d] - rx[2 * d]) + (cf[2 * d + 1] - rx[2 * d + 1]);
        q = d == 0 ? dx[0] * dx[0] : fmaf(dx[d], dx[d], q);
    }
    const float dt = cf[2 * D] - rt;
    if (KIND == kRate) {
        float mu = ex2_approx(fmaf(-dt, dt, -q));
        float xi = ex2_approx(fmaf(-k.rho, q, ra - cf[2 * D + 1]));
        if (!valid) {
            mu = 0.0f;
            xi = 0.0f;
        }
        part[0] += mu;
        acc[0] += mu;
        acc[0] += xi;
    } else if (KIND == kRateXi) {
        float mu = ex2_approx(fmaf(-dt, dt, -q));
        float xi = ex2_approx(fmaf(-k.rho, q, ra - cf[2 * D + 1]));
        if (!valid) {
            mu = 0.0f;
            xi = 0.0f;
        }
        part[0] += mu;
        acc[0] += mu;
        acc[1] += xi;
    } else if (KIND == kRateTheta) {
        const float dt2 = dt * dt;
        float mu = ex2_approx(-q - dt2);
        float xi = ex2_approx(fmaf(-k.rho, q, ra - cf[2 * D + 1]));
        if (!valid) {
            mu = 0.0f;
            xi = 0.0f;
        }
        part[0] += mu;
        part[1] = fmaf(mu, q, part[1]);
        part[2] = fmaf(mu, dt2, part[2]);
        acc[0] += mu;
        acc[1] += xi;
        acc[2] = fmaf(mu, q, acc[2]);
        acc[3] = fmaf(mu, dt2, acc[3]);
        acc[4] = fmaf(xi, dt, acc[4]);
        acc[5] = fmaf(xi, q, acc[5]);
    } else {
        // staged fields: 2D = time, 2D+1 = w_m, 2D+2 = b = kappa (t~_m - o) - C_m
        float mu = ex2_approx(fmaf(-dt, dt, -q));
        float xw = ex2_approx(fmaf(-k.rho, q, ra - cf[2 * D + 2]));
        if (!valid) {
            mu = 0.0f;
            xw = 0.0f;
        }
        float c = fmaf(mu, rw + cf[2 * D + 1], xw);
        if (KIND == kGradB) {
            const float cb = bmds::grad_coef(q * kb.qscale, y, kb.inv_sigma, kb.inv_s2);
            c = valid_b ? fmaf(cb, kb.cscale, c) : c;
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
            part[d] = fmaf(c, dx[d], part[d]);
            acc[d] = fmaf(-c, dx[d], acc[d]);
        }
    }
}

// 32 steps over one staged chunk.  pv points at this lane's entry of the
// warp's staged buffer ([NPP][64] float4).  MASKED chunks test every pair
// against the rows' tie ends (m >= tie_end excludes m <= n and tied times).
template <int KIND, int D, int R, bool MASKED>
__device__ __forceinline__ void chunk_steps(const float4 *__restrict__ pv, int src_lane, int lane, int m0,
                                            const int *__restrict__ te, const float (&rx)[R][2 * D],
                                            const float (&rt)[R], const float (&rw)[R], const float (&ra)[R],
                                            const PairConsts &k, float (&part)[R][KindTraits<KIND, D>::VR],
                                            float (&acc)[KindTraits<KIND, D>::VC], const BmdsIn &kb)
{
    using T = KindTraits<KIND, D>;
    // unrolled by 16: 1% shorter than 8 for the gradient pass at N = 1e5 on
    // GB300 (4 and 32 are slower; the arithmetic and its order are unchanged)
#pragma unroll(MASKED ? 1 : 16)
    for (int j = 0; j < 32; ++j) {
        float cf[4 * T::NPP];
#pragma unroll
        for (int p = 0; p < T::NPP; ++p) {
            const float4 v = pv[p * 64 + j];
            cf[4 * p + 0] = v.x;
            cf[4 * p + 1] = v.y;
            cf[4 * p + 2] = v.z;
            cf[4 * p + 3] = v.w;
        }
        const int m = m0 + ((lane + j) & 31);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const bool valid = MASKED ? (m >= te[32 * r + lane]) : true;
            // BMDS: every pair of distinct events once (m later in the
            // order than the row), padded columns excluded
            const bool valid_b = KIND == kGradB && MASKED ? (m < kb.n && m > kb.row0 + 32 * r + lane) : true;
            const float y = KIND == kGradB ? kb.ys[32 * 32 * r + ((lane + j) & 31)] : 0.0f;
            pair_update<KIND, D>(cf, rx[r], rt[r], rw[r], ra[r], k, valid, part[r], acc, kb, y, valid_b);
        }
#pragma unroll
        for (int v = 0; v < T::VC; ++v)
            acc[v] = __shfl_sync(0xffffffffu, acc[v], src_lane);
    }
}

// Dynamic shared memory of pair_kernel<KIND, D, R> with W warps, WC of
// them column groups (W / WC row groups; B = 32 R W / WC rows per block).
template <int KIND, int D, int R>
constexpr size_t pair_smem_bytes(int W, int WC)
{
    using T = KindTraits<KIND, D>;
    const int WR = W / WC;
    const size_t B = 32 * (size_t)R * WR;
    return (size_t)W * T::NPP * 64 * sizeof(float4)      // staged chunks
           + (size_t)WR * T::VC * B * sizeof(float)       // column totals of each row group
           + (size_t)WC * T::VC * B * sizeof(float)       // row totals of each column group
           + (size_t)W * 32 * R * sizeof(int)             // tie ends of each warp's rows
           + (KIND == kGradB ? (size_t)W * 2 * 32 * R * 32 * sizeof(float) : 0);  // each warp's two Y buffers
}

// One pair block {I, J} (I <= J) of set wi.set by the whole CTA: its warps
// form blockDim.x / 32 / WC row groups of 32 R rows of block I and WC column
// groups of B / WC columns of block J, so that at small N a block is swept
// by more warps (and ends sooner) without making the blocks, and with them
// the partial slots, smaller.  smem4 is the kernel's dynamic shared memory.
template <int KIND, int D, int R, int WC>
__device__ __forceinline__ void pair_item(const Work &w, const WorkItem wi, float4 *smem4)
{
    constexpr int wc = WC;
    using T = KindTraits<KIND, D>;
    constexpr int NP = nrec(D), NPP = T::NPP, VR = T::VR, VC = T::VC;
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wr = warps / wc, rg = warp / wc, cg = warp % wc;
    const int B = 32 * R * wr, CB = B / wc;
    float4 *priv = smem4 + warp * NPP * 64;
    float *colpart = reinterpret_cast<float *>(smem4 + warps * NPP * 64);  // [wr][VC][B]
    float *rowpart = colpart + (size_t)wr * VC * B;                        // [wc][VC][B]
    int *te_all = reinterpret_cast<int *>(rowpart + (size_t)wc * VC * B);  // [warps][32 R]
    int *s_te = te_all + warp * 32 * R;
    float *ysw = reinterpret_cast<float *>(te_all + warps * 32 * R) + (size_t)warp * 2 * 32 * R * 32;  // kGradB
    const int src_lane = (lane + 1) & 31;
#include "hk_pair_item.inc"
}

// Persistent pair kernel of one dimension: CTAs take pair blocks from the
// work list (an atomic counter; every thread decodes the block pair) until
// it is exhausted.
template <int KIND, int D, int R, int WC>
__global__ void __launch_bounds__(256)
    pair_kernel(Work w, Sched sc)
{
    constexpr int wc = WC;
    using T = KindTraits<KIND, D>;
    constexpr int NP = nrec(D), NPP = T::NPP, VR = T::VR, VC = T::VC;
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wr = warps / wc, rg = warp / wc, cg = warp % wc;
    const int B = 32 * R * wr, CB = B / wc;
    extern __shared__ float4 smem4[];
    float4 *priv = smem4 + warp * NPP * 64;
    float *colpart = reinterpret_cast<float *>(smem4 + warps * NPP * 64);  // [wr][VC][B]
    float *rowpart = colpart + (size_t)wr * VC * B;                        // [wc][VC][B]
    int *te_all = reinterpret_cast<int *>(rowpart + (size_t)wc * VC * B);  // [warps][32 R]
    int *s_te = te_all + warp * 32 * R;
    float *ysw = reinterpret_cast<float *>(te_all + warps * 32 * R) + (size_t)warp * 2 * 32 * R * 32;  // kGradB
    __shared__ int s_item;
    const int src_lane = (lane + 1) & 31;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(&w.pair_ctr[0], 1);
        __syncthreads();
        const int it = s_item;
        if (it >= sc.nitems)
            break;
        const WorkItem wi = decode_item(w.sets, sc, it);
#include "hk_pair_item.inc"
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(&w.pair_ctr[1], 1);
        if (done == (int)gridDim.x - 1) {
            w.pair_ctr[0] = 0;
            w.pair_ctr[1] = 0;
            __threadfence();
        }
    }
}

// The same over the work items of every dimension in one persistent launch:
// each item is dispatched on its set's dimension (one column group; every
// dimension's blocks are 32 rows_per_lane(d) x blockDim.x / 32 rows).  The
// kernel's register count is the largest any dimension needs.
template <int KIND>
__global__ void __launch_bounds__(256)
    pair_kernel_any_d(Work w, Sched sc)
{
    extern __shared__ float4 smem4[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(&w.pair_ctr[0], 1);
        __syncthreads();
        const int it = s_item;
        if (it >= sc.nitems)
            break;
        const WorkItem wi = decode_item(w.sets, sc, it);
        switch (w.sets[wi.set].d) {
        case 1: pair_item<KIND, 1, rows_per_lane(1), 1>(w, wi, smem4); break;
        case 2: pair_item<KIND, 2, rows_per_lane(2), 1>(w, wi, smem4); break;
        case 3: pair_item<KIND, 3, rows_per_lane(3), 1>(w, wi, smem4); break;
        case 4: pair_item<KIND, 4, rows_per_lane(4), 1>(w, wi, smem4); break;
        case 5: pair_item<KIND, 5, rows_per_lane(5), 1>(w, wi, smem4); break;
        case 6: pair_item<KIND, 6, rows_per_lane(6), 1>(w, wi, smem4); break;
        case 7: pair_item<KIND, 7, rows_per_lane(7), 1>(w, wi, smem4); break;
        default: pair_item<KIND, 8, rows_per_lane(8), 1>(w, wi, smem4); break;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(&w.pair_ctr[1], 1);
        if (done == (int)gridDim.x - 1) {
            w.pair_ctr[0] = 0;
            w.pair_ctr[1] = 0;
            __threadfence();
        }
    }
}

}  // namespace hk
