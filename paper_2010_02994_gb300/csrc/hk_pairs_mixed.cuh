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

#include "hk_internal.cuh"

namespace hk {

// kRateXi: the rate pass that also keeps the self-excitation sum of each row
// apart (plane 0: background terms, plane 1: self-excitation terms).
enum PairKind : int { kRate = 0, kRateTheta = 1, kGrad = 2, kRateXi = 3 };

template <int KIND, int D>
struct KindTraits {
    static constexpr int VR = KIND == kGrad ? D : (KIND == kRateTheta ? 3 : 1);   // values per row
    static constexpr int VC = KIND == kGrad ? D : (KIND == kRateTheta ? 6 : (KIND == kRateXi ? 2 : 1));  // per column
    // staged fields: coordinates (hi, lo), time, then b (rate kinds) or
    // w_m and b (gradient)
    static constexpr int NF = KIND == kGrad ? 2 * D + 3 : 2 * D + 2;
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

// c + k t for the two-word constant k = k_hi + k_lo (and c = c_hi + c_lo),
// with the error of one FP32 rounding of the result: the product's rounding
// error is recovered exactly by an FMA and added back with the low words.
__device__ __forceinline__ float kt_plus_c(float k_hi, float k_lo, float t, float c_hi, float c_lo)
{
    const float p = k_hi * t;
    const float e = fmaf(k_hi, t, -p);
    return (c_hi + p) + fmaf(k_lo, t, e + c_lo);
}

// One pair: its contributions to the row's values (part) and to the
// travelling column accumulator (acc).  cf holds the staged column fields.
template <int KIND, int D>
__device__ __forceinline__ void pair_update(const float *cf, const float *rx, float rt, float rw, float ra,
                                            const PairConsts &k, bool valid, float *part, float *acc)
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
        const float c = fmaf(mu, rw + cf[2 * D + 1], xw);
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
                                            float (&acc)[KindTraits<KIND, D>::VC])
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
            pair_update<KIND, D>(cf, rx[r], rt[r], rw[r], ra[r], k, valid, part[r], acc);
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
           + (size_t)W * 32 * R * sizeof(int);            // tie ends of each warp's rows
}

// Persistent pair kernel.  A CTA of W warps takes pair blocks {I, J} from the
// work list; its warps form W / WC row groups of 32 R rows of block I and WC
// column groups of B / WC columns of block J, so that at small N a block is
// swept by more warps (and ends sooner) without making the blocks, and with
// them the partial slots, smaller.
template <int KIND, int D, int R, int WC>
__global__ void __launch_bounds__(256)
    pair_kernel(Work w, const WorkItem *__restrict__ items, int nitems)
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
    __shared__ int s_item;
    const int src_lane = (lane + 1) & 31;

    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(&w.pair_ctr[0], 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems)
            break;
        const WorkItem wi = items[it];
        const SetDesc &S = w.sets[wi.set];
        const int I = wi.I, J = wi.J, n = S.n, npad = S.npad;
        const float4 *rec = w.rec + S.rec0;
        const float *w32 = w.w32 + S.row0;
        const float *cm32 = w.cm32 + S.row0;
        const PairConsts kc{S.rho, S.kappa, S.cxi1};
        float *P = (KIND == kGrad ? w.P2 + S.part2_0 : w.P1 + S.part0);

        // time origin: the middle row of block I
        float oh, ol;
        {
            const int io = min(I * B + B / 2, n - 1);
            const float4 v = rec[(int64_t)((2 * D) / 4) * npad + io];
            const float *c = reinterpret_cast<const float *>(&v);
            oh = c[(2 * D) % 4];
            ol = c[(2 * D) % 4 + 1];
        }
        // Optional skip of a block that is far apart in time: if even its
        // closest pair has both exponents <= -130, every kernel value of the
        // block flushes to zero in FP32 and its partials are exactly zero.
        bool skip = false;
        if (w.skip_far && I != J) {
            const int il = min(I * B + B - 1, n - 1), jf = J * B;
            const float4 vl = rec[(int64_t)((2 * D) / 4) * npad + il];
            const float4 vf = rec[(int64_t)((2 * D) / 4) * npad + jf];
            const float *cl = reinterpret_cast<const float *>(&vl);
            const float *cf0 = reinterpret_cast<const float *>(&vf);
            const float dtmin = ((cf0[(2 * D) % 4] - oh) + (cf0[(2 * D) % 4 + 1] - ol)) -
                                ((cl[(2 * D) % 4] - oh) + (cl[(2 * D) % 4 + 1] - ol));
            const float cmax = KIND == kGrad ? __int_as_float(w.set_cmmax[wi.set]) : kc.cxi;
            skip = dtmin * dtmin >= 130.0f && cmax - kc.kappa * dtmin <= -130.0f;
        }
        if (skip) {
            for (int c = threadIdx.x; c < B; c += blockDim.x)
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    P[((int64_t)J * VC + v) * npad + (int64_t)I * B + c] = 0.0f;
                    P[((int64_t)I * VC + v) * npad + (int64_t)J * B + c] = 0.0f;
                }
        } else {
            // this lane's rows
            float rx[R][2 * D], rt[R], rw[R], ra[R], part[R][VR], rs[R][VR], rc[R][VR];
            const int rbase = I * B + rg * 32 * R;
            int te_min = 0x7fffffff, te_max = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = rbase + 32 * r + lane;
                float f[4 * NP];
                load_rec<D>(rec, npad, row, f);
#pragma unroll
                for (int q = 0; q < 2 * D; ++q)
                    rx[r][q] = f[q];
                rt[r] = (f[2 * D] - oh) + (f[2 * D + 1] - ol);
                rw[r] = KIND == kGrad ? w32[row] : 0.0f;
                ra[r] = KIND == kGrad ? kt_plus_c(S.kappa, S.kappa_lo, rt[r], 0.0f, 0.0f)
                                      : kt_plus_c(S.kappa, S.kappa_lo, rt[r], S.cxi1, S.cxi1_lo);
                const int te = w.tie_end[S.row0 + row];
                s_te[32 * r + lane] = te;
                te_min = min(te_min, te);
                te_max = max(te_max, te);
#pragma unroll
                for (int v = 0; v < VR; ++v) {
                    rs[r][v] = 0.0f;
                    rc[r][v] = 0.0f;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                te_min = min(te_min, __shfl_xor_sync(0xffffffffu, te_min, o));
                te_max = max(te_max, __shfl_xor_sync(0xffffffffu, te_max, o));
            }
            const int cbase = J * B + cg * CB;
            // prefetch the first chunk's record for this lane
            float pf[4 * NP], pw = 0.0f, pc = 0.0f;
            {
                const int64_t col = (int64_t)cbase + lane;
                load_rec<D>(rec, npad, col, pf);
                if (KIND == kGrad) {
                    pw = w32[col];
                    pc = cm32[col];
                }
            }
            for (int c0 = 0; c0 < CB; c0 += 32) {
                // stage this chunk's records twice: entries lane and lane + 32
                {
                    float f[4 * NPP];
#pragma unroll
                    for (int q = 0; q < 4 * NPP; ++q)
                        f[q] = 0.0f;
#pragma unroll
                    for (int q = 0; q < 2 * D; ++q)
                        f[q] = pf[q];
                    f[2 * D] = (pf[2 * D] - oh) + (pf[2 * D + 1] - ol);
                    if (KIND == kGrad) {
                        f[2 * D + 1] = pw;
                        f[2 * D + 2] = kt_plus_c(S.kappa, S.kappa_lo, f[2 * D], -pc, 0.0f);
                    } else {
                        f[2 * D + 1] = kt_plus_c(S.kappa, S.kappa_lo, f[2 * D], 0.0f, 0.0f);
                    }
                    __syncwarp();
#pragma unroll
                    for (int p = 0; p < NPP; ++p) {
                        const float4 v = make_float4(f[4 * p], f[4 * p + 1], f[4 * p + 2], f[4 * p + 3]);
                        priv[p * 64 + lane] = v;
                        priv[p * 64 + lane + 32] = v;
                    }
                    __syncwarp();
                }
                if (c0 + 32 < CB) {
                    const int64_t col = (int64_t)cbase + c0 + 32 + lane;
                    load_rec<D>(rec, npad, col, pf);
                    if (KIND == kGrad) {
                        pw = w32[col];
                        pc = cm32[col];
                    }
                }
                const int m0 = cbase + c0;
                float *cp = colpart + (size_t)(rg * VC) * B + cg * CB + c0;
                if (m0 + 32 <= te_min) {  // every pair of this chunk is masked
#pragma unroll
                    for (int v = 0; v < VC; ++v)
                        cp[(size_t)v * B + lane] = 0.0f;
                    continue;
                }
                float acc[VC];
#pragma unroll
                for (int v = 0; v < VC; ++v)
                    acc[v] = 0.0f;
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int v = 0; v < VR; ++v)
                        part[r][v] = 0.0f;
                if (m0 < te_max)
                    chunk_steps<KIND, D, R, true>(priv + lane, src_lane, lane, m0, s_te, rx, rt, rw, ra, kc, part,
                                                  acc);
                else
                    chunk_steps<KIND, D, R, false>(priv + lane, src_lane, lane, m0, s_te, rx, rt, rw, ra, kc, part,
                                                   acc);
                // lane L now holds the total of column c0 + L
#pragma unroll
                for (int v = 0; v < VC; ++v)
                    cp[(size_t)v * B + lane] = acc[v];
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int v = 0; v < VR; ++v) {  // Kahan, once per chunk
                        const float y = part[r][v] - rc[r][v];
                        const float t = rs[r][v] + y;
                        rc[r][v] = (t - rs[r][v]) - y;
                        rs[r][v] = t;
                    }
            }
            // this column group's row totals, in the column-plane numbering
            float *rp = rowpart + (size_t)(cg * VC) * B;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int rr = rg * 32 * R + 32 * r + lane;
#pragma unroll
                for (int v = 0; v < VC; ++v)
                    rp[(size_t)v * B + rr] = 0.0f;
#pragma unroll
                for (int v = 0; v < VR; ++v)
                    rp[(size_t)row_plane<KIND>(v) * B + rr] = rs[r][v] - rc[r][v];
            }
            __syncthreads();
            // column totals over the row groups, row totals over the column
            // groups, both in group order
            for (int c = threadIdx.x; c < B; c += blockDim.x) {
#pragma unroll
                for (int v = 0; v < VC; ++v) {
                    float tot = 0.0f, rowv = 0.0f;
                    for (int q = 0; q < wr; ++q)
                        tot += colpart[((size_t)q * VC + v) * B + c];
                    for (int q = 0; q < wc; ++q)
                        rowv += rowpart[((size_t)q * VC + v) * B + c];
                    if (I != J) {
                        P[((int64_t)J * VC + v) * npad + (int64_t)I * B + c] = rowv;
                        P[((int64_t)I * VC + v) * npad + (int64_t)J * B + c] = tot;
                    } else {
                        P[((int64_t)I * VC + v) * npad + (int64_t)I * B + c] = rowv + tot;
                    }
                }
            }
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
