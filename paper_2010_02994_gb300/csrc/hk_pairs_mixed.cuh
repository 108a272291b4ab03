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
//   Pass 1 (rates): S_n += mu' for the earlier event, S_m += mu' + xi'' for
//     the later one; lambda_n = P_mu S_n.
//   Pass 2 (gradient): with w = 1/S and c = mu' (w_n + w_m) + xi''' w_m,
//     xi''' = xi'' rho (pass-2 constant c_xi2 = c_xi1 + log2 rho):
//     g~_n += c (x~_m - x~_n),  g~_m -= c (x~_m - x~_n);
//     d ell/d x_n = g~_n / (tau_x^2 kx).
//
// Tiling.  A CTA of W warps processes one pair block (I, J), I <= J, of
// B = 32 R W rows (block I) by B columns (block J) at a time, taking blocks
// from a persistent work list.  Each lane keeps R rows in registers for the
// whole block; the columns of block J are staged in shared memory with their
// times made relative to block I's middle row.  Columns are swept in chunks
// of 32: at step j lane L pairs its rows with column (L + j) mod 32 and adds
// that column's share into an accumulator that then moves to lane L - 1 by
// one shuffle, so after 32 steps every column's total over the warp's rows
// sits in one lane without any transpose.  Row sums are compensated (Kahan)
// once per chunk.  Per-warp column totals are summed over the warps at the
// end of the block, and the block's row and column totals go to one partial
// slot each (see hk_internal.cuh).  Pairs that must not count (m <= n in a
// diagonal block, exactly tied times) are removed by an index test only in
// the chunks that can contain them.
#pragma once

#include "hk_internal.cuh"

namespace hk {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int D>
struct PairConsts {
    float rho, kappa, cxi;
};

template <int D>
__device__ __forceinline__ void load_rec(const float4 *__restrict__ planes, int64_t stride, int64_t i,
                                         float (&f)[4 * nrec(D)])
{
#pragma unroll
    for (int p = 0; p < nrec(D); ++p) {
        float4 v = planes[(int64_t)p * stride + i];
        f[4 * p + 0] = v.x;
        f[4 * p + 1] = v.y;
        f[4 * p + 2] = v.z;
        f[4 * p + 3] = v.w;
    }
}

template <int D>
__device__ __forceinline__ void store_rec(float4 *planes, int64_t stride, int64_t i, const float (&f)[4 * nrec(D)])
{
#pragma unroll
    for (int p = 0; p < nrec(D); ++p)
        planes[(int64_t)p * stride + i] = make_float4(f[4 * p], f[4 * p + 1], f[4 * p + 2], f[4 * p + 3]);
}

// The two base-2 exponents of one pair; dx receives x~_col - x~_row.
template <int D>
__device__ __forceinline__ void pair_exponents(const float (&cf)[4 * nrec(D)], const float (&rx)[2 * D], float rt,
                                               const PairConsts<D> &k, float (&dx)[D], float &em, float &ex)
{
    float q;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        dx[d] = (cf[2 * d] - rx[2 * d]) + (cf[2 * d + 1] - rx[2 * d + 1]);
        q = d == 0 ? dx[0] * dx[0] : fmaf(dx[d], dx[d], q);
    }
    const float dt = cf[2 * D] - rt;
    em = fmaf(-dt, dt, -q);
    ex = fmaf(-k.rho, q, fmaf(-k.kappa, dt, k.cxi));
}

// -------------------------------------------------------------- pass 1 --

template <int D, bool MASKED>
__device__ __forceinline__ void pass1_chunk(const float4 *__restrict__ scol, int B, int c0, int lane, int m0,
                                            const float (&rx)[rows_per_lane(D)][2 * D],
                                            const float (&rt)[rows_per_lane(D)], const int (&rte)[rows_per_lane(D)],
                                            const PairConsts<D> &k, float (&part)[rows_per_lane(D)], float &acc)
{
    constexpr int R = rows_per_lane(D);
#pragma unroll 2
    for (int j = 0; j < 32; ++j) {
        const int cc = (lane + j) & 31;
        float cf[4 * nrec(D)];
        load_rec<D>(scol, B, c0 + cc, cf);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float dx[D], em, ex;
            pair_exponents<D>(cf, rx[r], rt[r], k, dx, em, ex);
            float mu = ex2_approx(em);
            float xi = ex2_approx(ex);
            if (MASKED) {
                const bool valid = m0 + cc >= rte[r];
                mu = valid ? mu : 0.0f;
                xi = valid ? xi : 0.0f;
            }
            part[r] += mu;
            acc += mu;
            acc += xi;
        }
        acc = __shfl_sync(0xffffffffu, acc, (lane + 1) & 31);
    }
}

template <int D>
__global__ void __launch_bounds__(256) pass1_mixed_kernel(Work w, const WorkItem *__restrict__ items, int nitems)
{
    constexpr int R = rows_per_lane(D);
    constexpr int NP = nrec(D);
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int B = 32 * R * warps;
    extern __shared__ float4 smem4[];
    float4 *scol = smem4;                                  // NP planes x B
    float *colpart = reinterpret_cast<float *>(smem4 + NP * B);  // [warps][B]
    __shared__ int s_item;

    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(&w.counters[0], 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems)
            break;
        const WorkItem wi = items[it];
        const SetDesc &S = w.sets[wi.set];
        const int I = wi.I, J = wi.J, n = S.n, npad = S.npad;
        const float4 *rec = w.rec + S.rec0;
        PairConsts<D> kc{S.rho, S.kappa, S.cxi1};

        // time origin: the middle row of block I
        float oh, ol;
        {
            const int io = min(I * B + B / 2, n - 1);
            const float4 v = rec[(int64_t)((2 * D) / 4) * npad + io];
            const float *c = reinterpret_cast<const float *>(&v);
            oh = c[(2 * D) % 4];
            ol = c[(2 * D) % 4 + 1];
        }
        // stage block J's columns
        for (int c = threadIdx.x; c < B; c += blockDim.x) {
            float f[4 * NP];
            load_rec<D>(rec, npad, (int64_t)J * B + c, f);
            f[2 * D] = (f[2 * D] - oh) + (f[2 * D + 1] - ol);
            f[2 * D + 1] = 0.0f;
            store_rec<D>(scol, B, c, f);
        }
        // this lane's rows
        float rx[R][2 * D], rt[R], part[R], rs[R], rc[R];
        int rte[R];
        const int rbase = I * B + warp * 32 * R;
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
            rte[r] = w.tie_end[S.row0 + row];
            te_min = min(te_min, rte[r]);
            te_max = max(te_max, rte[r]);
            rs[r] = 0.0f;
            rc[r] = 0.0f;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            te_min = min(te_min, __shfl_xor_sync(0xffffffffu, te_min, o));
            te_max = max(te_max, __shfl_xor_sync(0xffffffffu, te_max, o));
        }
        __syncthreads();

        for (int c0 = 0; c0 < B; c0 += 32) {
            const int m0 = J * B + c0;
            float *cp = colpart + warp * B + c0;
            if (m0 + 32 <= te_min) {  // every pair of this chunk is masked
                cp[lane] = 0.0f;
                continue;
            }
            float acc = 0.0f;
#pragma unroll
            for (int r = 0; r < R; ++r)
                part[r] = 0.0f;
            if (m0 < te_max)
                pass1_chunk<D, true>(scol, B, c0, lane, m0, rx, rt, rte, kc, part, acc);
            else
                pass1_chunk<D, false>(scol, B, c0, lane, m0, rx, rt, rte, kc, part, acc);
            cp[lane] = acc;
#pragma unroll
            for (int r = 0; r < R; ++r) {  // Kahan, once per chunk
                const float y = part[r] - rc[r];
                const float t = rs[r] + y;
                rc[r] = (t - rs[r]) - y;
                rs[r] = t;
            }
        }
        __syncthreads();
        float *P = w.P1 + S.part0;
        if (I != J) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                P[(int64_t)J * npad + rbase + 32 * r + lane] = rs[r] - rc[r];
            for (int c = threadIdx.x; c < B; c += blockDim.x) {
                float tot = 0.0f;
                for (int q = 0; q < warps; ++q)
                    tot += colpart[q * B + c];
                P[(int64_t)I * npad + (int64_t)J * B + c] = tot;
            }
        } else {
            float *rowbuf = reinterpret_cast<float *>(scol);
#pragma unroll
            for (int r = 0; r < R; ++r)
                rowbuf[warp * 32 * R + 32 * r + lane] = rs[r] - rc[r];
            __syncthreads();
            for (int c = threadIdx.x; c < B; c += blockDim.x) {
                float tot = rowbuf[c];
                for (int q = 0; q < warps; ++q)
                    tot += colpart[q * B + c];
                P[(int64_t)I * npad + (int64_t)I * B + c] = tot;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(&w.counters[1], 1);
        if (done == (int)gridDim.x - 1) {
            w.counters[0] = 0;
            w.counters[1] = 0;
            __threadfence();
        }
    }
}

// ------------------------------------------------ pass 1 with Theta sums --
// Besides the rate, every row collects the sums the parameter gradient needs
// (scaled units; the finalize kernel converts them): for the earlier event of
// a pair mu', mu' q, mu' dt^2; for the later one also xi'', xi'' dt, xi'' q.
// Partial planes per slot: 0 mu', 1 xi'', 2 mu' q, 3 mu' dt^2, 4 xi'' dt, 5 xi'' q.

template <int D, bool MASKED>
__device__ __forceinline__ void pass1_theta_chunk(const float4 *__restrict__ scol, int B, int c0, int lane, int m0,
                                                  const float (&rx)[rows_per_lane(D)][2 * D],
                                                  const float (&rt)[rows_per_lane(D)],
                                                  const int (&rte)[rows_per_lane(D)], const PairConsts<D> &k,
                                                  float (&part)[rows_per_lane(D)][3], float (&acc)[6])
{
    constexpr int R = rows_per_lane(D);
#pragma unroll 2
    for (int j = 0; j < 32; ++j) {
        const int cc = (lane + j) & 31;
        float cf[4 * nrec(D)];
        load_rec<D>(scol, B, c0 + cc, cf);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float q;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float dx = (cf[2 * d] - rx[r][2 * d]) + (cf[2 * d + 1] - rx[r][2 * d + 1]);
                q = d == 0 ? dx * dx : fmaf(dx, dx, q);
            }
            const float dt = cf[2 * D] - rt[r];
            const float dt2 = dt * dt;
            float mu = ex2_approx(-q - dt2);
            float xi = ex2_approx(fmaf(-k.rho, q, fmaf(-k.kappa, dt, k.cxi)));
            if (MASKED) {
                const bool valid = m0 + cc >= rte[r];
                mu = valid ? mu : 0.0f;
                xi = valid ? xi : 0.0f;
            }
            part[r][0] += mu;
            part[r][1] = fmaf(mu, q, part[r][1]);
            part[r][2] = fmaf(mu, dt2, part[r][2]);
            acc[0] += mu;
            acc[1] += xi;
            acc[2] = fmaf(mu, q, acc[2]);
            acc[3] = fmaf(mu, dt2, acc[3]);
            acc[4] = fmaf(xi, dt, acc[4]);
            acc[5] = fmaf(xi, q, acc[5]);
        }
#pragma unroll
        for (int v = 0; v < 6; ++v)
            acc[v] = __shfl_sync(0xffffffffu, acc[v], (lane + 1) & 31);
    }
}

template <int D>
__global__ void __launch_bounds__(256) pass1_theta_kernel(Work w, const WorkItem *__restrict__ items, int nitems)
{
    constexpr int R = rows_per_lane(D);
    constexpr int NP = nrec(D);
    constexpr int V = kPass1ThetaVals;
    constexpr int row_plane[3] = {0, 2, 3};
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int B = 32 * R * warps;
    extern __shared__ float4 smem4[];
    float4 *scol = smem4;
    const size_t scol_floats = (size_t)(NP * 4 > V ? NP * 4 : V) * B;
    float *colpart = reinterpret_cast<float *>(smem4) + scol_floats;  // [warps][V][B]
    __shared__ int s_item;

    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(&w.counters[0], 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems)
            break;
        const WorkItem wi = items[it];
        const SetDesc &S = w.sets[wi.set];
        const int I = wi.I, J = wi.J, n = S.n, npad = S.npad;
        const float4 *rec = w.rec + S.rec0;
        PairConsts<D> kc{S.rho, S.kappa, S.cxi1};
        float oh, ol;
        {
            const int io = min(I * B + B / 2, n - 1);
            const float4 v = rec[(int64_t)((2 * D) / 4) * npad + io];
            const float *c = reinterpret_cast<const float *>(&v);
            oh = c[(2 * D) % 4];
            ol = c[(2 * D) % 4 + 1];
        }
        for (int c = threadIdx.x; c < B; c += blockDim.x) {
            float f[4 * NP];
            load_rec<D>(rec, npad, (int64_t)J * B + c, f);
            f[2 * D] = (f[2 * D] - oh) + (f[2 * D + 1] - ol);
            f[2 * D + 1] = 0.0f;
            store_rec<D>(scol, B, c, f);
        }
        float rx[R][2 * D], rt[R], part[R][3], rs[R][3], rc[R][3];
        int rte[R];
        const int rbase = I * B + warp * 32 * R;
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
            rte[r] = w.tie_end[S.row0 + row];
            te_min = min(te_min, rte[r]);
            te_max = max(te_max, rte[r]);
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                rs[r][v] = 0.0f;
                rc[r][v] = 0.0f;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            te_min = min(te_min, __shfl_xor_sync(0xffffffffu, te_min, o));
            te_max = max(te_max, __shfl_xor_sync(0xffffffffu, te_max, o));
        }
        __syncthreads();
        for (int c0 = 0; c0 < B; c0 += 32) {
            const int m0 = J * B + c0;
            float *cp = colpart + (warp * V) * B + c0;
            if (m0 + 32 <= te_min) {
#pragma unroll
                for (int v = 0; v < V; ++v)
                    cp[v * B + lane] = 0.0f;
                continue;
            }
            float acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v)
                acc[v] = 0.0f;
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int v = 0; v < 3; ++v)
                    part[r][v] = 0.0f;
            if (m0 < te_max)
                pass1_theta_chunk<D, true>(scol, B, c0, lane, m0, rx, rt, rte, kc, part, acc);
            else
                pass1_theta_chunk<D, false>(scol, B, c0, lane, m0, rx, rt, rte, kc, part, acc);
#pragma unroll
            for (int v = 0; v < V; ++v)
                cp[v * B + lane] = acc[v];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const float y = part[r][v] - rc[r][v];
                    const float t = rs[r][v] + y;
                    rc[r][v] = (t - rs[r][v]) - y;
                    rs[r][v] = t;
                }
        }
        __syncthreads();
        float *P = w.P1 + S.part0;
        float *rowbuf = reinterpret_cast<float *>(scol);  // [V][B]
        for (int c = threadIdx.x; c < V * B; c += blockDim.x)
            rowbuf[c] = 0.0f;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int v = 0; v < 3; ++v)
                rowbuf[row_plane[v] * B + warp * 32 * R + 32 * r + lane] = rs[r][v] - rc[r][v];
        __syncthreads();
        if (I != J) {
            for (int c = threadIdx.x; c < B; c += blockDim.x) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    P[((int64_t)J * V + v) * npad + (int64_t)I * B + c] = rowbuf[v * B + c];
                    float tot = 0.0f;
                    for (int q = 0; q < warps; ++q)
                        tot += colpart[(q * V + v) * B + c];
                    P[((int64_t)I * V + v) * npad + (int64_t)J * B + c] = tot;
                }
            }
        } else {
            for (int c = threadIdx.x; c < B; c += blockDim.x) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    float tot = rowbuf[v * B + c];
                    for (int q = 0; q < warps; ++q)
                        tot += colpart[(q * V + v) * B + c];
                    P[((int64_t)I * V + v) * npad + (int64_t)I * B + c] = tot;
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(&w.counters[1], 1);
        if (done == (int)gridDim.x - 1) {
            w.counters[0] = 0;
            w.counters[1] = 0;
            __threadfence();
        }
    }
}

// -------------------------------------------------------------- pass 2 --

template <int D, bool MASKED>
__device__ __forceinline__ void pass2_chunk(const float4 *__restrict__ scol, int B, int c0, int lane, int m0,
                                            const float (&rx)[rows_per_lane(D)][2 * D],
                                            const float (&rt)[rows_per_lane(D)], const float (&rw)[rows_per_lane(D)],
                                            const int (&rte)[rows_per_lane(D)], const PairConsts<D> &k,
                                            float (&part)[rows_per_lane(D)][D], float (&acc)[D])
{
    constexpr int R = rows_per_lane(D);
#pragma unroll 2
    for (int j = 0; j < 32; ++j) {
        const int cc = (lane + j) & 31;
        float cf[4 * nrec(D)];
        load_rec<D>(scol, B, c0 + cc, cf);
        const float cw = cf[2 * D + 1];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float dx[D], em, ex;
            pair_exponents<D>(cf, rx[r], rt[r], k, dx, em, ex);
            float mu = ex2_approx(em);
            float xi = ex2_approx(ex);
            if (MASKED) {
                const bool valid = m0 + cc >= rte[r];
                mu = valid ? mu : 0.0f;
                xi = valid ? xi : 0.0f;
            }
            const float c = fmaf(mu, rw[r] + cw, xi * cw);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                part[r][d] = fmaf(c, dx[d], part[r][d]);
                acc[d] = fmaf(-c, dx[d], acc[d]);
            }
        }
#pragma unroll
        for (int d = 0; d < D; ++d)
            acc[d] = __shfl_sync(0xffffffffu, acc[d], (lane + 1) & 31);
    }
}

template <int D>
__global__ void __launch_bounds__(256) pass2_mixed_kernel(Work w, const WorkItem *__restrict__ items, int nitems)
{
    constexpr int R = rows_per_lane(D);
    constexpr int NP = nrec(D);
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int B = 32 * R * warps;
    extern __shared__ float4 smem4[];
    float4 *scol = smem4;
    float *colpart = reinterpret_cast<float *>(smem4 + NP * B);  // [warps][D][B]
    __shared__ int s_item;

    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(&w.counters[0], 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems)
            break;
        const WorkItem wi = items[it];
        const SetDesc &S = w.sets[wi.set];
        const int I = wi.I, J = wi.J, n = S.n, npad = S.npad;
        const float4 *rec = w.rec + S.rec0;
        const float *w32 = w.w32 + S.row0;
        PairConsts<D> kc{S.rho, S.kappa, S.cxi2};

        float oh, ol;
        {
            const int io = min(I * B + B / 2, n - 1);
            const float4 v = rec[(int64_t)((2 * D) / 4) * npad + io];
            const float *c = reinterpret_cast<const float *>(&v);
            oh = c[(2 * D) % 4];
            ol = c[(2 * D) % 4 + 1];
        }
        for (int c = threadIdx.x; c < B; c += blockDim.x) {
            float f[4 * NP];
            load_rec<D>(rec, npad, (int64_t)J * B + c, f);
            f[2 * D] = (f[2 * D] - oh) + (f[2 * D + 1] - ol);
            f[2 * D + 1] = w32[(int64_t)J * B + c];
            store_rec<D>(scol, B, c, f);
        }
        float rx[R][2 * D], rt[R], rw[R], part[R][D], rs[R][D], rc[R][D];
        int rte[R];
        const int rbase = I * B + warp * 32 * R;
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
            rw[r] = w32[row];
            rte[r] = w.tie_end[S.row0 + row];
            te_min = min(te_min, rte[r]);
            te_max = max(te_max, rte[r]);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                rs[r][d] = 0.0f;
                rc[r][d] = 0.0f;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            te_min = min(te_min, __shfl_xor_sync(0xffffffffu, te_min, o));
            te_max = max(te_max, __shfl_xor_sync(0xffffffffu, te_max, o));
        }
        __syncthreads();

        for (int c0 = 0; c0 < B; c0 += 32) {
            const int m0 = J * B + c0;
            float *cp = colpart + (warp * D) * B + c0;
            if (m0 + 32 <= te_min) {
#pragma unroll
                for (int d = 0; d < D; ++d)
                    cp[d * B + lane] = 0.0f;
                continue;
            }
            float acc[D];
#pragma unroll
            for (int d = 0; d < D; ++d)
                acc[d] = 0.0f;
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int d = 0; d < D; ++d)
                    part[r][d] = 0.0f;
            if (m0 < te_max)
                pass2_chunk<D, true>(scol, B, c0, lane, m0, rx, rt, rw, rte, kc, part, acc);
            else
                pass2_chunk<D, false>(scol, B, c0, lane, m0, rx, rt, rw, rte, kc, part, acc);
#pragma unroll
            for (int d = 0; d < D; ++d)
                cp[d * B + lane] = acc[d];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const float y = part[r][d] - rc[r][d];
                    const float t = rs[r][d] + y;
                    rc[r][d] = (t - rs[r][d]) - y;
                    rs[r][d] = t;
                }
        }
        __syncthreads();
        float *P = w.P2 + S.part2_0;
        if (I != J) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int d = 0; d < D; ++d)
                    P[((int64_t)J * D + d) * npad + rbase + 32 * r + lane] = rs[r][d] - rc[r][d];
            for (int c = threadIdx.x; c < B; c += blockDim.x) {
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    float tot = 0.0f;
                    for (int q = 0; q < warps; ++q)
                        tot += colpart[(q * D + d) * B + c];
                    P[((int64_t)I * D + d) * npad + (int64_t)J * B + c] = tot;
                }
            }
        } else {
            float *rowbuf = reinterpret_cast<float *>(scol);  // [D][B]
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int d = 0; d < D; ++d)
                    rowbuf[d * B + warp * 32 * R + 32 * r + lane] = rs[r][d] - rc[r][d];
            __syncthreads();
            for (int c = threadIdx.x; c < B; c += blockDim.x) {
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    float tot = rowbuf[d * B + c];
                    for (int q = 0; q < warps; ++q)
                        tot += colpart[(q * D + d) * B + c];
                    P[((int64_t)I * D + d) * npad + (int64_t)I * B + c] = tot;
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(&w.counters[1], 1);
        if (done == (int)gridDim.x - 1) {
            w.counters[0] = 0;
            w.counters[1] = 0;
            __threadfence();
        }
    }
}

template <int D>
size_t pass_smem_bytes_t(int pass, bool theta, int warps)
{
    const int B = 32 * rows_per_lane(D) * warps;
    const int vals = pass == 1 ? (theta ? kPass1ThetaVals : 1) : D;
    // staged columns (reused as the row buffer at the end of a block)
    const size_t scol_floats = (size_t)(nrec(D) * 4 > vals ? nrec(D) * 4 : vals) * B;
    return (scol_floats + (size_t)warps * vals * B) * sizeof(float);
}

}  // namespace hk
