// Bayesian multidimensional scaling (BMDS) likelihood of Section 2.2.3,
// Eq. (4), with its location and variance gradients: the second O(N^2)
// pairwise term of the BMDS-Hawkes posterior whose HMC needs both (Section 3).
// With observed distances y_nn', latent distances delta = |x_n - x_n'|,
// z = delta / sigma:
//   ell_B = N (1 - N) / 4 log(sigma2) - sum_{n > n'} r_nn',
//   r = (y - delta)^2 / (2 sigma2) + log Phi(z),
//   d ell_B / d x_n = sum_{n' != n} coef_nn' (x_n' - x_n),
//   coef = (phi(z) / (sigma Phi(z)) - (y - delta) / sigma2) / delta,
//   d ell_B / d sigma2 = N (1 - N) / (4 sigma2)
//       + sum_{n > n'} [(y - delta)^2 / (2 sigma2^2) + phi(z) delta / (2 sigma^3 Phi(z))].
//
// Work decomposition.  Rows and columns are cut into tiles of KT = 32 W
// events; one CTA (W warps) owns one tile pair (I, J), J <= I, so each
// unordered pair of distinct tiles is visited once.  Per 32-column chunk the
// CTA stages Y[rows of I][32 columns of J] in shared memory (read from the
// lower triangle only, coalesced) and the columns' coordinates; each warp
// then sweeps its 32 rows against the chunk in 32 rotated steps: at step s
// lane l pairs row l with column (l + s) mod 32, so every lane reads a
// different shared-memory bank, and the column accumulators travel one lane
// down per step by shuffle (after 32 steps lane l holds column l's sum).
// Off-diagonal tiles add each pair to the row side and to the column side;
// a diagonal tile evaluates both orders of its pairs on the row side only
// (the value is counted for the column below the row).
//
// Results go to partial slots with one writer each:
//   rowpart[p][v][r], v < D: row gradient, v = D: value, v = D + 1: sigma2 sum
//   colpart[p][k][c]: column gradient of tile J from tile pair p = (I, J), I > J,
// with p = I (I + 1) / 2 + J; the finalize kernel adds them in a fixed
// order, so every result is deterministic.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "hk_internal.cuh"

namespace hk {
namespace bmds {

constexpr int kCh = 32;     // columns per staged chunk
constexpr int kBatch = 16;  // FP32 Y loads issued together (half as many FP64)

template <typename F>
struct Consts {
    F inv_sigma, inv_s2, h2, h4, h3;  // 1/sigma, 1/sigma2, 1/(2 sigma2), 1/(2 sigma2^2), 1/(2 sigma^3)
};

template <typename F>
struct Args {
    const void *Y;  // double or float, row-major N x N
    const double *X;
    int64_t n;
    int d, T;
    Consts<F> k;
    F *rowpart;
    F *colpart;
    unsigned *status;
};

__host__ __device__ inline int64_t pair_index(int I, int J) { return (int64_t)I * (I + 1) / 2 + J; }

__device__ inline void pair_of(int64_t b, int &I, int &J)
{
    int i = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while (pair_index(i + 1, 0) <= b)
        ++i;
    while (pair_index(i, 0) > b)
        --i;
    I = i;
    J = (int)(b - pair_index(i, 0));
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Normal tail for z >= 0: Q(z) = 1 - Phi(z) = exp(-z^2 / 2) P(z) / B(z), where
// P / B (degrees 4 and 5) is a rational fit of the scaled tail
// Q(z) exp(z^2 / 2) on [0, 14]: weighted least squares made minimax by Lawson
// reweighting, relative error 6e-9 in exact arithmetic and about 3e-7 when
// evaluated in FP32 (the fit is made by gen_normal_tail.py beside this file).
// Beyond z = 14, exp(-z^2 / 2) is below the FP32 range, so P / B is evaluated
// at min(z, 14).
constexpr float kTailP[5] = {0.5f, 0.43723174929618835f, 0.1824471801519394f, 0.040367491543293f,
                             0.0040768226608633995f};
constexpr float kTailB[6] = {1.0f, 1.6723483800888062f, 1.1992309093475342f, 0.4673903286457062f,
                             0.10119310766458511f, 0.010218949988484383f};

// Terms of one pair in FP32.  q = |x_n - x_n'|^2, y the observed distance.
// With A = exp(-z^2/2) P and D = B - A (so Q = A / B and Phi = D / B), one
// reciprocal of B D gives Q, Phi and phi / Phi = exp(-z^2/2) B / (sqrt(2 pi) D).
// log Phi = log1p(-Q) takes its Taylor series below Q = 1/64 and the
// hardware log2 of Phi above.
__device__ __forceinline__ void pair_terms(float q, float y, const Consts<float> &k, float &val, float &ssum,
                                           float &coef)
{
    const float inv_delta = q > 0.0f ? rsqrtf(q) : 0.0f;  // coincident points: no gradient term
    const float delta = q * inv_delta;
    const float z = delta * k.inv_sigma;
    const float E = ex2_approx(z * (z * -0.72134752044448170f));  // exp(-z^2 / 2)
    const float zc = fminf(z, 14.0f);
    const float P = fmaf(fmaf(fmaf(fmaf(kTailP[4], zc, kTailP[3]), zc, kTailP[2]), zc, kTailP[1]), zc, kTailP[0]);
    const float B =
        fmaf(fmaf(fmaf(fmaf(fmaf(kTailB[5], zc, kTailB[4]), zc, kTailB[3]), zc, kTailB[2]), zc, kTailB[1]), zc,
             kTailB[0]);
    const float A = E * P;
    const float D = B - A;
    const float inv = rcp_approx(B * D);
    const float Q = A * D * inv;
    const float Phi = D * D * inv;
    const float ratio = (0.39894228040143268f * E) * (B * B * inv);  // phi(z) / Phi(z)
    const float series = -Q * fmaf(Q, fmaf(Q, fmaf(Q, 0.25f, 0.33333334f), 0.5f), 1.0f);
    const float log_Phi = Q < 0.015625f ? series : lg2_approx(Phi) * 0.69314718055994531f;
    const float e = y - delta;
    const float e2 = e * e;
    val = fmaf(e2, k.h2, log_Phi);
    ssum = fmaf(e2, k.h4, ratio * delta * k.h3);
    coef = (ratio * k.inv_sigma - e * k.inv_s2) * inv_delta;
}

// The gradient coefficient alone (coef above) in FP32, for the pair loop of
// the Hawkes gradient pass that also carries this term (the BMDS-Hawkes
// potential of Section 3): the same steps without log Phi and the value and
// variance sums.
__device__ __forceinline__ float grad_coef(float q, float y, float inv_sigma, float inv_s2)
{
    const float inv_delta = q > 0.0f ? rsqrtf(q) : 0.0f;
    const float delta = q * inv_delta;
    const float z = delta * inv_sigma;
    const float E = ex2_approx(z * (z * -0.72134752044448170f));
    const float zc = fminf(z, 14.0f);
    const float P = fmaf(fmaf(fmaf(fmaf(kTailP[4], zc, kTailP[3]), zc, kTailP[2]), zc, kTailP[1]), zc, kTailP[0]);
    const float B =
        fmaf(fmaf(fmaf(fmaf(fmaf(kTailB[5], zc, kTailB[4]), zc, kTailB[3]), zc, kTailB[2]), zc, kTailB[1]), zc,
             kTailB[0]);
    const float D = B - E * P;
    const float ratio = (0.39894228040143268f * E) * (B * rcp_approx(D));  // phi(z) / Phi(z)
    return (ratio * inv_sigma - (y - delta) * inv_s2) * inv_delta;
}

// The same terms with every operation in FP64.
__device__ __forceinline__ void pair_terms(double q, double y, const Consts<double> &k, double &val, double &ssum,
                                           double &coef)
{
    const double delta = sqrt(q);
    const double inv_delta = q > 0.0 ? 1.0 / delta : 0.0;
    const double z = delta * k.inv_sigma;
    const double tail = 0.5 * erfc(z * 0.70710678118654752440);
    const double ratio = exp(-0.5 * z * z) * 0.39894228040143267794 / (1.0 - tail);
    const double e = y - delta;
    val = e * e * k.h2 + log1p(-tail);
    ssum = e * e * k.h4 + ratio * delta * k.h3;
    coef = (ratio * k.inv_sigma - e * k.inv_s2) * inv_delta;
}

__device__ __forceinline__ float to_f(double v, float *) { return __double2float_rn(v); }
__device__ __forceinline__ double to_f(double v, double *) { return v; }

// Nearest float (ties to even) of a double by integer operations: the
// conversion instruction runs on the FP64 unit, which this GPU has few of.
// Magnitudes below 2^-126 give 0 (flush to zero), above the FP32 range
// infinity; infinities and NaN keep their class.
__device__ __forceinline__ float d2f_rn_int(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const unsigned int e = (unsigned int)(mag >> 52);
    const unsigned long long r = mag + 0x0fffffffull + ((mag >> 29) & 1ull);  // round 52 -> 23 mantissa bits
    unsigned int f = (unsigned int)(r >> 29) - (896u << 23);                   // exponent bias 1023 -> 127
    f = e < 897u ? 0u : f;
    f = e >= 1151u ? 0x7f800000u : f;
    f = (e == 2047u && mag != 0x7ff0000000000000ull) ? 0x7fc00000u : f;
    return __uint_as_float(f | sign);
}

// Observed distance as the kernel's type: FP64 input to FP32 by integer
// rounding, FP32 input as is (or widened exactly for the FP64 kernel).
__device__ __forceinline__ float y_to(double v, float *) { return d2f_rn_int(v); }
__device__ __forceinline__ float y_to(float v, float *) { return v; }
__device__ __forceinline__ double y_to(double v, double *) { return v; }
__device__ __forceinline__ double y_to(float v, double *) { return (double)v; }

// Column coordinate record in shared memory: two dimensions per record, as
// FP32 (hi, lo) pairs for the FP32 kernel and as doubles for the FP64 one.
template <typename F>
struct Rec;
template <>
struct Rec<float> {
    using type = float4;  // xh[2i], xl[2i], xh[2i+1], xl[2i+1]
};
template <>
struct Rec<double> {
    using type = double2;  // x[2i], x[2i+1]
};

__device__ __forceinline__ void rec_dx(const float4 &r, const float (&xh)[2], const float (&xl)[2], float &dx0,
                                       float &dx1)
{
    dx0 = (r.x - xh[0]) + (r.y - xl[0]);
    dx1 = (r.z - xh[1]) + (r.w - xl[1]);
}
__device__ __forceinline__ void rec_dx(const double2 &r, const double (&xh)[2], const double (&)[2], double &dx0,
                                       double &dx1)
{
    dx0 = r.x - xh[0];
    dx1 = r.y - xh[1];
}

__device__ __forceinline__ float4 make_rec(const double *v, float *)
{
    const float h0 = __double2float_rn(v[0]), h1 = __double2float_rn(v[1]);
    return make_float4(h0, __double2float_rn(v[0] - (double)h0), h1, __double2float_rn(v[1] - (double)h1));
}
__device__ __forceinline__ double2 make_rec(const double *v, double *) { return make_double2(v[0], v[1]); }

// Validity of the observed distances, tracked cheaply per element: the FP32
// kernel keeps the largest bit pattern of y + 0 (which maps -0 to +0); any
// negative, infinite or NaN y has a pattern above that of FLT_MAX.
__device__ __forceinline__ void track_y(float y, unsigned &acc)
{
    acc = max(acc, __float_as_uint(y + 0.0f));
}
__device__ __forceinline__ void track_y(double y, unsigned &acc)
{
    acc = (y >= 0.0 && y < INFINITY) ? acc : 0xffffffffu;
}
constexpr unsigned kYBitsMax = 0x7f7fffffu;

// One 32 x 32 block of a warp in 32 rotated steps: at step s lane l pairs its
// row with column (l + s) mod 32 of the chunk.  The lane's Y row is stored
// rotated (entry s is that column), and the column records are stored twice
// (entries j and j + 32), so step s reads fixed offsets from per-lane bases.
// MASKED handles ragged rows or columns and the diagonal tile; SYM adds the
// column side, whose accumulators move one lane down per step; VAL: the
// value and variance sums too (else the gradient coefficient alone, FP32).
template <typename F, int DS, bool MASKED, bool SYM, bool VAL>
__device__ __forceinline__ void sweep(int d, int lane, const F *__restrict__ yrow,
                                      const typename Rec<F>::type *__restrict__ xrec, const F (&xh)[DS],
                                      const F (&xl)[DS], const Consts<F> &k, int64_t row, int64_t c0, int64_t n,
                                      bool row_ok, F (&gp)[DS], F &vp, F &sp, F (&colacc)[DS])
{
    constexpr int NV = (DS + 1) / 2;
#pragma unroll 8
    for (int s = 0; s < kCh; ++s) {
        F dx[2 * NV];
        F q = F(0);
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            if (2 * i < d) {
                const typename Rec<F>::type r = xrec[i * 2 * kCh + s];
                const F h[2] = {xh[2 * i], 2 * i + 1 < DS ? xh[2 * i + 1] : F(0)};
                const F l[2] = {xl[2 * i], 2 * i + 1 < DS ? xl[2 * i + 1] : F(0)};
                rec_dx(r, h, l, dx[2 * i], dx[2 * i + 1]);
                q = fma(dx[2 * i], dx[2 * i], q);
                if (2 * i + 1 < d)
                    q = fma(dx[2 * i + 1], dx[2 * i + 1], q);
            } else {
                dx[2 * i] = dx[2 * i + 1] = F(0);
            }
        }
        F v = F(0), ss = F(0), cf;
        if constexpr (VAL)
            pair_terms(q, yrow[s], k, v, ss, cf);
        else
            cf = grad_coef(q, yrow[s], k.inv_sigma, k.inv_s2);
        if (MASKED) {
            const int64_t col = c0 + ((lane + s) & (kCh - 1));
            const bool ok = row_ok && col < n && col != row;
            const bool counted = ok && col < row;
            cf = ok ? cf : F(0);
            v = counted ? v : F(0);
            ss = counted ? ss : F(0);
        }
        vp += v;
        sp += ss;
#pragma unroll
        for (int c = 0; c < DS; ++c) {
            if (c < d) {
                gp[c] = fma(cf, dx[c], gp[c]);
                if (SYM)
                    colacc[c] = fma(-cf, dx[c], colacc[c]);
            }
        }
        if (SYM) {
#pragma unroll
            for (int c = 0; c < DS; ++c)
                if (c < d)
                    colacc[c] = __shfl_sync(0xffffffffu, colacc[c], (lane + 1) & (kCh - 1));
        }
    }
}

// D > 0: compile-time dimension; D == 0: runtime d (up to kMaxD).
// YT: element type of Y in memory (double or float).  VAL: the value and
// variance sums as well as the gradient (without them, FP32 only, their
// slots hold zeros: for callers that need the gradient alone).
template <typename F, typename YT, int D, int W, bool VAL = true>
__global__ void __launch_bounds__(32 * W) pairs_kernel(Args<F> a)
{
    using R = typename Rec<F>::type;
    constexpr int KT = 32 * W;
    constexpr int DS = D > 0 ? D : kMaxD;
    constexpr int NV = (DS + 1) / 2;
    constexpr int kYS = kCh + 1;  // padded stride of a rotated Y row
    constexpr bool HILO = sizeof(F) == 4;
    constexpr int kB = sizeof(YT) == 8 ? kBatch / 2 : kBatch;  // loads in flight per batch
    __shared__ F sY[KT * kYS];
    __shared__ R sxc[NV * 2 * kCh];
    __shared__ F scol[W * DS * kCh];

    const YT *__restrict__ Y = static_cast<const YT *>(a.Y);
    const int d = D > 0 ? D : a.d;
    int I, J;
    pair_of(blockIdx.x, I, J);
    const bool diag = I == J;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = a.n;
    const int64_t row = (int64_t)I * KT + threadIdx.x;
    const bool row_ok = row < n;
    const bool full_rows = (int64_t)(I + 1) * KT <= n;
    const int64_t p = pair_index(I, J);

    bool bad = false;
    unsigned ybits = 0;
    F xh[DS], xl[DS];
    {
        double v[DS];
#pragma unroll
        for (int c = 0; c < DS; ++c)
            v[c] = (c < d && row_ok) ? a.X[row * d + c] : 0.0;
#pragma unroll
        for (int c = 0; c < DS; ++c) {
            bad |= !isfinite(v[c]);
            xh[c] = to_f(v[c], (F *)nullptr);
            xl[c] = HILO ? to_f(v[c] - (double)xh[c], (F *)nullptr) : F(0);
        }
    }
    F g[DS];
#pragma unroll
    for (int c = 0; c < DS; ++c)
        g[c] = F(0);
    F val = F(0), ssum = F(0);

    for (int ch = 0; ch < W; ++ch) {
        const int64_t c0 = (int64_t)J * KT + ch * kCh;
        if (c0 >= n)
            break;
        __syncthreads();
        // Y below the diagonal: lane l reads column c0 + l of rows warp,
        // warp + W, ... (256 contiguous bytes per warp and row); element
        // (rr, cc) is stored at rotated position (cc - rr) mod 32 of row rr.
        // Loads go in batches of kBatch independent loads, then their stores.
        if (!diag && full_rows) {
            const int64_t stride = (int64_t)W * n;
            const YT *src = Y + ((int64_t)I * KT + warp) * n + c0 + lane;
#pragma unroll 1
            for (int b = 0; b < kCh / kB; ++b) {
                YT v[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    v[u] = __ldcs(src);
                    src += stride;
                }
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int rr = warp + (b * kB + u) * W;
                    const F y = y_to(v[u], (F *)nullptr);
                    track_y(y, ybits);
                    sY[rr * kYS + ((lane - rr) & (kCh - 1))] = y;
                }
            }
        } else {
#pragma unroll 1
            for (int b = 0; b < kCh / kB; ++b) {
                YT v[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int rr = warp + (b * kB + u) * W;
                    const int64_t gr = (int64_t)I * KT + rr, gc = c0 + lane;
                    v[u] = (gr < n && gr > gc) ? __ldcs(Y + gr * n + gc) : YT(0);
                }
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int rr = warp + (b * kB + u) * W;
                    const int64_t gr = (int64_t)I * KT + rr, gc = c0 + lane;
                    if (gr > gc) {
                        const F y = y_to(v[u], (F *)nullptr);
                        track_y(y, ybits);
                        sY[rr * kYS + ((lane - rr) & (kCh - 1))] = y;
                    }
                }
            }
            // diagonal tile: entries above the diagonal from Y[col][row];
            // thread t reads row I*KT + t of column c0 + cc (consecutive
            // threads along a row of Y)
            if (diag) {
#pragma unroll 1
                for (int b = 0; b < kCh / kB; ++b) {
                    YT v[kB];
#pragma unroll
                    for (int u = 0; u < kB; ++u) {
                        const int64_t gr = (int64_t)I * KT + threadIdx.x, gc = c0 + b * kB + u;
                        v[u] = (gc < n && gr < gc) ? __ldcs(Y + gc * n + gr) : YT(0);
                    }
#pragma unroll
                    for (int u = 0; u < kB; ++u) {
                        const int cc = b * kB + u;
                        const int64_t gr = (int64_t)I * KT + threadIdx.x, gc = c0 + cc;
                        if (gr < gc) {
                            const F y = y_to(v[u], (F *)nullptr);
                            track_y(y, ybits);
                            sY[threadIdx.x * kYS + ((cc - (int)threadIdx.x) & (kCh - 1))] = y;
                        }
                    }
                }
            }
        }
        // column records (one per thread: record i of column t), stored at
        // entries t and t + 32
        for (int e = threadIdx.x; e < NV * kCh; e += KT) {
            const int i = e / kCh, t = e % kCh;
            if (2 * i < d) {
                const int64_t col = c0 + t;
                double v[2];
                v[0] = col < n ? a.X[col * d + 2 * i] : 0.0;
                v[1] = (col < n && 2 * i + 1 < d) ? a.X[col * d + 2 * i + 1] : 0.0;
                const R r = make_rec(v, (F *)nullptr);
                sxc[i * 2 * kCh + t] = r;
                sxc[i * 2 * kCh + kCh + t] = r;
            }
        }
        __syncthreads();
        // warm L2 with this row's Y entries of the next chunk (off-diagonal tiles)
        if (!diag && row_ok && ch + 1 < W && c0 + kCh < n) {
            const YT *nxt = Y + row * n + c0 + kCh;
            constexpr int kLine = 128 / sizeof(YT);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(nxt));
            if (kLine < kCh && c0 + kCh + kLine < n)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nxt + kLine));
        }

        F gp[DS], colacc[DS];
#pragma unroll
        for (int c = 0; c < DS; ++c)
            gp[c] = colacc[c] = F(0);
        F vp = F(0), sp = F(0);
        const F *yrow = sY + threadIdx.x * kYS;
        const R *xrec = sxc + lane;
        const bool full = !diag && full_rows && c0 + kCh <= n;
        if (full)
            sweep<F, DS, false, true, VAL>(d, lane, yrow, xrec, xh, xl, a.k, row, c0, n, row_ok, gp, vp, sp, colacc);
        else if (!diag)
            sweep<F, DS, true, true, VAL>(d, lane, yrow, xrec, xh, xl, a.k, row, c0, n, row_ok, gp, vp, sp, colacc);
        else
            sweep<F, DS, true, false, VAL>(d, lane, yrow, xrec, xh, xl, a.k, row, c0, n, row_ok, gp, vp, sp, colacc);
#pragma unroll
        for (int c = 0; c < DS; ++c)
            g[c] += gp[c];
        val += vp;
        ssum += sp;
        if (!diag) {
#pragma unroll
            for (int c = 0; c < DS; ++c)
                if (c < d)
                    scol[(warp * DS + c) * kCh + lane] = colacc[c];
            __syncthreads();
            for (int e = threadIdx.x; e < d * kCh; e += KT) {
                const int c = e / kCh, cc = e % kCh;
                F s = F(0);
                for (int w2 = 0; w2 < W; ++w2)
                    s += scol[(w2 * DS + c) * kCh + cc];
                a.colpart[(p * d + c) * KT + ch * kCh + cc] = s;
            }
        }
    }
    F *rp = a.rowpart + p * (d + 2) * KT + threadIdx.x;
    for (int c = 0; c < d; ++c)
        rp[c * KT] = g[c];
    rp[d * KT] = val;
    rp[(d + 1) * KT] = ssum;
    if (bad || ybits > kYBitsMax)
        atomicOr(a.status, kStInvalidData);
}

}  // namespace bmds
}  // namespace hk
