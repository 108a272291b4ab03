// Row finalization in FP64: rates and log-likelihood (Eq. (1)), gradients
// (Appendix A), and the FP64 recomputation of rows whose mixed-precision
// rate is too small to trust in FP32.
//
// Mixed path.  S_n is the FP64 sum of the pair kernel's FP32 partial slots
// (fixed slot order).  A row with S_n < s_min (or not finite) is "flagged":
// FP32 kernel values below 2^-126 flush to zero, so such a row's rate could
// have lost a noticeable share of its terms.  Flagged rows get their rate,
// their own gradient, and their 1/lambda_n contribution to every other row's
// gradient from FP64 loops over all events; in the FP32 gradient pass their
// weight w_n is zero.  Flagged rows are listed per finalize CTA (segment) in
// row order, so every sum over them is also taken in a fixed order.
#include <algorithm>
#include <cmath>

#include "hk_internal.cuh"

namespace hk {

namespace {

constexpr int kT = kFinalizeThreads;

struct Nsum {
    double s = 0.0, c = 0.0;
    __device__ void add(double x)
    {
        const double t = s + x;
        if (!isfinite(t)) {
            s = t;
            c = 0.0;
            return;
        }
        if (fabs(s) >= fabs(x))
            c += (s - t) + x;
        else
            c += (x - t) + s;
        s = t;
    }
    __device__ double value() const { return isfinite(s) ? s + c : s; }
};

__device__ __forceinline__ int set_of_segment(const Work &w, int g)
{
    int lo = 0, hi = w.nsets - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (w.sets[mid].seg0 <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Fixed-order tree sum over the CTA (blockDim.x == kT).
__device__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// sum_{k < count} p[k * stride] of FP32 partials, added in the order
// k = 0, 1, ... with Kahan compensation in FP32 (FP64 adds run at 1/64 of
// the FP32 rate here), returned in FP64.  The error is about two FP32 units
// of sum |p_k|; the loads of sixteen consecutive terms are issued together.
__device__ __forceinline__ double ordered_strided_sum(const float *__restrict__ p, int count, int64_t stride)
{
    float s = 0.0f, c = 0.0f;
    int k = 0;
    for (; k + 16 <= count; k += 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u)
            v[u] = p[(int64_t)(k + u) * stride];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const float y = v[u] - c;
            const float t = s + y;
            c = (t - s) - y;
            s = t;
        }
    }
    for (; k < count; ++k) {
        const float y = p[(int64_t)k * stride] - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    return (double)s - (double)c;
}

// The same ordered compensated sums for NV values at once (value q at
// p[q * vstride + k * stride]): every value is added in the order
// k = 0, 1, ..., exactly as ordered_strided_sum does, but the loads of eight
// slots of all NV values are issued together, so a row's NV sums cost the
// memory round trips of one.
template <int NV>
__device__ __forceinline__ void ordered_strided_sums(const float *__restrict__ p, int64_t vstride, int count,
                                                     int64_t stride, double *out)
{
    float s[NV], c[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q)
        s[q] = c[q] = 0.0f;
    for (int k = 0; k < count; k += 8) {
        float v[8][NV];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int q = 0; q < NV; ++q)
                v[u][q] = (k + u < count) ? p[(int64_t)(k + u) * stride + (int64_t)q * vstride] : 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if (k + u < count) {
                    const float y = v[u][q] - c[q];
                    const float t = s[q] + y;
                    c[q] = (t - s[q]) - y;
                    s[q] = t;
                }
            }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q)
        out[q] = (double)s[q] - (double)c[q];
}

// Runtime value count 1..kMaxD dispatched to the compile-time version.
__device__ __forceinline__ void ordered_strided_sums_d(int nv, const float *__restrict__ p, int64_t vstride,
                                                       int count, int64_t stride, double *out)
{
    switch (nv) {
    case 1: ordered_strided_sums<1>(p, vstride, count, stride, out); break;
    case 2: ordered_strided_sums<2>(p, vstride, count, stride, out); break;
    case 3: ordered_strided_sums<3>(p, vstride, count, stride, out); break;
    case 4: ordered_strided_sums<4>(p, vstride, count, stride, out); break;
    case 5: ordered_strided_sums<5>(p, vstride, count, stride, out); break;
    case 6: ordered_strided_sums<6>(p, vstride, count, stride, out); break;
    case 7: ordered_strided_sums<7>(p, vstride, count, stride, out); break;
    default: ordered_strided_sums<8>(p, vstride, count, stride, out); break;
    }
}

struct PairFp64 {
    double a, b, c, Cmu, Cxi, omega, itx2, ih2;
    __device__ explicit PairFp64(const SetDesc &S)
    {
        const double two_pi = 6.283185307179586476925286766559;
        a = 0.5 / (S.tau_x * S.tau_x);
        b = 0.5 / (S.tau_t * S.tau_t);
        c = 0.5 / (S.h * S.h);
        Cmu = S.mu0 / (pow(S.tau_x, (double)S.d) * S.tau_t * pow(two_pi, 0.5 * (S.d + 1)));
        Cxi = S.theta * S.omega / (pow(S.h, (double)S.d) * pow(two_pi, 0.5 * S.d));
        omega = S.omega;
        itx2 = 1.0 / (S.tau_x * S.tau_x);
        ih2 = 1.0 / (S.h * S.h);
    }
};

// ------------------------------------------------------ finalize rows --

constexpr double kLog2e = 1.4426950408889634074;

// theta: which row sums the rate pass kept besides the rate (RateSums)
__global__ void __launch_bounds__(kT) finalize_rows_kernel(Work w, int fp64, int theta)
{
    __shared__ double sh[kT];
    __shared__ int wcount[kT / 32];
    const int g = blockIdx.x;
    const int s = set_of_segment(w, g);
    const SetDesc &S = w.sets[s];
    const int i = (g - S.seg0) * kT + threadIdx.x;
    const bool active = i < S.n;
    bool flagged = false;
    double lnl_v = 0.0;
    if (active) {
        const int64_t r = S.row0 + i;
        double lam, inv_sum = 0.0, log_sum = 0.0;
        if (fp64) {
            const int V = theta ? kPass1ThetaVals : 1;
            Nsum acc;
            Nsum th[kPass1ThetaVals];
            for (int sp = 0; sp < S.fsplit; ++sp) {
                const double *F = w.F1 + S.fpart0 + (int64_t)sp * V * S.npad + i;
                if (theta) {
                    for (int v = 0; v < kPass1ThetaVals; ++v)
                        th[v].add(F[(int64_t)v * S.npad]);
                } else {
                    acc.add(F[0]);
                }
            }
            if (theta) {
                for (int v = 0; v < kPass1ThetaVals; ++v)
                    w.theta_rows[r * kPass1ThetaVals + v] = th[v].value();
                lam = th[0].value() + th[1].value();
            } else {
                lam = acc.value();
            }
        } else if (theta == kSumsXi) {
            // background and self-excitation sums apart: the rate and sum_n' xi_nn'
            double v[kPass1XiVals];
            ordered_strided_sums<kPass1XiVals>(w.P1 + S.part0 + i, S.npad, S.nblk, (int64_t)kPass1XiVals * S.npad,
                                               v);
            const double sum = v[0] + v[1];
            flagged = !(sum >= S.s_min);
            lam = S.Pmu * sum;
            if (!flagged) {
                inv_sum = 1.0 / sum;
                log_sum = log(sum);
            }
            w.w32[r] = flagged ? 0.0f : (float)inv_sum;
            w.cm32[r] = flagged ? -INFINITY : (float)(S.cxi2_d - log_sum * kLog2e);
            w.theta_rows[r * kPass1ThetaVals + 1] = S.Pmu * v[1];
        } else if (theta) {
            double v[kMaxD];
            ordered_strided_sums<kPass1ThetaVals>(w.P1 + S.part0 + i, S.npad, S.nblk,
                                                  (int64_t)kPass1ThetaVals * S.npad, v);
            const double sum = v[0] + v[1];
            flagged = !(sum >= S.s_min);
            lam = S.Pmu * sum;
            if (!flagged) {
                inv_sum = 1.0 / sum;
                log_sum = log(sum);
            }
            w.w32[r] = flagged ? 0.0f : (float)inv_sum;
            w.cm32[r] = flagged ? -INFINITY : (float)(S.cxi2_d - log_sum * kLog2e);
            // natural units: sum mu, sum xi, sum mu r^2, sum mu dt^2, sum xi dt, sum xi r^2
            const double ikx2 = 1.0 / (S.kx * S.kx), ikt = 1.0 / S.kt;
            double *T = w.theta_rows + r * kPass1ThetaVals;
            T[0] = S.Pmu * v[0];
            T[1] = S.Pmu * v[1];
            T[2] = S.Pmu * v[2] * ikx2;
            T[3] = S.Pmu * v[3] * ikt * ikt;
            T[4] = S.Pmu * v[4] * ikt;
            T[5] = S.Pmu * v[5] * ikx2;
        } else {
            const double sum = ordered_strided_sum(w.P1 + S.part0 + i, S.nblk, S.npad);
            flagged = !(sum >= S.s_min);
            lam = S.Pmu * sum;
            if (!flagged) {
                inv_sum = 1.0 / sum;
                log_sum = log(sum);
            }
            w.w32[r] = flagged ? 0.0f : (float)inv_sum;
            w.cm32[r] = flagged ? -INFINITY : (float)(S.cxi2_d - log_sum * kLog2e);
        }
        if (!flagged) {
            // one FP64 division and one log per row (FP64 is a long-latency
            // path on this GPU): 1/lambda = (1/S) (1/Pmu), log lambda = log Pmu + log S
            w.lam64[r] = lam;
            w.w64[r] = fp64 ? 1.0 / lam : inv_sum * S.iPmu;
            lnl_v = (fp64 ? log(lam) : S.lPmu + log_sum) - w.Lam64[r];
            w.lnl[r] = lnl_v;
            if (!(lam > 0.0))
                atomicOr(&w.set_flags[s], 1);
        }
    }
    // bound on the gradient pass's column constants (for block skipping)
    if (!fp64) {
        float cmv = (active && !flagged) ? fmaxf(w.cm32[S.row0 + i], 0.0f) : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            cmv = fmaxf(cmv, __shfl_xor_sync(0xffffffffu, cmv, o));
        if ((threadIdx.x & 31) == 0 && cmv > 0.0f)
            atomicMax(&w.set_cmmax[s], __float_as_int(cmv));
    }
    // flagged rows of this segment, in row order
    const unsigned ball = __ballot_sync(0xffffffffu, flagged);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        wcount[wid] = __popc(ball);
    const double tot = block_sum(flagged ? 0.0 : lnl_v, sh);
    int off = 0;
    for (int q = 0; q < wid; ++q)
        off += wcount[q];
    if (flagged)
        w.seg_rows[(int64_t)g * kT + off + __popc(ball & ((1u << lane) - 1u))] = i;
    if (threadIdx.x == 0) {
        int cnt = 0;
        for (int q = 0; q < kT / 32; ++q)
            cnt += wcount[q];
        w.seg_count[g] = cnt;
        w.seg_sum[g] = tot;
        if (cnt)
            atomicAdd(&w.counters[2], cnt);
    }
}

// FP64 rate of one row, summed by the whole CTA in a fixed order.
__device__ double rate_fp64(const Work &w, const SetDesc &S, int i, double *sh)
{
    const PairFp64 k(S);
    const int64_t R0 = S.row0;
    const double tn = w.t64[R0 + i];
    Nsum acc;
    for (int m = threadIdx.x; m < S.n; m += kT) {
        const double tm = w.t64[R0 + m];
        if (tm == tn)
            continue;
        double r2 = 0.0;
        for (int q = 0; q < S.d; ++q) {
            const double df = w.x64[(R0 + i) * kMaxD + q] - w.x64[(R0 + m) * kMaxD + q];
            r2 += df * df;
        }
        const double dt = tn - tm;
        double v = k.Cmu * exp(-(r2 * k.a + dt * dt * k.b));
        if (tm < tn)
            v += k.Cxi * exp(-(k.omega * dt + r2 * k.c));
        acc.add(v);
    }
    return block_sum(acc.value(), sh);
}

// The six parameter-gradient row sums of one row in FP64 (natural units).
__device__ void theta_sums_fp64(const Work &w, const SetDesc &S, int i, double *sh, double *out6)
{
    const PairFp64 k(S);
    const int64_t R0 = S.row0;
    const double tn = w.t64[R0 + i];
    Nsum acc[kPass1ThetaVals];
    for (int m = threadIdx.x; m < S.n; m += kT) {
        const double tm = w.t64[R0 + m];
        if (tm == tn)
            continue;
        double r2 = 0.0;
        for (int q = 0; q < S.d; ++q) {
            const double df = w.x64[(R0 + i) * kMaxD + q] - w.x64[(R0 + m) * kMaxD + q];
            r2 += df * df;
        }
        const double dt = tn - tm;
        const double mu = k.Cmu * exp(-(r2 * k.a + dt * dt * k.b));
        acc[0].add(mu);
        acc[2].add(mu * r2);
        acc[3].add(mu * dt * dt);
        if (tm < tn) {
            const double xi = k.Cxi * exp(-(k.omega * dt + r2 * k.c));
            acc[1].add(xi);
            acc[4].add(xi * dt);
            acc[5].add(xi * r2);
        }
    }
    for (int q = 0; q < kPass1ThetaVals; ++q)
        out6[q] = block_sum(acc[q].value(), sh);
}

// Flagged rows get their rate in FP64; the last CTA to finish writes ell of
// every set: the segments' sums in order, then the flagged rows in order.
__global__ void __launch_bounds__(kT) fixup_rows_kernel(Work w, int total_segs, double *out_loglik, int theta)
{
    __shared__ double sh[kT];
    __shared__ int s_last;
    const int total_flagged = w.counters[2];
    if (total_flagged > 0) {
        int f = 0;  // flat index of the first flagged row of segment g
        for (int g = 0; g < total_segs; ++g) {
            const int cnt = w.seg_count[g];
            for (int k2 = 0; k2 < cnt; ++k2) {
                if ((f + k2) % (int)gridDim.x != (int)blockIdx.x)
                    continue;
                const int s = set_of_segment(w, g);
                const SetDesc &S = w.sets[s];
                const int i = w.seg_rows[(int64_t)g * kT + k2];
                const double lam = rate_fp64(w, S, i, sh);
                if (theta) {
                    double v6[kPass1ThetaVals];
                    theta_sums_fp64(w, S, i, sh, v6);
                    if (threadIdx.x == 0)
                        for (int q = 0; q < kPass1ThetaVals; ++q)
                            w.theta_rows[(S.row0 + i) * kPass1ThetaVals + q] = v6[q];
                }
                if (threadIdx.x == 0) {
                    const int64_t r = S.row0 + i;
                    w.lam64[r] = lam;
                    w.w64[r] = 1.0 / lam;
                    w.lnl[r] = log(lam) - w.Lam64[r];
                    if (!(lam > 0.0))
                        atomicOr(&w.set_flags[s], 1);
                }
            }
            f += cnt;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&w.counters[3], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    for (int s = 0; s < w.nsets; ++s) {
        const SetDesc &S = w.sets[s];
        double v = 0.0;
        for (int g = S.seg0 + threadIdx.x; g < S.seg0 + S.nseg; g += kT)
            v += w.seg_sum[g];
        double ell = block_sum(v, sh);
        if (threadIdx.x == 0) {
            if (total_flagged > 0) {
                for (int g = S.seg0; g < S.seg0 + S.nseg; ++g)
                    for (int k2 = 0; k2 < w.seg_count[g]; ++k2)
                        ell += w.lnl[S.row0 + w.seg_rows[(int64_t)g * kT + k2]];
            }
            w.set_loglik[s] = ell;
            if (out_loglik)
                out_loglik[s] = ell;
        }
    }
    if (threadIdx.x == 0)
        w.counters[3] = 0;
}

// ------------------------------------------------------ finalize grad --

// One thread per row: sum the gradient slots, add the FP64 contributions of
// the flagged rows' 1/lambda terms, write in the caller's order (and sorted,
// for the HMC integrator).
__global__ void __launch_bounds__(kT) finalize_grad_kernel(Work w, int fp64, double *out_grad, double *g_sorted)
{
    const int g = blockIdx.x;
    const int s = set_of_segment(w, g);
    const SetDesc &S = w.sets[s];
    const int i = (g - S.seg0) * kT + threadIdx.x;
    if (i >= S.n)
        return;
    const int d = S.d;
    const int64_t r = S.row0 + i;
    const bool zero_rate = (w.set_flags[s] & 1) != 0;
    double gv[kMaxD];
    if (fp64) {
#pragma unroll
        for (int q = 0; q < kMaxD; ++q) {
            if (q < d) {
                Nsum acc;
                for (int sp = 0; sp < S.fsplit; ++sp)
                    acc.add(w.F2[S.fpart2_0 + ((int64_t)sp * d + q) * S.npad + i]);
                gv[q] = acc.value();
            }
        }
    } else {
        if (zero_rate && i == 0)
            atomicOr(w.status, kStZeroRate);
        if (w.w32[r] == 0.0f)
            return;  // a flagged row: fixup_grad_kernel writes its gradient
        ordered_strided_sums_d(d, w.P2 + S.part2_0 + i, S.npad, S.nblk, (int64_t)d * S.npad, gv);
#pragma unroll
        for (int q = 0; q < kMaxD; ++q)
            if (q < d)
                gv[q] *= S.Cg;
        if (w.counters[2] > 0) {
            // contributions through the flagged rows' own rates:
            // w_n [mu_nm / tau_x^2 + xi_nm / h^2] (x_n - x_m), xi_nm when t_m < t_n
            const PairFp64 k(S);
            const double tm = w.t64[r];
            for (int gg = S.seg0; gg < S.seg0 + S.nseg; ++gg) {
                const int cnt = w.seg_count[gg];
                for (int k2 = 0; k2 < cnt; ++k2) {
                    const int nrow = w.seg_rows[(int64_t)gg * kT + k2];
                    if (nrow == i)
                        continue;
                    const int64_t rn = S.row0 + nrow;
                    const double tn = w.t64[rn];
                    if (tn == tm)
                        continue;
                    double r2 = 0.0;
                    for (int q = 0; q < d; ++q) {
                        const double df = w.x64[rn * kMaxD + q] - w.x64[r * kMaxD + q];
                        r2 += df * df;
                    }
                    const double dt = tn - tm;
                    double coef = k.Cmu * exp(-(r2 * k.a + dt * dt * k.b)) * k.itx2;
                    if (tm < tn)
                        coef += k.Cxi * exp(-(k.omega * dt + r2 * k.c)) * k.ih2;
                    coef *= w.w64[rn];
#pragma unroll
                    for (int q = 0; q < kMaxD; ++q)
                        if (q < d)
                            gv[q] += coef * (w.x64[rn * kMaxD + q] - w.x64[r * kMaxD + q]);
                }
            }
        }
    }
    if (zero_rate) {
#pragma unroll
        for (int q = 0; q < kMaxD; ++q)
            if (q < d)
                gv[q] = nan("");
        if (fp64 && i == 0)
            atomicOr(w.status, kStZeroRate);
    }
    const int src = w.perm[r];
    if (out_grad) {
#pragma unroll
        for (int q = 0; q < kMaxD; ++q)
            if (q < d)
                out_grad[S.x0 + (int64_t)src * d + q] = gv[q];
    }
    if (g_sorted) {
#pragma unroll
        for (int q = 0; q < kMaxD; ++q)
            if (q < d)
                g_sorted[r * kMaxD + q] = gv[q];
    }
}

// Own gradient of every flagged row, in FP64 over all events (the paper's
// Appendix A formula in its ordered form).
__global__ void __launch_bounds__(kT) fixup_grad_kernel(Work w, int total_segs, double *out_grad, double *g_sorted)
{
    __shared__ double sh[kT];
    if (w.counters[2] == 0)
        return;
    int f = 0;
    for (int g = 0; g < total_segs; ++g) {
        const int cnt = w.seg_count[g];
        for (int k2 = 0; k2 < cnt; ++k2) {
            if ((f + k2) % (int)gridDim.x != (int)blockIdx.x)
                continue;
            const int s = set_of_segment(w, g);
            const SetDesc &S = w.sets[s];
            const PairFp64 k(S);
            const int i = w.seg_rows[(int64_t)g * kT + k2];
            const int64_t R0 = S.row0, r = R0 + i;
            const double tn = w.t64[r], wn = w.w64[r];
            const bool zero_rate = (w.set_flags[s] & 1) != 0;
            const int src = w.perm[r];
            for (int q = 0; q < S.d; ++q) {
                Nsum acc;
                for (int m = threadIdx.x; m < S.n; m += kT) {
                    const double tm = w.t64[R0 + m];
                    if (tm == tn)
                        continue;
                    double r2 = 0.0;
                    for (int q2 = 0; q2 < S.d; ++q2) {
                        const double df = w.x64[r * kMaxD + q2] - w.x64[(R0 + m) * kMaxD + q2];
                        r2 += df * df;
                    }
                    const double dt = tn - tm;
                    const double wm = w.w64[R0 + m];
                    const double mu = k.Cmu * exp(-(r2 * k.a + dt * dt * k.b));
                    const double xi = k.Cxi * exp(-(k.omega * fabs(dt) + r2 * k.c));
                    const double coef = mu * (wn + wm) * k.itx2 + xi * (tm < tn ? wn : wm) * k.ih2;
                    acc.add(coef * (w.x64[(R0 + m) * kMaxD + q] - w.x64[r * kMaxD + q]));
                }
                double gq = block_sum(acc.value(), sh);
                if (zero_rate)
                    gq = nan("");
                if (threadIdx.x == 0) {
                    if (out_grad)
                        out_grad[S.x0 + (int64_t)src * S.d + q] = gq;
                    if (g_sorted)
                        g_sorted[r * kMaxD + q] = gq;
                }
            }
        }
        f += cnt;
    }
}

// d ell / d Theta of set 0 (Theta order mu0, tau_x, tau_t, theta, omega, h):
// per row, the rate-term sums divided by lambda_n plus the derivative of
// -Lambda_n; summed over rows in a fixed order.
// The six Theta-gradient sums over the rows (each row's terms need FP64
// normcdf, exp and divisions), split over kThetaParts CTAs so that the FP64
// work spreads over the SMs; each CTA writes its six compensated partials
// and theta_finish_kernel adds them in CTA order.
__global__ void __launch_bounds__(kT) theta_grad_kernel(Work w)
{
    __shared__ double sh[kT];
    const SetDesc &S = w.sets[0];
    const double D = (double)S.d;
    const double tx = S.tau_x, tt = S.tau_t, h = S.h, om = S.omega, th = S.theta, mu0 = S.mu0;
    const double T = w.t64[S.row0 + S.n - 1];
    const double inv_sqrt_2pi = 0.39894228040143267793994605993438;
    Nsum acc[6];
    for (int i = blockIdx.x * kT + threadIdx.x; i < S.n; i += gridDim.x * kT) {
        const int64_t r = S.row0 + i;
        const double *A = w.theta_rows + r * kPass1ThetaVals;
        const double lam = w.lam64[r];
        const double tn = w.t64[r];
        const double a = T - tn;
        const double ea = exp(-om * a);
        acc[0].add(A[0] / (mu0 * lam) - (normcdf(a / tt) - normcdf(-tn / tt)));
        acc[1].add((A[2] / (tx * tx * tx) - D * A[0] / tx) / lam);
        acc[2].add((A[3] / (tt * tt * tt) - A[0] / tt) / lam +
                   mu0 * inv_sqrt_2pi * (exp(-0.5 * (a / tt) * (a / tt)) * a + exp(-0.5 * (tn / tt) * (tn / tt)) * tn) /
                       (tt * tt));
        acc[3].add(A[1] / (th * lam) + expm1(-om * a));
        acc[4].add((A[1] / om - A[4]) / lam - th * a * ea);
        acc[5].add((A[5] / (h * h * h) - D * A[1] / h) / lam);
    }
    for (int q = 0; q < 6; ++q) {
        const double v = block_sum(acc[q].value(), sh);
        if (threadIdx.x == 0)
            w.theta_parts[blockIdx.x * kPass1ThetaVals + q] = v;
    }
}

__global__ void theta_finish_kernel(Work w, int parts, double *out6)
{
    const int q = threadIdx.x;
    if (q >= 6)
        return;
    Nsum acc;
    for (int b = 0; b < parts; ++b)
        acc.add(w.theta_parts[b * kPass1ThetaVals + q]);
    const bool zero_rate = (w.set_flags[0] & 1) != 0;
    out6[q] = zero_rate ? nan("") : acc.value();
}

// xi_n / lambda_n per event in the caller's order (the self-excitation
// probability of an event under the current state).
__global__ void self_excitation_kernel(Work w, double *out)
{
    const int g = blockIdx.x;
    const int s = set_of_segment(w, g);
    const SetDesc &S = w.sets[s];
    const int i = (g - S.seg0) * kT + threadIdx.x;
    if (i >= S.n)
        return;
    const int64_t r = S.row0 + i;
    const double lam = w.lam64[r];
    out[S.ev0 + w.perm[r]] = lam > 0.0 ? w.theta_rows[r * kPass1ThetaVals + 1] / lam : nan("");
}

}  // namespace

cudaError_t launch_finalize_rows(const Work &w, int32_t total_segs, bool fp64, int sums, cudaStream_t s)
{
    finalize_rows_kernel<<<total_segs, kT, 0, s>>>(w, fp64 ? 1 : 0, sums);
    return cudaGetLastError();
}

cudaError_t launch_fixup_rows(const Work &w, int32_t total_segs, int32_t grid, double *out_loglik, bool theta,
                              cudaStream_t s)
{
    fixup_rows_kernel<<<grid, kT, 0, s>>>(w, total_segs, out_loglik, theta ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_finalize_grad(const Work &w, int32_t total_segs, bool fp64, double *out_grad, double *g_sorted,
                                 cudaStream_t s)
{
    finalize_grad_kernel<<<total_segs, kT, 0, s>>>(w, fp64 ? 1 : 0, out_grad, g_sorted);
    return cudaGetLastError();
}

cudaError_t launch_fixup_grad(const Work &w, int32_t total_segs, int32_t grid, double *out_grad, double *g_sorted,
                              cudaStream_t s)
{
    fixup_grad_kernel<<<grid, kT, 0, s>>>(w, total_segs, out_grad, g_sorted);
    return cudaGetLastError();
}

cudaError_t launch_theta_grad(const Work &w, int64_t n, double *out6, cudaStream_t s)
{
    const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(kThetaParts, (n + kT - 1) / kT));
    theta_grad_kernel<<<parts, kT, 0, s>>>(w);
    theta_finish_kernel<<<1, 32, 0, s>>>(w, parts, out6);
    return cudaGetLastError();
}

cudaError_t launch_self_excitation(const Work &w, int32_t total_segs, double *out, cudaStream_t s)
{
    self_excitation_kernel<<<total_segs, kT, 0, s>>>(w, out);
    return cudaGetLastError();
}

}  // namespace hk
