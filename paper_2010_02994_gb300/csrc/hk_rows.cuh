// Per-row finalization used by the finalize kernels (hk_finalize.cu).
//
// Mixed path.  S_n is the sum of the pair kernel's FP32 partial slots,
// taken in slot order.  A row with S_n < s_min (or not finite) is "flagged":
// FP32 kernel values below 2^-126 flush to zero, so such a row's rate could
// have lost a noticeable share of its terms.  Flagged rows get their rate,
// their own gradient, and their 1/lambda_n contribution to every other row's
// gradient from FP64 loops over all events; in the FP32 gradient pass their
// weight w_n is zero.  Flagged rows are listed per segment of kSegRows rows
// in row order, so every sum over them is taken in a fixed order; so is the
// log-likelihood, summed per segment by one warp and then over the segments
// by one warp, whatever the CTA that does it.
#pragma once

#include <cmath>

#include "hk_internal.cuh"

namespace hk {

constexpr double kLog2eD = 1.4426950408889634074;

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

// Fixed-order tree sum over the first `nt` threads of the CTA (nt a power of
// two, every one of them calling); sh holds at least nt doubles.
__device__ __forceinline__ double cta_sum(double v, double *sh, int nt)
{
    __syncthreads();
    if ((int)threadIdx.x < nt)
        sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = nt / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Butterfly sum over the 32 lanes of a warp (the same order on every lane).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum_{k < count} p[k * stride] of FP32 partials, added in the order
// k = 0, 1, ... with Kahan compensation in FP32 (FP64 adds run at 1/64 of
// the FP32 rate here), returned in FP64.  The error is about two FP32 units
// of sum |p_k|; the loads of sixteen consecutive terms are issued together.
// Loads bypass L1: the slots may have been written by other SMs during the
// same launch.
__device__ __forceinline__ double ordered_strided_sum(const float *__restrict__ p, int count, int64_t stride)
{
    float s = 0.0f, c = 0.0f;
    int k = 0;
    for (; k + 16 <= count; k += 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u)
            v[u] = __ldcg(p + (int64_t)(k + u) * stride);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const float y = v[u] - c;
            const float t = s + y;
            c = (t - s) - y;
            s = t;
        }
    }
    for (; k < count; ++k) {
        const float y = __ldcg(p + (int64_t)k * stride) - c;
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
                v[u][q] = (k + u < count) ? __ldcg(p + (int64_t)(k + u) * stride + (int64_t)q * vstride) : 0.0f;
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

// FP64 constants of the two rate terms in natural units.
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

// Result of one row of the mixed rate finalization.
struct RowRate {
    bool flagged;
    double lnl;  // log lambda_n - Lambda_n (0 for flagged rows)
};

// Rate of row i of set s from its pass-1 slots (mixed path, no extra sums):
// lambda_n, 1/lambda_n (FP64 and FP32), the gradient pass's column constant,
// log lambda_n - Lambda_n, stored when `write`.  Flagged rows only get
// w32 = 0 and cm32 = -inf.
__device__ __forceinline__ RowRate finalize_rate_row(const Work &w, const SetDesc &S, int s, int i, bool write)
{
    const int64_t r = S.row0 + i;
    const double sum = ordered_strided_sum(w.P1 + S.part0 + i, S.nslot, S.npad);
    RowRate out{!(sum >= S.s_min), 0.0};
    if (!write)
        return out;
    if (out.flagged) {
        w.w32[r] = 0.0f;
        w.cm32[r] = -INFINITY;
        return out;
    }
    // one FP64 division and one log per row (FP64 is a long-latency path on
    // this GPU): 1/lambda = (1/S) (1/Pmu), log lambda = log Pmu + log S
    const double inv_sum = 1.0 / sum, log_sum = log(sum);
    const double lam = S.Pmu * sum;
    w.w32[r] = (float)inv_sum;
    w.cm32[r] = (float)(S.cxi2_d - log_sum * kLog2eD);
    w.lam64[r] = lam;
    w.w64[r] = inv_sum * S.iPmu;
    out.lnl = S.lPmu + log_sum - w.Lam64[r];
    w.lnl[r] = out.lnl;
    return out;
}

// One segment's log-likelihood sum and flagged-row list, by one warp from
// the segment's kSegRows = 64 values in row order (lnl[k], flagged[k] for
// row seg_first + k; rows past the set are given as not flagged, lnl 0):
// lane l adds rows l and l + 32, then a butterfly over the lanes.  Writes
// seg_sum[g], seg_count[g] and seg_rows[g * kSegRows ..] (set-relative rows)
// and marks set s as having flagged rows.
__device__ __forceinline__ void segment_finish(const Work &w, int s, int g, int seg_first, const double *lnl,
                                               const int *flagged)
{
    static_assert(kSegRows == 64, "a segment is two rows per lane of one warp");
    const int lane = threadIdx.x & 31;
    const bool f0 = flagged[lane] != 0, f1 = flagged[lane + 32] != 0;
    const double v = (f0 ? 0.0 : lnl[lane]) + (f1 ? 0.0 : lnl[lane + 32]);
    const double tot = warp_sum(v);
    const unsigned b0 = __ballot_sync(0xffffffffu, f0), b1 = __ballot_sync(0xffffffffu, f1);
    const unsigned below = (1u << lane) - 1u;
    if (f0)
        w.seg_rows[(int64_t)g * kSegRows + __popc(b0 & below)] = seg_first + lane;
    if (f1)
        w.seg_rows[(int64_t)g * kSegRows + __popc(b0) + __popc(b1 & below)] = seg_first + lane + 32;
    if (lane == 0) {
        const int cnt = __popc(b0) + __popc(b1);
        w.seg_count[g] = cnt;
        w.seg_sum[g] = tot;
        if (cnt)
            atomicOr(&w.set_flags[s], 2);
    }
}

// ell of set s from its segment sums and its flagged rows' log terms, by one
// warp: lane l adds the segments l, l + 32, ... in order, a butterfly adds the
// lanes, then lane 0 adds the flagged rows' terms in row order.  Writes
// set_loglik[s] and, when given, out_loglik[s].
__device__ __forceinline__ void set_loglik_finish(const Work &w, int s, double *out_loglik)
{
    const SetDesc &S = w.sets[s];
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int g = S.seg0 + lane; g < S.seg0 + S.nseg; g += 32)
        v += __ldcg(&w.seg_sum[g]);
    double ell = warp_sum(v);
    if (lane == 0) {
        if (__ldcg(&w.set_flags[s]) & 2)
            for (int g = S.seg0; g < S.seg0 + S.nseg; ++g) {
                const int cnt = __ldcg(&w.seg_count[g]);
                for (int k = 0; k < cnt; ++k)
                    ell += __ldcg(&w.lnl[S.row0 + __ldcg(&w.seg_rows[(int64_t)g * kSegRows + k])]);
            }
        w.set_loglik[s] = ell;
        if (out_loglik)
            out_loglik[s] = ell;
    }
}

// FP64 rate of row i of set S, summed by the first nt threads of the CTA in
// a fixed order (every thread of the CTA must call).
__device__ __forceinline__ double rate_fp64_cta(const Work &w, const SetDesc &S, int i, double *sh, int nt)
{
    const PairFp64 k(S);
    const int64_t R0 = S.row0;
    const double tn = w.t64[R0 + i];
    Nsum acc;
    for (int m = threadIdx.x; m < S.n && (int)threadIdx.x < nt; m += nt) {
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
    return cta_sum(acc.value(), sh, nt);
}

// The FP64 rate of a flagged row and what follows from it (every thread of
// the CTA must call; thread 0 stores).
__device__ __forceinline__ void fixup_rate_row(const Work &w, const SetDesc &S, int s, int i, double *sh, int nt)
{
    const double lam = rate_fp64_cta(w, S, i, sh, nt);
    if (threadIdx.x == 0) {
        const int64_t r = S.row0 + i;
        w.lam64[r] = lam;
        w.w64[r] = 1.0 / lam;
        w.lnl[r] = log(lam) - w.Lam64[r];
        if (!(lam > 0.0))
            atomicOr(&w.set_flags[s], 1);
    }
}

// Gradient of an unflagged row i of set s on the mixed path: its pass-2
// slots in slot order, scaled to natural units, plus the FP64 terms through
// the flagged rows' own rates (w_n [mu_nm / tau_x^2 + xi_nm / h^2] (x_n - x_m),
// xi_nm when t_m < t_n), in the caller's order (and sorted, for the HMC
// integrator).
__device__ __forceinline__ void finalize_grad_row(const Work &w, const SetDesc &S, int s, int i, double *out_grad,
                                                  double *g_sorted)
{
    const int d = S.d;
    const int64_t r = S.row0 + i;
    double gv[kMaxD];
    // all coordinates together: eight slots of each in flight per round trip
    ordered_strided_sums_d(d, w.P2 + S.part2_0 + i, S.npad, S.nslot, (int64_t)d * S.npad, gv);
#pragma unroll
    for (int q = 0; q < kMaxD; ++q)
        if (q < d)
            gv[q] *= S.Cg;
    if (w.set_flags[s] & 2) {
        const PairFp64 k(S);
        const double tm = w.t64[r];
        for (int gg = S.seg0; gg < S.seg0 + S.nseg; ++gg) {
            const int cnt = __ldcg(&w.seg_count[gg]);
            for (int k2 = 0; k2 < cnt; ++k2) {
                const int nrow = __ldcg(&w.seg_rows[(int64_t)gg * kSegRows + k2]);
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
                coef *= __ldcg(&w.w64[rn]);
#pragma unroll
                for (int q = 0; q < kMaxD; ++q)
                    if (q < d)
                        gv[q] += coef * (w.x64[rn * kMaxD + q] - w.x64[r * kMaxD + q]);
            }
        }
    }
    if (w.set_flags[s] & 1) {
#pragma unroll
        for (int q = 0; q < kMaxD; ++q)
            if (q < d)
                gv[q] = nan("");
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

// Own gradient of a flagged row, in FP64 over all events (Appendix A in its
// ordered form, plus the BMDS term of Eq. (4) when the gradient pass carried
// it), one pass over the events for every coordinate, summed by the first nt
// threads of the CTA in a fixed order (every thread of the CTA must call;
// thread 0 stores).
__device__ __forceinline__ void fixup_grad_row(const Work &w, const SetDesc &S, int s, int i, double *out_grad,
                                               double *g_sorted, double *sh, int nt)
{
    const PairFp64 k(S);
    const int64_t R0 = S.row0, r = R0 + i;
    const int d = S.d;
    const double tn = w.t64[r], wn = __ldcg(&w.w64[r]);
    const bool zero_rate = (w.set_flags[s] & 1) != 0;
    const int src = w.perm[r];
    Nsum acc[kMaxD];
    for (int m = threadIdx.x; m < S.n && (int)threadIdx.x < nt; m += nt) {
        const double tm = w.t64[R0 + m];
        if (tm == tn && (w.ysort == nullptr || m == i))
            continue;
        double r2 = 0.0;
        for (int q2 = 0; q2 < d; ++q2) {
            const double df = w.x64[r * kMaxD + q2] - w.x64[(R0 + m) * kMaxD + q2];
            r2 += df * df;
        }
        double coef = 0.0;
        if (tm != tn) {
            const double dt = tn - tm;
            const double wm = __ldcg(&w.w64[R0 + m]);
            const double mu = k.Cmu * exp(-(r2 * k.a + dt * dt * k.b));
            const double xi = k.Cxi * exp(-(k.omega * fabs(dt) + r2 * k.c));
            coef = mu * (wn + wm) * k.itx2 + xi * (tm < tn ? wn : wm) * k.ih2;
        }
        if (w.ysort) {
            // the BMDS term of a BMDS-Hawkes trajectory (every other event,
            // tied times included), from the same FP32 y as the pair kernel
            const double y = (double)w.ysort[(int64_t)i * S.npad + m];
            const double delta = sqrt(r2), inv_delta = r2 > 0.0 ? 1.0 / delta : 0.0;
            const double z = delta * w.bmds_inv_sigma_d;
            const double ratio = exp(-0.5 * z * z) * 0.39894228040143267794 / (1.0 - 0.5 * erfc(z * 0.70710678118654752440));
            coef += (ratio * w.bmds_inv_sigma_d - (y - delta) * w.bmds_inv_s2_d) * inv_delta;
        }
#pragma unroll
        for (int q = 0; q < kMaxD; ++q)
            if (q < d)
                acc[q].add(coef * (w.x64[(R0 + m) * kMaxD + q] - w.x64[r * kMaxD + q]));
    }
#pragma unroll
    for (int q = 0; q < kMaxD; ++q) {
        if (q >= d)
            break;
        double gq = cta_sum(acc[q].value(), sh, nt);
        if (zero_rate)
            gq = nan("");
        if (threadIdx.x == 0) {
            if (out_grad)
                out_grad[S.x0 + (int64_t)src * d + q] = gq;
            if (g_sorted)
                g_sorted[r * kMaxD + q] = gq;
        }
    }
}

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

}  // namespace hk
