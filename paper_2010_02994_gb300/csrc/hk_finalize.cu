// Row finalization in FP64 after each pair pass: rates, log-likelihood
// (Eq. (1)) and gradients (Appendix A), with the FP64 recompute of the rows
// whose mixed-precision rate is too small to trust in FP32 (hk_rows.cuh),
// the parameter gradient and the self-excitation probabilities.
//
// F CTAs of kSegRows threads finalize one segment of kSegRows rows (grid
// (segments, F)).  Each of them sums the segment's slots and so finds the
// same flagged rows; the first writes the rows' results, and the flagged
// rows' FP64 work is dealt round-robin to the F CTAs.  F is 1 when there are
// enough segments to fill the GPU (none of the paper-shaped workloads has a
// flagged row) and larger for small problems, so that data with many
// isolated events still spreads its FP64 recomputation over the SMs; no
// separate fixup launch is needed.  The CTA that finishes a set's last
// segment (a per-set ticket over all its CTAs) writes the set's ell, so the
// sets of a batch are summed in parallel.
#include <algorithm>
#include <cmath>

#include "hk_internal.cuh"
#include "hk_rows.cuh"

namespace hk {

namespace {

constexpr int kT = kFinalizeThreads;
static_assert(kT == kSegRows, "a standalone finalize CTA handles one segment");

// ------------------------------------------------------ finalize rows --


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
        out6[q] = cta_sum(acc[q].value(), sh, kT);
}

// One row per thread.  fp64: the FP64 path's slots; else the mixed path's,
// with the rate pass's extra row sums (RateSums: none, the six
// parameter-gradient sums, or the self-excitation sum apart).
__global__ void __launch_bounds__(kT) finalize_rows_kernel(Work w, int fp64, int sums, double *out_loglik, int ell)
{
    __shared__ double s_lnl[kT];
    __shared__ double sh[kT];
    __shared__ int s_fl[kT];
    __shared__ int s_last;
    const int g = blockIdx.x, f = blockIdx.y, F = gridDim.y;
    const bool writer = f == 0;
    const int s = set_of_segment(w, g);
    const SetDesc &S = w.sets[s];
    const int i = (g - S.seg0) * kT + threadIdx.x;
    const bool active = i < S.n;
    bool flagged = false;
    double lnl_v = 0.0;
    float cmv = 0.0f;
    if (active && !fp64 && sums == kSumsNone) {
        const RowRate rr = finalize_rate_row(w, S, s, i, writer);
        flagged = rr.flagged;
        lnl_v = rr.lnl;
        if (!flagged && writer)
            cmv = fmaxf(w.cm32[S.row0 + i], 0.0f);
    } else if (active && !writer) {
        // only the flag: the first CTA of the segment stores the results
        if (!fp64) {
            double v[kMaxD];
            if (sums == kSumsXi)
                ordered_strided_sums<kPass1XiVals>(w.P1 + S.part0 + i, S.npad, S.nslot,
                                                   (int64_t)kPass1XiVals * S.npad, v);
            else
                ordered_strided_sums<kPass1ThetaVals>(w.P1 + S.part0 + i, S.npad, S.nslot,
                                                      (int64_t)kPass1ThetaVals * S.npad, v);
            flagged = !(v[0] + v[1] >= S.s_min);
        }
    } else if (active) {
        const int64_t r = S.row0 + i;
        double lam, inv_sum = 0.0, log_sum = 0.0;
        if (fp64) {
            const int V = sums == kSumsTheta ? kPass1ThetaVals : 1;
            Nsum acc;
            Nsum th[kPass1ThetaVals];
            for (int sp = 0; sp < S.fsplit; ++sp) {
                const double *Fp = w.F1 + S.fpart0 + (int64_t)sp * V * S.npad + i;
                if (sums == kSumsTheta) {
                    for (int v = 0; v < kPass1ThetaVals; ++v)
                        th[v].add(Fp[(int64_t)v * S.npad]);
                } else {
                    acc.add(Fp[0]);
                }
            }
            if (sums == kSumsTheta) {
                for (int v = 0; v < kPass1ThetaVals; ++v)
                    w.theta_rows[r * kPass1ThetaVals + v] = th[v].value();
                lam = th[0].value() + th[1].value();
            } else {
                lam = acc.value();
            }
        } else {
            double v[kMaxD];
            if (sums == kSumsXi)
                ordered_strided_sums<kPass1XiVals>(w.P1 + S.part0 + i, S.npad, S.nslot,
                                                   (int64_t)kPass1XiVals * S.npad, v);
            else
                ordered_strided_sums<kPass1ThetaVals>(w.P1 + S.part0 + i, S.npad, S.nslot,
                                                      (int64_t)kPass1ThetaVals * S.npad, v);
            const double sum = v[0] + v[1];
            flagged = !(sum >= S.s_min);
            lam = S.Pmu * sum;
            if (!flagged) {
                inv_sum = 1.0 / sum;
                log_sum = log(sum);
            }
            w.w32[r] = flagged ? 0.0f : (float)inv_sum;
            w.cm32[r] = flagged ? -INFINITY : (float)(S.cxi2_d - log_sum * kLog2eD);
            if (!flagged)
                cmv = fmaxf(w.cm32[r], 0.0f);
            if (sums == kSumsXi) {
                w.theta_rows[r * kPass1ThetaVals + 1] = S.Pmu * v[1];
            } else {
                // natural units: sum mu, sum xi, sum mu r^2, sum mu dt^2, sum xi dt, sum xi r^2
                const double ikx2 = 1.0 / (S.kx * S.kx), ikt = 1.0 / S.kt;
                double *T = w.theta_rows + r * kPass1ThetaVals;
                T[0] = S.Pmu * v[0];
                T[1] = S.Pmu * v[1];
                T[2] = S.Pmu * v[2] * ikx2;
                T[3] = S.Pmu * v[3] * ikt * ikt;
                T[4] = S.Pmu * v[4] * ikt;
                T[5] = S.Pmu * v[5] * ikx2;
            }
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
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            cmv = fmaxf(cmv, __shfl_xor_sync(0xffffffffu, cmv, o));
        if ((threadIdx.x & 31) == 0 && cmv > 0.0f)
            atomicMax(&w.set_cmmax[s], __float_as_int(cmv));
    }
    s_lnl[threadIdx.x] = lnl_v;
    s_fl[threadIdx.x] = flagged ? 1 : 0;
    __syncthreads();
    if (writer && threadIdx.x < 32)
        segment_finish(w, s, g, (g - S.seg0) * kT, s_lnl, s_fl);
    __syncthreads();
    // this segment's flagged rows, in row order, dealt round-robin to the F
    // CTAs: FP64 rates over all events (and the six parameter-gradient sums
    // when the rate pass kept them)
    for (int k = 0, nf = 0; k < kT; ++k) {
        if (!s_fl[k] || nf++ % F != f)
            continue;
        const int fi = (g - S.seg0) * kT + k;
        if (sums == kSumsTheta || sums == kSumsXi) {
            double v6[kPass1ThetaVals];
            theta_sums_fp64(w, S, fi, sh, v6);
            if (threadIdx.x == 0)
                for (int q = 0; q < kPass1ThetaVals; ++q)
                    w.theta_rows[(S.row0 + fi) * kPass1ThetaVals + q] = v6[q];
        }
        fixup_rate_row(w, S, s, fi, sh, kT);
    }
    // the set's last segment writes its ell (when it is wanted: an HMC step
    // between the trajectory's ends needs only the rates)
    if (!ell)
        return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = atomicAdd(&w.set_done[s], 1) == S.nseg * F - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x < 32)
            set_loglik_finish(w, s, out_loglik);
        if (threadIdx.x == 0)
            w.set_done[s] = 0;
    }
}

// ------------------------------------------------------ finalize grad --

// One thread per row sums the gradient slots in a fixed order and writes the
// row's gradient in the caller's order (and sorted, for the HMC integrator);
// on the mixed path the FP64 terms through the flagged rows' rates are added,
// and the segment's flagged rows then get their own gradient in FP64 from the
// whole CTA.
__global__ void __launch_bounds__(kT) finalize_grad_kernel(Work w, int fp64, double *out_grad, double *g_sorted)
{
    __shared__ double sh[kT];
    const int g = blockIdx.x, f = blockIdx.y, F = gridDim.y;
    const int s = set_of_segment(w, g);
    const SetDesc &S = w.sets[s];
    const int i = (g - S.seg0) * kT + threadIdx.x;
    const bool zero_rate = (w.set_flags[s] & 1) != 0;
    if (i == 0 && f == 0 && zero_rate)
        atomicOr(w.status, kStZeroRate);
    if (fp64) {
        if (i >= S.n || f != 0)
            return;
        const int d = S.d;
        const int64_t r = S.row0 + i;
        double gv[kMaxD];
#pragma unroll
        for (int q = 0; q < kMaxD; ++q) {
            if (q < d) {
                Nsum acc;
                for (int sp = 0; sp < S.fsplit; ++sp)
                    acc.add(w.F2[S.fpart2_0 + ((int64_t)sp * d + q) * S.npad + i]);
                gv[q] = zero_rate ? nan("") : acc.value();
            }
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
        return;
    }
    if (f == 0 && i < S.n && w.w32[S.row0 + i] != 0.0f)
        finalize_grad_row(w, S, s, i, out_grad, g_sorted);
    // the segment's flagged rows, dealt round-robin to its F CTAs
    const int cnt = w.seg_count[g];
    for (int k = f; k < cnt; k += F)
        fixup_grad_row(w, S, s, w.seg_rows[(int64_t)g * kSegRows + k], out_grad, g_sorted, sh, kT);
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
        const double v = cta_sum(acc[q].value(), sh, kT);
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

// The partial slots of a set that a fold adds into: part 0 P1, 1 P2 (FP32),
// 2 F1, 3 F1 with the Theta sums, 4 F2 (FP64); V values per slot.
__device__ __forceinline__ float *fold_base(const Work &w, const SetDesc &S, int part, int &V, float *)
{
    V = part == 0 ? S.vpc : S.d;
    return part == 0 ? w.P1 + S.part0 : w.P2 + S.part2_0;
}

__device__ __forceinline__ double *fold_base(const Work &w, const SetDesc &S, int part, int &V, double *)
{
    V = part == 2 ? 1 : (part == 3 ? kPass1ThetaVals : S.d);
    return part == 4 ? w.F2 + S.fpart2_0 : w.F1 + S.fpart0;
}

// After a later phase of the pair schedule: each off-diagonal run of the
// launch's work list is one set and the nr rounds it had in the phase, whose
// partials went to the scratch slots nslot .. nslot + nr - 1; slot j < nr
// gets scratch slot nslot + j added, which is then cleared for the next
// phase.  Both are contiguous ranges of nr V npad values (blockIdx.y: the
// run).
template <typename T>
__global__ void __launch_bounds__(256) fold_slots_kernel(Work w, Sched sc, int part)
{
    const ItemRun ru = sc.runs[blockIdx.y];
    if (ru.diag)
        return;
    const SetDesc &S = w.sets[ru.set];
    int V;
    T *dst = fold_base(w, S, part, V, (T *)nullptr);
    T *src = dst + (int64_t)S.nslot * V * S.npad;
    const int64_t len = (int64_t)ru.nr * V * S.npad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        dst[i] += src[i];
        src[i] = T(0);
    }
}

}  // namespace

// CTAs per segment: enough for about four CTAs per SM in all (mixed path;
// the FP64 path has no flagged rows).
static int ctas_per_segment(const Work &w, int32_t total_segs, bool fp64)
{
    if (fp64)
        return 1;
    const int64_t want = 4LL * std::max(1, w.sm_count);
    return (int)std::min<int64_t>(32, std::max<int64_t>(1, (want + total_segs - 1) / total_segs));
}

cudaError_t launch_fold_slots(const Work &w, const Sched &sc, int part, cudaStream_t s)
{
    if (sc.nruns <= 0)
        return cudaSuccess;
    const dim3 grid((unsigned)std::max(1, (4 * std::max(1, w.sm_count) + sc.nruns - 1) / sc.nruns), (unsigned)sc.nruns);
    if (part <= 1)
        fold_slots_kernel<float><<<grid, 256, 0, s>>>(w, sc, part);
    else
        fold_slots_kernel<double><<<grid, 256, 0, s>>>(w, sc, part);
    return cudaGetLastError();
}

cudaError_t launch_finalize_rows(const Work &w, int32_t total_segs, bool fp64, int sums, double *out_loglik,
                                 cudaStream_t s, bool ell)
{
    const dim3 grid(total_segs, ctas_per_segment(w, total_segs, fp64));
    finalize_rows_kernel<<<grid, kT, 0, s>>>(w, fp64 ? 1 : 0, sums, out_loglik, ell ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_finalize_grad(const Work &w, int32_t total_segs, bool fp64, double *out_grad, double *g_sorted,
                                 cudaStream_t s)
{
    const dim3 grid(total_segs, ctas_per_segment(w, total_segs, fp64));
    finalize_grad_kernel<<<grid, kT, 0, s>>>(w, fp64 ? 1 : 0, out_grad, g_sorted);
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
