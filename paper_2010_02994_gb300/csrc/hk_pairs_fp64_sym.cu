// Symmetric FP64 pair kernels: the rate row sums of Eq. (1) (optionally with
// the six parameter-gradient sums) and the location gradient of Appendix A,
// every arithmetic step in double precision, each unordered pair evaluated
// once.
//
// Work: one CTA per pair block {E, L} (E <= L) of kSymRows time-sorted rows.
// Thread i owns row n = L*B + i (the later event of its pairs) and keeps
// its sums in registers; the columns m of block E are staged in shared
// memory.  Warp w covers the 32-column chunks in the order w, w+1, ...
// (mod W), one chunk per round with a CTA barrier between rounds, and in a
// chunk lane l meets column (l + s) mod 32 at step s while the column's
// running sums travel one lane down per step (a systolic shuffle), so after
// 32 steps lane l holds its own column's sums over the warp's 32 rows.  The
// round schedule gives every chunk one writer per round and a fixed order of
// warps.  Both blocks' rows receive the pair block's contribution in the
// slot of its round of the pair schedule (the diagonal block adds both
// directions into it): one writer per slot and launch, launches in order,
// and the fold and finalize kernels add the slots in a fixed order.
//
// Cost model.  On this GPU the FP64 pipe completes about 1.7 operations
// per SM per clock (DFMA, DADD and DMUL alike), some 70 times fewer than
// FP32 FMAs, so the kernels count FP64 operations and little else: tied or
// excluded pairs are decided on integer ranks (n >= tie_end[m] holds exactly
// for m < n with t_m < t_n), the exponentials are base-2 with the exponents
// folded into the constants and evaluated by Tang's table-driven method
// (exp2_neg, 7 FP64 operations), and work whose result rounds to zero is
// skipped, which leaves every sum unchanged: a term of a 32 x 32 chunk (a
// warp's rows against 32 columns) whose smallest time gap alone puts its
// exponent below -1076, and an exponential that no live lane of a warp
// needs above 2^-1076.  Every add and multiply is written as a fused multiply-add
// with a runtime one or negative zero (same results; the all-FMA stream
// measured 5% faster than the mixed one).  A pair costs at most 2D + 23 FP64
// operations in the rate pass and 4D + 23 in the gradient pass, against
// about 100 per unordered pair (D = 2) for the ordered kernels with CUDA's
// exp().
#include <climits>
#include <cmath>

#include "hk_exp2.cuh"
#include "hk_internal.cuh"

namespace hk {

namespace {

constexpr int kB = kSymRows;
constexpr int kW = kB / 32;
constexpr double kLog2eSym = 1.4426950408889634074;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double shfl_next(double v, int lane)
{
    return __shfl_sync(0xffffffffu, v, (lane + 1) & 31);
}

// Values per row kept by each kind: rate (mu, xi), the parameter-gradient
// sums, or the gradient.
template <int KIND, int D>
struct SymVals {
    static constexpr int R = KIND == 0 ? 2 : (KIND == 1 ? 6 : D);  // row values
    static constexpr int C = KIND == 0 ? 1 : (KIND == 1 ? 3 : D);  // column values
};

// Inputs of one warp's 32 x 32 pairs (its rows against one column chunk).
template <int D>
struct ChunkIn {
    const double *ct;
    const double (*cx)[kB];
    const double *cA;
    const int *cte;
    int base, lane, n_eff;
    double tn, An, Bn;
    double ap, bp, cp, wp;  // base-2 exponent constants
    unsigned long long r2_xi;
    double one, mz;
    const double *tab;
};

// The 32 steps of one chunk: at step s lane l meets column base + (l + s)
// mod 32, adds the pair's terms to its row sums and to the column sums it
// carries, and passes those one lane down.  MU / XI: whether the background
// / self-excitation term can be non-zero in this chunk at all.
template <int KIND, int D, bool MU, bool XI>
__device__ __forceinline__ void chunk_pairs(const ChunkIn<D> &in, const double (&xn)[D],
                                            double (&racc)[SymVals<KIND, D>::R], double (&cacc)[SymVals<KIND, D>::C])
{
    constexpr int VC = SymVals<KIND, D>::C;
    const double one = in.one, mz = in.mz;
#pragma unroll 2
    for (int s = 0; s < 32; ++s) {
        const int c = in.base + ((in.lane + s) & 31);
        double dx[D];
        dx[0] = fma(in.cx[0][c], one, -xn[0]);  // x_m - x_n
        double r2 = fma(dx[0], dx[0], mz);
#pragma unroll
        for (int q = 1; q < D; ++q) {
            dx[q] = fma(in.cx[q][c], one, -xn[q]);
            r2 = fma(dx[q], dx[q], r2);
        }
        const bool live = in.n_eff >= in.cte[c];
        // exact skips: an exponential that no live lane of the warp needs
        // above 2^-1076 is not evaluated (it would round to zero).  The
        // self-excitation exponent is at most -c' r^2, so r^2 above r2_xi
        // (compared as bit patterns: r^2 >= +0) rules it out before it is
        // formed.
        double dt = 0.0, mu = 0.0, xi = 0.0;
        bool any_mu = false, any_xi = false;
        if (MU) {
            dt = fma(in.tn, one, -in.ct[c]);  // t_n - t_m
            const double ym = fma(-dt, fma(dt, in.bp, mz), -fma(r2, in.ap, mz));
            any_mu = __any_sync(kFull, live && (unsigned)__double2hiint(ym) <= kHiNeg1076);
            if (any_mu) {  // warp-uniform: every lane makes the call
                const double e = exp2_neg(ym, in.tab, kFull, one, mz);
                mu = live ? e : 0.0;
            }
        }
        if (XI) {
            any_xi = __any_sync(kFull, live && (unsigned long long)__double_as_longlong(r2) <= in.r2_xi);
            if (any_xi) {
                if (!MU)
                    dt = fma(in.tn, one, -in.ct[c]);
                const double yx = fma(-in.wp, dt, -fma(r2, in.cp, mz));
                const double e = exp2_neg(yx, in.tab, kFull, one, mz);
                xi = live ? e : 0.0;
            }
        }
        if (KIND == 0) {
            if (any_mu) {
                racc[0] = fma(mu, one, racc[0]);
                cacc[0] = fma(mu, one, cacc[0]);
            }
            if (any_xi)
                racc[1] = fma(xi, one, racc[1]);
        } else if (KIND == 1) {
            if (any_mu) {
                const double dt2 = fma(dt, dt, mz);
                racc[0] = fma(mu, one, racc[0]);
                racc[2] = fma(mu, r2, racc[2]);
                racc[3] = fma(mu, dt2, racc[3]);
                cacc[0] = fma(mu, one, cacc[0]);
                cacc[1] = fma(mu, r2, cacc[1]);
                cacc[2] = fma(mu, dt2, cacc[2]);
            }
            if (any_xi) {
                racc[1] = fma(xi, one, racc[1]);
                racc[4] = fma(xi, dt, racc[4]);
                racc[5] = fma(xi, r2, racc[5]);
            }
        } else if (any_mu || any_xi) {
            // c_nm = mu (w_n + w_m) / tau_x^2 + xi w_n / h^2
            double coef;
            if (any_mu && any_xi)
                coef = fma(mu, fma(in.An, one, in.cA[c]), fma(xi, in.Bn, mz));
            else if (any_mu)
                coef = fma(mu, fma(in.An, one, in.cA[c]), mz);
            else
                coef = fma(xi, in.Bn, mz);
#pragma unroll
            for (int q = 0; q < D; ++q) {
                racc[q] = fma(coef, dx[q], racc[q]);
                cacc[q] = fma(-coef, dx[q], cacc[q]);
            }
        }
#pragma unroll
        for (int v = 0; v < VC; ++v)
            cacc[v] = shfl_next(cacc[v], in.lane);
    }
}

// KIND 0: rates, 1: rates with the parameter-gradient sums, 2: gradient.
template <int KIND, int D>
__global__ void __launch_bounds__(kB) sym_fp64_kernel(Work w, Sched sc, double one, double mz)
{
    constexpr int VR = SymVals<KIND, D>::R;
    constexpr int VC = SymVals<KIND, D>::C;
    const double *tab = kExp2Tab;  // 16 KB, read through L1
    __shared__ double ct[kB];
    __shared__ double cx[D][kB];
    __shared__ double cA[KIND == 2 ? kB : 1];
    __shared__ int cte[kB];
    __shared__ double csum[VC][kB];
    __shared__ WorkItem s_it;

    if (threadIdx.x == 0)
        s_it = decode_item(w.sets, sc, blockIdx.x);
    __syncthreads();
    const WorkItem it = s_it;
    const SetDesc &S = w.sets[it.set];
    const int E = it.I, L = it.J;
    const bool diag = E == L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t R0 = S.row0;
    // the block's slot (from its round of the pair schedule; a scratch slot
    // in a later phase)
    const int64_t slot = it.kind >> 2;
    if (L >= S.nblk) {
        // a pair with the schedule's empty team: block E's rows get a zero
        // partial, stored in a slot of phase 0 (a scratch slot is zero
        // already)
        const int m = E * kB + tid;
        if (!(it.kind & 2) && m < S.n) {
            if (KIND == 2)
#pragma unroll
                for (int q = 0; q < D; ++q)
                    w.F2[S.fpart2_0 + (slot * D + q) * S.npad + m] = 0.0;
            else
#pragma unroll
                for (int v = 0; v < (KIND == 1 ? kPass1ThetaVals : 1); ++v)
                    w.F1[S.fpart0 + (slot * (KIND == 1 ? kPass1ThetaVals : 1) + v) * S.npad + m] = 0.0;
        }
        return;
    }

    // exponent constants (base 2) and prefactors
    const double ap = 0.5 * kLog2eSym / (S.tau_x * S.tau_x);
    const double bp = 0.5 * kLog2eSym / (S.tau_t * S.tau_t);
    const double cp = 0.5 * kLog2eSym / (S.h * S.h);
    const double wp = S.omega * kLog2eSym;
    const double two_pi = 6.283185307179586476925286766559;
    const double Cmu = S.mu0 / (pow(S.tau_x, (double)D) * S.tau_t * pow(two_pi, 0.5 * (D + 1)));
    const double Cxi = S.theta * S.omega / (pow(S.h, (double)D) * pow(two_pi, 0.5 * D));
    const double Amu = Cmu / (S.tau_x * S.tau_x);  // gradient: mu / tau_x^2 per unit 1/lambda
    const double Bxi = Cxi / (S.h * S.h);
    // r^2 beyond which 2^(-c' r^2) < 2^-1076 (a relative margin covers the
    // rounding of c' r^2), as an unsigned bit pattern
    const unsigned long long r2_xi = (unsigned long long)__double_as_longlong(1076.0 / cp * (1.0 + 0x1p-40));

    {
        const int m = E * kB + tid;
        const bool ok = m < S.n;
        ct[tid] = ok ? w.t64[R0 + m] : 0.0;
#pragma unroll
        for (int q = 0; q < D; ++q)
            cx[q][tid] = ok ? w.x64[(R0 + m) * kMaxD + q] : 0.0;
        cte[tid] = ok ? w.tie_end[R0 + m] : INT_MAX;
        if (KIND == 2)
            cA[tid] = ok ? w.w64[R0 + m] * Amu : 0.0;
    }
    const int n = L * kB + tid;
    const bool row_ok = n < S.n;
    const int n_eff = row_ok ? n : -1;  // -1 >= tie_end never holds
    double tn = 0.0, xn[D], An = 0.0, Bn = 0.0;
#pragma unroll
    for (int q = 0; q < D; ++q)
        xn[q] = 0.0;
    if (row_ok) {
        tn = w.t64[R0 + n];
#pragma unroll
        for (int q = 0; q < D; ++q)
            xn[q] = w.x64[(R0 + n) * kMaxD + q];
        if (KIND == 2) {
            const double wn = w.w64[R0 + n];
            An = wn * Amu;
            Bn = wn * Bxi;
        }
    }
    double racc[VR];
#pragma unroll
    for (int v = 0; v < VR; ++v)
        racc[v] = 0.0;
    __syncthreads();

    // pair terms are zero (they round to zero in FP64) once the time gap
    // alone puts the exponent below -1076
    const double kFar = 1076.0 * (1.0 + 0x1p-40);
    for (int round = 0; round < kW; ++round) {
        const int chunk = (warp + round) & (kW - 1);
        const int base = chunk * 32;
        double cacc[VC];
#pragma unroll
        for (int v = 0; v < VC; ++v)
            cacc[v] = 0.0;
        // on the diagonal block the chunks after the warp's own hold no pair
        // m < n; round 0 (chunk == warp) always runs and initialises csum
        const bool active = !diag || chunk <= warp;
        if (active) {
            // the smallest time gap of the warp's rows and the chunk's columns:
            // its first row against its last valid column
            const int c_last = min(base + 31, S.n - 1 - E * kB);
            bool mu_on = false, xi_on = false;
            if (L * kB + warp * 32 < S.n && c_last >= base) {
                const double gap = __shfl_sync(kFull, tn, 0) - ct[c_last];
                mu_on = !(gap > 0.0 && gap * gap * bp > kFar);
                xi_on = !(gap > 0.0 && gap * wp > kFar);
            }
            const ChunkIn<D> in{ct, cx, cA, cte, base, lane, n_eff, tn, An, Bn, ap, bp, cp, wp, r2_xi, one, mz, tab};
            if (mu_on && xi_on)
                chunk_pairs<KIND, D, true, true>(in, xn, racc, cacc);
            else if (mu_on)
                chunk_pairs<KIND, D, true, false>(in, xn, racc, cacc);
            else if (xi_on)
                chunk_pairs<KIND, D, false, true>(in, xn, racc, cacc);
        }
#pragma unroll
        for (int v = 0; v < VC; ++v) {
            if (round == 0)
                csum[v][base + lane] = cacc[v];
            else if (active)
                csum[v][base + lane] += cacc[v];
        }
        __syncthreads();
    }

    // slot writes: the rows of L and the columns of E, both in the block's
    // slot (the diagonal block adds both directions into it)
    const int m = E * kB + tid;
    if (KIND == 0) {
        double *f = w.F1 + S.fpart0 + slot * S.npad;  // one value per slot
        double rv = Cmu * racc[0] + Cxi * racc[1];
        if (diag)
            rv += Cmu * csum[0][tid];
        if (row_ok)
            f[n] = rv;
        if (!diag && m < S.n)
            f[m] = Cmu * csum[0][tid];
    } else if (KIND == 1) {
        double rv[6] = {Cmu * racc[0], Cxi * racc[1], Cmu * racc[2], Cmu * racc[3], Cxi * racc[4], Cxi * racc[5]};
        const double cv[6] = {Cmu * csum[0][tid], 0.0, Cmu * csum[1][tid], Cmu * csum[2][tid], 0.0, 0.0};
        if (diag)
#pragma unroll
            for (int v = 0; v < 6; ++v)
                rv[v] += cv[v];
        double *f = w.F1 + S.fpart0 + slot * kPass1ThetaVals * S.npad;
        if (row_ok)
#pragma unroll
            for (int v = 0; v < 6; ++v)
                f[(int64_t)v * S.npad + n] = rv[v];
        if (!diag && m < S.n)
#pragma unroll
            for (int v = 0; v < 6; ++v)
                f[(int64_t)v * S.npad + m] = cv[v];
    } else {
        if (diag)
#pragma unroll
            for (int q = 0; q < D; ++q)
                racc[q] += csum[q][tid];
        double *f = w.F2 + S.fpart2_0 + slot * D * S.npad;
        if (row_ok)
#pragma unroll
            for (int q = 0; q < D; ++q)
                f[(int64_t)q * S.npad + n] = racc[q];
        if (!diag && m < S.n)
#pragma unroll
            for (int q = 0; q < D; ++q)
                f[(int64_t)q * S.npad + m] = csum[q][tid];
    }
}

template <int KIND>
cudaError_t launch_kind(int d, const Work &w, const Sched &sc, cudaStream_t s)
{
    if (sc.nitems <= 0)
        return cudaSuccess;
    const dim3 grid((unsigned)sc.nitems);
    // passed at run time so that the compiler keeps the fused forms
    const double one = 1.0, mz = -0.0;
    switch (d) {
    case 1: sym_fp64_kernel<KIND, 1><<<grid, kB, 0, s>>>(w, sc, one, mz); break;
    case 2: sym_fp64_kernel<KIND, 2><<<grid, kB, 0, s>>>(w, sc, one, mz); break;
    case 3: sym_fp64_kernel<KIND, 3><<<grid, kB, 0, s>>>(w, sc, one, mz); break;
    case 4: sym_fp64_kernel<KIND, 4><<<grid, kB, 0, s>>>(w, sc, one, mz); break;
    case 5: sym_fp64_kernel<KIND, 5><<<grid, kB, 0, s>>>(w, sc, one, mz); break;
    case 6: sym_fp64_kernel<KIND, 6><<<grid, kB, 0, s>>>(w, sc, one, mz); break;
    case 7: sym_fp64_kernel<KIND, 7><<<grid, kB, 0, s>>>(w, sc, one, mz); break;
    case 8: sym_fp64_kernel<KIND, 8><<<grid, kB, 0, s>>>(w, sc, one, mz); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pass1_fp64_sym(int d, const Work &w, const Sched &sc, bool theta, cudaStream_t s)
{
    return theta ? launch_kind<1>(d, w, sc, s) : launch_kind<0>(d, w, sc, s);
}

cudaError_t launch_pass2_fp64_sym(int d, const Work &w, const Sched &sc, cudaStream_t s)
{
    return launch_kind<2>(d, w, sc, s);
}

}  // namespace hk
