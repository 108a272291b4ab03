// Incremental Metropolis-within-Gibbs over event locations (Section 3: the
// location variables are updated block-wise by Metropolis-Hastings).
//
// Moving a block B of events from x_b to x*_b changes only the pair terms
// that involve some b in B.  Given the current rates lambda_m (Eq. (1),
// cached in FP64), the new rates are
//   m not in B:  lambda*_m = lambda_m + sum_{b in B} [k(m <- b at x*_b) - k(m <- b at x_b)],
//   m in B:      lambda*_m = sum_{m' != m} k(m <- m'), every m' at its new place,
// where k(m <- m') = mu_{mm'} + xi_{mm'} is event m' 's contribution to the rate
// at event m (Section 2.1).  The integrated rate does not depend on X, so
//   Delta ell = sum_m [log lambda*_m - log lambda_m],
// an O(|B| N) computation instead of the O(N^2) of a full evaluation.
//
// One launch per proposal: its first CTAs take the unmoved events (block
// membership, the |B| column updates, log1p(Delta_m / lambda_m) summed per
// CTA), the others the moved events (each moved event's new rate over all
// events, split over several CTAs), and the CTA that finishes last adds
// everything in a fixed order and, in step mode, takes the accept decision
// log u < Delta ell + log q-ratio and, on accept, the commit.  The rates live
// in two buffers; the device-side index of the current one flips on accept,
// so no call reads anything back to the host and a sequence of steps can be
// captured in a CUDA graph.  Rates, logs and decisions are FP64; the pair
// terms are FP64 or, in the mixed precision, FP32 (see State32 below).
#include <cuda_runtime.h>

#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "hawkes.h"
#include "hk_exp2.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDim = 8;
constexpr int kMaxBlock = 256;  // events moved together at most
constexpr int kRateTile = 128;
constexpr int kRateSplit = 16;

// status bits of the state
constexpr int kBadData = 1;      // non-finite input location or time, negative time
constexpr int kBadBlock = 2;     // index out of range or repeated in a block
constexpr int kBadProposal = 4;  // non-finite proposed location

struct Consts {
    double a, b, c;  // 1/(2 tau_x^2), 1/(2 tau_t^2), 1/(2 h^2)
    double a2, b2, c2, w2;  // a, b, c and omega times log2(e): the base-2 exponents
    double Cmu, Cxi, omega, mu0, tau_t, theta;
};

// For t >= 0 the bit pattern with the sign cleared (so -0 equals +0) orders
// like the value: the time indicators compare these keys.
__device__ __forceinline__ long long tkey(double v) { return __double_as_longlong(v) & 0x7fffffffffffffffLL; }

// Contribution of event (xs, ts) to the rate at event (xm, tm): the
// background term (both Gaussians, I[t != t_m]) and the self-excitation term
// (I[t < t_m]) of Section 2.1, in FP64 with base-2 exponents and the
// table-driven exp2.  An exponential whose exponent is below -1076 rounds to
// zero and is not evaluated (a warp skips it when none of its lanes needs it).
__device__ __forceinline__ double contrib(const double *xm, double tm, const double *xs, double ts, int d,
                                          const Consts &k)
{
    double r2 = 0.0;
    for (int q = 0; q < d; ++q) {
        const double df = xm[q] - xs[q];
        r2 = fma(df, df, r2);
    }
    const double dt = tm - ts;
    const long long km = tkey(tm), ks = tkey(ts);
    double v = 0.0;
    if (km != ks) {
        const double y = -fma(dt * k.b2, dt, r2 * k.a2);
        if ((unsigned)__double2hiint(y) <= hk::kHiNeg1076)
            v = k.Cmu * hk::exp2_neg_lane(y, hk::kExp2Tab);
    }
    if (ks < km) {
        const double y = -fma(k.w2, dt, r2 * k.c2);
        if ((unsigned)__double2hiint(y) <= hk::kHiNeg1076)
            v = fma(k.Cxi, hk::exp2_neg_lane(y, hk::kExp2Tab), v);
    }
    return v;
}

// ---------------------------------------------------- mixed precision --
//
// The pair terms in FP32: coordinates and times held as FP32 (hi, lo) pairs
// (hi the nearest float, lo the nearest float to the rest), differences
// taken as (hi - hi) + (lo - lo) (relative error a few 2^-24: when the hi
// parts cancel they are within an ulp and subtract exactly), exponentials
// on the MUFU (ex2.approx) with the prefactor as an FP32 factor, and
// compensated FP32 sums.  The tie indicators compare the FP64 times exactly,
// through their bit patterns.  Logs, rates and the decision stay FP64.
struct State32 {
    float *xh, *xl;         // n x d
    float *th, *tl;         // n
    float Cmu, Cxi;         // prefactors of the two kernels
    float a2, b2, c2, w2;   // a, b, c, omega times log2(e)
    double tau;             // rates below tau take the FP64 path (FP32 terms underflow)
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void split32(double v, float &h, float &l)
{
    h = __double2float_rn(v);
    l = __double2float_rn(v - (double)h);
}

struct Sum32 {  // compensated (Kahan) FP32 sum
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float u = s + y;
        c = (u - s) - y;
        s = u;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// contrib() in FP32: event s's contribution to the rate at event m.
template <int D>
__device__ __forceinline__ float contrib32(const float *xmh, const float *xml, float tmh, float tml, long long km,
                                           const float *xsh, const float *xsl, float tsh, float tsl, long long ks,
                                           const State32 &c)
{
    float r2 = 0.f;
#pragma unroll
    for (int q = 0; q < D; ++q) {
        const float dx = (xmh[q] - xsh[q]) + (xml[q] - xsl[q]);
        r2 = fmaf(dx, dx, r2);
    }
    const float dt = (tmh - tsh) + (tml - tsl);
    float v = 0.f;
    if (ks != km)
        v = c.Cmu * ex2_approx(-fmaf(r2, c.a2, dt * dt * c.b2));
    if (ks < km)
        v = fmaf(c.Cxi, ex2_approx(-fmaf(c.w2, dt, r2 * c.c2)), v);
    return v;
}

// FP32 copies of X and t; flag[0] is set when some |value| >= 2^100, where
// the FP32 differences could overflow (the state then stays on FP64).
__global__ void split_kernel(const double *__restrict__ X, const double *__restrict__ t, int64_t n, int d, float *xh,
                             float *xl, float *th, float *tl, int *flag)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * d; i += stride) {
        const double v = X[i];
        bad |= !(fabs(v) < 0x1p100);
        split32(v, xh[i], xl[i]);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = t[i];
        bad |= !(fabs(v) < 0x1p100);
        split32(v, th[i], tl[i]);
    }
    if (bad)
        atomicOr(flag, 1);
}

// Sum over a CTA of NT threads (a multiple of 32), valid in thread 0: a
// shuffle tree per warp, then one over the warp sums; the order is fixed, so
// the result is reproducible.  sh holds NT / 32 doubles.
template <int NT>
__device__ double cta_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    if constexpr (NT > 32) {
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0)
            sh[w] = v;
        __syncthreads();
        v = 0.0;
        if (w == 0) {
            v = l < NT / 32 ? sh[l] : 0.0;
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_down_sync(0xffffffffu, v, o);
        }
        __syncthreads();
    }
    return v;
}

// Whether this CTA is the last of `count` CTAs to get here: every CTA
// publishes its writes, then takes a ticket; the last one resets the counter
// for the next launch and may then read what all the others wrote.
__device__ bool last_cta_of(unsigned *ticket, unsigned count, int *flag)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned k = atomicAdd(ticket, 1u);
        *flag = k == count - 1;
        if (*flag)
            *ticket = 0u;
    }
    __syncthreads();
    const bool last = *flag;
    __syncthreads();  // flag is reused by the next call
    if (last)
        __threadfence();
    return last;
}

// log(lam_new / lam) with the extended-real convention for zero rates.
__device__ __forceinline__ double log_ratio(double lam, double lam_new, double delta)
{
    if (lam > 0.0)
        return log1p(delta / lam);
    return lam_new > 0.0 ? INFINITY : 0.0;
}

// ------------------------------------------------------------ full rates --

// Partial rate sums over one column split (ordered pairs), as in the FP64
// rate pass.
__global__ void __launch_bounds__(kRateTile) rates_kernel(const double *__restrict__ t, const double *__restrict__ X,
                                                          int64_t n, int d, Consts k, int fsplit,
                                                          double *__restrict__ part, int *status)
{
    __shared__ double st[kRateTile];
    __shared__ double sx[kRateTile * kMaxDim];
    const int64_t row = (int64_t)blockIdx.x * kRateTile + threadIdx.x;
    const int sp = blockIdx.y;
    const bool valid = row < n;
    double tn = 0.0, xn[kMaxDim];
    for (int q = 0; q < kMaxDim; ++q)
        xn[q] = 0.0;
    if (valid) {
        tn = t[row];
        bool bad = !(tn >= 0.0) || !isfinite(tn);
        for (int q = 0; q < d; ++q) {
            xn[q] = X[row * d + q];
            bad |= !isfinite(xn[q]);
        }
        if (bad && sp == 0)
            atomicOr(status, kBadData);
    }
    const int64_t tiles = (n + kRateTile - 1) / kRateTile;
    const int64_t per = (tiles + fsplit - 1) / fsplit;
    const int64_t lo = min(sp * per * kRateTile, n), hi = min((sp + 1) * per * kRateTile, n);
    double s = 0.0, c = 0.0;
    for (int64_t c0 = lo; c0 < hi; c0 += kRateTile) {
        const int cnt = (int)min((int64_t)kRateTile, hi - c0);
        __syncthreads();
        if (threadIdx.x < cnt) {
            st[threadIdx.x] = t[c0 + threadIdx.x];
            for (int q = 0; q < d; ++q)
                sx[threadIdx.x * kMaxDim + q] = X[(c0 + threadIdx.x) * d + q];
        }
        __syncthreads();
        if (!valid)
            continue;
        double acc = 0.0;
        for (int j = 0; j < cnt; ++j)
            acc += contrib(xn, tn, sx + j * kMaxDim, st[j], d, k);
        const double y = acc - c;  // compensated across tiles
        const double tt = s + y;
        c = (tt - s) - y;
        s = tt;
    }
    if (valid)
        part[(int64_t)sp * n + row] = s;
}

// T = max t_n (the end of the observation window), once per state.
__global__ void __launch_bounds__(kThreads) tmax_kernel(const double *__restrict__ t, int64_t n, double *T)
{
    __shared__ double sh[kThreads];
    double m = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += kThreads)
        m = fmax(m, t[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *T = sh[0];
}

// lambda_m from the splits (fixed order) into the current buffer and
// log lambda_m - Lambda_m summed per CTA; the last CTA adds the CTA sums in
// order into ell.  Small CTAs spread the FP64 logs and normal CDFs over every
// SM.
constexpr int kFinThreads = 64;

__global__ void __launch_bounds__(kFinThreads) rates_finish_kernel(const double *__restrict__ t, int64_t n,
                                                                   Consts k, int fsplit,
                                                                   const double *__restrict__ part,
                                                                   const double *__restrict__ Tmax, double *lam0,
                                                                   double *lam1, int *ctl, double *cpart,
                                                                   double *loglik)
{
    __shared__ double sh[kFinThreads / 32];
    __shared__ int flag;
    double *lam = ctl[0] ? lam1 : lam0;
    const double T = *Tmax;
    double acc = 0.0;
    const int64_t i = (int64_t)blockIdx.x * kFinThreads + threadIdx.x;
    if (i < n) {
        double l = 0.0;
        for (int sp = 0; sp < fsplit; ++sp)
            l += part[(int64_t)sp * n + i];
        lam[i] = l;
        const double a = T - t[i];
        const double Lam = k.mu0 * (normcdf(a / k.tau_t) - normcdf(-t[i] / k.tau_t)) - k.theta * expm1(-k.omega * a);
        acc = log(l) - Lam;
    }
    acc = cta_sum<kFinThreads>(acc, sh);
    if (threadIdx.x == 0)
        cpart[blockIdx.x] = acc;
    if (!last_cta_of(reinterpret_cast<unsigned *>(ctl + 2), gridDim.x, &flag))
        return;
    double v = 0.0;
    for (int c = threadIdx.x; c < (int)gridDim.x; c += kFinThreads)
        v += __ldcg(cpart + c);
    v = cta_sum<kFinThreads>(v, sh);
    if (threadIdx.x == 0)
        *loglik = v;
}

// ------------------------------------------------------------- proposal --

struct Block {
    int nb;
    const int64_t *idx;   // caller's device indices
    const double *xnew;   // caller's device proposals, nb x d
};

// The launch of one proposal.  CTAs [0, ncol) take 64 / lanes consecutive
// events each, `lanes` threads per event splitting its loop over the block
// (the column part); CTA ncol + b * splits + sp takes moved event b against
// events [sp * per, (sp + 1) * per) (the row part).
constexpr int kEvalThreads = 64;
constexpr int kRangeMax = 8192;  // events per row CTA at most (membership bitmap in shared memory)

struct Launch {
    int ncol, splits, lanes;
    int64_t per;
};

// For m in [lo, lo + cnt): set the bit of every moved event in the range; a
// bit found already set means a repeated index when `dup` is given.
__device__ void mark_block(const Block &B, int64_t n, int64_t lo, int64_t cnt, unsigned *bits, int *dup)
{
    for (int w = threadIdx.x; w < (int)((cnt + 31) / 32); w += kEvalThreads)
        bits[w] = 0u;
    __syncthreads();
    for (int b = threadIdx.x; b < B.nb; b += kEvalThreads) {
        const int64_t m = B.idx[b];
        if (m >= lo && m < lo + cnt && m < n) {
            const unsigned bit = 1u << ((m - lo) & 31);
            const unsigned old = atomicOr(bits + ((m - lo) >> 5), bit);
            if (dup && (old & bit))
                atomicOr(dup, kBadBlock);
        }
    }
    __syncthreads();
}

// Everything one proposal's launch needs.
struct EvalArgs {
    const double *t;
    double *X;
    int64_t n;
    Consts k;
    State32 m32;
    Block B;
    Launch L;
    double *lam0, *lam1;
    int *ctl;  // [0] current rate buffer, [1] status, [2] ticket, [3] FP32 range flag
    double *cpart, *rowpart, *bterm;
    unsigned *bticket;
    double *out_delta;
    bool step;
    const double *log_q_ratio, *log_u;
    int *accepted_out;
    double *loglik;
};

// Delta_m of an unmoved event m in FP64 over the whole block, reading the
// block from global memory (the FP64 path of the mixed precision).
template <int D>
__device__ double delta64(const double *xm, double tm, const EvalArgs &a)
{
    double dl = 0.0;
    for (int b = 0; b < a.B.nb; ++b) {
        const int64_t mb = a.B.idx[b];
        if (mb < 0 || mb >= a.n)
            continue;
        const double tb = a.t[mb];
        dl += contrib(xm, tm, a.B.xnew + (int64_t)b * D, tb, D, a.k) - contrib(xm, tm, a.X + mb * D, tb, D, a.k);
    }
    return dl;
}

// Position of event m in the block, or -1.
__device__ __forceinline__ int block_pos(const Block &B, int64_t m)
{
    for (int p = 0; p < B.nb; ++p)
        if (B.idx[p] == m)
            return p;
    return -1;
}

template <int D, bool MIXED>
__global__ void __launch_bounds__(kEvalThreads) eval_kernel(const EvalArgs a)
{
    constexpr int d = D;
    extern __shared__ __align__(16) unsigned char blk_raw[];  // the block, staged by the column part
    __shared__ unsigned bits[kRangeMax / 32];
    __shared__ double sh[kEvalThreads / 32];
    __shared__ double sl;
    __shared__ int flag, acc;
    const Block &B = a.B;
    const int64_t n = a.n;
    int *ctl = a.ctl, *status = ctl + 1;
    const int act = ctl[0];
    const bool use32 = MIXED && ctl[3] == 0;
    const double *lam = act ? a.lam1 : a.lam0;
    double *lam_new = act ? a.lam0 : a.lam1;
    const State32 &c32 = a.m32;
    if ((int)blockIdx.x < a.L.ncol) {
        // column part: every unmoved m of this CTA's range gets the change of
        // its rate, sum over b of k(m <- x*_b) - k(m <- x_b)
        const int ev = kEvalThreads / a.L.lanes;
        const int64_t lo = (int64_t)blockIdx.x * ev;
        double *sxo = reinterpret_cast<double *>(blk_raw), *sxn = sxo + B.nb * d, *stb = sxn + B.nb * d;
        float *soh = reinterpret_cast<float *>(blk_raw), *sol = soh + B.nb * d, *snh = sol + B.nb * d,
              *snl = snh + B.nb * d, *sth = snl + B.nb * d, *stl = sth + B.nb;
        long long *skey = reinterpret_cast<long long *>(stl + B.nb);  // 8-byte aligned: 4 nb (4 d + 2) bytes in
        for (int b = threadIdx.x; b < B.nb; b += kEvalThreads) {
            const int64_t m = B.idx[b];
            const bool ok = m >= 0 && m < n;
            bool bad = false;
            if (use32) {
                sth[b] = ok ? c32.th[m] : 0.f;
                stl[b] = ok ? c32.tl[m] : 0.f;
                skey[b] = ok ? tkey(a.t[m]) : 0;
                for (int q = 0; q < d; ++q) {
                    soh[b * d + q] = ok ? c32.xh[m * d + q] : 0.f;
                    sol[b * d + q] = ok ? c32.xl[m * d + q] : 0.f;
                    const double v = B.xnew[(int64_t)b * d + q];
                    bad |= !(fabs(v) < 0x1p100);
                    split32(v, snh[b * d + q], snl[b * d + q]);
                }
            } else {
                stb[b] = ok ? a.t[m] : 0.0;
                for (int q = 0; q < d; ++q) {
                    sxo[b * d + q] = ok ? a.X[m * d + q] : 0.0;
                    const double v = B.xnew[(int64_t)b * d + q];
                    bad |= !isfinite(v);
                    sxn[b * d + q] = v;
                }
            }
            if (blockIdx.x == 0) {
                if (!ok)
                    atomicOr(status, kBadBlock);
                if (bad)
                    atomicOr(status, kBadProposal);
            }
        }
        mark_block(B, n, lo, ev, bits, status);
        const int e = threadIdx.x / a.L.lanes, j = threadIdx.x % a.L.lanes;
        const int64_t m = lo + e;
        const bool mine = m < n && !((bits[e >> 5] >> (e & 31)) & 1u);
        double delta = 0.0;
        if (mine) {
            if (use32) {
                float xmh[D], xml[D];
                for (int q = 0; q < d; ++q) {
                    xmh[q] = c32.xh[m * d + q];
                    xml[q] = c32.xl[m * d + q];
                }
                const float tmh = c32.th[m], tml = c32.tl[m];
                const long long km = tkey(a.t[m]);
                Sum32 s;
                for (int b = j; b < B.nb; b += a.L.lanes)
                    s.add(contrib32<D>(xmh, xml, tmh, tml, km, snh + b * d, snl + b * d, sth[b], stl[b], skey[b], c32) -
                          contrib32<D>(xmh, xml, tmh, tml, km, soh + b * d, sol + b * d, sth[b], stl[b], skey[b], c32));
                delta = s.value();
            } else {
                double xm[D];
                for (int q = 0; q < d; ++q)
                    xm[q] = a.X[m * d + q];
                const double tm = a.t[m];
                for (int b = j; b < B.nb; b += a.L.lanes)
                    delta += contrib(xm, tm, sxn + b * d, stb[b], d, a.k) - contrib(xm, tm, sxo + b * d, stb[b], d, a.k);
            }
        }
        for (int o = a.L.lanes / 2; o > 0; o >>= 1)  // the event's lanes, in a fixed order
            delta += __shfl_down_sync(0xffffffffu, delta, o, a.L.lanes);
        double term = 0.0;
        if (mine && j == 0) {
            const double l = lam[m];
            // FP64 again where FP32 terms may underflow or where the move takes
            // away nearly all of the rate (the FP32 error would be magnified)
            if (use32 && (!(l >= c32.tau) || l + delta < l * 0x1p-10)) {
                double xm[D];
                for (int q = 0; q < d; ++q)
                    xm[q] = a.X[m * d + q];
                delta = delta64<D>(xm, a.t[m], a);
            }
            const double ln = l + delta;
            lam_new[m] = ln;
            term = log_ratio(l, ln, delta);
        }
        term = cta_sum<kEvalThreads>(term, sh);
        if (threadIdx.x == 0)
            a.cpart[blockIdx.x] = term;
    } else {
        // row part: moved event b's new rate over one range of events, the
        // moved ones at their proposed places
        const int r = (int)blockIdx.x - a.L.ncol;
        const int b = r / a.L.splits;
        const int64_t lo = min((int64_t)(r % a.L.splits) * a.L.per, n), cnt = min(a.L.per, n - lo);
        mark_block(B, n, lo, cnt, bits, nullptr);
        const int64_t mb = B.idx[b];
        const bool okb = mb >= 0 && mb < n;  // a bad index is reported by the column part
        double s = 0.0;
        if (okb && use32) {
            float xbh[D], xbl[D];
            for (int q = 0; q < d; ++q)
                split32(B.xnew[(int64_t)b * d + q], xbh[q], xbl[q]);
            const float tbh = c32.th[mb], tbl = c32.tl[mb];
            const long long kb = tkey(a.t[mb]);
            Sum32 acc32;
            for (int64_t jj = threadIdx.x; jj < cnt; jj += kEvalThreads) {
                const int64_t m = lo + jj;
                if (m == mb)
                    continue;
                float xh[D], xl[D];
                if ((bits[jj >> 5] >> (jj & 31)) & 1u) {
                    const int p = block_pos(B, m);
                    for (int q = 0; q < d; ++q)
                        split32(B.xnew[(int64_t)p * d + q], xh[q], xl[q]);
                } else {
                    for (int q = 0; q < d; ++q) {
                        xh[q] = c32.xh[m * d + q];
                        xl[q] = c32.xl[m * d + q];
                    }
                }
                acc32.add(contrib32<D>(xbh, xbl, tbh, tbl, kb, xh, xl, c32.th[m], c32.tl[m], tkey(a.t[m]), c32));
            }
            s = acc32.value();
        } else if (okb) {
            double xb[D];
            for (int q = 0; q < d; ++q)
                xb[q] = B.xnew[(int64_t)b * d + q];
            const double tb = a.t[mb];
            for (int64_t jj = threadIdx.x; jj < cnt; jj += kEvalThreads) {
                const int64_t m = lo + jj;
                if (m == mb)
                    continue;
                const double *xm = a.X + m * d;
                if ((bits[jj >> 5] >> (jj & 31)) & 1u)
                    xm = B.xnew + (int64_t)block_pos(B, m) * d;
                s += contrib(xb, tb, xm, a.t[m], d, a.k);
            }
        }
        s = cta_sum<kEvalThreads>(s, sh);
        if (threadIdx.x == 0)
            a.rowpart[r] = s;
        // the last of event b's CTAs adds its splits in order (lane-strided,
        // then a shuffle tree) and takes the log ratio of its rate
        if (last_cta_of(a.bticket + b, a.L.splits, &flag)) {
            if (threadIdx.x < 32) {
                double lnew = 0.0;
                for (int q = threadIdx.x; q < a.L.splits; q += 32)
                    lnew += __ldcg(a.rowpart + (int64_t)b * a.L.splits + q);
                for (int o = 16; o > 0; o >>= 1)
                    lnew += __shfl_down_sync(0xffffffffu, lnew, o);
                if (threadIdx.x == 0)
                    sl = lnew;
            }
            __syncthreads();
            if (use32 && okb && !(sl >= c32.tau)) {
                // FP32 terms may have underflowed: the whole rate again in FP64
                double xb[D];
                for (int q = 0; q < d; ++q)
                    xb[q] = B.xnew[(int64_t)b * d + q];
                const double tb = a.t[mb];
                double v = 0.0;
                for (int64_t m = threadIdx.x; m < n; m += kEvalThreads) {
                    if (m == mb)
                        continue;
                    const int p = block_pos(B, m);
                    v += contrib(xb, tb, p >= 0 ? B.xnew + (int64_t)p * d : a.X + m * d, a.t[m], d, a.k);
                }
                v = cta_sum<kEvalThreads>(v, sh);
                if (threadIdx.x == 0)
                    sl = v;
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                const double lnew = sl;
                double v = 0.0;
                if (okb) {
                    const double l = lam[mb];
                    lam_new[mb] = lnew;
                    v = (l > 0.0 && lnew > 0.0) ? log(lnew) - log(l) : log_ratio(l, lnew, lnew - l);
                }
                a.bterm[b] = v;
            }
        }
    }
    if (!last_cta_of(reinterpret_cast<unsigned *>(ctl + 2), gridDim.x, &flag))
        return;

    // Delta ell in a fixed order: the moved events' log ratios, then the
    // column partials; in step mode the decision and, on accept, the commit.
    double v = 0.0;
    for (int b = threadIdx.x; b < B.nb; b += kEvalThreads)
        v += __ldcg(a.bterm + b);
    for (int cc = threadIdx.x; cc < a.L.ncol; cc += kEvalThreads)
        v += __ldcg(a.cpart + cc);
    const double delta = cta_sum<kEvalThreads>(v, sh);
    if (threadIdx.x == 0) {
        const bool bad = *(volatile const int *)status != 0;
        const double dl = bad ? nan("") : delta;
        if (a.out_delta)
            *a.out_delta = dl;
        int ac = 0;
        if (a.step && !bad) {
            const double lhs = *a.log_u, rhs = dl + (a.log_q_ratio ? *a.log_q_ratio : 0.0);
            ac = (lhs < rhs) ? 1 : 0;  // NaN on either side rejects
        }
        acc = ac;
        if (a.accepted_out)
            *a.accepted_out = ac;
        if (ac) {
            *a.loglik += dl;
            ctl[0] = act ^ 1;
        }
    }
    __syncthreads();
    if (acc)
        for (int e = threadIdx.x; e < B.nb * d; e += kEvalThreads) {
            const int64_t i = B.idx[e / d] * d + e % d;
            const double x = B.xnew[e];
            a.X[i] = x;
            if (MIXED)
                split32(x, c32.xh[i], c32.xl[i]);
        }
}

__global__ void copy_rates_kernel(const double *lam0, const double *lam1, const int *active, int64_t n, double *out)
{
    const double *lam = *active ? lam1 : lam0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = lam[i];
}

// ------------------------------------------------------------ proposals --

// x - sin(x) on [0, 2 pi]; Taylor series below 0.5, where the difference
// would cancel.
__device__ double x_minus_sin(double x)
{
    if (x >= 0.5)
        return x - sin(x);
    const double x2 = x * x;
    double term = x * x2 / 6.0, sum = 0.0;
    for (int k = 1; k <= 7; ++k) {
        sum += term;
        term *= -x2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
    }
    return sum;
}

// log P(at least one of `tries` uniform draws from a disc of radius rho
// lands in a region of area A inside it)
__device__ double log_success(double A, double rho, int tries)
{
    const double p = A / (CUDART_PI * rho * rho);
    return p >= 1.0 ? 0.0 : log(-expm1((double)tries * log1p(-p)));
}

// The area of the intersection of discs of radii R and rho, centres c apart,
// is the sum of the two circular segments cut off by the common chord, each
// r^2 (2 theta - sin 2 theta) / 2 with theta = atan2(half-chord, signed
// distance of the chord from the centre).  lens_part returns one of them
// (which = 0: the prior circle's, 1: the disc's), so that two lanes evaluate
// a lens together; in the cases without a chord (no overlap, one disc inside
// the other) lane 0 carries the whole area.
__device__ double lens_part(double R, double rho, double c, int which)
{
    if (c >= R + rho)
        return 0.0;
    if (c <= fabs(R - rho)) {
        const double m = fmin(R, rho);
        return which == 0 ? CUDART_PI * m * m : 0.0;
    }
    const double d1 = (c * c + R * R - rho * rho) / (2.0 * c);
    const double d2 = c - d1;
    const double h = sqrt(fmax((R - d1) * (R + d1), 0.0));
    return which == 0 ? 0.5 * R * R * x_minus_sin(2.0 * atan2(h, d1))
                      : 0.5 * rho * rho * x_minus_sin(2.0 * atan2(h, d2));
}

// Lens proposals of Eq. (6) for a D = 2 block, four lanes per moved event:
// the two segments of each lens area on alternate lanes, the rejection tries
// four at a time (the first try inside the circle wins, as in a serial loop),
// and the four logs of the ratio side by side.  FP64 is a long-latency path
// on this GPU and these chains are most of a small block's step.  The
// block's log q-ratio is summed in a fixed order.
template <int NT>
__global__ void __launch_bounds__(NT) propose_circle_kernel(const double *__restrict__ X, int64_t n, Block B,
                                                            const double *__restrict__ centers,
                                                            const double *__restrict__ radii, double eps, int tries,
                                                            const double *__restrict__ u, double *X_new,
                                                            double *log_q_ratio, int *status)
{
    constexpr int G = 4;  // lanes per event
    __shared__ double sh[NT / 32];
    const int g = threadIdx.x & (G - 1), lane = threadIdx.x & 31;
    const unsigned gmask = 0xfu << (lane & ~(G - 1));
    double lq = 0.0;
    const int total = B.nb * G;
    for (int base = 0; base < total; base += NT) {  // uniform trip counts: every lane takes part in the shuffles
        const int e = (base + (int)threadIdx.x) / G;
        bool ok = false;
        double x0 = 0.0, x1 = 0.0, c0 = 0.0, c1 = 0.0, R = 0.0, rho = 0.0;
        if (e < B.nb) {
            const int64_t m = B.idx[e];
            if (m < 0 || m >= n) {
                if (g == 0)
                    atomicOr(status, kBadBlock);
            } else {
                x0 = X[m * 2];
                x1 = X[m * 2 + 1];
                c0 = centers[m * 2];
                c1 = centers[m * 2 + 1];
                R = radii[m];
                rho = R * eps;
                ok = true;
            }
        }
        double part = ok ? lens_part(R, rho, hypot(x0 - c0, x1 - c1), g & 1) : 0.0;
        const double A_x = part + __shfl_xor_sync(0xffffffffu, part, 1);
        if (ok && (!(R > 0.0) || !isfinite(R) || !(A_x > 0.0))) {
            if (g == 0)
                atomicOr(status, kBadProposal);
            ok = false;
        }
        double y0 = x0, y1 = x1;
        bool moved = false;
        for (int k0 = 0; k0 < tries; k0 += G) {
            const int k = k0 + g;
            bool inside = false;
            double z0 = 0.0, z1 = 0.0;
            if (ok && !moved && k < tries) {
                const double r = rho * sqrt(u[((int64_t)e * tries + k) * 2]);
                double sn, cs;
                sincospi(2.0 * u[((int64_t)e * tries + k) * 2 + 1], &sn, &cs);
                z0 = x0 + r * cs;
                z1 = x1 + r * sn;
                const double dx = z0 - c0, dy = z1 - c1;
                inside = dx * dx + dy * dy < R * R;
            }
            const unsigned hit = __ballot_sync(0xffffffffu, inside) & gmask;
            const int src = hit ? __ffs(hit) - 1 : lane;
            const double w0 = __shfl_sync(0xffffffffu, z0, src), w1 = __shfl_sync(0xffffffffu, z1, src);
            if (hit && !moved) {
                y0 = w0;
                y1 = w1;
                moved = true;
            }
        }
        part = moved ? lens_part(R, rho, hypot(y0 - c0, y1 - c1), g & 1) : 0.0;
        const double A_y = part + __shfl_xor_sync(0xffffffffu, part, 1);
        // lanes 0..3: log P(x*), log A(x*), log P(x), log A(x)
        double L = 0.0;
        if (moved)
            L = g == 0 ? log_success(A_y, rho, tries) : g == 1 ? log(A_y) : g == 2 ? log_success(A_x, rho, tries)
                                                                                  : log(A_x);
        const double L1 = __shfl_down_sync(0xffffffffu, L, 1), L2 = __shfl_down_sync(0xffffffffu, L, 2),
                     L3 = __shfl_down_sync(0xffffffffu, L, 3);
        if (ok && g == 0) {
            if (moved)
                lq += (L - L1) - (L2 - L3);
            X_new[(int64_t)e * 2] = y0;
            X_new[(int64_t)e * 2 + 1] = y1;
        }
    }
    lq = cta_sum<NT>(lq, sh);
    if (threadIdx.x == 0)
        *log_q_ratio = lq;
}

// Truncated-normal proposals inside the boxes of Eq. (2):
// x* = x + s Phi^{-1}(Phi(a) + u (Phi(b) - Phi(a))), and the log q-ratio
// sum log Z(x) - log Z(x*), Z(y) = Phi((hi - y)/s) - Phi((lo - y)/s).  Two
// adjacent lanes per coordinate, the even one for the lower wall and the odd
// one for the upper, so that the two normal CDFs of each stage and the two
// logs run side by side; FP64 on this GPU is a long-latency path, and this
// chain is most of a small block's step.
template <int NT>
__global__ void __launch_bounds__(NT) propose_box_kernel(const double *__restrict__ X, int64_t n, int d, Block B,
                                                         const double *__restrict__ lo, const double *__restrict__ hi,
                                                         double sd, double inv_sd, const double *__restrict__ u,
                                                         double *X_new, double *log_q_ratio, int *status)
{
    __shared__ double sh[NT / 32];
    double lq = 0.0;
    const int total = 2 * B.nb * d;
    for (int base = 0; base < total; base += NT) {  // uniform trip count: every lane takes part in the shuffles
        const int e2 = base + threadIdx.x;
        const bool active = e2 < total;
        const int e = e2 >> 1, upper = e2 & 1;
        bool ok = false;
        double x = 0.0, l = 0.0, h = 0.0;
        if (active) {
            const int b = e / d, q = e % d;
            const int64_t m = B.idx[b];
            if (m < 0 || m >= n) {
                if (!upper)
                    atomicOr(status, kBadBlock);
            } else {
                x = X[m * d + q];
                l = lo[m * d + q];
                h = hi[m * d + q];
                ok = l <= x && x <= h && sd > 0.0;
                if (!ok && !upper)
                    atomicOr(status, kBadProposal);
            }
        }
        const double wall = upper ? h : l;
        const double P = ok ? normcdf((wall - x) * inv_sd) : 0.0;
        const double Q = __shfl_xor_sync(0xffffffffu, P, 1);
        const double Pa = upper ? Q : P, Pb = upper ? P : Q;
        double y = x, L1 = 0.0;
        if (ok) {
            if (!upper)
                y = fmin(fmax(x + sd * normcdfinv(Pa + u[e] * (Pb - Pa)), l), h);
            else
                L1 = log(Pb - Pa);
        }
        y = __shfl_sync(0xffffffffu, y, threadIdx.x & ~1);
        const double Z = ok ? normcdf((wall - y) * inv_sd) : 0.0;
        const double Zo = __shfl_xor_sync(0xffffffffu, Z, 1);
        if (ok) {
            if (!upper)
                X_new[e] = y;
            else
                lq += L1 - log(Z - Zo);
        }
    }
    lq = cta_sum<NT>(lq, sh);
    if (threadIdx.x == 0)
        *log_q_ratio = lq;
}

bool params_ok(const hawkes_params *p)
{
    if (!p)
        return false;
    const double v[6] = {p->mu0, p->tau_x, p->tau_t, p->theta, p->omega, p->h};
    for (double x : v)
        if (!(x > 0.0) || !std::isfinite(x))
            return false;
    return true;
}

Consts make_consts(const hawkes_params &p, int d)
{
    const double two_pi = 6.283185307179586476925286766559;
    Consts k;
    k.a = 0.5 / (p.tau_x * p.tau_x);
    k.b = 0.5 / (p.tau_t * p.tau_t);
    k.c = 0.5 / (p.h * p.h);
    const double log2e = 1.4426950408889634074;
    k.a2 = k.a * log2e;
    k.b2 = k.b * log2e;
    k.c2 = k.c * log2e;
    k.w2 = p.omega * log2e;
    k.Cmu = p.mu0 / (std::pow(p.tau_x, d) * p.tau_t * std::pow(two_pi, 0.5 * (d + 1)));
    k.Cxi = p.theta * p.omega / (std::pow(p.h, d) * std::pow(two_pi, 0.5 * d));
    k.omega = p.omega;
    k.mu0 = p.mu0;
    k.tau_t = p.tau_t;
    k.theta = p.theta;
    return k;
}

int grid_for(int64_t n) { return (int)((n + kThreads - 1) / kThreads); }

}  // namespace

struct hawkes_mwg {
    int device = 0;
    int sms = 0;
    int64_t n = 0;
    int32_t d = 0;
    int32_t max_block = 0;
    Consts k{};
    std::string err;
    // device buffers
    double *t = nullptr, *X = nullptr, *lam0 = nullptr, *lam1 = nullptr;
    double *part = nullptr;     // rate splits: kRateSplit x n
    double *cpart = nullptr;    // per-CTA sums: ceil(n / 8)
    double *rowterm = nullptr;  // row partials: max_block x most splits
    double *loglik = nullptr;   // running ell
    double *Tmax = nullptr;     // max t
    double *bterm = nullptr;    // per moved event: log of its rate ratio (max_block)
    unsigned *bticket = nullptr;  // per moved event: last-CTA ticket of its row CTAs (max_block)
    int *ctl = nullptr;         // [0] current rate buffer, [1] status, [2] last-CTA ticket, [3] FP32 range flag
    hawkes_precision prec = HAWKES_PREC_FP64;
    State32 m32{};              // FP32 copies of X and t (mixed precision)
};

namespace {

hawkes_status fail(hawkes_mwg *s, hawkes_status st, const std::string &msg)
{
    if (s)
        s->err = msg;
    return st;
}

hawkes_status cuda_fail(hawkes_mwg *s, cudaError_t e, const char *where)
{
    cudaGetLastError();
    return fail(s, HAWKES_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define MWG_TRY(expr, where)                    \
    do {                                        \
        cudaError_t e_ = (expr);                \
        if (e_ != cudaSuccess)                  \
            return cuda_fail(s, e_, where);     \
    } while (0)

// FP32 copies of the current X and t and their range flag.
hawkes_status enqueue_split(hawkes_mwg *s, cudaStream_t st)
{
    MWG_TRY(cudaMemsetAsync(s->ctl + 3, 0, sizeof(int), st), "clear range flag");
    const int grid = (int)std::min<int64_t>(4 * (int64_t)s->sms, (s->n * s->d + kThreads - 1) / kThreads);
    split_kernel<<<std::max(grid, 1), kThreads, 0, st>>>(s->X, s->t, s->n, s->d, s->m32.xh, s->m32.xl, s->m32.th,
                                                         s->m32.tl, s->ctl + 3);
    MWG_TRY(cudaGetLastError(), "split kernel");
    return HAWKES_OK;
}

// The FP32 constants of the mixed precision, or false where they leave the
// range in which FP32 products and the underflow bound below hold.
bool make_state32(const Consts &k, State32 &c)
{
    const double log2e = 1.4426950408889634074;
    const double v[6] = {k.Cmu, k.Cxi, k.a * log2e, k.b * log2e, k.c * log2e, k.omega * log2e};
    for (double x : v)
        if (!(x >= 0x1p-100 && x <= 0x1p100))
            return false;
    c.Cmu = (float)v[0];
    c.Cxi = (float)v[1];
    c.a2 = (float)v[2];
    c.b2 = (float)v[3];
    c.c2 = (float)v[4];
    c.w2 = (float)v[5];
    // below tau, FP32 terms that flushed to zero (each < C 2^-126, at most
    // 2^30 of them) could reach 2^-36 of the rate
    c.tau = std::max(k.Cmu, k.Cxi) * 0x1p-60;
    return true;
}

hawkes_status enqueue_rates(hawkes_mwg *s, cudaStream_t st)
{
    const int64_t tiles = (s->n + kRateTile - 1) / kRateTile;
    int fsplit = (int)std::min<int64_t>(kRateSplit, std::max<int64_t>(1, (4 * s->sms + tiles - 1) / tiles));
    if (fsplit > tiles)
        fsplit = (int)tiles;
    rates_kernel<<<dim3((unsigned)tiles, fsplit), kRateTile, 0, st>>>(s->t, s->X, s->n, s->d, s->k, fsplit, s->part,
                                                                      s->ctl + 1);
    MWG_TRY(cudaGetLastError(), "rate kernel");
    const int64_t ncta = (s->n + kFinThreads - 1) / kFinThreads;
    rates_finish_kernel<<<(unsigned)ncta, kFinThreads, 0, st>>>(s->t, s->n, s->k, fsplit, s->part, s->Tmax, s->lam0,
                                                                  s->lam1, s->ctl, s->cpart, s->loglik);
    MWG_TRY(cudaGetLastError(), "rate finish kernel");
    return HAWKES_OK;
}

// CTAs per moved event in the row part: about two per SM in total, each with
// at least one event per thread and at most kRangeMax events.  (FP64 runs at
// 1/64 of the FP32 rate on this GPU, so one event's O(N) row must spread
// over many SMs.)
int64_t most_splits(int64_t n, int sms)
{
    return std::max<int64_t>(2 * (int64_t)sms + 1, (n + kRangeMax - 1) / kRangeMax);
}

// Threads per event in the column part: a power of two up to 8 and up to
// |B|, chosen so that a column CTA (64 / lanes events, 2|B| pair terms each)
// does about the work of a row CTA (`per` pair terms); the CTAs then finish
// together instead of the few SMs holding two column CTAs setting the time.
Launch plan_launch(const hawkes_mwg *s, int nb)
{
    Launch L;
    const int64_t want = (2 * (int64_t)s->sms + std::max(nb, 1) - 1) / std::max(nb, 1);
    const int64_t most = std::max<int64_t>(1, s->n / kEvalThreads);
    const int64_t need = (s->n + kRangeMax - 1) / kRangeMax;
    const int64_t splits = std::max(std::min(want, most), need);
    L.per = (s->n + splits - 1) / splits;
    L.splits = (int)((s->n + L.per - 1) / L.per);  // no empty range
    L.lanes = 1;
    while (L.lanes < 8 && 2 * L.lanes <= nb && 2 * kEvalThreads * (int64_t)nb >= 2 * L.lanes * L.per)
        L.lanes *= 2;
    const int ev = kEvalThreads / L.lanes;
    L.ncol = (int)((s->n + ev - 1) / ev);
    return L;
}

hawkes_status enqueue_proposal(hawkes_mwg *s, int32_t nb, const int64_t *idx, const double *X_new, bool step,
                               const double *log_q_ratio, const double *log_u, cudaStream_t st, double *out_delta,
                               int32_t *out_accepted)
{
    if (nb < 0 || nb > s->max_block)
        return fail(s, HAWKES_ERR_INVALID_ARG, "block size must be in [0, max_block]");
    if (nb > 0 && (!idx || !X_new))
        return fail(s, HAWKES_ERR_INVALID_ARG, "idx and X_new must be device pointers");
    if (step && !log_u)
        return fail(s, HAWKES_ERR_INVALID_ARG, "log_u must be a device pointer");
    MWG_TRY(cudaSetDevice(s->device), "cudaSetDevice");
    EvalArgs a;
    a.t = s->t;
    a.X = s->X;
    a.n = s->n;
    a.k = s->k;
    a.m32 = s->m32;
    a.B = Block{nb, idx, X_new};
    a.L = plan_launch(s, nb);
    a.lam0 = s->lam0;
    a.lam1 = s->lam1;
    a.ctl = s->ctl;
    a.cpart = s->cpart;
    a.rowpart = s->rowterm;
    a.bterm = s->bterm;
    a.bticket = s->bticket;
    a.out_delta = out_delta;
    a.step = step;
    a.log_q_ratio = log_q_ratio;
    a.log_u = log_u;
    a.accepted_out = out_accepted;
    a.loglik = s->loglik;
    const bool mixed = s->prec == HAWKES_PREC_MIXED;
    const int64_t grid = (int64_t)a.L.ncol + (int64_t)nb * a.L.splits;
    // the staged block: FP64 old and new places and times, or their FP32
    // (hi, lo) pairs and the time keys
    const size_t smem = mixed ? (size_t)nb * (16 * s->d + 16) : sizeof(double) * (size_t)nb * (2 * s->d + 1);
    switch (s->d * 2 + (mixed ? 1 : 0)) {
#define HK_MWG_EVAL(DD)                                                                   \
    case 2 * DD:                                                                          \
        eval_kernel<DD, false><<<(unsigned)grid, kEvalThreads, smem, st>>>(a);            \
        break;                                                                            \
    case 2 * DD + 1:                                                                      \
        eval_kernel<DD, true><<<(unsigned)grid, kEvalThreads, smem, st>>>(a);             \
        break;
        HK_MWG_EVAL(1)
        HK_MWG_EVAL(2)
        HK_MWG_EVAL(3)
        HK_MWG_EVAL(4)
        HK_MWG_EVAL(5)
        HK_MWG_EVAL(6)
        HK_MWG_EVAL(7)
        HK_MWG_EVAL(8)
#undef HK_MWG_EVAL
    default:
        return fail(s, HAWKES_ERR_INVALID_ARG, "dimension out of range");
    }
    MWG_TRY(cudaGetLastError(), "proposal kernel");
    return HAWKES_OK;
}

}  // namespace

extern "C" {

hawkes_status hawkes_mwg_create(int32_t device, const double *t, const double *X, int64_t n, int32_t d,
                                const hawkes_params *params, int32_t max_block, hawkes_stream stream,
                                hawkes_mwg **out)
{
    if (!out)
        return HAWKES_ERR_INVALID_ARG;
    *out = nullptr;
    if (!t || !X || n < 1 || n > ((int64_t)1 << 30) || d < 1 || d > kMaxDim || !params_ok(params) ||
        max_block < 1 || max_block > kMaxBlock)
        return HAWKES_ERR_INVALID_ARG;
    hawkes_mwg *s = new hawkes_mwg();
    s->device = device;
    s->n = n;
    s->d = d;
    s->max_block = max_block;
    s->k = make_consts(*params, d);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    auto bail = [&](hawkes_status code) {
        hawkes_mwg_destroy(s);
        return code;
    };
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return bail(HAWKES_ERR_CUDA);
    }
    const size_t ncta = (size_t)((n + 7) / 8);  // column CTAs of 8 events at the least
    if (cudaMalloc(&s->t, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&s->X, sizeof(double) * n * d) != cudaSuccess ||
        cudaMalloc(&s->lam0, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&s->lam1, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&s->part, sizeof(double) * (size_t)kRateSplit * n) != cudaSuccess ||
        cudaMalloc(&s->cpart, sizeof(double) * ncta) != cudaSuccess ||
        cudaMalloc(&s->rowterm, sizeof(double) * (size_t)max_block * most_splits(n, s->sms)) != cudaSuccess ||
        cudaMalloc(&s->loglik, sizeof(double)) != cudaSuccess || cudaMalloc(&s->Tmax, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&s->bterm, sizeof(double) * max_block) != cudaSuccess ||
        cudaMalloc(&s->bticket, sizeof(unsigned) * max_block) != cudaSuccess ||
        cudaMalloc(&s->m32.xh, sizeof(float) * n * d) != cudaSuccess ||
        cudaMalloc(&s->m32.xl, sizeof(float) * n * d) != cudaSuccess ||
        cudaMalloc(&s->m32.th, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&s->m32.tl, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&s->ctl, sizeof(int) * 4) != cudaSuccess) {
        cudaGetLastError();
        return bail(HAWKES_ERR_OOM);
    }
    if (cudaMemcpyAsync(s->t, t, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->X, X, sizeof(double) * n * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(s->ctl, 0, sizeof(int) * 4, st) != cudaSuccess ||
        cudaMemsetAsync(s->bticket, 0, sizeof(unsigned) * max_block, st) != cudaSuccess) {
        cudaGetLastError();
        return bail(HAWKES_ERR_CUDA);
    }
    tmax_kernel<<<1, kThreads, 0, st>>>(s->t, n, s->Tmax);
    if (cudaGetLastError() != cudaSuccess)
        return bail(HAWKES_ERR_CUDA);
    if (enqueue_rates(s, st) != HAWKES_OK)
        return bail(HAWKES_ERR_CUDA);
    *out = s;
    return HAWKES_OK;
}

void hawkes_mwg_destroy(hawkes_mwg *s)
{
    if (!s)
        return;
    cudaSetDevice(s->device);
    cudaFree(s->t);
    cudaFree(s->X);
    cudaFree(s->lam0);
    cudaFree(s->lam1);
    cudaFree(s->part);
    cudaFree(s->cpart);
    cudaFree(s->rowterm);
    cudaFree(s->loglik);
    cudaFree(s->Tmax);
    cudaFree(s->bterm);
    cudaFree(s->bticket);
    cudaFree(s->m32.xh);
    cudaFree(s->m32.xl);
    cudaFree(s->m32.th);
    cudaFree(s->m32.tl);
    cudaFree(s->ctl);
    delete s;
}

const char *hawkes_mwg_last_error(const hawkes_mwg *s) { return s ? s->err.c_str() : "null state"; }

hawkes_status hawkes_mwg_delta(hawkes_mwg *s, int32_t nb, const int64_t *idx, const double *X_new,
                               hawkes_stream stream, double *out_delta)
{
    if (!s)
        return HAWKES_ERR_INVALID_ARG;
    if (!out_delta)
        return fail(s, HAWKES_ERR_INVALID_ARG, "out_delta must be a device pointer");
    return enqueue_proposal(s, nb, idx, X_new, false, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream),
                            out_delta, nullptr);
}

hawkes_status hawkes_mwg_step(hawkes_mwg *s, int32_t nb, const int64_t *idx, const double *X_new,
                              const double *log_q_ratio, const double *log_u, hawkes_stream stream,
                              double *out_delta, int32_t *out_accepted)
{
    if (!s)
        return HAWKES_ERR_INVALID_ARG;
    return enqueue_proposal(s, nb, idx, X_new, true, log_q_ratio, log_u, reinterpret_cast<cudaStream_t>(stream),
                            out_delta, out_accepted);
}

hawkes_status hawkes_mwg_propose_circle(hawkes_mwg *s, int32_t nb, const int64_t *idx, const double *centers,
                                        const double *radii, double eps, int32_t tries, const double *u,
                                        hawkes_stream stream, double *X_new, double *log_q_ratio)
{
    if (!s)
        return HAWKES_ERR_INVALID_ARG;
    if (s->d != 2)
        return fail(s, HAWKES_ERR_INVALID_ARG, "circle proposals need D = 2");
    if (nb < 0 || nb > s->max_block || tries < 1 || !(eps > 0.0) || !std::isfinite(eps) || !log_q_ratio ||
        (nb > 0 && (!idx || !centers || !radii || !u || !X_new)))
        return fail(s, HAWKES_ERR_INVALID_ARG, "bad circle-proposal arguments");
    MWG_TRY(cudaSetDevice(s->device), "cudaSetDevice");
    const Block B{nb, idx, nullptr};
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (4 * nb <= 32)  // one warp: no cross-warp step in the q-ratio sum
        propose_circle_kernel<32><<<1, 32, 0, st>>>(s->X, s->n, B, centers, radii, eps, tries, u, X_new, log_q_ratio,
                                                    s->ctl + 1);
    else
        propose_circle_kernel<kThreads><<<1, kThreads, 0, st>>>(s->X, s->n, B, centers, radii, eps, tries, u, X_new,
                                                                log_q_ratio, s->ctl + 1);
    MWG_TRY(cudaGetLastError(), "circle proposals");
    return HAWKES_OK;
}

hawkes_status hawkes_mwg_propose_box(hawkes_mwg *s, int32_t nb, const int64_t *idx, const double *lo,
                                     const double *hi, double sd, const double *u, hawkes_stream stream,
                                     double *X_new, double *log_q_ratio)
{
    if (!s)
        return HAWKES_ERR_INVALID_ARG;
    if (nb < 0 || nb > s->max_block || !(sd > 0.0) || !std::isfinite(sd) || !log_q_ratio ||
        (nb > 0 && (!idx || !lo || !hi || !u || !X_new)))
        return fail(s, HAWKES_ERR_INVALID_ARG, "bad box-proposal arguments");
    MWG_TRY(cudaSetDevice(s->device), "cudaSetDevice");
    const Block B{nb, idx, nullptr};
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (2 * (int64_t)nb * s->d <= 32)
        propose_box_kernel<32><<<1, 32, 0, st>>>(s->X, s->n, s->d, B, lo, hi, sd, 1.0 / sd, u, X_new, log_q_ratio,
                                                 s->ctl + 1);
    else
        propose_box_kernel<kThreads><<<1, kThreads, 0, st>>>(s->X, s->n, s->d, B, lo, hi, sd, 1.0 / sd, u, X_new,
                                                             log_q_ratio, s->ctl + 1);
    MWG_TRY(cudaGetLastError(), "box proposals");
    return HAWKES_OK;
}

hawkes_status hawkes_mwg_refresh(hawkes_mwg *s, hawkes_stream stream)
{
    if (!s)
        return HAWKES_ERR_INVALID_ARG;
    MWG_TRY(cudaSetDevice(s->device), "cudaSetDevice");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (s->prec == HAWKES_PREC_MIXED) {
        const hawkes_status r = enqueue_split(s, st);
        if (r != HAWKES_OK)
            return r;
    }
    return enqueue_rates(s, st);
}

hawkes_status hawkes_mwg_set_precision(hawkes_mwg *s, hawkes_precision prec, hawkes_stream stream)
{
    if (!s)
        return HAWKES_ERR_INVALID_ARG;
    if (prec != HAWKES_PREC_MIXED && prec != HAWKES_PREC_FP64)
        return fail(s, HAWKES_ERR_INVALID_ARG, "unknown precision");
    if (prec == HAWKES_PREC_MIXED) {
        State32 c = s->m32;
        if (!make_state32(s->k, c))
            return fail(s, HAWKES_ERR_INVALID_ARG,
                        "mixed precision needs the kernel prefactors and scales within [2^-100, 2^100]");
        MWG_TRY(cudaSetDevice(s->device), "cudaSetDevice");
        const hawkes_status r = enqueue_split(s, reinterpret_cast<cudaStream_t>(stream));
        if (r != HAWKES_OK)
            return r;
        s->m32 = c;
    }
    s->prec = prec;
    return HAWKES_OK;
}

hawkes_status hawkes_mwg_read(hawkes_mwg *s, hawkes_stream stream, double *X_out, double *lam_out,
                              double *out_loglik)
{
    if (!s)
        return HAWKES_ERR_INVALID_ARG;
    MWG_TRY(cudaSetDevice(s->device), "cudaSetDevice");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (X_out)
        MWG_TRY(cudaMemcpyAsync(X_out, s->X, sizeof(double) * s->n * s->d, cudaMemcpyDeviceToDevice, st), "copy X");
    if (lam_out) {
        copy_rates_kernel<<<std::min(1024, grid_for(s->n)), kThreads, 0, st>>>(s->lam0, s->lam1, s->ctl, s->n,
                                                                                lam_out);
        MWG_TRY(cudaGetLastError(), "copy rates");
    }
    if (out_loglik)
        MWG_TRY(cudaMemcpyAsync(out_loglik, s->loglik, sizeof(double), cudaMemcpyDeviceToDevice, st), "copy ell");
    return HAWKES_OK;
}

hawkes_status hawkes_mwg_sync_status(hawkes_mwg *s, hawkes_stream stream)
{
    if (!s)
        return HAWKES_ERR_INVALID_ARG;
    MWG_TRY(cudaSetDevice(s->device), "cudaSetDevice");
    MWG_TRY(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)), "stream synchronize");
    int st = 0;
    MWG_TRY(cudaMemcpy(&st, s->ctl + 1, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    MWG_TRY(cudaMemset(s->ctl + 1, 0, sizeof(int)), "clear status");
    if (st & kBadData)
        return fail(s, HAWKES_ERR_INVALID_DATA, "non-finite location or time, or a negative time");
    if (st & kBadBlock)
        return fail(s, HAWKES_ERR_INVALID_DATA, "a block index is out of range or repeated");
    if (st & kBadProposal)
        return fail(s, HAWKES_ERR_INVALID_DATA,
                    "a proposed location is not finite (or, in mixed precision, has a coordinate of 2^100 or more)");
    s->err.clear();
    return HAWKES_OK;
}

}  // extern "C"
