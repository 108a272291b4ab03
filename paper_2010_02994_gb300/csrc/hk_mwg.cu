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
// Three launches per proposal: a column kernel (every m: block membership,
// the |B| column updates, log1p(Delta_m / lambda_m) summed per CTA), a row
// kernel (one CTA per moved event: its new rate over all events), and a
// one-CTA finish kernel (Delta ell in a fixed order; in step mode the accept
// decision log u < Delta ell + log q-ratio and, on accept, the commit).  The
// rates live in two buffers; the device-side index of the current one flips
// on accept, so no call reads anything back to the host and a sequence of
// steps can be captured in a CUDA graph.  Everything is FP64.
#include <cuda_runtime.h>

#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "hawkes.h"

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
    double Cmu, Cxi, omega, mu0, tau_t, theta;
};

// Contribution of event (xs, ts) to the rate at event (xm, tm): the
// background term (both Gaussians, I[t != t_m]) and the self-excitation term
// (I[t < t_m]) of Section 2.1.
__device__ __forceinline__ double contrib(const double *xm, double tm, const double *xs, double ts, int d,
                                          const Consts &k)
{
    double r2 = 0.0;
    for (int q = 0; q < d; ++q) {
        const double df = xm[q] - xs[q];
        r2 += df * df;
    }
    const double dt = tm - ts;
    double v = 0.0;
    if (tm != ts)
        v += k.Cmu * exp(-(r2 * k.a + dt * dt * k.b));
    if (ts < tm)
        v += k.Cxi * exp(-(k.omega * dt + r2 * k.c));
    return v;
}

template <int NT = kThreads>
__device__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
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

// lambda_m from the splits (fixed order) into the current buffer, and
// ell = sum log lambda - sum Lambda in one CTA.
__global__ void __launch_bounds__(kThreads) rates_finish_kernel(const double *__restrict__ t, int64_t n, Consts k,
                                                                int fsplit, const double *__restrict__ part,
                                                                double *lam0, double *lam1, const int *active,
                                                                double *loglik)
{
    __shared__ double sh[kThreads];
    double *lam = *active ? lam1 : lam0;
    double tmax = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += kThreads)
        tmax = fmax(tmax, t[i]);
    sh[threadIdx.x] = tmax;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    const double T = sh[0];
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) {
        double l = 0.0;
        for (int sp = 0; sp < fsplit; ++sp)
            l += part[(int64_t)sp * n + i];
        lam[i] = l;
        const double a = T - t[i];
        const double Lam = k.mu0 * (normcdf(a / k.tau_t) - normcdf(-t[i] / k.tau_t)) - k.theta * expm1(-k.omega * a);
        acc += log(l) - Lam;
    }
    const double ell = block_sum(acc, sh);
    if (threadIdx.x == 0)
        *loglik = ell;
}

// ------------------------------------------------------------- proposal --

struct Block {
    int nb;
    const int64_t *idx;   // caller's device indices
    const double *xnew;   // caller's device proposals, nb x d
};

// Every m: its position in the block (or -1), and for m outside the block
// the change of its rate and log1p(Delta_m / lambda_m), summed per CTA.
// Small CTAs, so that the FP64 work spreads over every SM.
constexpr int kColThreads = 64;

__global__ void __launch_bounds__(kColThreads) columns_kernel(const double *__restrict__ t,
                                                              const double *__restrict__ X, int64_t n, int d,
                                                              Consts k, Block B, double *lam0, double *lam1,
                                                              const int *active, int *pos, double *part, int *status)
{
    __shared__ double sh[kColThreads];
    __shared__ double sxo[kMaxBlock * kMaxDim], sxn[kMaxBlock * kMaxDim], stb[kMaxBlock];
    __shared__ int64_t sid[kMaxBlock];
    const double *lam = *active ? lam1 : lam0;
    double *lam_new = *active ? lam0 : lam1;
    for (int b = threadIdx.x; b < B.nb; b += kColThreads) {
        const int64_t m = B.idx[b];
        const bool ok = m >= 0 && m < n;
        sid[b] = ok ? m : -1;
        stb[b] = ok ? t[m] : 0.0;
        bool bad = false;
        for (int q = 0; q < d; ++q) {
            sxo[b * kMaxDim + q] = ok ? X[m * d + q] : 0.0;
            const double v = B.xnew[(int64_t)b * d + q];
            bad |= !isfinite(v);
            sxn[b * kMaxDim + q] = v;
        }
        if (blockIdx.x == 0) {
            if (!ok)
                atomicOr(status, kBadBlock);
            if (bad)
                atomicOr(status, kBadProposal);
        }
    }
    __syncthreads();
    double term = 0.0;
    const int64_t m = (int64_t)blockIdx.x * kColThreads + threadIdx.x;
    if (m < n) {
        int p = -1;
        for (int b = 0; b < B.nb; ++b)
            if (sid[b] == m) {
                if (p >= 0)
                    atomicOr(status, kBadBlock);  // repeated index
                p = b;
            }
        pos[m] = p;
        if (p < 0) {
            double xm[kMaxDim];
            for (int q = 0; q < d; ++q)
                xm[q] = X[m * d + q];
            const double tm = t[m];
            double delta = 0.0;
            for (int b = 0; b < B.nb; ++b)
                delta += contrib(xm, tm, sxn + b * kMaxDim, stb[b], d, k) -
                         contrib(xm, tm, sxo + b * kMaxDim, stb[b], d, k);
            const double l = lam[m];
            const double ln = l + delta;
            lam_new[m] = ln;
            term = log_ratio(l, ln, delta);
        }
    }
    term = block_sum<kColThreads>(term, sh);
    if (threadIdx.x == 0)
        part[blockIdx.x] = term;
}

// Moved event b's new rate over all events (moved ones at their proposed
// places), split over `splits` CTAs per event (grid b x split), each adding
// one contiguous range of events; the finish kernel adds the splits in order.
constexpr int kRowThreads = 64;

__global__ void __launch_bounds__(kRowThreads) rows_kernel(const double *__restrict__ t,
                                                           const double *__restrict__ X, int64_t n, int d, Consts k,
                                                           Block B, const int *pos, int splits, double *rowpart)
{
    __shared__ double sh[kRowThreads];
    const int b = blockIdx.x, sp = blockIdx.y;
    const int64_t mb = B.idx[b];
    const int64_t per = (n + splits - 1) / splits;
    const int64_t lo = min((int64_t)sp * per, n), hi = min(lo + per, n);
    double s = 0.0;
    if (mb >= 0 && mb < n) {  // a bad index is reported by the column kernel
        double xb[kMaxDim];
        for (int q = 0; q < d; ++q)
            xb[q] = B.xnew[(int64_t)b * d + q];
        const double tb = t[mb];
        for (int64_t m = lo + threadIdx.x; m < hi; m += kRowThreads) {
            if (m == mb)
                continue;
            const int p = pos[m];
            const double *xm = p >= 0 ? B.xnew + (int64_t)p * d : X + m * d;
            s += contrib(xb, tb, xm, t[m], d, k);
        }
    }
    s = block_sum<kRowThreads>(s, sh);
    if (threadIdx.x == 0)
        rowpart[(int64_t)b * splits + sp] = s;
}

// Delta ell in a fixed order: the moved events' new rates (their splits
// added in order) and log ratios, then the column partials; in step mode
// the accept decision and, on accept, the commit (moved locations, running
// ell, current-buffer flip).
__global__ void __launch_bounds__(kThreads) finish_kernel(int ncta, const double *__restrict__ part, Block B,
                                                          int64_t n, int splits, const double *__restrict__ rowpart,
                                                          double *lam0, double *lam1, const int *status,
                                                          double *out_delta, bool step, const double *log_q_ratio,
                                                          const double *log_u, int *accepted_out, double *X, int d,
                                                          int *active, double *loglik)
{
    __shared__ double sh[kThreads];
    __shared__ int acc;
    const double *lam = *active ? lam1 : lam0;
    double *lam_new = *active ? lam0 : lam1;
    double v = 0.0;
    for (int b = threadIdx.x; b < B.nb; b += kThreads) {
        const int64_t mb = B.idx[b];
        if (mb < 0 || mb >= n)
            continue;
        double lnew = 0.0;
        for (int sp = 0; sp < splits; ++sp)
            lnew += rowpart[(int64_t)b * splits + sp];
        const double l = lam[mb];
        lam_new[mb] = lnew;
        v += (l > 0.0 && lnew > 0.0) ? log(lnew) - log(l) : log_ratio(l, lnew, lnew - l);
    }
    for (int i = threadIdx.x; i < ncta; i += kThreads)
        v += part[i];
    const double delta = block_sum(v, sh);
    if (threadIdx.x == 0) {
        const bool bad = *(volatile const int *)status != 0;
        const double dl = bad ? nan("") : delta;
        if (out_delta)
            *out_delta = dl;
        int a = 0;
        if (step && !bad) {
            const double lhs = *log_u, rhs = dl + (log_q_ratio ? *log_q_ratio : 0.0);
            a = (lhs < rhs) ? 1 : 0;  // NaN on either side rejects
        }
        acc = a;
        if (accepted_out)
            *accepted_out = a;
        if (a) {
            *loglik += dl;
            *active ^= 1;
        }
    }
    __syncthreads();
    if (acc)
        for (int e = threadIdx.x; e < B.nb * d; e += kThreads) {
            const int b = e / d, q = e % d;
            X[B.idx[b] * d + q] = B.xnew[e];
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

// Area of the intersection of discs of radii R and rho, centres c apart:
// the two circular segments cut off by the common chord, each
// r^2 (2 theta - sin 2 theta) / 2 with theta = atan2(half-chord, signed
// distance of the chord from the centre).
__device__ double lens_area(double R, double rho, double c)
{
    if (c >= R + rho)
        return 0.0;
    if (c <= fabs(R - rho)) {
        const double m = fmin(R, rho);
        return CUDART_PI * m * m;
    }
    const double d1 = (c * c + R * R - rho * rho) / (2.0 * c);
    const double d2 = c - d1;
    const double h = sqrt(fmax((R - d1) * (R + d1), 0.0));
    return 0.5 * R * R * x_minus_sin(2.0 * atan2(h, d1)) + 0.5 * rho * rho * x_minus_sin(2.0 * atan2(h, d2));
}

// log P(at least one of `tries` uniform draws from a disc of radius rho
// lands in a region of area A inside it)
__device__ double log_success(double A, double rho, int tries)
{
    const double p = A / (CUDART_PI * rho * rho);
    return p >= 1.0 ? 0.0 : log(-expm1((double)tries * log1p(-p)));
}

// Lens proposals of Eq. (6) for a D = 2 block, one thread per moved event;
// the block's log q-ratio is summed in a fixed order.
__global__ void __launch_bounds__(kThreads) propose_circle_kernel(const double *__restrict__ X, int64_t n, Block B,
                                                                  const double *__restrict__ centers,
                                                                  const double *__restrict__ radii, double eps,
                                                                  int tries, const double *__restrict__ u,
                                                                  double *X_new, double *log_q_ratio, int *status)
{
    __shared__ double sh[kThreads];
    double lq = 0.0;
    for (int b = threadIdx.x; b < B.nb; b += kThreads) {
        const int64_t m = B.idx[b];
        if (m < 0 || m >= n) {
            atomicOr(status, kBadBlock);
            continue;
        }
        const double x0 = X[m * 2], x1 = X[m * 2 + 1], c0 = centers[m * 2], c1 = centers[m * 2 + 1];
        const double R = radii[m], rho = R * eps;
        const double A_x = lens_area(R, rho, hypot(x0 - c0, x1 - c1));
        if (!(R > 0.0) || !isfinite(R) || !(A_x > 0.0)) {
            atomicOr(status, kBadProposal);
            continue;
        }
        double y0 = x0, y1 = x1;
        for (int k = 0; k < tries; ++k) {
            const double r = rho * sqrt(u[((int64_t)b * tries + k) * 2]);
            double sn, cs;
            sincospi(2.0 * u[((int64_t)b * tries + k) * 2 + 1], &sn, &cs);
            const double z0 = x0 + r * cs, z1 = x1 + r * sn;
            const double dx = z0 - c0, dy = z1 - c1;
            if (dx * dx + dy * dy < R * R) {
                y0 = z0;
                y1 = z1;
                const double A_y = lens_area(R, rho, hypot(dx, dy));
                lq += (log_success(A_y, rho, tries) - log(A_y)) - (log_success(A_x, rho, tries) - log(A_x));
                break;
            }
        }
        X_new[(int64_t)b * 2] = y0;
        X_new[(int64_t)b * 2 + 1] = y1;
    }
    lq = block_sum(lq, sh);
    if (threadIdx.x == 0)
        *log_q_ratio = lq;
}

// Truncated-normal proposals inside the boxes of Eq. (2), one thread per
// coordinate: x* = x + s Phi^{-1}(Phi(a) + u (Phi(b) - Phi(a))), and the
// log q-ratio sum log Z(x) - log Z(x*), Z(y) = Phi((hi - y)/s) - Phi((lo - y)/s).
__global__ void __launch_bounds__(kThreads) propose_box_kernel(const double *__restrict__ X, int64_t n, int d,
                                                               Block B, const double *__restrict__ lo,
                                                               const double *__restrict__ hi, double sd,
                                                               const double *__restrict__ u, double *X_new,
                                                               double *log_q_ratio, int *status)
{
    __shared__ double sh[kThreads];
    double lq = 0.0;
    for (int e = threadIdx.x; e < B.nb * d; e += kThreads) {
        const int b = e / d, q = e % d;
        const int64_t m = B.idx[b];
        if (m < 0 || m >= n) {
            atomicOr(status, kBadBlock);
            continue;
        }
        const double x = X[m * d + q], l = lo[m * d + q], h = hi[m * d + q];
        if (!(l <= x && x <= h) || !(sd > 0.0)) {
            atomicOr(status, kBadProposal);
            continue;
        }
        const double Pa = normcdf((l - x) / sd), Pb = normcdf((h - x) / sd);
        const double y = fmin(fmax(x + sd * normcdfinv(Pa + u[e] * (Pb - Pa)), l), h);
        X_new[e] = y;
        lq += log(Pb - Pa) - log(normcdf((h - y) / sd) - normcdf((l - y) / sd));
    }
    lq = block_sum(lq, sh);
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
    double *part = nullptr;     // max(kRateSplit * n, column-kernel CTAs)
    double *rowterm = nullptr;  // row-kernel partials: max_block x (2 SMs + 1)
    double *loglik = nullptr;   // running ell
    int *ctl = nullptr;         // [0] current rate buffer, [1] status
    int *pos = nullptr;         // n
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

hawkes_status enqueue_rates(hawkes_mwg *s, cudaStream_t st)
{
    const int64_t tiles = (s->n + kRateTile - 1) / kRateTile;
    int fsplit = (int)std::min<int64_t>(kRateSplit, std::max<int64_t>(1, (4 * s->sms + tiles - 1) / tiles));
    if (fsplit > tiles)
        fsplit = (int)tiles;
    rates_kernel<<<dim3((unsigned)tiles, fsplit), kRateTile, 0, st>>>(s->t, s->X, s->n, s->d, s->k, fsplit, s->part,
                                                                      s->ctl + 1);
    MWG_TRY(cudaGetLastError(), "rate kernel");
    rates_finish_kernel<<<1, kThreads, 0, st>>>(s->t, s->n, s->k, fsplit, s->part, s->lam0, s->lam1, s->ctl,
                                                s->loglik);
    MWG_TRY(cudaGetLastError(), "rate finish kernel");
    return HAWKES_OK;
}

// CTAs per moved event in the row kernel: about two per SM in total, each
// with at least one event per thread.  (FP64 runs at 1/64 of the FP32 rate
// on this GPU, so one event's O(N) row must spread over many SMs.)
int row_splits(const hawkes_mwg *s, int nb)
{
    const int64_t want = (2 * (int64_t)s->sms + std::max(nb, 1) - 1) / std::max(nb, 1);
    const int64_t most = std::max<int64_t>(1, s->n / kRowThreads);
    return (int)std::max<int64_t>(1, std::min(want, most));
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
    const Block B{nb, idx, X_new};
    const int ncta = (int)((s->n + kColThreads - 1) / kColThreads);
    columns_kernel<<<ncta, kColThreads, 0, st>>>(s->t, s->X, s->n, s->d, s->k, B, s->lam0, s->lam1, s->ctl, s->pos,
                                                 s->part, s->ctl + 1);
    MWG_TRY(cudaGetLastError(), "column kernel");
    const int splits = row_splits(s, nb);
    if (nb > 0) {
        rows_kernel<<<dim3(nb, splits), kRowThreads, 0, st>>>(s->t, s->X, s->n, s->d, s->k, B, s->pos, splits,
                                                           s->rowterm);
        MWG_TRY(cudaGetLastError(), "row kernel");
    }
    finish_kernel<<<1, kThreads, 0, st>>>(ncta, s->part, B, s->n, splits, s->rowterm, s->lam0, s->lam1, s->ctl + 1,
                                          out_delta, step, log_q_ratio, log_u, out_accepted, s->X, s->d, s->ctl,
                                          s->loglik);
    MWG_TRY(cudaGetLastError(), "finish kernel");
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
    const size_t part_n = std::max<size_t>((size_t)kRateSplit * n, (size_t)((n + kColThreads - 1) / kColThreads));
    if (cudaMalloc(&s->t, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&s->X, sizeof(double) * n * d) != cudaSuccess ||
        cudaMalloc(&s->lam0, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&s->lam1, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&s->part, sizeof(double) * part_n) != cudaSuccess ||
        cudaMalloc(&s->rowterm, sizeof(double) * (size_t)max_block * (2 * s->sms + 1)) != cudaSuccess ||
        cudaMalloc(&s->loglik, sizeof(double)) != cudaSuccess || cudaMalloc(&s->ctl, sizeof(int) * 2) != cudaSuccess ||
        cudaMalloc(&s->pos, sizeof(int) * n) != cudaSuccess) {
        cudaGetLastError();
        return bail(HAWKES_ERR_OOM);
    }
    if (cudaMemcpyAsync(s->t, t, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->X, X, sizeof(double) * n * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(s->ctl, 0, sizeof(int) * 2, st) != cudaSuccess) {
        cudaGetLastError();
        return bail(HAWKES_ERR_CUDA);
    }
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
    cudaFree(s->rowterm);
    cudaFree(s->loglik);
    cudaFree(s->ctl);
    cudaFree(s->pos);
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
    propose_circle_kernel<<<1, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        s->X, s->n, Block{nb, idx, nullptr}, centers, radii, eps, tries, u, X_new, log_q_ratio, s->ctl + 1);
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
    propose_box_kernel<<<1, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        s->X, s->n, s->d, Block{nb, idx, nullptr}, lo, hi, sd, u, X_new, log_q_ratio, s->ctl + 1);
    MWG_TRY(cudaGetLastError(), "box proposals");
    return HAWKES_OK;
}

hawkes_status hawkes_mwg_refresh(hawkes_mwg *s, hawkes_stream stream)
{
    if (!s)
        return HAWKES_ERR_INVALID_ARG;
    MWG_TRY(cudaSetDevice(s->device), "cudaSetDevice");
    return enqueue_rates(s, reinterpret_cast<cudaStream_t>(stream));
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
        return fail(s, HAWKES_ERR_INVALID_DATA, "a proposed location is not finite");
    s->err.clear();
    return HAWKES_OK;
}

}  // extern "C"
