// FP64 pair kernels: the rate row sums of Eq. (1) and the location gradient
// of Appendix A with every operation in double precision.
//
// Each CTA owns kFp64Rows consecutive (time-sorted) rows of one set and one
// of fsplit column ranges; it walks its range in tiles staged in shared
// memory and writes one partial per row to its split's slot.  The finalize
// kernels add the fsplit partials in a fixed order.  Pairs are ordered: row n
// evaluates mu_nn' and xi_nn' from their definitions (one exp each, with the
// spatial and temporal Gaussians merged into a single exponent).  CUDA's
// exp() supplies the exponentials.
#include <cmath>

#include "hk_internal.cuh"

namespace hk {

namespace {

constexpr int kTile = kFp64Rows;

struct Nsum {
    double s = 0.0, c = 0.0;
    __device__ void add(double x)
    {
        const double t = s + x;
        if (fabs(s) >= fabs(x))
            c += (s - t) + x;
        else
            c += (x - t) + s;
        s = t;
    }
    __device__ double value() const { return isfinite(s) ? s + c : s; }
};

struct Fp64Consts {
    double a, b, c;       // 1/(2 tau_x^2), 1/(2 tau_t^2), 1/(2 h^2)
    double Cmu, Cxi;      // mu0/(tau_x^D tau_t (2pi)^((D+1)/2)),  theta omega/(h^D (2pi)^(D/2))
    double omega;
};

__device__ Fp64Consts make_consts(const SetDesc &S)
{
    Fp64Consts k;
    const double two_pi = 6.283185307179586476925286766559;
    k.a = 0.5 / (S.tau_x * S.tau_x);
    k.b = 0.5 / (S.tau_t * S.tau_t);
    k.c = 0.5 / (S.h * S.h);
    k.Cmu = S.mu0 / (pow(S.tau_x, (double)S.d) * S.tau_t * pow(two_pi, 0.5 * (S.d + 1)));
    k.Cxi = S.theta * S.omega / (pow(S.h, (double)S.d) * pow(two_pi, 0.5 * S.d));
    k.omega = S.omega;
    return k;
}

// Column range [lo, hi) of split sp out of fsplit, in whole tiles.
__device__ __forceinline__ void split_range(int n, int fsplit, int sp, int &lo, int &hi)
{
    const int tiles = (n + kTile - 1) / kTile;
    const int per = (tiles + fsplit - 1) / fsplit;
    lo = min(sp * per * kTile, n);
    hi = min((sp + 1) * per * kTile, n);
}

template <bool THETA>
__global__ void __launch_bounds__(kTile) pass1_fp64_kernel(Work w, int set_lo)
{
    const SetDesc &S = w.sets[set_lo + blockIdx.y];
    const int n = S.n, d = S.d;
    const int nrt = (n + kTile - 1) / kTile;
    const int rt = blockIdx.x / S.fsplit, sp = blockIdx.x % S.fsplit;
    if (rt >= nrt)
        return;
    __shared__ double st[kTile];
    __shared__ double sx[kTile * kMaxD];
    const Fp64Consts k = make_consts(S);
    const int row = rt * kTile + threadIdx.x;
    const bool valid = row < n;
    const int64_t R0 = S.row0;
    double tn = 0.0, xn[kMaxD];
    for (int q = 0; q < kMaxD; ++q)
        xn[q] = 0.0;
    if (valid) {
        tn = w.t64[R0 + row];
        for (int q = 0; q < d; ++q)
            xn[q] = w.x64[(R0 + row) * kMaxD + q];
    }
    int lo, hi;
    split_range(n, S.fsplit, sp, lo, hi);
    constexpr int V = THETA ? kPass1ThetaVals : 1;
    Nsum tot[V];
    for (int c0 = lo; c0 < hi; c0 += kTile) {
        const int cnt = min(kTile, hi - c0);
        __syncthreads();
        if (threadIdx.x < cnt) {
            st[threadIdx.x] = w.t64[R0 + c0 + threadIdx.x];
            for (int q = 0; q < d; ++q)
                sx[threadIdx.x * kMaxD + q] = w.x64[(R0 + c0 + threadIdx.x) * kMaxD + q];
        }
        __syncthreads();
        if (!valid)
            continue;
        double part[V];
        for (int v = 0; v < V; ++v)
            part[v] = 0.0;
        for (int j = 0; j < cnt; ++j) {
            const double tm = st[j];
            double r2 = 0.0;
            for (int q = 0; q < d; ++q) {
                const double df = xn[q] - sx[j * kMaxD + q];
                r2 += df * df;
            }
            const double dt = tn - tm;
            double mu = 0.0, xi = 0.0;
            if (tn != tm)
                mu = k.Cmu * exp(-(r2 * k.a + dt * dt * k.b));
            if (tm < tn)
                xi = k.Cxi * exp(-(k.omega * dt + r2 * k.c));
            if (THETA) {
                part[0] += mu;
                part[1] += xi;
                part[2] += mu * r2;
                part[3] += mu * dt * dt;
                part[4] += xi * dt;
                part[5] += xi * r2;
            } else {
                part[0] += mu + xi;
            }
        }
        for (int v = 0; v < V; ++v)
            tot[v].add(part[v]);
    }
    if (valid)
        for (int v = 0; v < V; ++v)
            w.F1[S.fpart0 + ((int64_t)sp * V + v) * S.npad + row] = tot[v].value();
}

__global__ void __launch_bounds__(kTile) pass2_fp64_kernel(Work w, int set_lo)
{
    const SetDesc &S = w.sets[set_lo + blockIdx.y];
    const int n = S.n, d = S.d;
    const int nrt = (n + kTile - 1) / kTile;
    const int rt = blockIdx.x / S.fsplit, sp = blockIdx.x % S.fsplit;
    if (rt >= nrt)
        return;
    __shared__ double st[kTile];
    __shared__ double sw[kTile];
    __shared__ double sx[kTile * kMaxD];
    const Fp64Consts k = make_consts(S);
    const double itx2 = 1.0 / (S.tau_x * S.tau_x), ih2 = 1.0 / (S.h * S.h);
    const int row = rt * kTile + threadIdx.x;
    const bool valid = row < n;
    const int64_t R0 = S.row0;
    double tn = 0.0, wn = 0.0, xn[kMaxD];
    for (int q = 0; q < kMaxD; ++q)
        xn[q] = 0.0;
    if (valid) {
        tn = w.t64[R0 + row];
        wn = w.w64[R0 + row];
        for (int q = 0; q < d; ++q)
            xn[q] = w.x64[(R0 + row) * kMaxD + q];
    }
    int lo, hi;
    split_range(n, S.fsplit, sp, lo, hi);
    Nsum tot[kMaxD];
    for (int c0 = lo; c0 < hi; c0 += kTile) {
        const int cnt = min(kTile, hi - c0);
        __syncthreads();
        if (threadIdx.x < cnt) {
            st[threadIdx.x] = w.t64[R0 + c0 + threadIdx.x];
            sw[threadIdx.x] = w.w64[R0 + c0 + threadIdx.x];
            for (int q = 0; q < d; ++q)
                sx[threadIdx.x * kMaxD + q] = w.x64[(R0 + c0 + threadIdx.x) * kMaxD + q];
        }
        __syncthreads();
        if (!valid)
            continue;
        double part[kMaxD];
        for (int q = 0; q < kMaxD; ++q)
            part[q] = 0.0;
        for (int j = 0; j < cnt; ++j) {
            const double tm = st[j];
            if (tm == tn)
                continue;  // both indicators vanish (includes n' = n)
            double r2 = 0.0;
            for (int q = 0; q < d; ++q) {
                const double df = xn[q] - sx[j * kMaxD + q];
                r2 += df * df;
            }
            const double dt = tn - tm;
            const double wm = sw[j];
            const double mu = k.Cmu * exp(-(r2 * k.a + dt * dt * k.b));
            const double xi = k.Cxi * exp(-(k.omega * fabs(dt) + r2 * k.c));
            // xi_{nn'} lives in lambda_n when t_m < t_n, xi_{n'n} in lambda_m otherwise
            const double coef = mu * (wn + wm) * itx2 + xi * (tm < tn ? wn : wm) * ih2;
            for (int q = 0; q < d; ++q)
                part[q] += coef * (sx[j * kMaxD + q] - xn[q]);
        }
        for (int q = 0; q < d; ++q)
            tot[q].add(part[q]);
    }
    if (valid)
        for (int q = 0; q < d; ++q)
            w.F2[S.fpart2_0 + ((int64_t)sp * d + q) * S.npad + row] = tot[q].value();
}

}  // namespace

cudaError_t launch_pass1_fp64(const Work &w, int32_t set_lo, int32_t set_hi, int32_t max_fsplit, int64_t max_nblk,
                              bool theta, cudaStream_t s)
{
    dim3 grid((unsigned)(max_nblk * max_fsplit), (unsigned)(set_hi - set_lo));
    if (theta)
        pass1_fp64_kernel<true><<<grid, kTile, 0, s>>>(w, set_lo);
    else
        pass1_fp64_kernel<false><<<grid, kTile, 0, s>>>(w, set_lo);
    return cudaGetLastError();
}

cudaError_t launch_pass2_fp64(const Work &w, int32_t set_lo, int32_t set_hi, int32_t max_fsplit, int64_t max_nblk,
                              cudaStream_t s)
{
    dim3 grid((unsigned)(max_nblk * max_fsplit), (unsigned)(set_hi - set_lo));
    pass2_fp64_kernel<<<grid, kTile, 0, s>>>(w, set_lo);
    return cudaGetLastError();
}

}  // namespace hk
