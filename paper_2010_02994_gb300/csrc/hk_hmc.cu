// HMC over the event locations (Section 3; Neal 2011): leapfrog updates with
// reflection at box walls, Hamiltonian and accept step, all in FP64.
//
// The state lives in time-sorted row order (x64, with p and the box walls
// gathered into the same order).  Updates use explicitly rounded FP64
// multiplies and adds (no fused multiply-add), in the order
//   p <- p + (eps/2) g,   x <- x + eps p,   reflect,
// so that a trajectory repeats bit for bit given the same gradients.
#include <cmath>

#include "hk_internal.cuh"

namespace hk {

namespace {

__device__ __forceinline__ int set_of_row(const Work &w, const int64_t *set_row0, int64_t r)
{
    int lo = 0, hi = w.nsets - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (set_row0[mid] <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void split_hilo(double v, float &hi, float &lo)
{
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

// dst (sorted rows, stride kMaxD) <- src (caller order, row-major, width d)
__global__ void gather_sorted_kernel(Work w, const int64_t *set_row0, const double *__restrict__ src,
                                     double *__restrict__ dst, int64_t total_rows, double pad)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const SetDesc &S = w.sets[set_of_row(w, set_row0, r)];
        const int64_t i = r - S.row0;
        for (int k = 0; k < kMaxD; ++k) {
            double v = pad;
            if (i < S.n && k < S.d)
                v = src[S.x0 + (int64_t)w.perm[r] * S.d + k];
            dst[r * kMaxD + k] = v;
        }
    }
}

// Reflection at the walls of [lo, hi]; returns false if 1000 mirror steps
// did not bring the coordinate inside.
__device__ bool reflect(double &x, double &p, double lo, double hi)
{
    for (int it = 0; it < 1000; ++it) {
        if (x < lo) {
            x = __dsub_rn(__dmul_rn(2.0, lo), x);
            p = -p;
        } else if (x > hi) {
            x = __dsub_rn(__dmul_rn(2.0, hi), x);
            p = -p;
        } else {
            return true;
        }
    }
    return false;
}

// kicks = number of (eps/2) g half-kicks before the drift (1 for the first
// step, 2 afterwards: the previous step's closing kick and this step's
// opening kick, done as two separate roundings).  Repacks the mixed-path
// records of the moved coordinates when `repack`.  The first CTA also clears
// the per-evaluation control words (per-set flags and skip bounds) for the
// evaluation that follows the drift.
__global__ void kick_drift_kernel(Work w, const int64_t *set_row0, double *__restrict__ p,
                                  const double *__restrict__ g, const double *__restrict__ lo,
                                  const double *__restrict__ hi, const double *__restrict__ eps_dev,
                                  int64_t total_rows, int kicks, int repack, int32_t *refl_bad)
{
    if (blockIdx.x == 0) {
        for (int k = threadIdx.x; k < w.nsets; k += blockDim.x) {
            w.set_flags[k] = 0;
            w.set_cmmax[k] = 0;
        }
    }
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int set = set_of_row(w, set_row0, r);
        const SetDesc &S = w.sets[set];
        const int64_t i = r - S.row0;
        if (i >= S.n)
            continue;
        const double eps = eps_dev[set];
        const double half = __dmul_rn(0.5, eps);
        bool bad = false;
        float f[2 * kMaxD];
        for (int k = 0; k < S.d; ++k) {
            const int64_t e = r * kMaxD + k;
            double pk = p[e], xk = w.x64[e];
            const double gk = g[e];
            for (int q = 0; q < kicks; ++q)
                pk = __dadd_rn(pk, __dmul_rn(half, gk));
            xk = __dadd_rn(xk, __dmul_rn(eps, pk));
            if (lo)
                bad |= !reflect(xk, pk, lo[e], hi[e]);
            p[e] = pk;
            w.x64[e] = xk;
            if (repack)
                split_hilo(xk * S.kx, f[2 * k], f[2 * k + 1]);
        }
        if (repack) {
            for (int pl = 0; pl < nrec(S.d); ++pl) {
                float4 v = w.rec[S.rec0 + (int64_t)pl * S.npad + i];
                float *c = reinterpret_cast<float *>(&v);
                for (int q = 0; q < 4; ++q)
                    if (4 * pl + q < 2 * S.d)
                        c[q] = f[4 * pl + q];
                w.rec[S.rec0 + (int64_t)pl * S.npad + i] = v;
            }
        }
        if (bad)
            atomicOr(&refl_bad[set], 1);
    }
}

__global__ void kick_kernel(Work w, const int64_t *set_row0, double *__restrict__ p, const double *__restrict__ g,
                            const double *__restrict__ eps_dev, int64_t total_rows)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int set = set_of_row(w, set_row0, r);
        const SetDesc &S = w.sets[set];
        if (r - S.row0 >= S.n)
            continue;
        const double half = __dmul_rn(0.5, eps_dev[set]);
        for (int k = 0; k < S.d; ++k) {
            const int64_t e = r * kMaxD + k;
            p[e] = __dadd_rn(p[e], __dmul_rn(half, g[e]));
        }
    }
}

// H = -ell + sum p^2/2 of every set.  The FP64 sum of p^2/2 is split over
// kEnergyParts CTAs per set (FP64 is 1/64 of the FP32 rate here, so one SM
// per set would dominate a short trajectory step); each writes a
// compensated partial, and a one-CTA-per-set kernel adds them in order.
__global__ void __launch_bounds__(256) energy_parts_kernel(Work w, const double *__restrict__ p, double *parts)
{
    __shared__ double sh[256];
    const int set = blockIdx.x, part = blockIdx.y;
    const SetDesc &S = w.sets[set];
    const int64_t total = (int64_t)S.n * S.d;
    const int64_t per = (total + kEnergyParts - 1) / kEnergyParts;
    const int64_t lo = min((int64_t)part * per, total), hi = min(lo + per, total);
    double s = 0.0, c = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int64_t r = S.row0 + i / S.d;
        const double v = p[r * kMaxD + i % S.d];
        const double x = __dmul_rn(0.5, __dmul_rn(v, v));
        const double t = s + x;
        c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    sh[threadIdx.x] = s + c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        parts[set * kEnergyParts + part] = sh[0];
}

__global__ void energy_finish_kernel(Work w, const double *__restrict__ parts, double *H_out)
{
    const int set = blockIdx.x * blockDim.x + threadIdx.x;
    if (set >= w.nsets)
        return;
    double k = 0.0;
    for (int q = 0; q < kEnergyParts; ++q)
        k += parts[set * kEnergyParts + q];
    H_out[set] = -w.set_loglik[set] + k;
}

__global__ void accept_kernel(const double *H0, const double *H1, const double *log_u, const int32_t *refl_bad,
                              int32_t *accepted, int nsets)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsets)
        return;
    const double h0 = H0[s], h1 = H1[s];
    accepted[s] = (refl_bad[s] == 0 && isfinite(h0) && isfinite(h1) && log_u[s] < h0 - h1) ? 1 : 0;
}

__global__ void scatter_kernel(Work w, const int64_t *set_row0, const double *__restrict__ Xs,
                               double *__restrict__ X_out, const int32_t *__restrict__ accepted, int64_t total_rows)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int set = set_of_row(w, set_row0, r);
        const SetDesc &S = w.sets[set];
        const int64_t i = r - S.row0;
        if (i >= S.n || accepted[set] == 0)
            continue;
        for (int k = 0; k < S.d; ++k)
            X_out[S.x0 + (int64_t)w.perm[r] * S.d + k] = Xs[r * kMaxD + k];
    }
}

// Sorted rows (stride kMaxD) to the caller's order (row-major, width d),
// for every row of every set.
__global__ void to_caller_kernel(Work w, const int64_t *set_row0, const double *__restrict__ Xs,
                                 double *__restrict__ X_out, int64_t total_rows)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const SetDesc &S = w.sets[set_of_row(w, set_row0, r)];
        if (r - S.row0 >= S.n)
            continue;
        for (int k = 0; k < S.d; ++k)
            X_out[S.x0 + (int64_t)w.perm[r] * S.d + k] = Xs[r * kMaxD + k];
    }
}

// g_sorted += g (caller order; g null: nothing) and, once, set_loglik[0] +=
// *ell_add (ell_add null: nothing): folds a second potential term (BMDS, evaluated in the caller's
// order) into the Hawkes gradient and log-likelihood that the leapfrog and
// energy read.
__global__ void add_caller_term_kernel(Work w, const int64_t *set_row0, const double *__restrict__ g,
                                       double *__restrict__ g_sorted, int64_t total_rows, const double *ell_add)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && ell_add)
        w.set_loglik[0] += *ell_add;
    if (g == nullptr)  // the value alone
        return;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const SetDesc &S = w.sets[set_of_row(w, set_row0, r)];
        if (r - S.row0 >= S.n)
            continue;
        for (int k = 0; k < S.d; ++k)
            g_sorted[r * kMaxD + k] += g[S.x0 + (int64_t)w.perm[r] * S.d + k];
    }
}

// Element-wise HMC kernels run 64-thread CTAs: their FP64 updates are few
// per row, and small CTAs spread them over every SM (FP64 is 1/64 of the
// FP32 rate on this GPU).
constexpr int kElemThreads = 64;

int grid_for(int64_t n)
{
    int64_t g = (n + kElemThreads - 1) / kElemThreads;
    if (g < 1)
        g = 1;
    if (g > 8192)
        g = 8192;
    return (int)g;
}

}  // namespace

cudaError_t launch_gather_sorted(const Work &w, const int64_t *set_row0, const double *src, double *dst,
                                 int64_t total_rows, double pad, cudaStream_t s)
{
    gather_sorted_kernel<<<grid_for(total_rows), kElemThreads, 0, s>>>(w, set_row0, src, dst, total_rows, pad);
    return cudaGetLastError();
}

cudaError_t launch_kick_drift(const Work &w, const int64_t *set_row0, double *p, const double *g, const double *lo,
                              const double *hi, const double *eps_dev, int64_t total_rows, int kicks, bool repack,
                              int32_t *refl_bad, cudaStream_t s)
{
    kick_drift_kernel<<<grid_for(total_rows), kElemThreads, 0, s>>>(w, set_row0, p, g, lo, hi, eps_dev, total_rows, kicks,
                                                           repack ? 1 : 0, refl_bad);
    return cudaGetLastError();
}

cudaError_t launch_kick(const Work &w, const int64_t *set_row0, double *p, const double *g, const double *eps_dev,
                        int64_t total_rows, cudaStream_t s)
{
    kick_kernel<<<grid_for(total_rows), kElemThreads, 0, s>>>(w, set_row0, p, g, eps_dev, total_rows);
    return cudaGetLastError();
}

cudaError_t launch_energy(const Work &w, const double *p, double *H_out, double *parts, cudaStream_t s)
{
    energy_parts_kernel<<<dim3(w.nsets, kEnergyParts), 256, 0, s>>>(w, p, parts);
    energy_finish_kernel<<<(w.nsets + 127) / 128, 128, 0, s>>>(w, parts, H_out);
    return cudaGetLastError();
}

cudaError_t launch_accept(const double *H0, const double *H1, const double *log_u, const int32_t *refl_bad,
                          int32_t *accepted, int nsets, cudaStream_t s)
{
    accept_kernel<<<(nsets + 127) / 128, 128, 0, s>>>(H0, H1, log_u, refl_bad, accepted, nsets);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const Work &w, const int64_t *set_row0, const double *Xs, double *X_out,
                           const int32_t *accepted, int64_t total_rows, cudaStream_t s)
{
    scatter_kernel<<<grid_for(total_rows), kElemThreads, 0, s>>>(w, set_row0, Xs, X_out, accepted, total_rows);
    return cudaGetLastError();
}

cudaError_t launch_to_caller(const Work &w, const int64_t *set_row0, const double *Xs, double *X_out,
                             int64_t total_rows, cudaStream_t s)
{
    to_caller_kernel<<<grid_for(total_rows), kElemThreads, 0, s>>>(w, set_row0, Xs, X_out, total_rows);
    return cudaGetLastError();
}

cudaError_t launch_add_caller_term(const Work &w, const int64_t *set_row0, const double *g, double *g_sorted,
                                   int64_t total_rows, const double *ell_add, cudaStream_t s)
{
    add_caller_term_kernel<<<grid_for(total_rows), kElemThreads, 0, s>>>(w, set_row0, g, g_sorted, total_rows, ell_add);
    return cudaGetLastError();
}

}  // namespace hk
